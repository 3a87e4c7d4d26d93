"""Argument checks of the binning entry points and the tracker's device.

The kernels write keys[np], perm[np] and offsets[nblocks + 1] into caller
arrays, so a wrong size, type or device must be refused before any launch:
by the binding (sizes, dtypes, devices of torch tensors) and by the library
itself (a pointer that is not device memory of the current device).
"""
import ctypes
import math

import pytest
import torch

import paper_2107_01104_gb300 as trk

pytestmark = pytest.mark.gpu
L = 2 * math.pi


def _pos(n, N=32):
    g = torch.Generator(device="cpu").manual_seed(n)
    return (torch.rand((3, n), generator=g, dtype=torch.float64) * L).cuda()


@pytest.mark.parametrize("what", ["offsets_short", "offsets_int64", "keys_short", "perm_cpu", "nonfinite_empty"])
def test_static_binning_refuses_bad_outputs(what):
    N, n = 32, 1000
    pos = _pos(n, N)
    nb = (N // 8) ** 3
    kw = {}
    if what == "offsets_short":
        kw["offsets"] = torch.empty(nb, dtype=torch.int32, device="cuda")
    elif what == "offsets_int64":
        kw["offsets"] = torch.empty(nb + 1, dtype=torch.int64, device="cuda")
    elif what == "keys_short":
        kw["keys"] = torch.empty(n - 1, dtype=torch.int32, device="cuda")
    elif what == "perm_cpu":
        kw["perm"] = torch.empty(n, dtype=torch.int32)
    else:
        kw["nonfinite"] = torch.empty(0, dtype=torch.int32, device="cuda")
    with pytest.raises((ValueError, TypeError)):
        trk.tracker_bin_static(pos, N, L, **kw)


def test_tracker_bin_refuses_short_offsets():
    t = trk.Tracker(32, family=trk.TRK_LAGRANGE, I=4, storage=trk.TRK_F32)
    pos = _pos(500)
    with pytest.raises(ValueError):
        trk.tracker_bin(t.h, pos, offsets=torch.empty(8, dtype=torch.int32, device="cuda"))
    t.close()


def test_library_refuses_host_pointers():
    """Called through the C ABI directly: a host array as an output is refused
    with TRK_EINVAL (the library checks where each pointer lives) and nothing
    is launched."""
    lib = trk.load_library()
    N, n = 32, 100
    pos = _pos(n, N)
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    offsets_host = torch.empty((N // 8) ** 3 + 1, dtype=torch.int32).pin_memory()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.tracker_bin_static(n, ctypes.c_void_p(pos.data_ptr()), N, L, 8, 8, 8, ctypes.c_void_p(keys.data_ptr()),
                                ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(offsets_host.data_ptr()), None, st)
    assert rc == trk.TRK_EINVAL
    assert "device memory" in trk.tracker_last_error()
    t = trk.Tracker(N, family=trk.TRK_LAGRANGE, I=4, storage=trk.TRK_F32)
    rc = lib.tracker_bin(t.h, n, ctypes.c_void_p(pos.data_ptr()), None, ctypes.c_void_p(perm.data_ptr()),
                         ctypes.c_void_p(offsets_host.data_ptr()))
    assert rc == trk.TRK_EINVAL
    t.close()


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs two visible GPUs")
def test_tracker_refuses_another_current_device():
    """A tracker made on device 0, called with device 1 current through the C
    ABI, returns TRK_EINVAL before touching either GPU."""
    lib = trk.load_library()
    with torch.cuda.device(0):
        t = trk.Tracker(32, family=trk.TRK_LAGRANGE, I=4, storage=trk.TRK_F32)
    with torch.cuda.device(1):
        assert lib.tracker_sync(t.h) == trk.TRK_EINVAL
        assert "device" in trk.tracker_last_error()
    t.close()
