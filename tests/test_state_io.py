"""Tracer-set state files (host code, no GPU): round trips, the documented
byte layout and checksum, and the failure modes (corruption, truncation,
trailing bytes, argument errors)."""
import os
import struct

import numpy as np
import pytest
import torch

import paper_2107_01104_gb300 as trk

MASK = (1 << 64) - 1


def fnv_words(data: bytes, h: int = 14695981039346656037) -> int:
    """The documented checksum, written out independently: 64-bit words, then tail bytes."""
    n8 = len(data) // 8 * 8
    for (w,) in struct.iter_unpack("<Q", data[:n8]):
        h = ((h ^ w) * 1099511628211) & MASK
    for b in data[n8:]:
        h = ((h ^ b) * 1099511628211) & MASK
    return h


def make(np_, scheme, seed=0):
    g = torch.Generator().manual_seed(seed)
    pos = torch.rand((3, np_), generator=g, dtype=torch.float64) * 7 - 1
    rhs = torch.randn((scheme, 3, np_), generator=g, dtype=torch.float32) if scheme else None
    return pos, rhs


def write(path, pos, rhs, scheme, hv=0, **kw):
    args = dict(step=17, time=0.085, dt=0.005, N=64, L=2 * np.pi, family=trk.TRK_SPLINE, I=6, m=2)
    args.update(kw)
    trk.tracker_state_write(str(path), pos, rhs, scheme, hv, **args)


@pytest.mark.parametrize("scheme,hv", [(trk.TRK_RK2, 0), (trk.TRK_AB2, 1), (trk.TRK_AB3, 1), (trk.TRK_AB4, 3)])
@pytest.mark.parametrize("np_", [0, 1, 1001])
def test_round_trip(tmp_path, scheme, hv, np_):
    pos, rhs = make(np_, scheme)
    f = tmp_path / "s.trk"
    write(f, pos, rhs, scheme, hv)
    p2, r2, info = trk.tracker_state_read(str(f))
    assert torch.equal(pos, p2)
    assert (r2 is None) == (rhs is None) and (rhs is None or torch.equal(rhs, r2))
    assert info == {"N": 64, "L": 2 * np.pi, "family": trk.TRK_SPLINE, "I": 6, "m": 2, "np": np_, "scheme": scheme,
                    "history_valid": hv, "step": 17, "time": 0.085, "dt": 0.005}
    assert trk.tracker_state_read_info(str(f)) == info


def test_byte_layout_and_checksums(tmp_path):
    np_, scheme = 37, trk.TRK_AB3
    pos, rhs = make(np_, scheme, 1)
    f = tmp_path / "s.trk"
    write(f, pos, rhs, scheme, 2)
    b = f.read_bytes()
    assert len(b) == 96 + 24 * np_ + 4 * 6 * np_
    assert b[:8] == b"TRKSTAT1"
    version, hbytes, N, fam, I, m, L, n, sch, hv, step, time, dt, psum, hsum = struct.unpack_from(
        "<IIiiiidqiiqddQQ", b, 8)
    assert (version, hbytes, N, fam, I, m, n, sch, hv, step) == (1, 96, 64, 1, 6, 2, np_, scheme, 2, 17)
    assert (L, time, dt) == (2 * np.pi, 0.085, 0.005)
    payload = b[96:]
    assert payload[:24 * np_] == pos.numpy().tobytes()                  # [3][np] float64, caller order
    assert payload[24 * np_:] == rhs.numpy().tobytes()                  # [3(k-1)][np] float32
    assert psum == fnv_words(payload)
    assert hsum == fnv_words(b[:88])


def test_corruption_and_truncation_detected(tmp_path):
    pos, rhs = make(100, trk.TRK_AB2, 2)
    f = tmp_path / "s.trk"
    write(f, pos, rhs, trk.TRK_AB2, 1)
    good = f.read_bytes()
    cases = {
        "payload bit": good[:500] + bytes([good[500] ^ 1]) + good[501:],
        "header bit": good[:50] + bytes([good[50] ^ 4]) + good[51:],
        "truncated payload": good[:-3],
        "truncated header": good[:40],
        "trailing bytes": good + b"\0",
        "magic": b"XRKSTAT1" + good[8:],
    }
    for name, data in cases.items():
        g = tmp_path / "bad.trk"
        g.write_bytes(data)
        with pytest.raises(trk.TrackerError) as e:
            trk.tracker_state_read(str(g))
        assert e.value.status == trk.TRK_EIO, name
    with pytest.raises(trk.TrackerError) as e:
        trk.tracker_state_read(str(tmp_path / "missing.trk"))
    assert e.value.status == trk.TRK_EIO


def test_argument_errors(tmp_path):
    pos, rhs = make(10, trk.TRK_AB2, 3)
    with pytest.raises(trk.TrackerError) as e:
        write(tmp_path / "a.trk", pos, rhs, trk.TRK_AB2, 2)              # AB2 keeps one entry
    assert e.value.status == trk.TRK_EINVAL
    with pytest.raises(trk.TrackerError) as e:
        write(tmp_path / "b.trk", pos, None, 7, 0)                     # unknown scheme
    assert e.value.status == trk.TRK_EINVAL
    with pytest.raises(ValueError):
        write(tmp_path / "c.trk", pos, None, trk.TRK_AB2, 0)           # AB2 needs its history
    with pytest.raises(trk.TrackerError) as e:
        write(tmp_path / "no" / "such" / "dir.trk", pos, rhs, trk.TRK_AB2, 1)
    assert e.value.status == trk.TRK_EIO
    assert not (tmp_path / "no").exists()
    # buffers of the wrong particle count
    write(tmp_path / "d.trk", pos, rhs, trk.TRK_AB2, 1)
    lib = trk.load_library()
    buf = torch.empty((3, 11), dtype=torch.float64)
    info = trk.trk_state_info()
    import ctypes
    rc = lib.tracker_state_read(os.fsencode(str(tmp_path / "d.trk")), 11, ctypes.c_void_p(buf.data_ptr()), None,
                                ctypes.byref(info))
    assert rc == trk.TRK_EINVAL


def test_failed_write_keeps_existing_file(tmp_path):
    pos, rhs = make(50, trk.TRK_AB2, 4)
    f = tmp_path / "s.trk"
    write(f, pos, rhs, trk.TRK_AB2, 1)
    before = f.read_bytes()
    with pytest.raises(trk.TrackerError):
        write(f, pos, rhs, trk.TRK_AB2, 5)                              # rejected before any byte is written
    assert f.read_bytes() == before
    assert [p.name for p in tmp_path.iterdir()] == ["s.trk"]            # no temporary left behind
