"""tracker_bin_static: binning for callers that cannot allocate device memory.

It must give exactly what tracker_bin gives (binning is bit-exact), on two
calls in a row, even though every call reuses the same fixed scratch array
inside the library.  This file is collected last so that a run stopping at its
first failure has already run every other test; it also passes on its own in a
fresh process.
"""
import math

import numpy as np
import pytest
import torch

import paper_2107_01104_gb300 as trk

pytestmark = pytest.mark.gpu
L = 2 * math.pi


def positions(n, seed, N):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-L, 2 * L, (3, n))
    pos[:, : n // 10] = rng.integers(-N, 2 * N, (3, n // 10)) * (L / N)     # on nodes
    return torch.from_numpy(pos).cuda()


@pytest.mark.parametrize("N,block", [(64, (8, 8, 8)), (256, (8, 8, 8)), (32, (32, 32, 1))])
def test_static_binning_matches_tracker_bin_twice(N, block):
    t = trk.Tracker(N, family=trk.TRK_LAGRANGE, I=4, storage=trk.TRK_F32)
    if block != (8, 8, 8):
        trk.tracker_set_block(t.h, *block)
    # two calls in a row: a large one, then a smaller one whose result must not
    # depend on what the first call left in the shared scratch array
    for n, seed in ((200_003, 1), (70_001, 2)):
        pos = positions(n, seed, N)
        k_ref, p_ref, o_ref = t.bin(pos)
        flag = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        k, p, o = trk.tracker_bin_static(pos, N, L, block, nonfinite=flag)
        torch.cuda.synchronize()
        assert torch.equal(k, k_ref)
        assert torch.equal(p, p_ref)
        assert torch.equal(o, o_ref)
        assert int(flag.item()) == 0
    t.sync()
    t.close()


def test_static_binning_flags_nonfinite_and_rejects_oversize():
    N = 32
    pos = positions(1000, 3, N)
    pos[1, 5] = float("nan")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    trk.tracker_bin_static(pos, N, L, nonfinite=flag)
    torch.cuda.synchronize()
    assert int(flag.item()) == 1
    big = torch.zeros((3, (1 << 18) + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(trk.TrackerError) as e:
        trk.tracker_bin_static(big, N, L)
    assert e.value.status == trk.TRK_EINVAL
    # a clean call afterwards clears the flag
    pos[1, 5] = 0.5
    trk.tracker_bin_static(pos, N, L, nonfinite=flag)
    torch.cuda.synchronize()
    assert int(flag.item()) == 0
