"""GPU: the column step kernel against the block step kernel and the oracle.

The column kernel (float32 fields, I = 4 and 6) performs the same floating-
point operations in the same order as the block kernel, so the two must agree
bit for bit after any number of steps.  The cases cover crowded slabs (more
than 64 particles in a cell block: the unpipelined extra batches), sparse and
empty column segments, the smallest grid (N = 16, two blocks per axis), edge
positions (on nodes and one ulp from cell faces) and the RK2 stage-2 point
leaving the staged planes (slow path).  The oracle comparisons of the default
path are in test_gpu_parity.py; here the slow path is also checked against it.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2107_01104_gb300 as trk
import synth

pytestmark = pytest.mark.gpu
L = 2 * math.pi
DEV = "cuda"


def tracker(N, I, m, field, kind):
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=I, m=m, storage=trk.TRK_F32)
    t.set_step_kernel(kind)
    t.set_field(torch.from_numpy(field).to(DEV))
    return t


def positions(kind, N, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return rng.uniform(0.0, L, (3, n))
    if kind == "cluster":                      # every particle in cell block 0
        return rng.uniform(1e-3, 8 * L / N - 1e-3, (3, n))
    if kind == "slab":                         # one x3 slab of blocks only: most column segments empty
        p = rng.uniform(0.0, L, (3, n))
        p[2] = rng.uniform(3 * 8 * L / N, 4 * 8 * L / N, n)
        return p
    # edges: nodes, +-1 ulp of faces, unwrapped far outside [0, L)
    p = rng.uniform(-L, 2 * L, (3, n))
    q = n // 4
    delta = L / N
    p[:, :q] = rng.integers(-N, 2 * N, (3, q)) * delta
    faces = rng.integers(0, N + 1, (3, q)) * delta
    p[:, q:2 * q] = np.nextafter(faces, np.where(rng.random((3, q)) < 0.5, -np.inf, np.inf))
    return p


def run(N, I, m, field, pos, kind, scheme, steps, dt, cfl=False):
    t = tracker(N, I, m, field, kind)
    p = torch.from_numpy(pos).to(DEV)
    k = scheme + 1
    rhs = torch.zeros((max(k - 1, 1), 3, pos.shape[1]), dtype=torch.float32, device=DEV)
    if scheme != trk.TRK_RK2:
        t.advance(p, dt, 2, scheme, rhs=rhs, history_valid=0)
        t.advance(p, dt, steps - 2, scheme, rhs=rhs, history_valid=min(2, k - 1))
    else:
        t.advance(p, dt, steps, scheme)
    if cfl:
        with pytest.raises(trk.TrackerError) as e:
            t.sync()
        assert e.value.status == trk.TRK_ECFL
    else:
        t.sync()
    return p.cpu(), rhs.cpu()


CASES = [
    (16, 200, "uniform"),       # 2 blocks per axis, nseg = 2
    (32, 20000, "uniform"),     # ~312 particles per block: extra batches in every slab
    (64, 5000, "uniform"),      # ~10 per block, some empty blocks
    (64, 3000, "slab"),         # empty column segments
    (32, 3000, "cluster"),      # all in one block
    (32, 4000, "edges"),
    (128, 1 << 17, "uniform"),  # 32 per block, the benchmark density
]


@pytest.mark.parametrize("I,m", [(4, 1), (6, 2), (6, 3)])
@pytest.mark.parametrize("scheme", [trk.TRK_RK2, trk.TRK_AB2, trk.TRK_AB3, trk.TRK_AB4])
@pytest.mark.parametrize("N,n,layout", CASES)
def test_column_bit_identical_to_block(I, m, scheme, N, n, layout):
    field = synth.velocity_field_np(N, min(10, N // 3), 300 + N).astype(np.float32)
    pos = positions(layout, N, n, 11)
    steps, dt = 6, 4e-3
    pb, rb = run(N, I, m, field, pos, trk.TRK_STEP_BLOCK, scheme, steps, dt)
    pc, rc = run(N, I, m, field, pos, trk.TRK_STEP_COLUMN, scheme, steps, dt)
    assert torch.equal(pb, pc)
    if scheme != trk.TRK_RK2:
        assert torch.equal(rb, rc)


def test_column_cfl_slow_path_matches_oracle():
    """Stage-2 points several cells away: gathered from global memory, flagged, still exact."""
    N, n, dt = 32, 1500, 5e-3
    field = (synth.velocity_field_np(N, 10, 81) * 30.0).astype(np.float32)
    pos = synth.uniform_particles_np(n, 7)
    t = tracker(N, 6, 2, field, trk.TRK_STEP_COLUMN)
    p = torch.from_numpy(pos).to(DEV)
    t.advance(p, dt, 2, trk.TRK_RK2)
    with pytest.raises(trk.TrackerError) as e:
        t.sync()
    assert e.value.status == trk.TRK_ECFL
    ref = oracle.advance(field.astype(np.float64), pos, dt, 2, trk.TRK_SPLINE, 6, 2)
    # float32 weights and sums, |u| up to ~100: 2e-6 relative to the field rms (30) per stage
    assert np.abs(p.cpu().numpy() - ref).max() <= 5 * 2e-6 * 30.0 * dt * 2
    pb, _ = run(N, 6, 2, field, pos, trk.TRK_STEP_BLOCK, trk.TRK_RK2, 2, dt, cfl=True)
    assert torch.equal(p.cpu(), pb)


def test_column_nonfinite_flagged():
    N = 32
    field = synth.velocity_field_np(N, 10, 82).astype(np.float32)
    pos = synth.uniform_particles_np(400, 8)
    pos[1, 17] = np.nan
    pos[0, 3] = np.inf
    t = tracker(N, 4, 1, field, trk.TRK_STEP_COLUMN)
    p = torch.from_numpy(pos).to(DEV)
    t.advance(p, 1e-3, 2, trk.TRK_RK2)
    with pytest.raises(trk.TrackerError) as e:
        t.sync()
    assert e.value.status == trk.TRK_ENONFINITE
    ok = np.ones(400, bool)
    ok[[3, 17]] = False
    ref = oracle.advance(field.astype(np.float64), pos[:, ok], 1e-3, 2, trk.TRK_SPLINE, 4, 1)
    assert np.abs(p.cpu().numpy()[:, ok] - ref).max() <= 5 * 2e-6 * 1e-3 * 2


def test_step_kernel_selection():
    f = synth.velocity_field_np(16, 5, 1).astype(np.float32)
    t64 = trk.Tracker(16, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F64)
    with pytest.raises(trk.TrackerError) as e:
        t64.set_step_kernel(trk.TRK_STEP_COLUMN)
    assert e.value.status == trk.TRK_EINVAL
    t64.set_step_kernel(trk.TRK_STEP_BLOCK)
    t8 = trk.Tracker(16, family=trk.TRK_SPLINE, I=8, m=3, storage=trk.TRK_F32)
    with pytest.raises(trk.TrackerError):
        t8.set_step_kernel(trk.TRK_STEP_COLUMN)
    t6 = tracker(16, 6, 2, f, trk.TRK_STEP_COLUMN)
    with pytest.raises(trk.TrackerError):
        t6.set_step_kernel(7)
    t6.set_step_kernel(trk.TRK_STEP_AUTO)
    # a block shape other than 8^3 has no column kernel
    t6.close()
    t6 = tracker(16, 6, 2, f, trk.TRK_STEP_AUTO)
    trk.tracker_set_block(t6.h, 16, 16, 1)
    with pytest.raises(trk.TrackerError):
        t6.set_step_kernel(trk.TRK_STEP_COLUMN)
