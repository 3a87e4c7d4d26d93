"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Same-input comparisons give the oracle exactly the field values the library
stores (float32, or hi + lo of the split-bf16 pair, promoted to float64), so
the difference measures the library's arithmetic alone.  Tolerances:
  binning                     bit-exact keys, permutation and offsets
  float64 storage             1e-12 relative: max error <= 1e-12 x max|field|
                              (the separable float64 sum rounds in a different
                              order than the oracle's direct quadruple loop)
  float32 / split-bf16        max error <= 2e-6 x field rms (float32 weights
                              and sums, same input)
  split-bf16 vs float64 field rms error <= 1e-5 x field rms (hi + lo keeps
                              about 2^-18 of each value, so the max error over
                              many particles can exceed 1e-5 where |u| ~ 4)
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

KERNELS = [
    (trk.TRK_LAGRANGE, 4, 0), (trk.TRK_LAGRANGE, 6, 0), (trk.TRK_LAGRANGE, 8, 0),
    (trk.TRK_SPLINE, 4, 1), (trk.TRK_SPLINE, 6, 2), (trk.TRK_SPLINE, 8, 3),
    (trk.TRK_SPLINE, 4, 2), (trk.TRK_SPLINE, 6, 3), (trk.TRK_SPLINE, 8, 4),   # degree I+1 variants
    (trk.TRK_SPLINE, 6, 0), (trk.TRK_SPLINE, 8, 1),
]
STORAGES = [trk.TRK_F64, trk.TRK_F32, trk.TRK_BF16X2]
TOL = {trk.TRK_F64: 1e-12, trk.TRK_F32: 2e-6, trk.TRK_BF16X2: 2e-6}


def stored(field: np.ndarray, storage: int) -> np.ndarray:
    """The values the library holds for `field` in `storage` (float64 array)."""
    if storage == trk.TRK_F64:
        return field
    f32 = field.astype(np.float32)
    if storage == trk.TRK_F32:
        return f32.astype(np.float64)
    hi, lo = synth.bf16_split(torch.from_numpy(f32))
    return hi.double().numpy() + lo.double().numpy()


def edge_positions(N, n, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-L, 2 * L, (3, n))
    delta = L / N
    q = n // 8
    k = rng.integers(-N, 2 * N, (3, q))
    pos[:, :q] = k * delta                                            # on nodes
    faces = rng.integers(0, N + 1, (3, q)) * delta
    pos[:, q:2 * q] = np.nextafter(faces, np.where(rng.random((3, q)) < 0.5, -np.inf, np.inf))  # +-1 ulp of faces
    if n >= 2 * q + 16:
        pos[:, 2 * q:2 * q + 16] = pos[:, :16]                        # duplicates
    return pos


def make_tracker(N, family, I, m, storage, field):
    t = trk.Tracker(N, family=family, I=I, m=m, storage=storage)
    t.set_field(torch.from_numpy(field).to(DEV))
    return t


@pytest.mark.parametrize("N,n", [(16, 0), (16, 1), (16, 37), (64, 5000), (64, 100003), (256, 70001)])
def test_binning_bit_exact(N, n):
    pos = edge_positions(N, max(n, 1), 11 + N)[:, :n]
    t = trk.Tracker(N, family=trk.TRK_LAGRANGE, I=4, storage=trk.TRK_F32)
    keys, perm, offsets = t.bin(torch.from_numpy(np.ascontiguousarray(pos)).to(DEV))
    t.sync()
    rk, rp, ro = oracle.bin_particles(pos, N, (8, 8, 8))
    np.testing.assert_array_equal(keys.cpu().numpy(), rk)
    np.testing.assert_array_equal(perm.cpu().numpy(), rp)
    np.testing.assert_array_equal(offsets.cpu().numpy(), ro)


@pytest.mark.parametrize("B", [(64, 64, 1), (4, 2, 8), (1, 1, 1), (16, 16, 16)])
def test_binning_other_block_shapes(B):
    N = 64
    pos = edge_positions(N, 20000, 5)
    t = trk.Tracker(N, family=trk.TRK_LAGRANGE, I=4, storage=trk.TRK_F32)
    trk.tracker_set_block(t.h, *B)
    keys, perm, offsets = t.bin(torch.from_numpy(pos).to(DEV))
    rk, rp, ro = oracle.bin_particles(pos, N, B)
    np.testing.assert_array_equal(keys.cpu().numpy(), rk)
    np.testing.assert_array_equal(perm.cpu().numpy(), rp)
    np.testing.assert_array_equal(offsets.cpu().numpy(), ro)


@pytest.mark.parametrize("family,I,m", KERNELS)
@pytest.mark.parametrize("storage", STORAGES)
def test_interpolate_parity(family, I, m, storage):
    N, n = 32, 4099
    field = synth.velocity_field_np(N, 10, 77)
    pos = edge_positions(N, n, 3)
    t = make_tracker(N, family, I, m, storage, field)
    out = t.interpolate(torch.from_numpy(pos).to(DEV), out_dtype=torch.float64)
    t.sync()
    ref = oracle.interp(stored(field, storage), pos, family, I, m)
    err = np.abs(out.cpu().numpy() - ref).max()
    scale = np.abs(field).max() if storage == trk.TRK_F64 else np.sqrt(np.mean(field ** 2))
    assert err <= TOL[storage] * scale, err
    if storage == trk.TRK_BF16X2:
        truth = oracle.interp(field, pos, family, I, m)
        d = out.cpu().numpy() - truth
        assert np.sqrt(np.mean(d ** 2)) <= 1e-5 * np.sqrt(np.mean(field ** 2))
        assert np.abs(d).max() <= 2.0 ** -17 * np.abs(field).max() * 2.0
    if storage == trk.TRK_F32:
        # against the float64 field itself: the storage rounding (2^-24
        # relative per value) is inside the same 2e-6 x rms bar
        truth = oracle.interp(field, pos, family, I, m)
        assert np.abs(out.cpu().numpy() - truth).max() <= 2e-6 * np.sqrt(np.mean(field ** 2))


@pytest.mark.parametrize("C", [1, 2, 4, 9, 12])
def test_interpolate_component_chunks(C):
    N, n = 32, 3001
    rng = np.random.default_rng(C)
    field = rng.standard_normal((C, N, N, N))
    pos = rng.uniform(0, L, (3, n))
    t = make_tracker(N, trk.TRK_SPLINE, 8, 3, trk.TRK_F32, field)
    out = t.interpolate(torch.from_numpy(pos).to(DEV), out_dtype=torch.float32)
    ref = oracle.interp(stored(field, trk.TRK_F32), pos, trk.TRK_SPLINE, 8, 3)
    assert np.abs(out.cpu().numpy() - ref).max() <= 4e-6 * field.std() * 3


@pytest.mark.parametrize("family,I,m", [(trk.TRK_LAGRANGE, 4, 0), (trk.TRK_SPLINE, 6, 2), (trk.TRK_SPLINE, 8, 3),
                                        (trk.TRK_SPLINE, 6, 3)])
@pytest.mark.parametrize("storage", [trk.TRK_F64, trk.TRK_F32])
def test_interpolate_gradient_parity(family, I, m, storage):
    N, n = 32, 2000
    field = synth.velocity_field_np(N, 10, 78)
    pos = edge_positions(N, n, 4)
    t = make_tracker(N, family, I, m, storage, field)
    out = t.interpolate(torch.from_numpy(pos).to(DEV), out_dtype=torch.float64, deriv=True)
    ref = oracle.interp(stored(field, storage), pos, family, I, m, deriv=True).reshape(9, n)
    tol = (1e-11 if storage == trk.TRK_F64 else 4e-6) * N / L
    assert np.abs(out.cpu().numpy() - ref).max() <= tol


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("family,I,m", [(trk.TRK_SPLINE, 6, 2), (trk.TRK_LAGRANGE, 4, 0), (trk.TRK_SPLINE, 8, 3)])
def test_rk2_parity(storage, family, I, m):
    N, n, dt, steps = 32, 3000, 5e-3, 6
    field = synth.velocity_field_np(N, 10, 79)
    pos = edge_positions(N, n, 5)
    t = make_tracker(N, family, I, m, storage, field)
    p = torch.from_numpy(pos).to(DEV)
    t.advance(p, dt, steps, trk.TRK_RK2)
    t.sync()
    ref = oracle.advance(stored(field, storage), pos, dt, steps, family, I, m, scheme=oracle.RK2)
    tol = 1e-11 if storage == trk.TRK_F64 else 5 * 2e-6 * dt * steps
    assert np.abs(p.cpu().numpy() - ref).max() <= tol


@pytest.mark.parametrize("storage", [trk.TRK_F64, trk.TRK_F32])
def test_ab2_parity_and_history(storage):
    N, n, dt = 32, 2500, 4e-3
    field = synth.velocity_field_np(N, 10, 80)
    pos = edge_positions(N, n, 6)
    t = make_tracker(N, trk.TRK_SPLINE, 6, 2, storage, field)
    p = torch.from_numpy(pos).to(DEV)
    rhs = torch.zeros((3, n), dtype=torch.float32, device=DEV)
    t.advance(p, dt, 3, trk.TRK_AB2, rhs=rhs, history_valid=False)
    t.advance(p, dt, 4, trk.TRK_AB2, rhs=rhs, history_valid=True)
    t.sync()
    ref, ref_rhs = oracle.advance(stored(field, storage), pos, dt, 7, trk.TRK_SPLINE, 6, 2, scheme=oracle.AB2)
    # the library keeps the AB2 history in float32 (documented)
    tol = 1e-7 if storage == trk.TRK_F64 else 5 * 2e-6 * dt * 7
    assert np.abs(p.cpu().numpy() - ref).max() <= tol
    assert np.abs(rhs.cpu().numpy() - ref_rhs).max() <= 2e-6 * 3


@pytest.mark.parametrize("N,layout", [(64, "uniform"), (256, "uniform"), (64, "cluster"), (32, "slices")])
def test_interpolate_large_sets(N, layout):
    """Interpolation of more than 2^20 particles (counting-sort binning with
    the permutation read by the kernels): every output of the block and the
    direct kernel bit-identical on all particles, and against the oracle on a
    sample.  Ragged count; a cluster where one cell block holds every
    particle; x3 slices (the block shape N x N x 1, direct kernel only)."""
    n = (1 << 20) + 12345
    rng = np.random.default_rng(N)
    field = synth.velocity_field_np(N, min(10, N // 3), 85)
    if layout == "cluster":
        pos = rng.uniform(0.01, 8 * L / N - 0.01, (3, n))
    else:
        pos = rng.uniform(-L, 2 * L, (3, n))
    p = torch.from_numpy(pos).to(DEV)
    outs = []
    for kind in (trk.TRK_STEP_BLOCK, trk.TRK_STEP_DIRECT):
        t = make_tracker(N, trk.TRK_SPLINE, 6, 2, trk.TRK_F32, field)
        if layout == "slices":
            trk.tracker_set_block(t.h, N, N, 1)
        t.set_step_kernel(kind)
        if layout == "slices" and kind == trk.TRK_STEP_BLOCK:
            t.close()
            continue
        outs.append(t.interpolate(p, out_dtype=torch.float64).cpu())
        t.sync()
        t.close()
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    ix = rng.choice(n, 3000, replace=False)
    ref = oracle.interp(stored(field, trk.TRK_F32), pos[:, ix], trk.TRK_SPLINE, 6, 2)
    assert np.abs(outs[0].numpy()[:, ix] - ref).max() <= 2e-6 * np.sqrt(np.mean(field ** 2))


def test_cfl_violation_takes_exact_slow_path():
    N, n = 32, 500
    field = synth.velocity_field_np(N, 10, 81) * 30.0     # |dt u| >> delta
    pos = synth.uniform_particles_np(n, 7)
    t = make_tracker(N, trk.TRK_SPLINE, 6, 2, trk.TRK_F64, field)
    p = torch.from_numpy(pos).to(DEV)
    t.advance(p, 5e-3, 2, trk.TRK_RK2)
    with pytest.raises(trk.TrackerError) as e:
        t.sync()
    assert e.value.status == trk.TRK_ECFL
    ref = oracle.advance(field, pos, 5e-3, 2, trk.TRK_SPLINE, 6, 2)
    assert np.abs(p.cpu().numpy() - ref).max() <= 1e-10


def test_nonfinite_position_is_flagged_not_faulted():
    N = 32
    field = synth.velocity_field_np(N, 10, 82)
    pos = synth.uniform_particles_np(100, 8)
    pos[1, 17] = np.nan
    pos[0, 3] = np.inf
    t = make_tracker(N, trk.TRK_LAGRANGE, 4, 0, trk.TRK_F32, field)
    out = t.interpolate(torch.from_numpy(pos).to(DEV))
    with pytest.raises(trk.TrackerError) as e:
        t.sync()
    assert e.value.status == trk.TRK_ENONFINITE
    ok = np.ones(100, bool); ok[[3, 17]] = False
    ref = oracle.interp(stored(field, trk.TRK_F32), pos[:, ok], trk.TRK_LAGRANGE, 4, 0)
    assert np.abs(out.cpu().numpy()[:, ok] - ref).max() <= 2e-6
    t.sync()    # flags were cleared


def test_empty_and_single():
    N = 16
    field = synth.velocity_field_np(N, 5, 83)
    t = make_tracker(N, trk.TRK_SPLINE, 4, 1, trk.TRK_F32, field)
    e = torch.empty((3, 0), dtype=torch.float64, device=DEV)
    assert t.interpolate(e).shape == (3, 0)
    t.advance(e, 1e-3, 3)
    one = torch.tensor([[0.1], [6.2], [3.3]], dtype=torch.float64, device=DEV)
    out = t.interpolate(one, out_dtype=torch.float64)
    ref = oracle.interp(stored(field, trk.TRK_F32), one.cpu().numpy(), trk.TRK_SPLINE, 4, 1)
    assert np.abs(out.cpu().numpy() - ref).max() <= 2e-6
    t.sync()


def test_dense_cluster_exceeds_one_batch():
    """More particles in one block than threads per CTA: batches of 256 reuse the halo."""
    N, n = 32, 3000
    field = synth.velocity_field_np(N, 10, 84)
    rng = np.random.default_rng(9)
    pos = rng.uniform(1e-3, 8 * L / N - 1e-3, (3, n))          # cells 0..7: all inside block 0
    t = make_tracker(N, trk.TRK_SPLINE, 8, 3, trk.TRK_F32, field)
    out = t.interpolate(torch.from_numpy(pos).to(DEV), out_dtype=torch.float64)
    ref = oracle.interp(stored(field, trk.TRK_F32), pos, trk.TRK_SPLINE, 8, 3)
    assert np.abs(out.cpu().numpy() - ref).max() <= 2e-6
    p = torch.from_numpy(pos).to(DEV)
    t.advance(p, 5e-3, 3)
    ref = oracle.advance(stored(field, trk.TRK_F32), pos, 5e-3, 3, trk.TRK_SPLINE, 8, 3)
    assert np.abs(p.cpu().numpy() - ref).max() <= 5 * 2e-6 * 5e-3 * 3


def test_config1_small_plain_method():
    """32^3 float64 field |k| <= 8, 1e4 tracers, Lagrange I=4, one RK2 step dt=1e-3."""
    N = 32
    field = synth.velocity_field_np(N, 8, 1000)
    pos = synth.uniform_particles_np(10_000, 1)
    t = make_tracker(N, trk.TRK_LAGRANGE, 4, 0, trk.TRK_F64, field)
    p = torch.from_numpy(pos).to(DEV)
    u = t.interpolate(p, out_dtype=torch.float64)
    t.advance(p, 1e-3, 1, trk.TRK_RK2)
    t.sync()
    np.testing.assert_allclose(u.cpu().numpy(), oracle.interp(field, pos, trk.TRK_LAGRANGE, 4, 0), rtol=0, atol=1e-12)
    np.testing.assert_allclose(p.cpu().numpy(), oracle.advance(field, pos, 1e-3, 1, trk.TRK_LAGRANGE, 4, 0),
                               rtol=0, atol=1e-13)


def _sync_allow_cfl(t):
    """A CFL flag marks particles that took the exact slow path; it is not an error here."""
    try:
        t.sync()
    except trk.TrackerError as e:
        if e.status != trk.TRK_ECFL:
            raise


@pytest.mark.parametrize("kind", [trk.TRK_STEP_AUTO, trk.TRK_STEP_COLUMN, trk.TRK_STEP_DIRECT])
def test_config2_full_size_sampled(kind):
    """256^3 float32 field |k| <= 85, 2^20 tracers, spline I=6 (m=2), RK2 dt=5e-3, re-binned every step,
    in the launch configuration bench.py times (AUTO: 8 steps, so the kernels are timed and one kept).
    Binning checked bit-exactly for all particles; trajectories on a 3000-particle sample."""
    N, n, dt, steps = 256, 1 << 20, 5e-3, 8
    field = synth.velocity_field_np(N, 85, 1001).astype(np.float32)
    pos = synth.uniform_particles_np(n, 2)
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_step_kernel(kind)
    t.set_field(torch.from_numpy(field).to(DEV))
    p = torch.from_numpy(pos).to(DEV)
    keys, perm, offsets = t.bin(p)
    rk, rp, ro = oracle.bin_particles(pos, N, (8, 8, 8))
    np.testing.assert_array_equal(perm.cpu().numpy(), rp)
    np.testing.assert_array_equal(offsets.cpu().numpy(), ro)
    t.advance(p, dt, steps, trk.TRK_RK2)
    _sync_allow_cfl(t)
    if kind == trk.TRK_STEP_AUTO:
        assert t.last_step_kernel() in (trk.TRK_STEP_COLUMN, trk.TRK_STEP_DIRECT)
    sample = np.random.default_rng(0).choice(n, 3000, replace=False)
    ref = oracle.advance(field.astype(np.float64), pos[:, sample], dt, steps, trk.TRK_SPLINE, 6, 2)
    assert np.abs(p.cpu().numpy()[:, sample] - ref).max() <= 5 * 2e-6 * dt * steps


def test_config2_full_size_column_and_direct_identical():
    """The two step kernels the timing chooses between give the same bits at full size."""
    N, n, dt, steps = 256, 1 << 20, 5e-3, 3
    field = synth.velocity_field_np(N, 85, 1001).astype(np.float32)
    pos = synth.uniform_particles_np(n, 2)
    res = []
    for kind in (trk.TRK_STEP_COLUMN, trk.TRK_STEP_DIRECT):
        t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
        t.set_step_kernel(kind)
        t.set_field(torch.from_numpy(field).to(DEV))
        p = torch.from_numpy(pos).to(DEV)
        t.advance(p, dt, steps, trk.TRK_RK2)
        _sync_allow_cfl(t)
        res.append(p.cpu())
        t.close()
    assert torch.equal(res[0], res[1])
