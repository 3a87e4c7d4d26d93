"""GPU adjoint (tracker_adjoint, autograd) against the oracle's adjoint and finite differences.

Tolerance (the stated bar): gradients within 1e-6 relative of the oracle
gradient, in the 2-norm over all entries; same-input mode (the oracle gets the
field values the library stores)."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2107_01104_gb300 as trk
from paper_2107_01104_gb300.autograd import advect
import synth

pytestmark = pytest.mark.gpu
FAM, I, M = trk.TRK_SPLINE, 6, 2
L = 2 * math.pi


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def stored(field, storage):
    return field if storage == trk.TRK_F64 else field.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("storage", [trk.TRK_F64, trk.TRK_F32])
@pytest.mark.parametrize("steps,ckpt", [(6, 4), (5, 5), (3, 1)])
def test_adjoint_matches_oracle(storage, steps, ckpt):
    N, n, dt = 32, 600, 5e-3
    field = synth.velocity_field_np(N, 10, 90)
    pos = synth.uniform_particles_np(n, 9)
    fs = stored(field, storage)
    t = trk.Tracker(N, family=FAM, I=I, m=M, storage=storage)
    t.set_field(torch.from_numpy(field).cuda())
    posT = oracle.advance(fs, pos, dt, steps, FAM, I, M)
    lam = 2 * posT
    gpos_ref, gf_ref = oracle.adjoint_rk2(fs, pos, lam, dt, steps, FAM, I, M)
    gf = torch.zeros((3, N, N, N), dtype=torch.float64, device="cuda")
    gpos, _ = t.adjoint(torch.from_numpy(pos).cuda(), torch.from_numpy(lam).cuda(), dt, steps, ckpt, grad_field=gf)
    t.sync()
    tol = 1e-10 if storage == trk.TRK_F64 else 1e-6
    assert rel(gpos.cpu().numpy(), gpos_ref) <= tol
    assert rel(gf.cpu().numpy(), gf_ref) <= tol


def test_adjoint_against_gpu_finite_differences():
    """Central differences (h = 1e-6) of the float64 GPU forward on sampled coordinates."""
    N, n, dt, steps = 32, 40, 5e-3, 4
    field = synth.velocity_field_np(N, 10, 91)
    pos = synth.uniform_particles_np(n, 10)
    t = trk.Tracker(N, family=FAM, I=I, m=M, storage=trk.TRK_F64)
    t.set_field(torch.from_numpy(field).cuda())

    def fwd(p):
        x = torch.from_numpy(p).cuda()
        t.advance(x, dt, steps)
        return x.cpu().numpy()

    XT = fwd(pos)
    gpos, _ = t.adjoint(torch.from_numpy(pos).cuda(), torch.from_numpy(2 * XT).cuda(), dt, steps, 2)
    g = gpos.cpu().numpy()
    h = 1e-6
    for a in range(3):
        e = np.zeros_like(pos); e[a] = h
        fd = ((fwd(pos + e) ** 2).sum(0) - (fwd(pos - e) ** 2).sum(0)) / (2 * h)   # particle p's own term
        np.testing.assert_allclose(g[a], fd, rtol=2e-6, atol=2e-7)


def test_autograd_function():
    N, n, dt, steps = 32, 300, 5e-3, 4
    field = synth.velocity_field_np(N, 10, 92)
    pos = synth.uniform_particles_np(n, 11)
    t = trk.Tracker(N, family=FAM, I=I, m=M, storage=trk.TRK_F64)
    p0 = torch.from_numpy(pos).cuda().requires_grad_(True)
    f = torch.from_numpy(field).cuda().requires_grad_(True)
    loss = (advect(p0, f, t, dt, steps, ckpt_every=2) ** 2).sum()
    loss.backward()
    posT = oracle.advance(field, pos, dt, steps, FAM, I, M)
    gpos_ref, gf_ref = oracle.adjoint_rk2(field, pos, 2 * posT, dt, steps, FAM, I, M)
    assert abs(loss.item() - (posT ** 2).sum()) <= 1e-10 * (posT ** 2).sum()
    assert rel(p0.grad.cpu().numpy(), gpos_ref) <= 1e-10
    assert rel(f.grad.cpu().numpy(), gf_ref) <= 1e-10


def test_autograd_two_fields_on_one_tracker():
    """Two advect() calls with different fields share one tracker before
    backward: the first graph's gradients must be those of its own field
    (the backward pass restores it), not of the field set by the second."""
    N, n, dt, steps = 32, 200, 5e-3, 3
    fa = synth.velocity_field_np(N, 10, 95)
    fb = synth.velocity_field_np(N, 10, 96)
    pos = synth.uniform_particles_np(n, 12)
    t = trk.Tracker(N, family=FAM, I=I, m=M, storage=trk.TRK_F64)
    p0 = torch.from_numpy(pos).cuda().requires_grad_(True)
    f_a = torch.from_numpy(fa).cuda().requires_grad_(True)
    f_b = torch.from_numpy(fb).cuda().requires_grad_(True)
    loss_a = (advect(p0, f_a, t, dt, steps, ckpt_every=2) ** 2).sum()
    loss_b = (advect(p0, f_b, t, dt, steps, ckpt_every=2) ** 2).sum()
    loss_a.backward()
    ga_pos = p0.grad.cpu().numpy().copy()
    p0.grad = None
    loss_b.backward()
    for field, g_pos, f_t in ((fa, ga_pos, f_a), (fb, p0.grad.cpu().numpy(), f_b)):
        posT = oracle.advance(field, pos, dt, steps, FAM, I, M)
        gpos_ref, gf_ref = oracle.adjoint_rk2(field, pos, 2 * posT, dt, steps, FAM, I, M)
        assert rel(g_pos, gpos_ref) <= 1e-10
        assert rel(f_t.grad.cpu().numpy(), gf_ref) <= 1e-10


def _periodic_cell_distance(cells, c0, N):
    """Largest per-axis periodic distance (in cells) of each particle's cell from c0."""
    d = np.abs(cells - np.asarray(c0)[:, None]) % N
    return np.minimum(d, N - d).max(axis=0)


def test_config5_full_size_sampled():
    """256^3 float32 field, 2^22 tracers, spline I=6, 20 RK2 steps, checkpoints every 5,
    loss = sum |X_T|^2.  Position gradients on a particle sample (the loss
    separates over particles).  The field gradient of the whole 2^22-tracer run
    on sampled grid nodes: only tracers whose stencils reach a node add to its
    gradient, so the oracle's adjoint over the tracers that start within reach
    of the sampled nodes gives those nodes' exact values.  Reach: a tracer moves
    at most T max|u| (T = 20 dt, max|u| bounded by the largest stored value
    times the kernel's Lebesgue constant), plus the stencil half-width I/2 and
    one cell for the stage-2 point."""
    N, n, dt, steps = 256, 1 << 22, 5e-3, 20
    field = synth.velocity_field_np(N, 85, 1004).astype(np.float32)
    fs = field.astype(np.float64)
    pos = synth.uniform_particles_np(n, 5)
    t = trk.Tracker(N, family=FAM, I=I, m=M, storage=trk.TRK_F32)
    t.set_field(torch.from_numpy(field).cuda())
    p = torch.from_numpy(pos).cuda()
    x = p.clone()
    t.advance(x, dt, steps)
    lam = 2 * x
    gf = torch.zeros((3, N, N, N), dtype=torch.float64, device="cuda")
    gpos, _ = t.adjoint(p, lam, dt, steps, 5, grad_field=gf)
    try:
        t.sync()
    except trk.TrackerError as e:
        assert e.status == trk.TRK_ECFL       # a few fast points take the exact slow path
    sample = np.random.default_rng(0).choice(n, 512, replace=False)
    ps = pos[:, sample]
    posT = oracle.advance(fs, ps, dt, steps, FAM, I, M)
    gref, _ = oracle.adjoint_rk2(fs, ps, 2 * posT, dt, steps, FAM, I, M, with_field=False)
    assert rel(gpos.cpu().numpy()[:, sample], gref) <= 1e-6
    # field gradient of the full run on 16 nodes in a 3^3 neighbourhood
    rng = np.random.default_rng(1)
    c0 = rng.integers(0, N, 3)
    nodes = (c0[:, None] + rng.integers(-1, 2, (3, 16))) % N
    lebesgue = max(np.abs(oracle.weights(FAM, I, M, tt)).sum() for tt in np.linspace(0, 1, 201))
    reach = np.abs(fs).max() * lebesgue * dt * steps * N / L + I // 2 + 2
    cells, _ = oracle.split(pos, N)
    near = np.nonzero(_periodic_cell_distance(cells, c0, N) <= np.ceil(reach) + 1)[0]
    assert 0 < near.size < n // 4
    pn = pos[:, near]
    posT = oracle.advance(fs, pn, dt, steps, FAM, I, M)
    _, gf_ref = oracle.adjoint_rk2(fs, pn, 2 * posT, dt, steps, FAM, I, M)
    got = gf.cpu().numpy()[:, nodes[2], nodes[1], nodes[0]]
    want = gf_ref[:, nodes[2], nodes[1], nodes[0]]
    assert np.abs(want).max() > 0
    assert rel(got, want) <= 1e-6


@pytest.mark.parametrize("storage,I_,m_", [(trk.TRK_F32, 6, 2), (trk.TRK_F64, 4, 1), (trk.TRK_F32, 8, 3)])
@pytest.mark.parametrize("N,n,layout", [(16, 300, "uniform"), (32, 4000, "uniform"), (32, 2000, "cluster")])
def test_field_gradient_scratch_and_atomic_paths_agree(monkeypatch, storage, I_, m_, N, n, layout):
    """The per-block partial sums + node gather (default) and the float64
    atomics per halo node (forced by a zero scratch budget) give the same
    field gradient to rounding; both match the oracle.  N = 16 with I = 8 has halos wider
    than the grid (a block's halo holds two periodic images of some nodes)."""
    dt, steps, ckpt = 5e-3, 3, 2
    field = synth.velocity_field_np(N, min(10, N // 3), 92)
    rng = np.random.default_rng(11)
    if layout == "uniform":
        pos = rng.uniform(0, L, (3, n))
    else:                                   # every particle in cell block 0
        pos = rng.uniform(0.01, 8 * L / N - 0.01, (3, n))
    fs = stored(field, storage)
    posT = oracle.advance(fs, pos, dt, steps, FAM, I_, m_)
    lam = 2 * posT
    gpos_ref, gf_ref = oracle.adjoint_rk2(fs, pos, lam, dt, steps, FAM, I_, m_)
    out = {}
    for mode in ("scratch", "atomic"):
        if mode == "atomic":
            monkeypatch.setenv("TRK_ADJ_SCRATCH_BYTES", "0")
        t = trk.Tracker(N, family=FAM, I=I_, m=m_, storage=storage)
        t.set_field(torch.from_numpy(field).cuda())
        gf = torch.zeros((3, N, N, N), dtype=torch.float64, device="cuda")
        gpos, _ = t.adjoint(torch.from_numpy(pos).cuda(), torch.from_numpy(lam).cuda(), dt, steps, ckpt,
                            grad_field=gf)
        t.sync()
        out[mode] = (gpos.cpu().numpy(), gf.cpu().numpy())
        t.close()
    tol = 1e-10 if storage == trk.TRK_F64 else 1e-6
    for mode in out:
        assert rel(out[mode][0], gpos_ref) <= tol, mode
        assert rel(out[mode][1], gf_ref) <= tol, mode
    assert np.array_equal(out["scratch"][0], out["atomic"][0])
    # both paths add each block's contributions in the storage precision, in
    # different orders (atomics into the scratch slab vs a shared-memory
    # accumulator): they agree to the adjoint tolerance of 1e-6 relative
    assert rel(out["scratch"][1], out["atomic"][1]) <= (1e-14 if storage == trk.TRK_F64 else 1e-6)


def stored_any(field, storage):
    if storage != trk.TRK_BF16X2:
        return stored(field, storage)
    hi, lo = synth.bf16_split(torch.from_numpy(field.astype(np.float32)))
    return hi.double().numpy() + lo.double().numpy()


@pytest.mark.parametrize("storage", [trk.TRK_F64, trk.TRK_F32, trk.TRK_BF16X2])
@pytest.mark.parametrize("I_,m_", [(4, 1), (6, 2), (8, 3)])
@pytest.mark.parametrize("layout", ["sparse", "cluster"])
def test_direct_adjoint_matches_oracle(storage, I_, m_, layout):
    """The direct adjoint (no halos; float64 atomic adds straight into the
    field gradient), forced, on a sparse set and on one crowded block."""
    N, dt, steps, ckpt = 32, 5e-3, 4, 2
    rng = np.random.default_rng(12)
    if layout == "sparse":
        pos = rng.uniform(0, L, (3, 60))
    else:
        pos = rng.uniform(0.01, 8 * L / N - 0.01, (3, 500))
    field = synth.velocity_field_np(N, 10, 93)
    fs = stored_any(field, storage)
    posT = oracle.advance(fs, pos, dt, steps, FAM, I_, m_)
    lam = 2 * posT
    gpos_ref, gf_ref = oracle.adjoint_rk2(fs, pos, lam, dt, steps, FAM, I_, m_)
    t = trk.Tracker(N, family=FAM, I=I_, m=m_, storage=storage)
    t.set_step_kernel(trk.TRK_STEP_DIRECT)
    t.set_field(torch.from_numpy(field).cuda())
    gf = torch.zeros((3, N, N, N), dtype=torch.float64, device="cuda")
    gpos, _ = t.adjoint(torch.from_numpy(pos).cuda(), torch.from_numpy(lam).cuda(), dt, steps, ckpt, grad_field=gf)
    t.sync()
    tol = 1e-10 if storage == trk.TRK_F64 else 1e-6
    assert rel(gpos.cpu().numpy(), gpos_ref) <= tol
    assert rel(gf.cpu().numpy(), gf_ref) <= tol


@pytest.mark.parametrize("storage", [trk.TRK_F64, trk.TRK_F32])
def test_direct_and_halo_adjoints_agree(storage):
    N, n, dt, steps, ckpt = 32, 3000, 5e-3, 3, 2
    field = synth.velocity_field_np(N, 10, 94)
    pos = synth.uniform_particles_np(n, 14)
    lam = 2 * pos
    out = []
    for kind in (trk.TRK_STEP_DIRECT, trk.TRK_STEP_BLOCK):
        t = trk.Tracker(N, family=FAM, I=I, m=M, storage=storage)
        t.set_step_kernel(kind)
        t.set_field(torch.from_numpy(field).cuda())
        gf = torch.zeros((3, N, N, N), dtype=torch.float64, device="cuda")
        gpos, _ = t.adjoint(torch.from_numpy(pos).cuda(), torch.from_numpy(lam).cuda(), dt, steps, ckpt,
                            grad_field=gf)
        t.sync()
        out.append((gpos.cpu().numpy(), gf.cpu().numpy()))
        t.close()
    assert np.array_equal(out[0][0], out[1][0])          # the position gradient: same float64 arithmetic
    assert rel(out[0][1], out[1][1]) <= (1e-14 if storage == trk.TRK_F64 else 1e-6)
