"""GPU: the direct path (stencils gathered from global memory, no halo) for
sparse particle sets.

Per particle it performs the same floating-point operations in the same order
as the block kernel, so positions, AB histories and interpolated values must
agree bit for bit; at the paper's sparse density (about 1.5e-3 tracers per
grid cell) it is also checked against the oracle.  The automatic choice picks
it below 0.05 particles per cell where a column kernel exists (and times the
two between 0.01 and 0.25), else below 0.25.
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

STORAGES = [trk.TRK_F64, trk.TRK_F32, trk.TRK_BF16X2]
KERNELS = [(4, 1), (6, 2), (8, 3), (6, 3)]


def stored(field, storage):
    if storage == trk.TRK_F64:
        return field
    f32 = field.astype(np.float32)
    if storage == trk.TRK_F32:
        return f32.astype(np.float64)
    hi, lo = synth.bf16_split(torch.from_numpy(f32))
    return hi.double().numpy() + lo.double().numpy()


def positions(layout, N, n, seed):
    rng = np.random.default_rng(seed)
    if layout == "uniform":
        return rng.uniform(0.0, L, (3, n))
    if layout == "cluster":                        # many particles in one cell block
        return rng.uniform(1e-3, 8 * L / N - 1e-3, (3, n))
    p = rng.uniform(-L, 2 * L, (3, n))             # edges: nodes and +-1 ulp of faces, unwrapped
    q = n // 4
    delta = L / N
    p[:, :q] = rng.integers(-N, 2 * N, (3, q)) * delta
    faces = rng.integers(0, N + 1, (3, q)) * delta
    p[:, q:2 * q] = np.nextafter(faces, np.where(rng.random((3, q)) < 0.5, -np.inf, np.inf))
    return p


def advance(N, I, m, storage, field, pos, kind, scheme, steps, dt):
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=I, m=m, storage=storage)
    t.set_step_kernel(kind)
    t.set_field(torch.from_numpy(field).to(DEV))
    p = torch.from_numpy(pos).to(DEV)
    k = scheme + 1
    rhs = torch.zeros((max(k - 1, 1), 3, pos.shape[1]), dtype=torch.float32, device=DEV)
    if scheme != trk.TRK_RK2:
        t.advance(p, dt, 2, scheme, rhs=rhs, history_valid=0)
        t.advance(p, dt, steps - 2, scheme, rhs=rhs, history_valid=min(2, k - 1))
    else:
        t.advance(p, dt, steps, scheme)
    t.sync()
    return p.cpu(), rhs.cpu()


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("I,m", KERNELS)
@pytest.mark.parametrize("scheme", [trk.TRK_RK2, trk.TRK_AB2, trk.TRK_AB4])
@pytest.mark.parametrize("N,n,layout", [(32, 300, "uniform"), (32, 3000, "cluster"), (64, 5000, "edges"),
                                        (16, 1, "uniform"), (64, 257, "uniform")])
def test_direct_bit_identical_to_block(storage, I, m, scheme, N, n, layout):
    field = synth.velocity_field_np(N, min(10, N // 3), 400 + N)
    pos = positions(layout, N, n, 21)
    steps, dt = 5, 4e-3
    pb, rb = advance(N, I, m, storage, field, pos, trk.TRK_STEP_BLOCK, scheme, steps, dt)
    pd, rd = advance(N, I, m, storage, field, pos, trk.TRK_STEP_DIRECT, scheme, steps, dt)
    assert torch.equal(pb, pd)
    if scheme != trk.TRK_RK2:
        assert torch.equal(rb, rd)


@pytest.mark.parametrize("storage", [trk.TRK_F32, trk.TRK_BF16X2])
@pytest.mark.parametrize("I,m", [(4, 1), (6, 2), (8, 3)])
@pytest.mark.parametrize("scheme", [trk.TRK_RK2, trk.TRK_AB4])
def test_direct_texture_and_plain_loads_agree(monkeypatch, storage, I, m, scheme):
    """The 16-byte node loads go through a texture object where the node-major
    copy is small enough (by default at most four times the L2 size, as here),
    else through plain loads (TRK_NM_TEXTURE_BYTES=0 forces these): the same
    bits either way, stepping and interpolating."""
    N, n = 64, 5000
    field = synth.velocity_field_np(N, 10, 470)
    pos = positions("edges", N, n, 23)
    res = []
    for cap in (None, "0"):
        if cap is None:
            monkeypatch.delenv("TRK_NM_TEXTURE_BYTES", raising=False)
        else:
            monkeypatch.setenv("TRK_NM_TEXTURE_BYTES", cap)
        p, r = advance(N, I, m, storage, field, pos, trk.TRK_STEP_DIRECT, scheme, 5, 4e-3)
        t = trk.Tracker(N, family=trk.TRK_SPLINE, I=I, m=m, storage=storage)
        t.set_step_kernel(trk.TRK_STEP_DIRECT)
        t.set_field(torch.from_numpy(field).to(DEV))
        u = t.interpolate(torch.from_numpy(pos).to(DEV), out_dtype=torch.float64, deriv=True).cpu()
        t.sync()
        assert t.field_texture() == (cap is None)
        res.append((p, r, u))
    for other in res[1:]:
        for a, b in zip(res[0], other):
            assert torch.equal(a, b)


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("I,m", KERNELS)
@pytest.mark.parametrize("C,deriv", [(3, 0), (3, 1), (9, 0), (4, 1), (12, 0), (6, 1)])
def test_direct_interpolation_bit_identical_to_block(storage, I, m, C, deriv):
    N, n = 32, 2000
    rng = np.random.default_rng(C)
    field = rng.standard_normal((C, N, N, N))
    pos = positions("edges", N, n, 22)
    outs = []
    for kind in (trk.TRK_STEP_BLOCK, trk.TRK_STEP_DIRECT):
        t = trk.Tracker(N, family=trk.TRK_SPLINE, I=I, m=m, storage=storage)
        t.set_step_kernel(kind)
        t.set_field(torch.from_numpy(field).to(DEV))
        outs.append(t.interpolate(torch.from_numpy(pos).to(DEV), out_dtype=torch.float64, deriv=bool(deriv)).cpu())
        t.sync()
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("storage", STORAGES)
def test_direct_at_paper_density_matches_oracle(storage):
    """1.5e-3 tracers per cell (the paper's production runs): AUTO picks the direct path."""
    N = 64
    n = int(1.5e-3 * N ** 3)
    field = synth.velocity_field_np(N, 20, 401)
    pos = synth.uniform_particles_np(n, 23)
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=storage)
    t.set_field(torch.from_numpy(field).to(DEV))
    assert t.step_kernel_for(n) == trk.TRK_STEP_DIRECT
    u = t.interpolate(torch.from_numpy(pos).to(DEV), out_dtype=torch.float64)
    p = torch.from_numpy(pos).to(DEV)
    dt, steps = 4e-3, 6
    t.advance(p, dt, steps, trk.TRK_RK2)
    t.sync()
    f = stored(field, storage)
    rms = np.sqrt(np.mean(field ** 2))
    scale = np.abs(field).max() * 1e-12 if storage == trk.TRK_F64 else 2e-6 * rms
    assert np.abs(u.cpu().numpy() - oracle.interp(f, pos, trk.TRK_SPLINE, 6, 2)).max() <= scale
    ref = oracle.advance(f, pos, dt, steps, trk.TRK_SPLINE, 6, 2)
    assert np.abs(p.cpu().numpy() - ref).max() <= 5 * scale * dt * steps


@pytest.mark.parametrize("N,n,shapes", [
    (32, 200, ((8, 8, 8), (32, 32, 1))),                 # x3 slices
    (128, 5000, ((8, 8, 8), (2, 2, 2), (1, 1, 1))),      # 2^18 and 2^21 blocks: the multi-CTA count scan
])
def test_direct_any_block_shape(N, n, shapes):
    """The direct path needs no 8^3 cell blocks: with other groupings the results are the same."""
    field = synth.velocity_field_np(N, 10, 402).astype(np.float32)
    pos = synth.uniform_particles_np(n, 24)
    res = []
    for shape in shapes:
        t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
        trk.tracker_set_block(t.h, *shape)
        t.set_step_kernel(trk.TRK_STEP_DIRECT)
        t.set_field(torch.from_numpy(field).to(DEV))
        p = torch.from_numpy(pos).to(DEV)
        t.advance(p, 4e-3, 4, trk.TRK_RK2)
        t.sync()
        res.append(p.cpu())
    for r in res[1:]:
        assert torch.equal(res[0], r)


def test_direct_cfl_flag():
    """Stage-2 points more than one cell away raise TRK_ECFL; the result is still exact."""
    N, n, dt = 32, 600, 5e-3
    field = (synth.velocity_field_np(N, 10, 81) * 30.0).astype(np.float32)
    pos = synth.uniform_particles_np(n, 7)
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_step_kernel(trk.TRK_STEP_DIRECT)
    t.set_field(torch.from_numpy(field).to(DEV))
    p = torch.from_numpy(pos).to(DEV)
    t.advance(p, dt, 2, trk.TRK_RK2)
    with pytest.raises(trk.TrackerError) as e:
        t.sync()
    assert e.value.status == trk.TRK_ECFL
    ref = oracle.advance(field.astype(np.float64), pos, dt, 2, trk.TRK_SPLINE, 6, 2)
    assert np.abs(p.cpu().numpy() - ref).max() <= 5 * 2e-6 * 30.0 * dt * 2
    # one cell per stage at most: no flag
    p = torch.from_numpy(pos).to(DEV)
    t.advance(p, 1e-4, 2, trk.TRK_RK2)
    t.sync()


def test_automatic_choice():
    N = 64
    f = synth.velocity_field_np(N, 5, 1)
    t32 = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    thr = int(0.05 * N ** 3)
    assert t32.step_kernel_for(0) == trk.TRK_STEP_DIRECT
    assert t32.step_kernel_for(thr - 1) == trk.TRK_STEP_DIRECT
    assert t32.step_kernel_for(thr + 1) == trk.TRK_STEP_COLUMN
    # without a column kernel: block vs direct by a threshold per storage
    t64 = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F64)
    assert t64.step_kernel_for(thr + 1) == trk.TRK_STEP_DIRECT
    assert t64.step_kernel_for(N ** 3 // 4 - 1) == trk.TRK_STEP_DIRECT
    assert t64.step_kernel_for(N ** 3 // 4 + 1) == trk.TRK_STEP_BLOCK
    t8 = trk.Tracker(N, family=trk.TRK_SPLINE, I=8, m=3, storage=trk.TRK_F32)
    assert t8.step_kernel_for(N ** 3 // 4 + 1) == trk.TRK_STEP_BLOCK
    assert t8.step_kernel_for(N ** 3 // 8) == trk.TRK_STEP_DIRECT
    tb = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_BF16X2)
    assert tb.step_kernel_for(N ** 3 // 8) == trk.TRK_STEP_DIRECT
    assert tb.step_kernel_for(N ** 3 // 4 + 1) == trk.TRK_STEP_BLOCK
    t64.set_step_kernel(trk.TRK_STEP_DIRECT)
    assert t64.step_kernel_for(10 ** 9) == trk.TRK_STEP_DIRECT
    t32.set_step_kernel(trk.TRK_STEP_BLOCK)
    assert t32.step_kernel_for(1) == trk.TRK_STEP_BLOCK
    with pytest.raises(trk.TrackerError):
        t32.step_kernel_for(-1)
    del f


@pytest.mark.parametrize("storage", [trk.TRK_F32, trk.TRK_BF16X2])
def test_direct_sees_a_replaced_field(storage):
    """The direct path of a float32 or split-bf16 tracker reads a node-major copy
    of the field: after set_field it must gather the new values (interpolation
    and steps)."""
    N, n = 32, 500
    fa = synth.velocity_field_np(N, 10, 410).astype(np.float32)
    fb = synth.velocity_field_np(N, 10, 411).astype(np.float32)
    pos = synth.uniform_particles_np(n, 25)
    td = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=storage)
    td.set_step_kernel(trk.TRK_STEP_DIRECT)
    tb = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=storage)
    tb.set_step_kernel(trk.TRK_STEP_BLOCK)
    x = torch.from_numpy(pos).to(DEV)
    for f in (fa, fb, fa):
        for t in (td, tb):
            t.set_field(torch.from_numpy(f).to(DEV))
        ud = td.interpolate(x, out_dtype=torch.float64)
        ub = tb.interpolate(x, out_dtype=torch.float64)
        pd, pb = x.clone(), x.clone()
        td.advance(pd, 4e-3, 3, trk.TRK_RK2)
        tb.advance(pb, 4e-3, 3, trk.TRK_RK2)
        td.sync()
        tb.sync()
        assert torch.equal(ud, ub)
        assert torch.equal(pd, pb)


@pytest.mark.parametrize("scheme", [trk.TRK_RK2, trk.TRK_AB4])
def test_automatic_choice_by_timing(scheme):
    """At 1/16 per cell (inside the timed range) the first call of >= 6 steps
    times both kernels and keeps one; the results equal the block kernel's and
    the decision is reused."""
    N = 64
    n = N ** 3 // 16
    field = synth.velocity_field_np(N, 20, 412).astype(np.float32)
    pos = synth.uniform_particles_np(n, 26)
    res = []
    for kind in (trk.TRK_STEP_AUTO, trk.TRK_STEP_BLOCK):
        t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
        t.set_step_kernel(kind)
        t.set_field(torch.from_numpy(field).to(DEV))
        assert t.last_step_kernel() == trk.TRK_STEP_AUTO
        p = torch.from_numpy(pos).to(DEV)
        k = scheme + 1
        h = torch.zeros((max(k - 1, 1), 3, n), dtype=torch.float32, device=DEV)
        kw = dict(rhs=h, history_valid=0) if scheme else {}
        t.advance(p, 4e-3, 8, scheme, **kw)
        chosen = t.last_step_kernel()
        if scheme:
            kw["history_valid"] = k - 1
        t.advance(p, 4e-3, 7, scheme, **kw)
        t.sync()
        if kind == trk.TRK_STEP_AUTO:
            assert chosen in (trk.TRK_STEP_COLUMN, trk.TRK_STEP_DIRECT)
            assert t.last_step_kernel() == chosen                      # cached
        else:
            assert chosen == trk.TRK_STEP_BLOCK
        res.append((p.cpu(), h.cpu()))
    assert torch.equal(res[0][0], res[1][0])
    assert torch.equal(res[0][1], res[1][1])


def test_no_timing_for_short_calls():
    N = 64
    n = N ** 3 // 16
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_field(torch.from_numpy(synth.velocity_field_np(N, 5, 413).astype(np.float32)).to(DEV))
    p = torch.from_numpy(synth.uniform_particles_np(n, 27)).to(DEV)
    t.advance(p, 4e-3, 5, trk.TRK_RK2)
    t.sync()
    assert t.last_step_kernel() == t.step_kernel_for(n)


@pytest.mark.parametrize("storage", [trk.TRK_F32, trk.TRK_BF16X2])
@pytest.mark.parametrize("C,deriv", [(3, 0), (3, 1), (12, 0)])
def test_interpolation_choice_by_timing(storage, C, deriv):
    """Inside the timed density range the first AUTO call runs both kernels and
    keeps one; every call gives the block kernel's values."""
    N, n = 32, 4099
    rng = np.random.default_rng(40 + C)
    field = rng.standard_normal((C, N, N, N)).astype(np.float32)
    x = torch.from_numpy(synth.uniform_particles_np(n, 28)).to(DEV)
    ta = trk.Tracker(N, family=trk.TRK_SPLINE, I=8, m=3, storage=storage)
    ta.set_field(torch.from_numpy(field).to(DEV))
    tb = trk.Tracker(N, family=trk.TRK_SPLINE, I=8, m=3, storage=storage)
    tb.set_step_kernel(trk.TRK_STEP_BLOCK)
    tb.set_field(torch.from_numpy(field).to(DEV))
    ref = tb.interpolate(x, deriv=bool(deriv))
    for _ in range(2):   # timed, then cached
        assert torch.equal(ta.interpolate(x, deriv=bool(deriv)), ref)
    ta.sync()


def test_split_bf16_copy_follows_the_component_count():
    """Split-bf16 fields: the direct kernel's node-major copy holds one 16-byte
    record per node and chunk of three components; a field with another
    component count replaces it (and a count that is not a multiple of three
    is read from the component-major field)."""
    N, n = 32, 1500
    rng = np.random.default_rng(77)
    x = torch.from_numpy(positions("uniform", N, n, 31)).to(DEV)
    td = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_BF16X2)
    td.set_step_kernel(trk.TRK_STEP_DIRECT)
    tb = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_BF16X2)
    tb.set_step_kernel(trk.TRK_STEP_BLOCK)
    for C in (3, 12, 4, 6, 3):
        f = torch.from_numpy(rng.standard_normal((C, N, N, N)).astype(np.float32)).to(DEV)
        td.set_field(f)
        tb.set_field(f)
        for deriv in (False, True):
            assert torch.equal(td.interpolate(x, deriv=deriv), tb.interpolate(x, deriv=deriv)), (C, deriv)
        assert td.field_texture() == (C == 3)
    td.sync()
    tb.sync()
