"""Batched AB2 advection (one persistent launch per step for all sets) against the oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2107_01104_gb300 as trk
import synth

pytestmark = pytest.mark.gpu
L = 2 * math.pi


def run_sets(t, specs, dt, steps):
    sets = []
    for sp in specs:
        n = sp["np"]
        pos = torch.from_numpy(sp["pos"]).cuda()
        rhs = torch.zeros((3, n), dtype=torch.float32, device="cuda")
        out = torch.zeros((9 if sp["deriv"] else 3, n), dtype=torch.float32, device="cuda")
        sets.append(dict(pos=pos, rhs=rhs, out=out, family=sp["family"], I=sp["I"], m=sp["m"], deriv=sp["deriv"]))
    t.advance_batched(sets, dt, steps, history_valid=False)
    try:
        t.sync()
    except trk.TrackerError as e:
        assert e.status == trk.TRK_ECFL
    return sets


@pytest.mark.parametrize("storage", [trk.TRK_F32, trk.TRK_BF16X2])
def test_batched_sets_match_oracle(storage):
    N, dt, steps = 32, 4e-3, 6
    field = synth.velocity_field_np(N, 10, 95)
    f32 = field.astype(np.float32)
    if storage == trk.TRK_F32:
        fs = f32.astype(np.float64)
    else:
        hi, lo = synth.bf16_split(torch.from_numpy(f32))
        fs = hi.double().numpy() + lo.double().numpy()
    rng = np.random.default_rng(1)
    specs = [
        dict(np=0, family=trk.TRK_SPLINE, I=4, m=1, deriv=0),
        dict(np=10, family=trk.TRK_LAGRANGE, I=4, m=0, deriv=0),
        dict(np=300, family=trk.TRK_SPLINE, I=6, m=2, deriv=1),
        dict(np=5000, family=trk.TRK_SPLINE, I=8, m=3, deriv=0),
        dict(np=20000, family=trk.TRK_SPLINE, I=6, m=3, deriv=1),
    ]
    for sp in specs:
        sp["pos"] = rng.uniform(-L, 2 * L, (3, sp["np"]))
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=storage)
    t.set_field(torch.from_numpy(f32).cuda())
    sets = run_sets(t, specs, dt, steps)
    for sp, st in zip(specs, sets):
        if sp["np"] == 0:
            continue
        ref, ref_rhs = oracle.advance(fs, sp["pos"], dt, steps, sp["family"], sp["I"], sp["m"], scheme=oracle.AB2)
        assert np.abs(st["pos"].cpu().numpy() - ref).max() <= 5 * 2e-6 * dt * steps
        assert np.abs(st["rhs"].cpu().numpy() - ref_rhs).max() <= 3 * 2e-6
        # per-step outputs hold the last step's values, at the position before it
        prev, _ = oracle.advance(fs, sp["pos"], dt, steps - 1, sp["family"], sp["I"], sp["m"], scheme=oracle.AB2)
        if sp["deriv"]:
            g = oracle.interp(fs, prev, sp["family"], sp["I"], sp["m"], deriv=True).reshape(9, -1)
            assert np.abs(st["out"].cpu().numpy() - g).max() <= 4e-6 * N / L * 3
        else:
            u = oracle.interp(fs, prev, sp["family"], sp["I"], sp["m"])
            assert np.abs(st["out"].cpu().numpy() - u).max() <= 3 * 2e-6


@pytest.mark.parametrize("storage", [trk.TRK_F32, trk.TRK_BF16X2])
def test_batched_texture_and_plain_loads_agree(monkeypatch, storage):
    """The batched kernel's direct items read the node-major copy by plain
    loads whether or not the tracker made a texture object over it (by
    default for a copy this small; TRK_NM_TEXTURE_BYTES=0: none): the
    texture setting must not change a bit of the results (and whichever path
    each set takes, direct and halo-staged agree bit for bit)."""
    N, dt, steps = 32, 4e-3, 4
    f32 = synth.velocity_field_np(N, 10, 97).astype(np.float32)
    rng = np.random.default_rng(2)
    specs = [dict(np=12, family=trk.TRK_SPLINE, I=8, m=3, deriv=1),
             dict(np=40, family=trk.TRK_LAGRANGE, I=6, m=0, deriv=0),
             dict(np=3000, family=trk.TRK_SPLINE, I=4, m=1, deriv=1)]
    for sp in specs:
        sp["pos"] = rng.uniform(-L, 2 * L, (3, sp["np"]))
    res = []
    for cap in (None, "0"):
        if cap is None:
            monkeypatch.delenv("TRK_NM_TEXTURE_BYTES", raising=False)
        else:
            monkeypatch.setenv("TRK_NM_TEXTURE_BYTES", cap)
        t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=storage)
        t.set_field(torch.from_numpy(f32).cuda())
        sets = run_sets(t, specs, dt, steps)
        assert t.field_texture() == (cap is None)   # the first call makes the copy (it times both paths per set)
        res.append([st[k].cpu() for st in sets for k in ("pos", "rhs", "out")])
        t.close()
    for other in res[1:]:
        for a, b in zip(res[0], other):
            assert torch.equal(a, b)


def test_batched_equals_single_set_path():
    N, dt, steps = 32, 4e-3, 5
    field = synth.velocity_field_np(N, 10, 96).astype(np.float32)
    pos = synth.uniform_particles_np(7000, 3)
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_field(torch.from_numpy(field).cuda())
    sets = run_sets(t, [dict(np=7000, pos=pos, family=trk.TRK_SPLINE, I=6, m=2, deriv=0)], dt, steps)
    p = torch.from_numpy(pos).cuda()
    rhs = torch.zeros((3, 7000), dtype=torch.float32, device="cuda")
    t.advance(p, dt, steps, trk.TRK_AB2, rhs=rhs)
    t.sync()
    assert np.abs(sets[0]["pos"].cpu().numpy() - p.cpu().numpy()).max() <= 1e-12
    assert np.abs(sets[0]["rhs"].cpu().numpy() - rhs.cpu().numpy()).max() <= 1e-6


def _ab2_error_bound(fs, pos, dt, steps, family, I, m, eps, rho):
    """First-order bound on |X_gpu - X_oracle| per tracer after `steps` AB2
    steps from `pos` (Euler first step), for velocity evaluations in error by
    at most eps (float32 weights and sums) and a float32 history rounded by at
    most rho.

    The error made at step n enters X_{n+1} with weight c_n dt (c_0 = 1, then
    3/2) and, through the stored u_n, X_{n+2} with weight dt/2; from there it
    is carried to step S by the Jacobian J_{S<-k} = dX_S/dX_k of the oracle's
    own AB2 map (history held), which this function takes by central
    differences (h = 1e-6) of the oracle from each state of its trajectory:
        |e_S| <= sum_n dt (c_n eps ||J_{S<-n+1}|| + (eps + rho)/2 ||J_{S<-n+2}||).
    The errors are ~1e-8 of a cell, so the linearisation is exact to far
    below the bound's own size."""
    npart = pos.shape[1]
    xs, hs = [pos], [np.zeros_like(pos)]
    x, rhs = pos, None
    for n in range(steps):
        x, rhs = oracle.advance(fs, x, dt, 1, family, I, m, scheme=oracle.AB2, rhs=rhs, history_valid=n > 0)
        xs.append(x)
        hs.append(rhs)
    h = 1e-6
    jn = np.ones((steps + 1, npart))                   # ||J_{S<-k}||_2 per tracer, k = 0 .. S
    for k in range(1, steps):
        xk = np.concatenate([xs[k] + h * e[:, None] for e in np.vstack([np.eye(3), -np.eye(3)])], axis=1)
        hk = np.tile(hs[k], (1, 6))
        xe, _ = oracle.advance(fs, xk, dt, steps - k, family, I, m, scheme=oracle.AB2, rhs=hk, history_valid=True)
        xe = xe.reshape(3, 6, npart)
        jac = (xe[:, :3] - xe[:, 3:]) / (2 * h)        # [3 out][3 in][np]
        jn[k] = np.linalg.norm(np.moveaxis(jac, 2, 0), ord=2, axis=(1, 2))
    bound = np.zeros(npart)
    for n in range(steps):
        c = 1.0 if n == 0 else 1.5
        bound += dt * c * eps * jn[n + 1]
        if n + 2 <= steps:
            bound += dt * 0.5 * (eps + rho) * jn[n + 2]
    return bound, jn.max()


def test_config4_full_size_sampled():
    """512^3 float32 field (|k| <= 170), 8 sets of 1e3 .. 2e7 tracers, I cycling 4/6/8,
    3- or 9-component outputs alternating, 50 AB2 steps (one step, then 49 more
    with the history valid); a sample of every set vs the oracle.

    The first call's per-step outputs (u, or grad u, at the caller's positions)
    are compared element by element at the small-size tolerances.  The final
    positions of every sampled tracer are compared with twice its first-order
    bound from _ab2_error_bound (eps = 2e-6 x field rms, the float32 arithmetic
    bar; rho = 2^-24 x the largest |u|, the float32 history); the factor 2
    covers the second-order terms and the difference between the Jacobians
    along the GPU's and the oracle's trajectories."""
    N, dt, steps = 512, 2e-3, 50
    u = synth.velocity_field_torch(N, 170, 1003, out_dtype=torch.float32)
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_field(u)
    sizes = [1000, 10_000, 30_000, 100_000, 1_000_000, 3_000_000, 10_000_000, 20_000_000]
    specs = []
    for s, n in enumerate(sizes):
        I = (4, 6, 8)[s % 3]
        specs.append(dict(np=n, family=trk.TRK_SPLINE, I=I, m=I // 2 - 1, deriv=s % 2,
                          pos=synth.uniform_particles_np(n, 10 + s)))
    sets = run_sets(t, specs, dt, 1)
    fs = u.double().cpu().numpy()
    del u
    rms = float(np.sqrt(np.mean(fs ** 2)))
    rng = np.random.default_rng(0)
    idx = [rng.choice(sp["np"], 64, replace=False) for sp in specs]
    for sp, st, ix in zip(specs, sets, idx):
        x0 = sp["pos"][:, ix]
        if sp["deriv"]:
            g = oracle.interp(fs, x0, sp["family"], sp["I"], sp["m"], deriv=True).reshape(9, -1)
            assert np.abs(st["out"].cpu().numpy()[:, ix] - g).max() <= 4e-6 * N / L * 3
        else:
            uo = oracle.interp(fs, x0, sp["family"], sp["I"], sp["m"])
            assert np.abs(st["out"].cpu().numpy()[:, ix] - uo).max() <= 3 * 2e-6 * rms
    t.advance_batched(sets, dt, steps - 1, history_valid=True)
    try:
        t.sync()
    except trk.TrackerError as e:
        assert e.status == trk.TRK_ECFL
    umax = float(np.abs(fs).max())
    for sp, st, ix in zip(specs, sets, idx):
        x0 = sp["pos"][:, ix]
        ref, _ = oracle.advance(fs, x0, dt, steps, sp["family"], sp["I"], sp["m"], scheme=oracle.AB2)
        lebesgue = max(np.abs(oracle.weights(sp["family"], sp["I"], sp["m"], tt)).sum()
                       for tt in np.linspace(0, 1, 101))
        bound, _ = _ab2_error_bound(fs, x0, dt, steps, sp["family"], sp["I"], sp["m"], 2e-6 * rms,
                                    2.0 ** -24 * umax * lebesgue)
        err = np.abs(st["pos"].cpu().numpy()[:, ix] - ref).max(axis=0)
        assert np.all(err <= 2 * bound), (sp["np"], sp["I"], (err / bound).max())
