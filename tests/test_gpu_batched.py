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


def test_config4_full_size_sampled():
    """512^3 float32 field (|k| <= 170), 8 sets of 1e3 .. 2e7 tracers, I cycling 4/6/8,
    3- or 9-component outputs alternating, 50 AB2 steps; a sample of every set vs the oracle."""
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
    sets = run_sets(t, specs, dt, steps)
    fs = u.double().cpu().numpy()
    del u
    rng = np.random.default_rng(0)
    for sp, st in zip(specs, sets):
        idx = rng.choice(sp["np"], 64, replace=False)
        ref, _ = oracle.advance(fs, sp["pos"][:, idx], dt, steps, sp["family"], sp["I"], sp["m"], scheme=oracle.AB2)
        assert np.abs(st["pos"].cpu().numpy()[:, idx] - ref).max() <= 5 * 2e-6 * dt * steps * 10
