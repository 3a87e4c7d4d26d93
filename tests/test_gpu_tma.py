"""Tensor-copy (TMA) halo staging of the block kernel against the cp.async
staging and the oracle.

Both stagings put the same field values in shared memory (the tensor copy in a
padded box, the element copies in the conflict-free layout), and the
contraction reads them in the same order, so the outputs and trajectories
must agree bit for bit; both are also checked against the oracle at the
stated tolerances.  Covered: kernel widths 4, 6, 8, float32 and float64
storage, interpolation with 3, 4 and 12 components (chunks of three, the last
one partial), values and gradients, RK2 (stage-2 margin box) and AB2 steps,
and a 16^3 grid whose halos with I = 8 are wider than the grid.
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


def stored(field, storage):
    return field if storage == trk.TRK_F64 else field.astype(np.float32).astype(np.float64)


def positions(N, n, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-L, 2 * L, (3, n))
    q = n // 8
    pos[:, :q] = rng.integers(-N, 2 * N, (3, q)) * (L / N)      # on nodes
    return pos


def run_both(N, family, I, m, storage, field, fn):
    out = {}
    for hc in (trk.TRK_HALO_ASYNC, trk.TRK_HALO_TMA):
        t = trk.Tracker(N, family=family, I=I, m=m, storage=storage)
        t.set_step_kernel(trk.TRK_STEP_BLOCK)
        t.set_halo_copy(hc)
        t.set_field(torch.from_numpy(field).cuda())
        out[hc] = fn(t)
        t.sync()
        if hc == trk.TRK_HALO_TMA and field.shape[0] >= 3:
            assert t.halo_copy(False) == trk.TRK_HALO_TMA and t.halo_copy(True) == trk.TRK_HALO_TMA
        t.close()
    return out[trk.TRK_HALO_ASYNC], out[trk.TRK_HALO_TMA]


@pytest.mark.parametrize("storage", [trk.TRK_F32, trk.TRK_F64])
@pytest.mark.parametrize("family,I,m", [(trk.TRK_LAGRANGE, 4, 0), (trk.TRK_SPLINE, 6, 2), (trk.TRK_SPLINE, 8, 3)])
@pytest.mark.parametrize("C,deriv", [(3, False), (4, False), (12, False), (3, True)])
def test_tma_interpolation_matches_cp_async_and_oracle(storage, family, I, m, C, deriv):
    N, n = 32, 5003
    rng = np.random.default_rng(C + I)
    field = synth.velocity_field_np(N, 10, 70) if C == 3 else rng.standard_normal((C, N, N, N))
    pos = positions(N, n, I)
    p = torch.from_numpy(pos).cuda()
    a, b = run_both(N, family, I, m, storage, field,
                    lambda t: t.interpolate(p, out_dtype=torch.float64, deriv=deriv).cpu())
    assert torch.equal(a, b)
    ref = oracle.interp(stored(field, storage), pos, family, I, m, deriv=deriv).reshape(b.shape)
    scale = np.abs(field).max() if storage == trk.TRK_F64 else np.sqrt(np.mean(field ** 2))
    # random (non-smooth) fields for C != 3: the float32 bar of the chunked-component test
    f32_bar = 2e-6 if C == 3 else 1.2e-5
    tol = (1e-12 if storage == trk.TRK_F64 else f32_bar) * scale * (N / L * 2 if deriv else 1)
    assert np.abs(b.numpy() - ref).max() <= tol


@pytest.mark.parametrize("storage", [trk.TRK_F32, trk.TRK_F64])
@pytest.mark.parametrize("family,I,m", [(trk.TRK_LAGRANGE, 4, 0), (trk.TRK_SPLINE, 6, 2), (trk.TRK_SPLINE, 8, 3)])
@pytest.mark.parametrize("scheme", [trk.TRK_RK2, trk.TRK_AB2])
def test_tma_steps_match_cp_async_and_oracle(storage, family, I, m, scheme):
    N, n, dt, steps = 32, 6000, 5e-3, 5
    field = synth.velocity_field_np(N, 10, 71)
    pos = positions(N, n, 20 + I)

    def run(t):
        p = torch.from_numpy(pos).cuda()
        rhs = torch.zeros((3, n), dtype=torch.float32, device="cuda") if scheme == trk.TRK_AB2 else None
        t.advance(p, dt, steps, scheme, rhs=rhs)
        return p.cpu()

    a, b = run_both(N, family, I, m, storage, field, run)
    assert torch.equal(a, b)
    ref = oracle.advance(stored(field, storage), pos, dt, steps, family, I, m, scheme=scheme)
    if scheme == trk.TRK_AB2:
        ref = ref[0]
    tol = (1e-11 if scheme == trk.TRK_RK2 else 1e-7) if storage == trk.TRK_F64 else 5 * 2e-6 * dt * steps
    assert np.abs(b.numpy() - ref).max() <= tol


def test_tma_halo_wider_than_grid():
    """16^3 with I = 8: the RK2 halo (17 nodes) is wider than the grid; the
    box reads ghost layers on both sides and zero fill beyond the padding."""
    N, n, dt, steps = 16, 3000, 5e-3, 4
    field = synth.velocity_field_np(N, 5, 72)
    pos = positions(N, n, 30)

    def run(t):
        u = t.interpolate(torch.from_numpy(pos).cuda(), out_dtype=torch.float64).cpu()
        p = torch.from_numpy(pos).cuda()
        t.advance(p, dt, steps)
        return torch.cat([u, p.cpu()])

    a, b = run_both(N, trk.TRK_SPLINE, 8, 3, trk.TRK_F32, field, run)
    assert torch.equal(a, b)
    fs = stored(field, trk.TRK_F32)
    assert np.abs(b[:3].numpy() - oracle.interp(fs, pos, trk.TRK_SPLINE, 8, 3)).max() <= 2e-6
    ref = oracle.advance(fs, pos, dt, steps, trk.TRK_SPLINE, 8, 3)
    assert np.abs(b[3:].numpy() - ref).max() <= 5 * 2e-6 * dt * steps


@pytest.mark.parametrize("C", [3, 12])
def test_tma_crowded_block_several_batches(C):
    """More particles in one cell block than one CTA batch (256): the halo of a
    single chunk stays in place for the later batches (no new copy is awaited),
    several chunks are copied again per batch."""
    N, n = 32, 1500
    rng = np.random.default_rng(40 + C)
    field = rng.standard_normal((C, N, N, N))
    pos = rng.uniform(1e-3, 8 * L / N - 1e-3, (3, n))      # cells 0..7: all in block 0
    p = torch.from_numpy(pos).cuda()

    def run(t):
        u = t.interpolate(p, out_dtype=torch.float64).cpu()
        if C != 3:
            return u
        q = p.clone()
        t.advance(q, 5e-3, 3)
        return torch.cat([u, q.cpu()])

    a, b = run_both(N, trk.TRK_SPLINE, 8, 3, trk.TRK_F32, field, run)
    assert torch.equal(a, b)
    ref = oracle.interp(stored(field, trk.TRK_F32), pos, trk.TRK_SPLINE, 8, 3)
    assert np.abs(b[:C].numpy() - ref).max() <= 1.2e-5 * np.sqrt(np.mean(field ** 2))


def test_tma_falls_back_without_a_map():
    """Split-bf16 storage and fields of fewer than three components have no
    tensor map: TRK_HALO_TMA then stages with the register / cp.async copies."""
    t = trk.Tracker(32, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_BF16X2)
    t.set_halo_copy(trk.TRK_HALO_TMA)
    t.set_field(torch.from_numpy(synth.velocity_field_np(32, 10, 73)).cuda())
    assert t.halo_copy(False) == trk.TRK_HALO_ASYNC
    t.close()
    t = trk.Tracker(32, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_halo_copy(trk.TRK_HALO_TMA)
    t.set_field(torch.zeros((2, 32, 32, 32), dtype=torch.float32).cuda())
    assert t.halo_copy(False) == trk.TRK_HALO_ASYNC
    t.close()
