"""GPU: Adams-Bashforth of orders 2-4 against the oracle.

Same-input comparisons (the oracle gets the stored field values).  The
library keeps the rhs history in float32 (the oracle in float64), which adds
up to ~1e-7 relative per history value; the tolerance is that of the float32
field (2e-6 of the field rms per interpolation) times the steps, plus the
history rounding weighted by the largest AB weight sum (|beta| <= 6.25 for
AB4).
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


def stored(field, storage):
    if storage == trk.TRK_F64:
        return field
    f32 = field.astype(np.float32)
    if storage == trk.TRK_F32:
        return f32.astype(np.float64)
    hi, lo = synth.bf16_split(torch.from_numpy(f32))
    return hi.double().numpy() + lo.double().numpy()


@pytest.mark.parametrize("scheme", [trk.TRK_AB2, trk.TRK_AB3, trk.TRK_AB4])
@pytest.mark.parametrize("storage,I,m", [(trk.TRK_F32, 6, 2), (trk.TRK_F32, 4, 1), (trk.TRK_F64, 6, 2),
                                         (trk.TRK_BF16X2, 8, 3)])
@pytest.mark.parametrize("first", [1, 2, 3])
def test_ab_matches_oracle_across_calls(scheme, storage, I, m, first):
    """`first` steps from no history, then the rest with the returned history."""
    k = scheme + 1
    N, n, dt, steps = 32, 3000, 4e-3, 9
    field = synth.velocity_field_np(N, 10, 95)
    pos = synth.uniform_particles_np(n, 12)
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=I, m=m, storage=storage)
    t.set_field(torch.from_numpy(field).to(DEV))
    p = torch.from_numpy(pos).to(DEV)
    rhs = torch.zeros((k - 1, 3, n), dtype=torch.float32, device=DEV)
    t.advance(p, dt, first, scheme, rhs=rhs, history_valid=0)
    t.advance(p, dt, steps - first, scheme, rhs=rhs, history_valid=min(first, k - 1))
    t.sync()
    ref, ref_rhs = oracle.advance(stored(field, storage), pos, dt, steps, trk.TRK_SPLINE, I, m, scheme=scheme)
    ref_rhs = np.asarray(ref_rhs).reshape(k - 1, 3, n)
    tol = (5 * 2e-6 + 6.25 * 1.2e-7 * 4) * dt * steps if storage != trk.TRK_F64 else 6.25 * 1.2e-7 * 4 * dt * steps
    assert np.abs(p.cpu().numpy() - ref).max() <= tol
    assert np.abs(rhs.cpu().numpy() - ref_rhs).max() <= 4 * 2e-6 * 4


@pytest.mark.parametrize("scheme", [trk.TRK_AB3, trk.TRK_AB4])
def test_ab_partial_history_and_start_up(scheme):
    """Fewer steps than k - 1: the history returned has the new entries first and
    zeros beyond; the first steps equal those of the lower order."""
    k = scheme + 1
    N, n, dt = 16, 500, 5e-3
    field = synth.velocity_field_np(N, 5, 96).astype(np.float32)
    pos = synth.uniform_particles_np(n, 13)
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_field(torch.from_numpy(field).to(DEV))
    p = torch.from_numpy(pos).to(DEV)
    rhs = torch.zeros((k - 1, 3, n), dtype=torch.float32, device=DEV)
    t.advance(p, dt, 1, scheme, rhs=rhs, history_valid=0)
    q = torch.from_numpy(pos).to(DEV)
    r2 = torch.zeros((k - 2, 3, n) if k > 3 else (3, n), dtype=torch.float32, device=DEV)
    t.advance(q, dt, 1, scheme - 1, rhs=r2, history_valid=0)
    t.sync()
    assert torch.equal(p, q)                                    # one Euler step either way
    h = rhs.cpu().numpy()
    assert np.abs(h[0]).max() > 0 and np.all(h[1:] == 0)


def test_ab_argument_errors():
    N = 16
    field = synth.velocity_field_np(N, 5, 97).astype(np.float32)
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_field(torch.from_numpy(field).to(DEV))
    p = torch.from_numpy(synth.uniform_particles_np(10, 1)).to(DEV)
    rhs = torch.zeros((2, 3, 10), dtype=torch.float32, device=DEV)
    with pytest.raises(trk.TrackerError) as e:
        t.advance(p, 1e-3, 1, trk.TRK_AB3, rhs=rhs, history_valid=3)
    assert e.value.status == trk.TRK_EINVAL
    with pytest.raises(ValueError):
        t.advance(p, 1e-3, 1, trk.TRK_AB4, rhs=rhs, history_valid=0)   # AB4 needs 3 entries
    with pytest.raises(trk.TrackerError):
        trk.tracker_advance(t.h, p, 1e-3, 1, 7, None, 0)               # unknown scheme
