"""GPU: restart from a state file continues a run bit for bit.

A run of S steps is compared with the same run stopped after s steps, written
to a state file in caller order, read back into a fresh tracker and advanced
by the remaining S - s steps (with the AB history and its valid count taken
from the file)."""
import numpy as np
import pytest
import torch

import paper_2107_01104_gb300 as trk
import synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


def tracker(N, field, kind):
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_step_kernel(kind)
    t.set_field(torch.from_numpy(field).to(DEV))
    return t


@pytest.mark.parametrize("kind", [trk.TRK_STEP_COLUMN, trk.TRK_STEP_DIRECT, trk.TRK_STEP_BLOCK])
@pytest.mark.parametrize("scheme,first", [(trk.TRK_RK2, 4), (trk.TRK_AB2, 1), (trk.TRK_AB4, 2), (trk.TRK_AB4, 5)])
def test_restart_is_bit_identical(tmp_path, kind, scheme, first):
    N, n, dt, S = 32, 3000, 4e-3, 9
    field = synth.velocity_field_np(N, 10, 500).astype(np.float32)
    pos = synth.uniform_particles_np(n, 31)
    k = scheme + 1
    rows = (k - 1, 3, n) if scheme else (1, 3, n)

    t = tracker(N, field, kind)
    p = torch.from_numpy(pos).to(DEV)
    h = torch.zeros(rows, dtype=torch.float32, device=DEV)
    t.advance(p, dt, S, scheme, rhs=h if scheme else None, history_valid=0)
    t.sync()

    t1 = tracker(N, field, kind)
    q = torch.from_numpy(pos).to(DEV)
    g = torch.zeros(rows, dtype=torch.float32, device=DEV)
    t1.advance(q, dt, first, scheme, rhs=g if scheme else None, history_valid=0)
    t1.sync()
    hv = min(first, k - 1) if scheme else 0
    f = tmp_path / "run.trk"
    t1.save_state(str(f), q, g if scheme else None, scheme, hv, step=first, time=first * dt, dt=dt)
    t1.close()

    t2 = tracker(N, field, kind)
    q2, g2, info = t2.load_state(str(f))
    assert (info["step"], info["history_valid"], info["dt"]) == (first, hv, dt)
    t2.advance(q2, info["dt"], S - info["step"], scheme, rhs=g2, history_valid=info["history_valid"])
    t2.sync()
    assert torch.equal(p, q2)
    if scheme:
        assert torch.equal(h, g2)


def test_load_state_checks_grid_and_kernel(tmp_path):
    t = trk.Tracker(32, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    pos = torch.from_numpy(synth.uniform_particles_np(10, 1))
    t.save_state(str(tmp_path / "a.trk"), pos)
    other = trk.Tracker(32, family=trk.TRK_SPLINE, I=4, m=1, storage=trk.TRK_F32)
    with pytest.raises(ValueError):
        other.load_state(str(tmp_path / "a.trk"))
    p, r, info = t.load_state(str(tmp_path / "a.trk"))
    assert r is None and torch.equal(p.cpu(), pos)
