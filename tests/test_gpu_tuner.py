"""The time-step tuner: timed choice of the step kernel and its launch shape.

Every candidate (column kernel segments, direct-kernel binning block edges,
the block kernel's halo copy) must give bit-identical trajectories, so the
tuned run is compared bit for bit with runs fixed to each candidate and to
the untuned default; decisions are remembered and, through TRK_TUNE_CACHE,
persisted across trackers.
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


def _run(N, storage, field, pos, steps, tuning=None, scheme=trk.TRK_RK2, dt=5e-3):
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=storage)
    if tuning is not None:
        t.set_tuning(**tuning)
    t.set_field(torch.from_numpy(field).cuda())
    p = torch.from_numpy(pos).cuda()
    rhs = torch.zeros((3, pos.shape[1]), dtype=torch.float32, device="cuda") if scheme == trk.TRK_AB2 else None
    t.advance(p, dt, steps, scheme, rhs=rhs)
    try:
        t.sync()
    except trk.TrackerError as e:
        assert e.status == trk.TRK_ECFL
    info = t.tuning()
    t.close()
    return p.cpu(), info


CASES = {
    # (N, particles per cell, storage): candidates the tuner times
    # (direct: edges 8/16 x 256/128 particles per CTA)
    "column_and_direct": (128, 1 / 16, trk.TRK_F32),    # column 8/16, direct
    "dense_all_kernels": (64, 1 / 2, trk.TRK_F32),      # column 8 (N/8 = 8 slabs), block tma/async, direct
    "sparse_direct_only": (256, 1 / 200, trk.TRK_F32),  # direct
    "no_column_float64": (128, 1 / 16, trk.TRK_F64),    # block tma/async, direct
}


def _candidates(N, dens, storage):
    """The tuner's candidates and a few more launch shapes, all fixed in turn."""
    c = []
    if dens >= 0.01 and storage == trk.TRK_F32:
        c += [dict(step_kernel=trk.TRK_STEP_COLUMN, column_segment=s) for s in (4, 8, 16) if s <= N // 8]
    c += [dict(step_kernel=trk.TRK_STEP_BLOCK, halo_copy=h) for h in (trk.TRK_HALO_TMA, trk.TRK_HALO_ASYNC)]
    c += [dict(step_kernel=trk.TRK_STEP_DIRECT, direct_block=b) for b in (4, 8, 16, 32)]
    c += [dict(step_kernel=trk.TRK_STEP_DIRECT, direct_block=b, direct_particles=128) for b in (8, 16)]
    c += [dict(step_kernel=trk.TRK_STEP_DIRECT, direct_block=8, direct_particles=64)]
    return c


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("scheme", [trk.TRK_RK2, trk.TRK_AB2])
def test_tuned_run_is_bit_identical_to_every_candidate(case, scheme):
    N, dens, storage = CASES[case]
    n = int(dens * N ** 3)
    steps = 16
    field = synth.velocity_field_np(N, N // 3, 60 + N)
    pos = synth.uniform_particles_np(n, 61)
    tuned, info = _run(N, storage, field, pos, steps, scheme=scheme)
    assert info["source"] == trk.TRK_TUNE_TIMED, info
    # the untuned default (the density rule) and every candidate, fixed
    default, dinfo = _run(N, storage, field, pos, 5, tuning=None, scheme=scheme)   # too few steps to time
    assert dinfo["source"] == trk.TRK_TUNE_DEFAULT
    for cand in _candidates(N, dens, storage):
        got, cinfo = _run(N, storage, field, pos, steps, tuning=cand, scheme=scheme)
        assert cinfo["source"] == trk.TRK_TUNE_FIXED
        assert cinfo["step_kernel"] == cand["step_kernel"]
        assert torch.equal(got, tuned), (case, cand)
    short, _ = _run(N, storage, field, pos, 5, tuning=_candidates(N, dens, storage)[0], scheme=scheme)
    assert torch.equal(short, default)
    # and the tuned trajectory against the oracle on a sample
    fs = field if storage == trk.TRK_F64 else field.astype(np.float32).astype(np.float64)
    ix = np.random.default_rng(0).choice(n, 200, replace=False)
    ref = oracle.advance(fs, pos[:, ix], 5e-3, steps, trk.TRK_SPLINE, 6, 2, scheme=scheme)
    ref = ref[0] if scheme == trk.TRK_AB2 else ref
    tol = 1e-7 if storage == trk.TRK_F64 else 5 * 2e-6 * 5e-3 * steps
    assert np.abs(tuned.numpy()[:, ix] - ref).max() <= tol


def test_tuning_is_remembered_and_persisted(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("TRK_TUNE_CACHE", str(cache))
    N, n = 128, 128 ** 3 // 16
    field = synth.velocity_field_np(N, 42, 62).astype(np.float32)
    pos = synth.uniform_particles_np(n, 63)
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_field(torch.from_numpy(field).cuda())
    p = torch.from_numpy(pos).cuda()
    t.advance(p, 5e-3, 16)
    first = t.tuning()
    t.advance(p, 5e-3, 16)
    again = t.tuning()
    t.close()
    assert first["source"] == trk.TRK_TUNE_TIMED and again["source"] == trk.TRK_TUNE_CACHED
    assert {k: first[k] for k in first if k != "source"} == {k: again[k] for k in again if k != "source"}
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("advance2 N=128 ")
    # a new tracker (as in a new process) reads the file and times nothing
    t2 = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t2.set_field(torch.from_numpy(field).cuda())
    q = torch.from_numpy(pos).cuda()
    t2.advance(q, 5e-3, 16)
    third = t2.tuning()
    t2.close()
    assert third["source"] == trk.TRK_TUNE_CACHED
    assert third["step_kernel"] == first["step_kernel"]
    # malformed lines and shapes this tracker cannot run are ignored
    cache.write_text("garbage\nadvance2 N=128 x|3 7 8 1 256\nadvance2 N=128 y|3 8 8 1\n" + "\n".join(lines) + "\n")
    t3 = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t3.set_field(torch.from_numpy(field).cuda())
    t3.advance(torch.from_numpy(pos).cuda(), 5e-3, 16)
    assert t3.tuning()["source"] == trk.TRK_TUNE_CACHED
    t3.close()


def test_tuned_block_edge_bins_bit_exactly():
    """The block edge the tuner picked for the direct path, given to the oracle:
    binning by cubes of that edge (tracker_bin with that block shape) equals the
    oracle's stable binning bit for bit, for the tracers the tuner ran on."""
    N, n = 128, 128 ** 3 // 32
    field = synth.velocity_field_np(N, 42, 64).astype(np.float32)
    pos = synth.uniform_particles_np(n, 65)
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    t.set_field(torch.from_numpy(field).cuda())
    t.advance(torch.from_numpy(pos).cuda(), 5e-3, 16)
    info = t.tuning()
    assert info["source"] == trk.TRK_TUNE_TIMED
    B = info["direct_block"] if info["step_kernel"] == trk.TRK_STEP_DIRECT else 8
    trk.tracker_set_block(t.h, B, B, B)
    keys, perm, offsets = t.bin(torch.from_numpy(pos).cuda())
    rk, rp, ro = oracle.bin_particles(pos, N, (B, B, B))
    np.testing.assert_array_equal(keys.cpu().numpy(), rk)
    np.testing.assert_array_equal(perm.cpu().numpy(), rp)
    np.testing.assert_array_equal(offsets.cpu().numpy(), ro)
    t.close()


@pytest.mark.parametrize("bad", [dict(step_kernel=trk.TRK_STEP_DIRECT, direct_block=3),
                                 dict(step_kernel=trk.TRK_STEP_DIRECT, direct_block=512),
                                 dict(step_kernel=trk.TRK_STEP_COLUMN, column_segment=128),
                                 dict(step_kernel=trk.TRK_STEP_AUTO),
                                 dict(step_kernel=trk.TRK_STEP_DIRECT, direct_particles=100),
                                 dict(step_kernel=trk.TRK_STEP_BLOCK, halo_copy=trk.TRK_HALO_AUTO)])
def test_set_tuning_rejects_invalid_shapes(bad):
    t = trk.Tracker(256, family=trk.TRK_SPLINE, I=6, m=2, storage=trk.TRK_F32)
    with pytest.raises(trk.TrackerError) as e:
        t.set_tuning(**bad)
    assert e.value.status == trk.TRK_EINVAL
    t.close()
