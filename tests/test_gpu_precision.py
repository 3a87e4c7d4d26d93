"""The precision configuration at its full size, against the FP64 oracle.

1024^3 grid, velocity u (3 components) and its spectral gradient (9
components, d u_k / d x_j from i k_j u_hat_k), stored as float32 and as split
bf16 hi + lo pairs, |k| <= 340, 2^27 uniform tracers with float64 positions,
spline kernel I = 8 (m = 3), interpolation of u and of u + grad u (12
components).  Eq. (triple_sum) of Sec. 2.2 at every tracer; the outputs of a
10^5-tracer subsample are compared element by element with the oracle's
direct quadruple sum over the same stencil nodes.

Two oracle inputs per storage (the readings of the tolerances):
  same input  the values the library stores (float32, or float64(hi) +
              float64(lo)): max error <= 2e-6 x the rms of the component
              group (u, or grad u); the library's float32 weights and sums
              alone;
  truth       the float64 field: float32 storage max error <= 2e-6 x rms,
              split bf16 rms error <= 1e-5 x rms.

The float64 field never exists whole on the host: it is made on the GPU one
component at a time and only the subsample's stencil nodes (512 per tracer
and component) are gathered for the oracle.  Both interpolation kernels the
tracker chooses between (one CTA per cell block with a shared-memory halo,
and direct stencil gathers) are run explicitly, and the automatic choice once.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2107_01104_gb300 as trk
import synth

pytestmark = pytest.mark.gpu

N, KMAX, NPART, NSUB, I8, M8 = 1024, 340, 1 << 27, 100_000, 8, 3
SEED_FIELD, SEED_POS = 1002, 3


@pytest.fixture(scope="module")
def c3():
    dev = torch.device("cuda")
    pos = synth.uniform_particles_torch(NPART, SEED_POS, device=dev)
    sub = pos[:, :NSUB].cpu().numpy()
    cell, frac = oracle.split(sub, N)
    rel = np.arange(1 - I8 // 2, I8 // 2 + 1)
    c1 = (cell[0][:, None] + rel[None, :]) % N
    c2 = (cell[1][:, None] + rel[None, :]) % N
    c3_ = (cell[2][:, None] + rel[None, :]) % N
    idx = ((c3_[:, :, None, None] * N + c2[:, None, :, None]) * N + c1[:, None, None, :]).reshape(NSUB, -1)
    idx_t = torch.from_numpy(idx).to(dev)
    f12 = torch.empty((12, N, N, N), dtype=torch.float32, device=dev)
    ref = {"truth": np.empty((12, NSUB)), "f32": np.empty((12, NSUB)), "bf16x2": np.empty((12, NSUB))}
    rms = np.empty(12)
    for i, comp in enumerate(synth.velocity_components_torch(N, KMAX, SEED_FIELD, device=dev)):
        f12[i] = comp.to(torch.float32)
        rms[i] = float(torch.sqrt(torch.mean(comp * comp)))
        flat = comp.reshape(-1)
        st_truth = flat[idx_t].cpu().numpy()
        del comp, flat
        g32 = f12[i].reshape(-1)[idx_t]
        hi, lo = synth.bf16_split(g32)
        st_f32 = g32.double().cpu().numpy()
        st_bf = (hi.double() + lo.double()).cpu().numpy()
        del g32, hi, lo
        for key, st in (("truth", st_truth), ("f32", st_f32), ("bf16x2", st_bf)):
            ref[key][i] = oracle.interp_stencil(frac, st.reshape(NSUB, 1, I8, I8, I8), oracle.SPLINE, I8, M8)[0]
    del idx_t
    torch.cuda.empty_cache()
    rms_u = float(np.sqrt(np.mean(rms[:3] ** 2)))
    rms_g = float(np.sqrt(np.mean(rms[3:] ** 2)))
    yield dict(pos=pos, f12=f12, ref=ref, rms_u=rms_u, rms_g=rms_g)
    del f12, pos
    torch.cuda.empty_cache()


def _check(out, c3, storage_key, C):
    got = out[:, :NSUB].double().cpu().numpy()
    groups = [(slice(0, 3), c3["rms_u"])] + ([(slice(3, 12), c3["rms_g"])] if C == 12 else [])
    for sl, r in groups:
        same = got[sl] - c3["ref"][storage_key][sl]
        assert np.abs(same).max() <= 2e-6 * r, (storage_key, C, sl, np.abs(same).max() / r)
        truth = got[sl] - c3["ref"]["truth"][sl]
        if storage_key == "f32":
            assert np.abs(truth).max() <= 2e-6 * r, (C, sl, np.abs(truth).max() / r)
        else:
            assert np.sqrt(np.mean(truth ** 2)) <= 1e-5 * r, (C, sl, np.sqrt(np.mean(truth ** 2)) / r)


@pytest.mark.parametrize("storage_key,storage", [("f32", trk.TRK_F32), ("bf16x2", trk.TRK_BF16X2)])
@pytest.mark.parametrize("C", [3, 12])
def test_config3_full_size(c3, storage_key, storage, C):
    t = trk.Tracker(N, family=trk.TRK_SPLINE, I=I8, m=M8, storage=storage)
    t.set_field(c3["f12"][:C])
    out = torch.empty((C, NPART), dtype=torch.float32, device="cuda")
    chosen = []
    for kind in (trk.TRK_STEP_AUTO, trk.TRK_STEP_BLOCK, trk.TRK_STEP_DIRECT):
        t.set_step_kernel(kind)
        out.fill_(float("nan"))
        t.interpolate(c3["pos"], out=out)
        t.sync()
        chosen.append(t.last_step_kernel())
        assert bool(torch.isfinite(out).all())
        _check(out, c3, storage_key, C)
    assert chosen[0] in (trk.TRK_STEP_BLOCK, trk.TRK_STEP_DIRECT)
    assert chosen[1:] == [trk.TRK_STEP_BLOCK, trk.TRK_STEP_DIRECT]
    t.close()
    del out
    torch.cuda.empty_cache()
