"""Pins for the oracle's discrete RK2 adjoint: central finite differences of
the oracle's own forward map, and the transpose (dot-product) identity of the
field-to-particle interpolation operator."""
import math

import numpy as np

import oracle
import synth

L = 2 * math.pi
FAM, I, M = oracle.SPLINE, 6, 2      # C^2 kernel, so finite differences are well defined


def small_case(np_=12, N=16, steps=4, seed=0):
    f = synth.velocity_field_np(N, 5, 1000 + seed)
    pos = synth.uniform_particles_np(np_, seed)
    return f, pos, 0.05, steps


def loss(f, pos, dt, steps):
    out = oracle.advance(f, pos, dt, steps, FAM, I, M)
    return out, (out ** 2).sum(axis=0)      # per-particle terms |X_p(T)|^2


def test_position_gradient_matches_central_differences():
    f, pos, dt, steps = small_case()
    out, _ = loss(f, pos, dt, steps)
    gpos, _ = oracle.adjoint_rk2(f, pos, 2 * out, dt, steps, FAM, I, M, with_field=False)
    h = 1e-6
    for a in range(3):
        e = np.zeros_like(pos); e[a] = h
        _, lp = loss(f, pos + e, dt, steps)
        _, lm = loss(f, pos - e, dt, steps)
        fd = (lp - lm) / (2 * h)          # particle p's own loss term, d/dX0[a, p]
        np.testing.assert_allclose(gpos[a], fd, rtol=2e-6, atol=2e-7)


def test_field_gradient_matches_central_differences():
    f, pos, dt, steps = small_case(np_=6, steps=3)
    out, _ = loss(f, pos, dt, steps)
    _, gf = oracle.adjoint_rk2(f, pos, 2 * out, dt, steps, FAM, I, M)
    N = f.shape[-1]
    c, _ = oracle.split(pos, N)
    h = 1e-6
    rng = np.random.default_rng(3)
    checked = 0
    for trial in range(12):
        p = rng.integers(pos.shape[1])
        k = rng.integers(3)
        node = [(c[a, p] + rng.integers(-2, 4)) % N for a in range(3)]
        fp = f.copy(); fp[k, node[2], node[1], node[0]] += h
        fm = f.copy(); fm[k, node[2], node[1], node[0]] -= h
        fd = (loss(fp, pos, dt, steps)[1].sum() - loss(fm, pos, dt, steps)[1].sum()) / (2 * h)
        g = gf[k, node[2], node[1], node[0]]
        assert abs(g - fd) < 1e-6 * max(1.0, abs(fd)) + 1e-7, (g, fd)
        checked += abs(fd) > 1e-4
    assert checked >= 4


def test_interpolation_transpose_identity():
    """With a zero field one Heun step has X' = X and dLoss/dfield = dt W(X)^T lambda."""
    N = 16
    rng = np.random.default_rng(4)
    pos = rng.uniform(-L, 2 * L, (3, 40))
    lam = rng.standard_normal((3, 40))
    zero = np.zeros((3, N, N, N))
    dt = 0.1
    gpos, gf = oracle.adjoint_rk2(zero, pos, lam, dt, 1, FAM, I, M)
    np.testing.assert_allclose(gpos, lam, atol=1e-15)
    df = rng.standard_normal((3, N, N, N))
    lhs = (oracle.interp(df, pos, FAM, I, M) * lam).sum()          # <W df, lambda>
    rhs = (df * gf).sum() / dt                                       # <df, W^T lambda>
    assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))
