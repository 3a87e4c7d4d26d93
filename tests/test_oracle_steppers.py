"""Pins for the oracle's time steppers for Eq. (tracers).

Uniform flow advects exactly; a linear (solid-body rotation) field is
reproduced exactly by every kernel away from the periodic seam, so the
discrete RK2 and AB2 maps have closed forms in 3x3 matrices; the global error
against the exact rotation falls like dt^2.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle

L = 2 * math.pi


def linear_field(N, A, xc):
    x = np.arange(N) * (L / N)
    X3, X2, X1 = np.meshgrid(x, x, x, indexing="ij")
    R = np.stack([X1 - xc[0], X2 - xc[1], X3 - xc[2]])
    return np.einsum("kj,jabc->kabc", A, R)


A_ROT = np.array([[0.0, -1.0, 0.3], [1.0, 0.0, -0.2], [-0.3, 0.2, 0.0]])  # antisymmetric: rotation
XC = np.array([math.pi, math.pi, math.pi])


@pytest.mark.parametrize("scheme", [oracle.RK2, oracle.AB2])
def test_uniform_flow_is_exact(scheme):
    N = 16
    u0 = np.array([0.7, -1.1, 0.35])
    f = np.broadcast_to(u0[:, None, None, None], (3, N, N, N)).copy()
    pos = np.random.default_rng(0).uniform(0, L, (3, 100))
    dt, steps = 0.01, 37
    res = oracle.advance(f, pos, dt, steps, oracle.SPLINE, 6, 2, scheme=scheme)
    out = res[0] if scheme == oracle.AB2 else res
    np.testing.assert_allclose(out, pos + steps * dt * u0[:, None], atol=1e-12)


@pytest.mark.parametrize("family,I,m", [(oracle.LAGRANGE, 4, 0), (oracle.SPLINE, 6, 2), (oracle.SPLINE, 8, 3)])
def test_rk2_rotation_closed_form(family, I, m):
    N = 32
    f = linear_field(N, A_ROT, XC)
    rng = np.random.default_rng(1)
    pos = XC[:, None] + rng.uniform(-0.6, 0.6, (3, 50))
    h, n = 0.02, 25
    out = oracle.advance(f, pos, h, n, family, I, m, scheme=oracle.RK2)
    M = np.eye(3) + h * A_ROT + 0.5 * h * h * A_ROT @ A_ROT
    ref = XC[:, None] + np.linalg.matrix_power(M, n) @ (pos - XC[:, None])
    np.testing.assert_allclose(out, ref, atol=1e-12)


def test_ab2_rotation_recurrence():
    N = 32
    f = linear_field(N, A_ROT, XC)
    rng = np.random.default_rng(2)
    pos = XC[:, None] + rng.uniform(-0.6, 0.6, (3, 40))
    h, n = 0.02, 20
    out, rhs = oracle.advance(f, pos, h, n, oracle.SPLINE, 6, 2, scheme=oracle.AB2)
    # AB2 with a forward-Euler first step, written on the deviation y = X - xc
    y_prev = pos - XC[:, None]
    y = y_prev + h * A_ROT @ y_prev
    for _ in range(n - 1):
        y, y_prev = y + h * (1.5 * A_ROT @ y - 0.5 * A_ROT @ y_prev), y
    np.testing.assert_allclose(out, XC[:, None] + y, atol=1e-12)
    np.testing.assert_allclose(rhs, A_ROT @ y_prev, atol=1e-12)


def test_ab2_history_continues():
    N = 16
    f = linear_field(N, A_ROT, XC)
    pos = XC[:, None] + np.random.default_rng(3).uniform(-0.4, 0.4, (3, 30))
    a, ra = oracle.advance(f, pos, 0.03, 10, oracle.LAGRANGE, 4, 0, scheme=oracle.AB2)
    b, rb = oracle.advance(f, pos, 0.03, 4, oracle.LAGRANGE, 4, 0, scheme=oracle.AB2)
    b, rb = oracle.advance(f, b, 0.03, 6, oracle.LAGRANGE, 4, 0, scheme=oracle.AB2, rhs=rb, history_valid=True)
    np.testing.assert_allclose(a, b, atol=1e-14)
    np.testing.assert_allclose(ra, rb, atol=1e-14)


@pytest.mark.parametrize("scheme", [oracle.RK2, oracle.AB2])
def test_global_error_is_second_order(scheme):
    N = 32
    f = linear_field(N, A_ROT, XC)
    pos = XC[:, None] + np.random.default_rng(4).uniform(-0.5, 0.5, (3, 20))
    T = 0.8
    exact = XC[:, None] + scipy.linalg.expm(T * A_ROT) @ (pos - XC[:, None])
    errs = []
    for n in (20, 40, 80):
        res = oracle.advance(f, pos, T / n, n, oracle.SPLINE, 6, 2, scheme=scheme)
        out = res[0] if scheme == oracle.AB2 else res
        errs.append(np.abs(out - exact).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.25), (errs, orders)


# ---------------------------------------------------------------------------
# Higher-order Adams-Bashforth (AB3, AB4)
# ---------------------------------------------------------------------------
def ab_weights_textbook(q):
    """Adams-Bashforth weights of order q from their definition: the integral
    over one step (s in [0, 1]) of the Lagrange basis polynomials on the past
    nodes s = 0, -1, ..., -(q-1) (newest first)."""
    nodes = -np.arange(q, dtype=float)
    w = []
    for j in range(q):
        p = np.poly1d([1.0])
        for i in range(q):
            if i != j:
                p = p * np.poly1d([1.0, -nodes[i]]) / (nodes[j] - nodes[i])
        P = p.integ()
        w.append(P(1.0) - P(0.0))
    return np.array(w)


@pytest.mark.parametrize("scheme,k", [(oracle.AB2, 2), (oracle.AB3, 3), (oracle.AB4, 4)])
def test_ab_weights_match_their_definition(scheme, k):
    """One step in a uniform field u with a chosen history isolates each weight:
    X' - X = dt (beta_0 u + sum_j beta_j H_{j-1})."""
    N, dt = 16, 0.1
    u0 = np.array([0.25, 0.0, 0.0])
    f = np.broadcast_to(u0[:, None, None, None], (3, N, N, N)).copy()
    pos = np.array([[1.0], [2.0], [3.0]])
    for hv in range(k):                      # history length -> order q = hv + 1
        q = hv + 1
        got = []
        # beta_0 from a zero history, beta_j from a unit history entry j-1 on axis 1
        out, _ = oracle.advance(f, pos, dt, 1, oracle.SPLINE, 4, 1, scheme=scheme,
                                rhs=np.zeros((k - 1, 3, 1)), history_valid=hv)
        got.append((out[0, 0] - pos[0, 0]) / (dt * u0[0]))
        for j in range(1, q):
            H = np.zeros((k - 1, 3, 1))
            H[j - 1, 1, 0] = 1.0
            out, _ = oracle.advance(f, pos, dt, 1, oracle.SPLINE, 4, 1, scheme=scheme, rhs=H, history_valid=hv)
            got.append((out[1, 0] - pos[1, 0]) / dt)
        np.testing.assert_allclose(got, ab_weights_textbook(q), rtol=0, atol=1e-13)


@pytest.mark.parametrize("scheme,k", [(oracle.AB3, 3), (oracle.AB4, 4)])
def test_ab_global_error_order_with_exact_history(scheme, k):
    """Rotation field, history taken from the exact solution: global error ~ dt^k."""
    N = 32
    f = linear_field(N, A_ROT, XC)
    pos = XC[:, None] + np.random.default_rng(5).uniform(-0.5, 0.5, (3, 20))
    T = 0.8
    y0 = pos - XC[:, None]
    exact = XC[:, None] + scipy.linalg.expm(T * A_ROT) @ y0
    errs = []
    for n in (16, 32, 64):
        h = T / n
        H = np.stack([A_ROT @ scipy.linalg.expm(-(e + 1) * h * A_ROT) @ y0 for e in range(k - 1)])
        out, _ = oracle.advance(f, pos, h, n, oracle.SPLINE, 6, 2, scheme=scheme, rhs=H, history_valid=k - 1)
        errs.append(np.abs(out - exact).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - k) < 0.3), (errs, orders)


@pytest.mark.parametrize("scheme,k", [(oracle.AB3, 3), (oracle.AB4, 4)])
def test_ab_start_up_uses_lower_orders(scheme, k):
    """Without history the first k-1 steps of ABk are those of AB(k-1)."""
    N = 16
    f = linear_field(N, A_ROT, XC)
    pos = XC[:, None] + np.random.default_rng(6).uniform(-0.4, 0.4, (3, 25))
    hi, _ = oracle.advance(f, pos, 0.03, k - 1, oracle.SPLINE, 4, 1, scheme=scheme)
    lo, _ = oracle.advance(f, pos, 0.03, k - 1, oracle.SPLINE, 4, 1, scheme=scheme - 1)
    np.testing.assert_array_equal(hi, lo)


@pytest.mark.parametrize("scheme,k", [(oracle.AB3, 3), (oracle.AB4, 4)])
def test_ab_history_continues(scheme, k):
    N = 16
    f = linear_field(N, A_ROT, XC)
    pos = XC[:, None] + np.random.default_rng(7).uniform(-0.4, 0.4, (3, 30))
    a, ra = oracle.advance(f, pos, 0.03, 11, oracle.LAGRANGE, 4, 0, scheme=scheme)
    for first in (1, 2, 5):
        b, rb = oracle.advance(f, pos, 0.03, first, oracle.LAGRANGE, 4, 0, scheme=scheme)
        b, rb = oracle.advance(f, b, 0.03, 11 - first, oracle.LAGRANGE, 4, 0, scheme=scheme, rhs=rb,
                               history_valid=min(first, k - 1))
        np.testing.assert_allclose(a, b, atol=1e-14)
        np.testing.assert_allclose(ra, rb, atol=1e-14)


@pytest.mark.parametrize("scheme", [oracle.AB3, oracle.AB4])
def test_ab_uniform_flow_is_exact(scheme):
    N = 16
    u0 = np.array([0.7, -1.1, 0.35])
    f = np.broadcast_to(u0[:, None, None, None], (3, N, N, N)).copy()
    pos = np.random.default_rng(8).uniform(0, L, (3, 100))
    out, rhs = oracle.advance(f, pos, 0.01, 37, oracle.SPLINE, 6, 2, scheme=scheme)
    np.testing.assert_allclose(out, pos + 37 * 0.01 * u0[:, None], atol=1e-12)
    np.testing.assert_allclose(rhs, np.broadcast_to(u0[None, :, None], rhs.shape), atol=1e-14)
