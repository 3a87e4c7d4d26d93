"""Pins for the oracle's interpolation kernels beta_i (Sec. 2.2).

Each check compares against something other than the oracle itself: textbook
closed forms (Lagrange weights at t = 1/2, the Keys/Catmull-Rom cubic
convolution kernel, centred finite-difference coefficients), polynomial
reproduction, partition of unity and the smoothness order.
"""
import numpy as np
import pytest

import oracle

KERNELS = [(oracle.LAGRANGE, I, 0) for I in (4, 6, 8)] + [
    (oracle.SPLINE, I, m) for I in (4, 6, 8) for m in range(0, I // 2 + 1)
]
TS = np.linspace(0.0, 1.0, 23)


def reproduced_degree(family, I, m):
    n = I // 2 - 1
    return I - 1 if family == oracle.LAGRANGE else min(2 * n, 2 * m + 1)


def nodes(I):
    return np.arange(1 - I // 2, I // 2 + 1, dtype=np.float64)


@pytest.mark.parametrize("family,I,m", KERNELS)
def test_partition_of_unity(family, I, m):
    for t in TS:
        assert abs(oracle.weights(family, I, m, t).sum() - 1.0) < 1e-12


@pytest.mark.parametrize("family,I,m", KERNELS)
def test_interpolates_nodes(family, I, m):
    e0 = np.zeros(I); e0[I // 2 - 1] = 1.0
    e1 = np.zeros(I); e1[I // 2] = 1.0
    np.testing.assert_allclose(oracle.weights(family, I, m, 0.0), e0, atol=1e-12)
    np.testing.assert_allclose(oracle.weights(family, I, m, 1.0), e1, atol=1e-12)


@pytest.mark.parametrize("family,I,m", KERNELS)
def test_polynomial_reproduction_degree(family, I, m):
    """Reproduces x^q exactly for q <= d and not for q = d + 1 (pins d)."""
    d = reproduced_degree(family, I, m)
    x = nodes(I)
    for q in range(0, d + 2):
        err = max(abs(oracle.weights(family, I, m, t) @ x ** q - t ** q) for t in TS)
        if q <= d:
            assert err < 1e-11, (q, err)
        else:
            assert err > 1e-6, (q, err)


def test_lagrange_midpoint_textbook():
    # Lagrange weights at the cell centre (textbook values of centred interpolation)
    exp = {
        4: [-1, 9, 9, -1],
        6: [3, -25, 150, 150, -25, 3],
        8: [-5, 49, -245, 1225, 1225, -245, 49, -5],
    }
    den = {4: 16, 6: 256, 8: 2048}
    for I in (4, 6, 8):
        np.testing.assert_allclose(oracle.weights(oracle.LAGRANGE, I, 0, 0.5),
                                   np.array(exp[I], float) / den[I], rtol=0, atol=1e-15)


def keys_kernel(x, a=-0.5):
    x = abs(x)
    if x <= 1:
        return (a + 2) * x ** 3 - (a + 3) * x ** 2 + 1
    if x < 2:
        return a * x ** 3 - 5 * a * x ** 2 + 8 * a * x - 4 * a
    return 0.0


def test_spline_I4_m1_is_catmull_rom():
    """n=1, m=1 is the Keys (a = -1/2) cubic convolution kernel (Catmull-Rom)."""
    for t in TS:
        ref = [keys_kernel(t - i) for i in nodes(4)]
        np.testing.assert_allclose(oracle.weights(oracle.SPLINE, 4, 1, t), ref, atol=1e-14)


def test_spline_m0_is_linear():
    for I in (4, 6, 8):
        for t in TS:
            w = oracle.weights(oracle.SPLINE, I, 0, t)
            ref = np.zeros(I); ref[I // 2 - 1] = 1 - t; ref[I // 2] = t
            np.testing.assert_allclose(w, ref, atol=1e-14)


def poly_coeffs_of_weights(family, I, m, deg):
    """Monomial coefficients of each beta_i, recovered by exact-degree fitting."""
    ts = 0.5 - 0.5 * np.cos(np.pi * (np.arange(deg + 1) + 0.5) / (deg + 1))
    W = np.array([oracle.weights(family, I, m, t) for t in ts])  # (deg+1, I)
    V = np.vander(ts, deg + 1, increasing=True)
    return np.linalg.solve(V, W)  # (deg+1, I): coeff[s][i]


def deriv_at(coeffs, q, t):
    """q-th derivative of sum_s coeffs[s] t^s at t (vectorised over columns)."""
    out = np.zeros(coeffs.shape[1])
    for s in range(q, coeffs.shape[0]):
        f = 1.0
        for r in range(q):
            f *= (s - r)
        out += f * coeffs[s] * t ** (s - q)
    return out


@pytest.mark.parametrize("I,m", [(I, m) for I in (4, 6, 8) for m in range(1, I // 2 + 1)])
def test_spline_smoothness_order(I, m):
    """The spline interpolant is C^m across cell faces and not C^(m+1)."""
    deg = max(2 * m + 1, I - 1)
    co = poly_coeffs_of_weights(oracle.SPLINE, I, m, deg)
    rng = np.random.default_rng(5)
    y = rng.standard_normal(I + 1)  # values on nodes -n .. n+2; cell A = [0,1], cell B = [1,2]
    for q in range(0, m + 2):
        left = deriv_at(co, q, 1.0) @ y[:I]     # cell A at t=1 (nodes -n..n+1)
        right = deriv_at(co, q, 0.0) @ y[1:]    # cell B at t=0 (nodes 1-n..n+2)
        if q <= m:
            assert abs(left - right) < 1e-8 * (1 + abs(left)), (q, left, right)
        else:
            # one order beyond the matched one, the one-sided derivatives differ for generic data
            assert abs(left - right) > 1e-6, (q, left, right)


CENTRED_D1 = {1: [-1, 0, 1], 2: [1, -8, 0, 8, -1], 3: [-1, 9, -45, 0, 45, -9, 1]}
CENTRED_D1_DEN = {1: 2, 2: 12, 3: 60}
CENTRED_D2 = {1: [1, -2, 1], 2: [-1, 16, -30, 16, -1], 3: [2, -27, 270, -490, 270, -27, 2]}
CENTRED_D2_DEN = {1: 1, 2: 12, 3: 180}


@pytest.mark.parametrize("I,m", [(I, m) for I in (4, 6, 8) for m in range(1, I // 2 + 1)])
def test_spline_node_derivatives_are_centred_differences(I, m):
    """Node derivatives equal the textbook centred (2n+1)-point differences."""
    n = I // 2 - 1
    deg = max(2 * m + 1, I - 1)
    co = poly_coeffs_of_weights(oracle.SPLINE, I, m, deg)
    d1 = deriv_at(co, 1, 0.0)  # weights on nodes -n..n+1
    ref1 = np.zeros(I); ref1[:2 * n + 1] = np.array(CENTRED_D1[n], float) / CENTRED_D1_DEN[n]
    np.testing.assert_allclose(d1, ref1, atol=1e-9)
    if m >= 2:
        d2 = deriv_at(co, 2, 0.0)
        ref2 = np.zeros(I); ref2[:2 * n + 1] = np.array(CENTRED_D2[n], float) / CENTRED_D2_DEN[n]
        np.testing.assert_allclose(d2, ref2, atol=1e-8)


@pytest.mark.parametrize("family,I,m", KERNELS)
def test_derivative_weights_match_finite_differences(family, I, m):
    h = 1e-6
    for t in np.linspace(0.05, 0.95, 7):
        _, db = oracle.weights(family, I, m, t, deriv=True)
        fd = (oracle.weights(family, I, m, t + h) - oracle.weights(family, I, m, t - h)) / (2 * h)
        np.testing.assert_allclose(db, fd, atol=2e-8)
