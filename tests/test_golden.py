"""The oracle against the cited reference values in tests/golden/ (no GPU).

Each fixture holds exact rationals from a published closed form or table,
with its citation in the file header: the Adams-Bashforth coefficients of
orders 1-4, the Lagrange weights at the cell midpoint for I = 4, 6, 8, and
the cubic convolution kernel (a = -1/2) that the I = 4, m = 1 spline must
equal."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                out.append([Fraction(x) for x in line.split()])
    return out


def test_fixtures_are_consistent():
    """Every weight row sums to one (partition of unity / consistency of the scheme)."""
    for r in rows("adams_bashforth_coefficients.txt"):
        assert sum(r[1:]) == 1 and len(r) == int(r[0]) + 1
    for r in rows("lagrange_midpoint_weights.txt"):
        assert sum(r[1:]) == 1 and len(r) == int(r[0]) + 1
    for r in rows("keys_cubic_convolution.txt"):
        assert sum(r[1:]) == 1 and len(r) == 5


@pytest.mark.parametrize("row", rows("lagrange_midpoint_weights.txt"), ids=lambda r: f"I{int(r[0])}")
def test_lagrange_midpoint_weights(row):
    I = int(row[0])
    got = oracle.weights(oracle.LAGRANGE, I, 0, 0.5)
    np.testing.assert_allclose(got, [float(x) for x in row[1:]], rtol=0, atol=2e-16 * I)


@pytest.mark.parametrize("row", rows("keys_cubic_convolution.txt"), ids=lambda r: f"t{float(r[0])}")
def test_spline_I4_m1_is_the_cubic_convolution_kernel(row):
    got = oracle.weights(oracle.SPLINE, 4, 1, float(row[0]))
    np.testing.assert_allclose(got, [float(x) for x in row[1:]], rtol=0, atol=1e-15)


def ab_step_weights(scheme, k, q):
    """Weights of one oracle step of order q (history length q - 1), isolated by
    a uniform field for beta_0 and one unit history entry per older weight."""
    N, dt = 16, 0.125
    u0 = 0.25
    f = np.zeros((3, N, N, N))
    f[0] = u0
    pos = np.array([[1.0], [2.0], [3.0]])
    hv = q - 1
    out, _ = oracle.advance(f, pos, dt, 1, oracle.SPLINE, 4, 1, scheme=scheme,
                            rhs=np.zeros((max(k - 1, 1), 3, 1)), history_valid=hv)
    w = [(out[0, 0] - pos[0, 0]) / (dt * u0)]
    for j in range(1, q):
        H = np.zeros((k - 1, 3, 1))
        H[j - 1, 1, 0] = 1.0
        out, _ = oracle.advance(f, pos, dt, 1, oracle.SPLINE, 4, 1, scheme=scheme, rhs=H, history_valid=hv)
        w.append((out[1, 0] - pos[1, 0]) / dt)
    return w


@pytest.mark.parametrize("row", rows("adams_bashforth_coefficients.txt"), ids=lambda r: f"order{int(r[0])}")
def test_adams_bashforth_coefficients(row):
    """Order q is the AB4 scheme with q - 1 valid history entries (start-up
    uses the lower orders), and the AB(q) scheme with a full history."""
    q = int(row[0])
    exp = [float(x) for x in row[1:]]
    np.testing.assert_allclose(ab_step_weights(oracle.AB4, 4, q), exp, rtol=0, atol=1e-13)
    if q >= 2:
        scheme = {2: oracle.AB2, 3: oracle.AB3, 4: oracle.AB4}[q]
        np.testing.assert_allclose(ab_step_weights(scheme, q, q), exp, rtol=0, atol=1e-13)
