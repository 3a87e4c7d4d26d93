"""Pins for the oracle's cell split, binning and triple sum (Sec. 2.2, Sec. 3.3.1).

References other than the oracle: exact geometry of the split, numpy's stable
argsort, polynomial reproduction, separable (tensor-product) fields against
scipy's 1-D Lagrange interpolation, the Keys kernel, convergence order on a
single Fourier mode, and analytic derivatives.
"""
import math

import numpy as np
import pytest
import scipy.interpolate

import oracle

L = 2 * math.pi


def test_split_geometry_and_ranges():
    N = 8
    delta = L / N
    rng = np.random.default_rng(0)
    xs = np.concatenate([
        np.arange(-2 * N, 3 * N) * delta,                     # on nodes, several periods
        rng.uniform(-20, 20, 500),                           # anywhere, negatives, > 2pi
        [-1e-300, -5e-324, 0.0, 5e-324, L, -L, 1e6, -1e6],    # tiny, wrap, large
    ])
    faces = np.arange(0, N + 1) * delta
    xs = np.concatenate([xs, np.nextafter(faces, -np.inf), np.nextafter(faces, np.inf)])
    pos = np.stack([xs, xs[::-1], np.roll(xs, 7)])
    c, t = oracle.split(pos, N)
    assert c.min() >= 0 and c.max() < N
    assert t.min() >= 0.0 and t.max() <= 1.0
    # (c + t) delta == X (mod 2 pi) to rounding
    rec = (c + t) * delta
    d = np.remainder(rec - pos + L / 2, L) - L / 2
    assert np.abs(d).max() < 1e-9 * (1 + np.abs(pos).max())


def test_split_rejects_nonfinite():
    pos = np.zeros((3, 4)); pos[1, 2] = np.nan
    with pytest.raises(FloatingPointError):
        oracle.split(pos, 16)
    pos[1, 2] = np.inf
    with pytest.raises(FloatingPointError):
        oracle.split(pos, 16)


@pytest.mark.parametrize("B", [(1, 1, 1), (2, 2, 2), (4, 2, 8), (8, 8, 1), (16, 16, 1)])
def test_binning_is_stable_sort_by_block(B):
    N = 16
    rng = np.random.default_rng(1)
    np_ = 3000
    pos = rng.uniform(-L, 2 * L, (3, np_))
    pos[:, :40] = pos[:, 40:80]            # duplicates: ties must keep incoming order
    keys, perm, offsets = oracle.bin_particles(pos, N, B)
    c, _ = oracle.split(pos, N)
    nb = (N // B[0], N // B[1], N // B[2])
    ref_keys = ((c[2] // B[2]) * nb[1] + c[1] // B[1]) * nb[0] + c[0] // B[0]
    np.testing.assert_array_equal(keys, ref_keys)
    np.testing.assert_array_equal(perm, np.argsort(keys, kind="stable"))
    counts = np.bincount(keys, minlength=nb[0] * nb[1] * nb[2])
    np.testing.assert_array_equal(offsets, np.concatenate([[0], np.cumsum(counts)]))
    assert offsets[-1] == np_


def test_binning_slices_like_the_paper():
    # B1 = B2 = N: one group per x3 slice (the slice ordering of Sec. 3.3.1)
    N = 8
    rng = np.random.default_rng(2)
    pos = rng.uniform(0, L, (3, 500))
    keys, perm, offsets = oracle.bin_particles(pos, N, (N, N, 1))
    c, _ = oracle.split(pos, N)
    np.testing.assert_array_equal(keys, c[2])
    assert np.all(np.diff(c[2][perm]) >= 0)


KERNELS = [(oracle.LAGRANGE, I, 0) for I in (4, 6, 8)] + [(oracle.SPLINE, 4, 1), (oracle.SPLINE, 6, 2),
                                                          (oracle.SPLINE, 8, 3), (oracle.SPLINE, 6, 1)]


def degree(family, I, m):
    return I - 1 if family == oracle.LAGRANGE else min(I - 2, 2 * m + 1)


def grid(N):
    return np.arange(N) * (L / N)


@pytest.mark.parametrize("family,I,m", KERNELS)
def test_constant_field(family, I, m):
    N = 16
    f = np.empty((3, N, N, N)); f[0] = 1.5; f[1] = -2.0; f[2] = 0.25
    pos = np.random.default_rng(3).uniform(-L, 2 * L, (3, 200))
    out = oracle.interp(f, pos, family, I, m)
    np.testing.assert_allclose(out, np.array([1.5, -2.0, 0.25])[:, None] * np.ones((1, 200)), atol=1e-13)


@pytest.mark.parametrize("family,I,m", KERNELS)
def test_polynomial_field_reproduced_on_local_window(family, I, m):
    """A tensor polynomial of degree <= d per axis is reproduced exactly away from the seam."""
    N = 32
    d = degree(family, I, m)
    x = grid(N)
    X3, X2, X1 = np.meshgrid(x, x, x, indexing="ij")
    c0 = np.pi
    p = lambda a, b, c: ((a - c0) ** d + 0.3 * (a - c0)) * (1 + (b - c0) ** max(d - 1, 0)) * ((c - c0) ** 2 + 0.5)
    f = np.stack([p(X1, X2, X3), p(X2, X3, X1), p(X3, X1, X2)])
    rng = np.random.default_rng(4)
    pos = rng.uniform(c0 - 1.2, c0 + 1.2, (3, 300))      # stencils stay inside [0, 2pi)
    out = oracle.interp(f, pos, family, I, m)
    ref = np.stack([p(pos[0], pos[1], pos[2]), p(pos[1], pos[2], pos[0]), p(pos[2], pos[0], pos[1])])
    np.testing.assert_allclose(out, ref, rtol=1e-10, atol=1e-10)
    # gradient: derivative of the reproduced polynomial
    g = oracle.interp(f, pos, family, I, m, deriv=True)
    h = 1e-6
    for j in range(3):
        e = np.zeros((3, 1)); e[j] = h
        fd = (np.stack([p((pos + e)[0], (pos + e)[1], (pos + e)[2])]) -
              np.stack([p((pos - e)[0], (pos - e)[1], (pos - e)[2])])) / (2 * h)
        np.testing.assert_allclose(g[0, j], fd[0], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("I", [4, 6, 8])
def test_lagrange_separable_field_vs_scipy(I):
    """f = a(x1) b(x2) c(x3): the triple sum is the product of three 1-D Lagrange interpolants."""
    N = 16
    x = grid(N)
    a, b, c = np.sin(x) + 0.2, np.cos(2 * x), np.exp(np.sin(x))
    f = np.einsum("k,j,i->kji", c, b, a)[None]
    rng = np.random.default_rng(5)
    pos = rng.uniform(0, L, (3, 50))
    out = oracle.interp(f, pos, oracle.LAGRANGE, I, 0)[0]
    delta = L / N

    def lag1(vals, X):
        cc = int(np.floor(X / delta))
        idx = np.arange(cc + 1 - I // 2, cc + I // 2 + 1)
        poly = scipy.interpolate.BarycentricInterpolator((idx - cc).astype(float), vals[idx % N])
        return poly(X / delta - cc)

    ref = np.array([lag1(a, p[0]) * lag1(b, p[1]) * lag1(c, p[2]) for p in pos.T])
    np.testing.assert_allclose(out, ref, rtol=1e-9, atol=1e-10)


def test_spline_I4_m1_separable_is_keys_convolution():
    N = 16
    x = grid(N)
    a, b, c = np.sin(3 * x), np.cos(x) + 1, np.sin(x) ** 2
    f = np.einsum("k,j,i->kji", c, b, a)[None]
    pos = np.random.default_rng(6).uniform(0, L, (3, 40))
    out = oracle.interp(f, pos, oracle.SPLINE, 4, 1)[0]
    delta = L / N

    def keys(s):
        s = abs(s)
        return 1.5 * s ** 3 - 2.5 * s ** 2 + 1 if s <= 1 else (-0.5 * s ** 3 + 2.5 * s ** 2 - 4 * s + 2 if s < 2 else 0.0)

    def conv(vals, X):
        g = X / delta
        return sum(vals[j % N] * keys(g - j) for j in range(int(np.floor(g)) - 3, int(np.floor(g)) + 4))

    ref = np.array([conv(a, p[0]) * conv(b, p[1]) * conv(c, p[2]) for p in pos.T])
    np.testing.assert_allclose(out, ref, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("family,I,m", KERNELS)
def test_fourier_mode_convergence_order(family, I, m):
    """Error on sin(k.x) falls like delta^(d+1)."""
    k = np.array([1, 2, 1])
    pos = np.random.default_rng(7).uniform(0, L, (3, 400))
    exact = np.sin(k @ pos)
    errs = []
    Ns = [16, 32, 64]
    for N in Ns:
        x = grid(N)
        X3, X2, X1 = np.meshgrid(x, x, x, indexing="ij")
        f = np.sin(k[0] * X1 + k[1] * X2 + k[2] * X3)[None]
        errs.append(np.abs(oracle.interp(f, pos, family, I, m)[0] - exact).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    expected = degree(family, I, m) + 1
    assert orders[-1] > expected - 0.6, (errs, orders, expected)
    assert orders[-1] < expected + 1.0, (errs, orders, expected)


def test_nodes_give_grid_values():
    N = 16
    rng = np.random.default_rng(8)
    f = rng.standard_normal((2, N, N, N))
    cells = rng.integers(-N, 2 * N, (3, 100))
    pos = cells * (L / N)
    for fam, I, m in [(oracle.LAGRANGE, 6, 0), (oracle.SPLINE, 8, 3)]:
        out = oracle.interp(f, pos, fam, I, m)
        ref = f[:, cells[2] % N, cells[1] % N, cells[0] % N]
        np.testing.assert_allclose(out, ref, atol=1e-12)


def test_stencil_entry_matches_dense():
    N = 16
    rng = np.random.default_rng(9)
    f = rng.standard_normal((3, N, N, N))
    pos = rng.uniform(-L, 2 * L, (3, 64))
    I = 6
    c, t = oracle.split(pos, N)
    rel = np.arange(1 - I // 2, I // 2 + 1)
    st = np.empty((64, 3, I, I, I))
    for p in range(64):
        i3 = (c[2, p] + rel) % N
        i2 = (c[1, p] + rel) % N
        i1 = (c[0, p] + rel) % N
        st[p] = f[:, i3][:, :, i2][:, :, :, i1]
    a = oracle.interp_stencil(t, st, oracle.SPLINE, I, 2)
    b = oracle.interp(f, pos, oracle.SPLINE, I, 2)
    np.testing.assert_allclose(a, b, atol=1e-13)
