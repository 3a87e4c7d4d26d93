"""Seeded input generator: divergence-free, unit rms, Kolmogorov-like slope, deterministic."""
import numpy as np

import synth


def test_field_is_solenoidal_and_normalised():
    N = 32
    u, g = synth.velocity_field_np(N, 10, 1234, with_grad=True)
    assert u.shape == (3, N, N, N) and g.shape == (9, N, N, N)
    assert abs(np.sqrt(np.mean(u * u)) - 1.0) < 1e-12
    div = g[0] + g[4] + g[8]               # du1/dx1 + du2/dx2 + du3/dx3
    assert np.abs(div).max() < 1e-10 * np.abs(g).max()
    # spectral gradient agrees with a finite difference of the field
    dx = 2 * np.pi / N
    fd = (np.roll(u[0], -1, axis=2) - np.roll(u[0], 1, axis=2)) / (2 * dx)
    assert np.abs(fd - g[0]).max() < 0.2 * np.abs(g[0]).max()


def test_spectrum_slope():
    N = 64
    u = synth.velocity_field_np(N, 21, 7)
    uh = np.fft.rfftn(u, axes=(1, 2, 3))
    k3 = np.fft.fftfreq(N, 1 / N)[:, None, None]
    k2 = np.fft.fftfreq(N, 1 / N)[None, :, None]
    k1 = np.fft.rfftfreq(N, 1 / N)[None, None, :]
    kk = np.sqrt(k1 ** 2 + k2 ** 2 + k3 ** 2)
    e = (np.abs(uh) ** 2).sum(0)
    w = np.where(k1 == 0, 1.0, 2.0)
    shells = np.arange(3, 20)
    E = np.array([(e * w)[(kk >= s - 0.5) & (kk < s + 0.5)].sum() for s in shells])
    slope = np.polyfit(np.log(shells), np.log(E), 1)[0]
    assert -2.1 < slope < -1.3, slope
    assert (e * w)[kk > 21.5].sum() < 1e-20 * e.sum()


def test_seeded_and_in_box():
    a = synth.uniform_particles_np(1000, 3)
    b = synth.uniform_particles_np(1000, 3)
    np.testing.assert_array_equal(a, b)
    assert a.min() >= 0 and a.max() < 2 * np.pi
    np.testing.assert_array_equal(synth.velocity_field_np(16, 4, 9), synth.velocity_field_np(16, 4, 9))
