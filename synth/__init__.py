"""Seeded synthetic inputs: periodic random velocity fields and uniform tracers.

This module only makes inputs.  It holds none of the tracking method's
arithmetic (no cell split, no weights, no interpolation, no time stepping), so
both the CUDA path and the CPU oracle may use it.

The paper's DNS fields are not available; they are stood in for by a
divergence-free random Fourier field on [0, 2pi)^3 with a Kolmogorov-like
shell spectrum (the velocity of Sec. 2.1 is obtained in Fourier space from a
solenoidal vorticity by the Biot-Savart law, so it is divergence free):

* modes 1 <= |k| <= kmax, complex Gaussian amplitudes from a seeded generator,
* projected on k . u_hat = 0,
* scaled to |u_hat| ~ |k|^(-11/6), i.e. shell energy E(k) ~ k^(-5/3),
* transformed with an inverse real FFT (Hermitian symmetry implied),
* scaled by one common factor so the rms over the three components is 1.

The gradient (when asked for) is the spectral derivative
d u_k / d x_j = IFFT[i k_j u_hat_k], in the order grad[3*k + j].

Array layout: field[C][N][N][N] with x3 the slowest and x1 the fastest axis.
Grids up to N = 256 are made with numpy on the host; larger grids need the
torch CUDA path (:func:`velocity_field_torch`).  The two random streams differ,
so a given (N, seed) always uses the path its size selects.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def _spectrum_np(N: int, kmax: float, seed: int):
    rng = np.random.default_rng(seed)
    shape = (3, N, N, N // 2 + 1)
    uh = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    k3 = np.fft.fftfreq(N, 1.0 / N)[:, None, None]
    k2 = np.fft.fftfreq(N, 1.0 / N)[None, :, None]
    k1 = np.fft.rfftfreq(N, 1.0 / N)[None, None, :]
    kk = k1 * k1 + k2 * k2 + k3 * k3
    kvec = (np.broadcast_to(k1, kk.shape), np.broadcast_to(k2, kk.shape), np.broadcast_to(k3, kk.shape))
    shell = (kk >= 1.0) & (kk <= kmax * kmax)
    ksafe = np.where(kk > 0, kk, 1.0)
    kdotu = kvec[0] * uh[0] + kvec[1] * uh[1] + kvec[2] * uh[2]
    for a in range(3):
        uh[a] = uh[a] - kvec[a] * kdotu / ksafe
    amp = np.where(shell, ksafe ** (-11.0 / 12.0), 0.0)  # |u_hat| ~ k^(-11/6), k = sqrt(kk)
    uh *= amp[None]
    return uh, kvec


def velocity_field_np(N: int, kmax: float, seed: int, with_grad: bool = False):
    """Velocity u[3][N][N][N] (float64), optionally with grad[9][N][N][N]."""
    uh, kvec = _spectrum_np(N, kmax, seed)
    u = np.fft.irfftn(uh, s=(N, N, N), axes=(1, 2, 3))
    scale = 1.0 / math.sqrt(float(np.mean(u * u)))
    u *= scale
    if not with_grad:
        return u
    g = np.empty((9, N, N, N), np.float64)
    for k in range(3):
        for j in range(3):
            g[3 * k + j] = np.fft.irfftn(1j * kvec[j] * uh[k], s=(N, N, N), axes=(0, 1, 2)) * scale
    return u, g


def velocity_field_torch(N: int, kmax: float, seed: int, device="cuda", with_grad: bool = False,
                         out_dtype=None):
    """Same recipe on a torch device (float64 transforms).  For N > 256.

    Components are produced one at a time so the peak memory stays near one
    complex half-spectrum per component.  ``out_dtype`` (e.g. torch.float32)
    converts each component as it is produced.
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    k_full = torch.fft.fftfreq(N, 1.0 / N, device=device, dtype=torch.float64)
    k_half = torch.fft.rfftfreq(N, 1.0 / N, device=device, dtype=torch.float64)
    k3 = k_full[:, None, None]
    k2 = k_full[None, :, None]
    k1 = k_half[None, None, :]
    kk = k1 * k1 + k2 * k2 + k3 * k3
    shell = (kk >= 1.0) & (kk <= kmax * kmax)
    ksafe = torch.where(kk > 0, kk, torch.ones_like(kk))
    shape = (N, N, N // 2 + 1)
    uh = []
    for _ in range(3):
        re = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
        im = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
        uh.append(torch.complex(re, im))
    kvec = (k1, k2, k3)
    kdotu = k1 * uh[0] + k2 * uh[1] + k3 * uh[2]
    for a in range(3):
        uh[a] = uh[a] - kvec[a] * kdotu / ksafe
    del kdotu
    amp = torch.where(shell, ksafe ** (-11.0 / 12.0), torch.zeros_like(ksafe))
    del kk, shell, ksafe
    for a in range(3):
        uh[a] = uh[a] * amp
    del amp
    odt = out_dtype or torch.float64
    comps = []
    sumsq = 0.0
    for a in range(3):
        ua = torch.fft.irfftn(uh[a], s=(N, N, N))
        sumsq += float((ua * ua).sum())
        comps.append(ua.to(odt))
        del ua
    scale = 1.0 / math.sqrt(sumsq / (3.0 * N ** 3))
    u = torch.empty((3, N, N, N), dtype=odt, device=device)
    for a in range(3):
        u[a] = comps[a] * scale
    del comps
    if not with_grad:
        return u
    grad = torch.empty((9, N, N, N), dtype=odt, device=device)
    for k in range(3):
        for j in range(3):
            grad[3 * k + j] = (torch.fft.irfftn(1j * kvec[j] * uh[k], s=(N, N, N)) * scale).to(odt)
    return u, grad


def velocity_components_torch(N: int, kmax: float, seed: int, device="cuda", with_grad: bool = True):
    """Yield the float64 components of :func:`velocity_field_torch` one at a time.

    Order: u1, u2, u3, then d u_k / d x_j as 3k + j.  Same spectrum, seed and
    scaling as velocity_field_torch, so the values agree with it; only one
    real-space component is held at a time (for grids whose float64 copy does
    not fit at once).
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    k_full = torch.fft.fftfreq(N, 1.0 / N, device=device, dtype=torch.float64)
    k_half = torch.fft.rfftfreq(N, 1.0 / N, device=device, dtype=torch.float64)
    k3 = k_full[:, None, None]
    k2 = k_full[None, :, None]
    k1 = k_half[None, None, :]
    kk = k1 * k1 + k2 * k2 + k3 * k3
    shell = (kk >= 1.0) & (kk <= kmax * kmax)
    ksafe = torch.where(kk > 0, kk, torch.ones_like(kk))
    shape = (N, N, N // 2 + 1)
    uh = []
    for _ in range(3):
        re = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
        im = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
        uh.append(torch.complex(re, im))
    kvec = (k1, k2, k3)
    kdotu = k1 * uh[0] + k2 * uh[1] + k3 * uh[2]
    for a in range(3):
        uh[a] = uh[a] - kvec[a] * kdotu / ksafe
    del kdotu
    amp = torch.where(shell, ksafe ** (-11.0 / 12.0), torch.zeros_like(ksafe))
    del kk, shell, ksafe
    for a in range(3):
        uh[a] = uh[a] * amp
    del amp
    sumsq = 0.0
    for a in range(3):
        ua = torch.fft.irfftn(uh[a], s=(N, N, N))
        sumsq += float((ua * ua).sum())
        del ua
    scale = 1.0 / math.sqrt(sumsq / (3.0 * N ** 3))
    for a in range(3):
        yield torch.fft.irfftn(uh[a], s=(N, N, N)) * scale
    if with_grad:
        for k in range(3):
            for j in range(3):
                yield torch.fft.irfftn(1j * kvec[j] * uh[k], s=(N, N, N)) * scale


def uniform_particles_np(n: int, seed: int) -> np.ndarray:
    """Tracer positions pos[3][n] (float64), uniform in [0, 2pi)^3."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, TWO_PI, size=(3, n))


def uniform_particles_torch(n: int, seed: int, device="cuda"):
    """Tracer positions pos[3][n] (torch float64), uniform in [0, 2pi)^3, generated on ``device``."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.rand((3, n), generator=g, device=device, dtype=torch.float64) * TWO_PI


def velocity_field(N: int, kmax: float, seed: int, with_grad: bool = False):
    """numpy field for N <= 256 (the host path); see module docstring."""
    if N > 256:
        raise ValueError("N > 256 fields are made on the GPU with velocity_field_torch")
    return velocity_field_np(N, kmax, seed, with_grad)


def bf16_split(x):
    """Split a float32 torch tensor into bfloat16 (hi, lo) with hi + lo ~= x.

    hi = RN_bf16(x), lo = RN_bf16(x - hi).  This is the storage format the
    library's split-BF16 mode is specified to hold; the oracle consumes
    float64(hi) + float64(lo) in same-input comparisons.
    """
    import torch

    hi = x.to(torch.bfloat16)
    lo = (x - hi.to(torch.float32)).to(torch.bfloat16)
    return hi, lo
