"""Seeded synthetic input fields.

This module is shared by the tests, the benchmark and the CPU oracle's checks.
It only draws random numbers and shapes spectra; it contains none of the
compressor's arithmetic.  Every generator is deterministic for a given seed
and device (numpy generators for CPU-only use, torch generators otherwise).

Stand-ins for the paper's application data (the cosmology, climate and plasma
datasets of its "Application impact" section are not available):

* ``sinusoids_2d``      -- a sum of random-phase sinusoids plus small noise.
* ``gaussian_random_field`` -- an isotropic Gaussian random field whose
  shell-averaged energy spectrum falls off as ``|k|^-beta`` (Kolmogorov
  turbulence has ``beta = 5/3``), synthesised by filtering white noise in
  Fourier space; normalised to unit variance.
* ``blobs_field``       -- a random field plus localized Gaussian blobs.
* ``advected_field``    -- a sequence of timesteps: a base field shifted in
  Fourier space, damped at high wavenumbers, plus a small fresh innovation.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def sinusoids_2d(n0: int, n1: int, nwaves: int = 8, kmax: int = 16,
                 noise: float = 1e-3, seed: int = 0) -> np.ndarray:
    """Sum of ``nwaves`` unit-amplitude plane waves on ``[0,1]^2`` sampled at
    ``n0 x n1`` points, wavenumbers drawn from ``1..kmax`` per axis, phases
    uniform in ``[0, 2pi)``, plus ``N(0, noise^2)`` noise.  float64."""
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 1.0, n0)[:, None]
    y = np.linspace(0.0, 1.0, n1)[None, :]
    u = np.zeros((n0, n1))
    for _ in range(nwaves):
        kx, ky = rng.integers(1, kmax + 1, size=2)
        phi = rng.uniform(0.0, 2.0 * math.pi)
        u += np.sin(2.0 * math.pi * (kx * x + ky * y) + phi)
    u += rng.normal(0.0, noise, size=u.shape)
    return u


def _spectral_filter(shape, beta: float, device, dtype=torch.float64):
    """Amplitude filter sqrt(P(|k|)) for a D-dimensional isotropic field whose
    shell-averaged spectrum is E(k) ~ k^-beta, i.e. spectral density
    P(k) ~ k^-(beta + D - 1).  k = 0 is removed."""
    D = len(shape)
    grids = []
    for d, n in enumerate(shape):
        if d == D - 1:
            k = torch.fft.rfftfreq(n, d=1.0 / n, dtype=dtype, device=device)
        else:
            k = torch.fft.fftfreq(n, d=1.0 / n, dtype=dtype, device=device)
        view = [1] * D
        view[d] = -1
        grids.append(k.view(view) ** 2)
    k2 = grids[0]
    for g in grids[1:]:
        k2 = k2 + g
    k2 = k2.clone()
    zero = k2 == 0
    k2[zero] = 1.0
    expo = beta + D - 1.0
    amp = k2 ** (-expo / 4.0)          # sqrt(k^-expo) = (k^2)^(-expo/4)
    amp[zero] = 0.0
    return amp


def gaussian_random_field(shape, beta: float = 5.0 / 3.0, seed: int = 1,
                          device="cpu", out_dtype=torch.float32) -> torch.Tensor:
    """Isotropic Gaussian random field (periodic FFT synthesis in float64),
    unit variance, returned as ``out_dtype`` on ``device``."""
    shape = tuple(int(s) for s in shape)
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    white = torch.randn(shape, generator=g, dtype=torch.float64)
    white = white.to(device)
    W = torch.fft.rfftn(white)
    del white
    W *= _spectral_filter(shape, beta, device)
    u = torch.fft.irfftn(W, s=shape)
    del W
    u -= u.mean()
    u /= u.std()
    return u.to(out_dtype)


def blobs_field(shape, nblobs: int = 50, beta: float = 5.0 / 3.0, seed: int = 5,
                device="cpu", out_dtype=torch.float32) -> torch.Tensor:
    """Random-field background plus ``nblobs`` Gaussian blobs with widths
    uniform in [2, 20] cells and amplitudes of +-10 background std."""
    u = gaussian_random_field(shape, beta, seed, device, torch.float64)
    rng = np.random.default_rng(seed + 7919)
    axes = [torch.arange(n, dtype=torch.float64, device=device) for n in shape]
    for _ in range(nblobs):
        c = [rng.uniform(0, n - 1) for n in shape]
        sig = rng.uniform(2.0, 20.0)
        amp = rng.choice([-10.0, 10.0])
        # separable Gaussian: product of 1D factors
        fac = None
        for d, (a, cd) in enumerate(zip(axes, c)):
            f = torch.exp(-0.5 * ((a - cd) / sig) ** 2)
            view = [1] * len(shape)
            view[d] = -1
            f = f.view(view)
            fac = f if fac is None else fac * f
        u += amp * fac
    return u.to(out_dtype)


def advected_field(shape, t: int, beta: float = 5.0 / 3.0, seed: int = 0,
                   velocity=(0.7, 1.3, 0.5), innovation: float = 0.05,
                   decay_steps: float = 50.0, device="cpu",
                   out_dtype=torch.float32) -> torch.Tensor:
    """Timestep ``t`` of a field advected at ``velocity`` cells/step (a phase
    shift in Fourier space), damped so the Nyquist mode decays by e^-1 over
    ``decay_steps`` steps, plus ``innovation`` x a fresh field (seed 1000+t)."""
    shape = tuple(int(s) for s in shape)
    D = len(shape)
    base = gaussian_random_field(shape, beta, seed, device, torch.float64)
    U = torch.fft.rfftn(base)
    del base
    phase = None
    k2 = None
    for d, n in enumerate(shape):
        if d == D - 1:
            k = torch.fft.rfftfreq(n, d=1.0 / n, dtype=torch.float64, device=device)
        else:
            k = torch.fft.fftfreq(n, d=1.0 / n, dtype=torch.float64, device=device)
        view = [1] * D
        view[d] = -1
        kd = k.view(view)
        ph = 2.0 * math.pi * kd / n * velocity[d % len(velocity)] * t
        phase = ph if phase is None else phase + ph
        k2 = kd ** 2 if k2 is None else k2 + kd ** 2
    kny2 = sum((n / 2.0) ** 2 for n in shape)
    nu = 1.0 / (kny2 * decay_steps)
    U *= torch.polar(torch.exp(-nu * k2 * t), -phase)
    u = torch.fft.irfftn(U, s=shape)
    del U
    if innovation:
        u += innovation * gaussian_random_field(shape, beta, 1000 + t, device,
                                                torch.float64)
    return u.to(out_dtype)


def uneven_shapes(count: int = 64, lo: int = 33, hi: int = 300, seed: int = 100):
    """``count`` 3D shapes with each extent uniform in ``lo..hi`` and a
    spectrum exponent uniform in [2, 11/3] per field (returned as pairs)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        shp = tuple(int(x) for x in rng.integers(lo, hi + 1, size=3))
        beta = float(rng.uniform(2.0, 11.0 / 3.0))
        out.append((shp, beta))
    return out
