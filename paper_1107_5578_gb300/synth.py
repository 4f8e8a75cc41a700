"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no diffraction arithmetic: it only draws fields.  Every generator is a
pure function of its seed, built on numpy's Philox counter-based generator so that the same
seed gives the same bits on x86_64 and aarch64.  Fields are produced in float64/complex128;
callers cast to complex64 for the GPU path.

Workload recipes (the paper's own inputs -- Lena images, a hologram bitmap, point clouds --
are not available, so these stand in for them):
  * random_field         amplitude ~ U[0,1), phase ~ U[0, 2 pi)         (512^2 ASM case)
  * masked_gaussian      Bernoulli(p) mask times exp(-r^2 / (2 sigma^2)) about (N/2, N/2)
                         (2048^2 Fresnel z-stack case, sigma = 400 px, p = 0.5)
  * random_phase_field   unit amplitude, phase ~ U[0, 2 pi)              (4096^2 precision case)
  * hologram_problem     phase ~ U[0, 2 pi) on 1080 x 1920 plus a smooth target made of 20
                         random Gaussians (phase-only hologram optimisation)
  * serving_requests     Poisson arrivals with mixed N, type, z, wavelength and pitch
  * gs_problem           GS kinoform input: amplitude sqrt(I) of a smooth test image I in
                         [0, 1] (30 Gaussians, sigma ~ U[N/64, N/8], peaks ~ U[0.3, 1], plus
                         two bright bars) and the initial random phase U[0, 2 pi)
  * gaussian_beam        exp(-r^2 / w0^2) about a given centre (closed-form test beam)
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def random_field(n: int, seed: int, ny: int | None = None) -> np.ndarray:
    ny = n if ny is None else ny
    g = rng(seed)
    amp = g.random((ny, n))
    ph = g.random((ny, n)) * (2.0 * np.pi)
    return amp * np.exp(1j * ph)


def random_phase_field(n: int, seed: int) -> np.ndarray:
    g = rng(seed)
    return np.exp(1j * (g.random((n, n)) * (2.0 * np.pi)))


def masked_gaussian(n: int, seed: int, sigma_px: float = 400.0, p: float = 0.5) -> np.ndarray:
    g = rng(seed)
    mask = (g.random((n, n)) < p).astype(np.float64)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    r2 = (x - n / 2) ** 2 + (y - n / 2) ** 2
    return (mask * np.exp(-r2 / (2.0 * sigma_px ** 2))).astype(np.complex128)


def gaussian_beam(n: int, pitch: float, w0: float, cx: float | None = None,
                  cy: float | None = None) -> np.ndarray:
    cx = n / 2 if cx is None else cx
    cy = n / 2 if cy is None else cy
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    r2 = ((x - cx) * pitch) ** 2 + ((y - cy) * pitch) ** 2
    return np.exp(-r2 / w0 ** 2).astype(np.complex128)


def hologram_problem(seed: int, h: int = 1080, w: int = 1920, n_gauss: int = 20):
    """Initial phase [h][w] ~ U[0, 2 pi) and an unnormalised smooth target [h][w] >= 0.

    Target: n_gauss Gaussians, centres uniform in the window, sigma ~ U[20, 120] px,
    peak ~ U[0.5, 1].  The caller rescales the target to the energy of its initial field.
    """
    g = rng(seed)
    phi = g.random((h, w)) * (2.0 * np.pi)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    tgt = np.zeros((h, w))
    for _ in range(n_gauss):
        cy, cx = g.random() * h, g.random() * w
        s = 20.0 + 100.0 * g.random()
        a = 0.5 + 0.5 * g.random()
        tgt += a * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2.0 * s * s))
    return phi, tgt


SERVING_SIZES = (256, 512, 1024, 2048, 4096)
SERVING_WEIGHTS = (0.3, 0.3, 0.2, 0.15, 0.05)
SERVING_WAVELENGTHS = (450e-9, 532e-9, 633e-9)


def serving_requests(n_req: int, seed: int, rate_hz: float = 2000.0,
                     sizes=SERVING_SIZES, weights=SERVING_WEIGHTS):
    """Open-loop Poisson request stream: arrival time (s), N, type (0 ASM / 1 Fresnel), z,
    wavelength, pitch, and a field-pool index.  Types are 70 % ASM, 30 % Fresnel."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate_hz, size=n_req)
    t = np.cumsum(gaps) - gaps[0]
    n = g.choice(np.asarray(sizes), size=n_req, p=np.asarray(weights) / np.sum(weights))
    kind = (g.random(n_req) < 0.3).astype(np.int64)
    z = 0.01 + 0.49 * g.random(n_req)
    lam = g.choice(np.asarray(SERVING_WAVELENGTHS), size=n_req)
    pitch = 4e-6 + 6e-6 * g.random(n_req)
    pool = g.integers(0, 1 << 30, size=n_req)
    return {"t": t, "n": n, "kind": kind, "z": z, "lam": lam, "pitch": pitch, "pool": pool}


def gs_problem(n: int, seed: int, n_gauss: int = 30):
    """(amplitude [n][n] >= 0, field0 = amplitude * exp(i phase0)) for the GS kinoform loop."""
    g = rng(seed)
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    img = np.zeros((n, n))
    for _ in range(n_gauss):
        cy, cx = g.random() * n, g.random() * n
        s = n / 64.0 + (n / 8.0 - n / 64.0) * g.random()
        a = 0.3 + 0.7 * g.random()
        img += a * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2.0 * s * s))
    img[n // 4:n // 4 + max(1, n // 32), n // 8:7 * n // 8] += 1.0
    img[n // 8:7 * n // 8, 3 * n // 4:3 * n // 4 + max(1, n // 32)] += 1.0
    img /= img.max()
    amp = np.sqrt(img)
    phase0 = g.random((n, n)) * (2.0 * np.pi)
    return amp, amp * np.exp(1j * phase0)
