"""FP64 CPU oracle for FFT-based scalar diffraction (CWO++, Shimobaba et al.).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this package; the product path never does.  It shares no code with
the CUDA library.  The arithmetic lives in ``cwo_oracle.c`` (plain C, double precision); this
module compiles it with gcc on first use and wraps it with ctypes.  The composites below (the
z-stack and the hologram loss gradient) only call those C functions in the order the paper's
usage describes.

Pins (each checked by the ``-m "not gpu"`` tests, none of them by re-calling this code):
  * ``fft``            -- direct DFT on every size 1..64 and numpy.fft as a third opinion
  * ``dft``            -- closed forms: delta -> ones, pure tone -> scaled delta (fixes the sign)
  * ``propagate``      -- Fresnel: brute-force direct sum and the Gaussian-beam closed form;
                          ASM: brute-force kernel sum, plane-wave phase exp(ikz), z = 0 identity,
                          Gaussian-beam Hankel quadrature, Parseval, z then -z
  * adjoint flag       -- dot-product test <A x, y> = <x, A^H y>
  * ``hologram_grad``  -- central finite differences
  * ``gs_run``         -- z = 0 fixed point, zero iterations = one propagation plus the phase
                          constraint, unit-amplitude kinoform, and on the circular (unitary)
                          grid the error-reduction property: the object-plane amplitude error
                          never increases from one iteration to the next
  * ``propagate_shifted`` -- no shift and no window = ``propagate``; on the circular grid a shift
                          of whole pixels is an exact translation; the window removes the
                          spectrum outside it
  * ``fresnel_fourier``-- the literal double sum of Eq. fre_fourier3 on tiny grids, the Gaussian
                          closed form on the destination grid, energy conservation
  * ``shifted_fresnel``-- the literal Fresnel sum at arbitrary destination pitches and offsets,
                          the convolution form at equal pitches, the off-axis Gaussian closed form
  * ``band_limit``     -- the limit is where the transfer phase's slope reaches the Nyquist rate
                          of the padded frequency grid (finite differences of the phase)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cwo_oracle.c")
_LIB = os.path.join(_HERE, "_cwo_oracle.so")

# flag and type values of cwo_oracle.c
ADJOINT = 1
NO_PAD = 2
FULL_OUTPUT = 4
LITERAL_SCALE = 8
ANGULAR = 0
FRESNEL_CONV = 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile cwo_oracle.c into _cwo_oracle.so with gcc (OpenMP on, IEEE arithmetic)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.c_void_p
            L, D, I, U = ctypes.c_long, ctypes.c_double, ctypes.c_int, ctypes.c_uint
            lib.orc_dft.argtypes = [dp, dp, L, I]
            lib.orc_dft.restype = None
            lib.orc_fft.argtypes = [dp, L, I]
            lib.orc_fft.restype = I
            lib.orc_fft2.argtypes = [dp, L, L, I]
            lib.orc_fft2.restype = I
            lib.orc_asm_transfer.argtypes = [dp, L, L, D, D, D, D]
            lib.orc_asm_transfer.restype = None
            lib.orc_propagate.argtypes = [dp, dp, L, L, D, D, D, D, I, U]
            lib.orc_propagate.restype = I
            lib.orc_propagate_direct.argtypes = [dp, dp, L, L, D, D, D, D, I, U]
            lib.orc_propagate_direct.restype = I
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = I
            lib.orc_set_threads.argtypes = [I]
            lib.orc_set_threads.restype = None
            _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def max_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().orc_max_threads())


def set_threads(n: int) -> None:
    """Threads for the oracle's parallel loops from now on (timing; results do not depend on it)."""
    _load().orc_set_threads(int(n))


def dft(x, sign: int = -1) -> np.ndarray:
    """Direct O(n^2) DFT, X[k] = sum_j x[j] exp(sign 2 pi i j k / n)."""
    x = _c128(x)
    out = np.empty_like(x)
    _load().orc_dft(x.ctypes.data, out.ctypes.data, x.size, sign)
    return out


def fft(x, sign: int = -1) -> np.ndarray:
    """Textbook radix-2 FFT (unscaled)."""
    a = _c128(x).copy()
    if _load().orc_fft(a.ctypes.data, a.size, sign) != 0:
        raise ValueError("orc_fft: length must be a power of two")
    return a


def fft2(x, sign: int = -1) -> np.ndarray:
    a = _c128(x).copy()
    if _load().orc_fft2(a.ctypes.data, a.shape[0], a.shape[1], sign) != 0:
        raise ValueError("orc_fft2: sides must be powers of two")
    return a


def asm_transfer(px: int, py: int, dx: float, dy: float, lam: float, z: float) -> np.ndarray:
    """H_A of Eq. ang2 on the [py][px] frequency grid (0 where evanescent)."""
    H = np.empty((py, px), dtype=np.complex128)
    _load().orc_asm_transfer(H.ctypes.data, px, py, dx, dy, lam, z)
    return H


def propagate(u1, dx: float, dy: float, lam: float, z: float, kind: int = ANGULAR,
              flags: int = 0) -> np.ndarray:
    """Pad, FFT, multiply by H, inverse FFT, crop (one [ny][nx] field, complex128)."""
    u1 = _c128(u1)
    ny, nx = u1.shape
    shape = (2 * ny, 2 * nx) if (flags & FULL_OUTPUT and not flags & NO_PAD) else (ny, nx)
    u2 = np.empty(shape, dtype=np.complex128)
    st = _load().orc_propagate(u1.ctypes.data, u2.ctypes.data, nx, ny, dx, dy, lam, z, kind, flags)
    if st != 0:
        raise ValueError(f"orc_propagate failed with status {st}")
    return u2


def propagate_direct(u1, dx: float, dy: float, lam: float, z: float, kind: int = ANGULAR,
                     flags: int = 0) -> np.ndarray:
    """Brute-force linear-convolution sum (tiny grids, N <= 64)."""
    u1 = _c128(u1)
    ny, nx = u1.shape
    u2 = np.empty_like(u1)
    st = _load().orc_propagate_direct(u1.ctypes.data, u2.ctypes.data, nx, ny, dx, dy, lam, z, kind, flags)
    if st != 0:
        raise ValueError(f"orc_propagate_direct failed with status {st}")
    return u2


def propagate_stack(u1, dx: float, dy: float, lam: float, zs, kind: int = ANGULAR,
                    flags: int = 0) -> np.ndarray:
    """3-D field by stacking 2-D diffractions along z (Section "Three-dimensional diffraction
    calculations"): one independent propagation of the same source per plane."""
    return np.stack([propagate(u1, dx, dy, lam, float(z), kind, flags) for z in zs])


def hologram_loss_grad(phi, canvas: tuple, offset: tuple, target, dx: float, lam: float,
                       z: float):
    """Loss and gradient of the phase-only hologram objective.

    x = exp(i phi) placed at ``offset`` (row, col) inside a zero canvas, U = A x with A the
    padded angular-spectrum propagation, loss L = mean over the phi-sized window of
    (|U|^2 - T)^2.  With r = (2/M)(|U|^2 - T) on the window (0 elsewhere), the chain rule
    gives dL/dphi = 2 Re(-i conj(x) [A^H (r U)]) restricted to the window.
    """
    phi = np.asarray(phi, dtype=np.float64)
    h, w = phi.shape
    oy, ox = offset
    cy, cx = canvas
    x = np.zeros((cy, cx), dtype=np.complex128)
    x[oy:oy + h, ox:ox + w] = np.exp(1j * phi)
    U = propagate(x, dx, dx, lam, z, ANGULAR)
    Uw = U[oy:oy + h, ox:ox + w]
    I_ = np.abs(Uw) ** 2
    M = I_.size
    diff = I_ - np.asarray(target, dtype=np.float64)
    loss = float(np.sum(diff * diff) / M)
    g = np.zeros((cy, cx), dtype=np.complex128)
    g[oy:oy + h, ox:ox + w] = (2.0 / M) * diff * Uw
    back = propagate(g, dx, dx, lam, z, ANGULAR, ADJOINT)
    grad = 2.0 * np.real(-1j * np.conj(x[oy:oy + h, ox:ox + w]) * back[oy:oy + h, ox:ox + w])
    return loss, grad


def phase_only(u) -> np.ndarray:
    """The phase constraint of the GS iteration: keep the phase, set the amplitude to one
    (a pixel of zero amplitude has phase 0, i.e. becomes 1).  Section "GS algorithm"."""
    u = _c128(u)
    m = np.abs(u)
    out = np.ones_like(u)
    nz = m > 0
    out[nz] = u[nz] / m[nz]
    return out


def gs_run(amplitude, field0, dx: float, dy: float, lam: float, z: float, iterations: int,
           flags: int = 0):
    """Gerchberg-Saxton kinoform iteration with the angular spectrum method, in the order of
    Section "GS algorithm": propagate the object field (amplitude with its initial phase) by +z
    and keep the phase (kinoform); then, per iteration, propagate the kinoform by -z, replace
    the amplitude by the object amplitude (amplitude constraint), propagate by +z and keep the
    phase (phase constraint).  Returns (kinoform, reconstructed intensity |ASM(-z) kinoform|^2).
    ``flags`` is passed to every propagation (NO_PAD gives the circular, unitary variant)."""
    a1 = np.asarray(amplitude, dtype=np.float64)
    u = phase_only(propagate(field0, dx, dy, lam, z, ANGULAR, flags))
    for _ in range(int(iterations)):
        back = propagate(u, dx, dy, lam, -z, ANGULAR, flags)
        obj = a1 * phase_only(back)
        u = phase_only(propagate(obj, dx, dy, lam, z, ANGULAR, flags))
    rec = propagate(u, dx, dy, lam, -z, ANGULAR, flags)
    return u, np.abs(rec) ** 2


def gs_amplitude_errors(amplitude, field0, dx: float, dy: float, lam: float, z: float,
                        iterations: int, flags: int = 0) -> np.ndarray:
    """|| |ASM(-z) kinoform_k| - amplitude || after k = 0 .. iterations GS iterations (the
    object-plane error of the error-reduction view of the iteration)."""
    a1 = np.asarray(amplitude, dtype=np.float64)
    errs = []
    u = phase_only(propagate(field0, dx, dy, lam, z, ANGULAR, flags))
    for k in range(int(iterations) + 1):
        back = propagate(u, dx, dy, lam, -z, ANGULAR, flags)
        errs.append(float(np.linalg.norm(np.abs(back) - a1)))
        if k == iterations:
            break
        u = phase_only(propagate(a1 * phase_only(back), dx, dy, lam, z, ANGULAR, flags))
    return np.array(errs)


def signed_freqs(p: int, pitch: float) -> np.ndarray:
    """Frequencies of the bins of a length-p axis: kt / (p pitch), kt = k (k < p/2) else k - p."""
    k = np.arange(p)
    return np.where(k < p // 2, k, k - p) / (p * pitch)


def rect(x) -> np.ndarray:
    """Rect(x) = 1 for |x| <= 1/2, else 0 (the window edge counts as inside)."""
    return (np.abs(np.asarray(x, dtype=np.float64)) <= 0.5).astype(np.float64)


def shifted_asm_transfer(px: int, py: int, dx: float, dy: float, lam: float, z: float,
                         ox: float = 0.0, oy: float = 0.0, cx: float = 0.0, wx: float = 0.0,
                         cy: float = 0.0, wy: float = 0.0) -> np.ndarray:
    """Shifted angular spectrum transfer function (Section "Shifted angular spectrum method",
    Eqs. shift_ang1 and shift_ang2 with the imaginary unit restored): H_A of Eq. ang2 times
    exp(i 2 pi (ox fx + oy fy)) times Rect((fx - cx) / wx) Rect((fy - cy) / wy); a width <= 0
    means no window on that axis.  Frequencies on the padded grid (signed_freqs)."""
    H = asm_transfer(px, py, dx, dy, lam, z)
    fx = signed_freqs(px, dx)[None, :]
    fy = signed_freqs(py, dy)[:, None]
    H = H * np.exp(2j * np.pi * (ox * fx + oy * fy))
    if wx > 0:
        H = H * rect((fx - cx) / wx)
    if wy > 0:
        H = H * rect((fy - cy) / wy)
    return H


def propagate_shifted(u1, dx: float, dy: float, lam: float, z: float, ox: float = 0.0, oy: float = 0.0,
                      cx: float = 0.0, wx: float = 0.0, cy: float = 0.0, wy: float = 0.0,
                      flags: int = 0) -> np.ndarray:
    """Shifted ASM propagation: pad to 2N (NO_PAD: circular on N), FFT2, multiply by the shifted
    and windowed transfer function, inverse FFT2, crop (FULL_OUTPUT: keep the padded grid).
    ADJOINT multiplies by conj(H)."""
    u1 = _c128(u1)
    ny, nx = u1.shape
    if flags & NO_PAD:
        py, px = ny, nx
        g = u1.copy()
    else:
        py, px = 2 * ny, 2 * nx
        g = np.zeros((py, px), dtype=np.complex128)
        g[:ny, :nx] = u1
    H = shifted_asm_transfer(px, py, dx, dy, lam, z, ox, oy, cx, wx, cy, wy)
    if flags & ADJOINT:
        H = np.conj(H)
    G = fft2(g, -1) * H
    out = fft2(G, +1) / (px * py)
    if flags & FULL_OUTPUT or flags & NO_PAD:
        return out
    return out[:ny, :nx]


def band_limit(nx: int, ny: int, dx: float, dy: float, lam: float, z: float):
    """On-axis band limit of the angular spectrum method (Matsushima and Shimobaba, "Band-limited
    angular spectrum method", Opt. Express 17, 19662 (2009)): on the padded grid with frequency
    pitch df = 1/(P pitch) the transfer function's phase is sampled without aliasing for
    |f| <= 1 / (lam sqrt((2 df z)^2 + 1)).  Returns (wx, wy): the full widths of the Rect
    windows centred on zero frequency."""
    dfx = 1.0 / (2 * nx * dx)
    dfy = 1.0 / (2 * ny * dy)
    ux = 1.0 / (lam * np.sqrt((2 * dfx * z) ** 2 + 1.0))
    uy = 1.0 / (lam * np.sqrt((2 * dfy * z) ** 2 + 1.0))
    return 2.0 * ux, 2.0 * uy


def _centred(n: int) -> np.ndarray:
    """Centred sample indices m - n/2 of an n-point axis (the array's element n/2 is the axis)."""
    return np.arange(n) - n // 2


def _coeff(dx: float, dy: float, lam: float, z: float, flags: int) -> complex:
    # exp(i 2 pi z / lam) / (i lam z), with the area element dx dy of the discretised integral
    # unless LITERAL_SCALE (the same reading as the convolution form)
    c = np.exp(2j * np.pi * np.fmod(z / lam, 1.0)) / (1j * lam * z)
    return c if flags & LITERAL_SCALE else c * dx * dy


def fresnel_fourier(u1, dx: float, dy: float, lam: float, z: float, flags: int = 0) -> np.ndarray:
    """Fresnel diffraction in Fourier form (Section "The Fresnel diffraction (Fourier form)",
    Eqs. fre_fourier2 and fre_fourier3; the y integration variable of Eq. fre_fourier1 read as
    y1): multiply by the source chirp exp(i pi (x1^2 + y1^2) / (lam z)), take the centred DFT,
    multiply by C and the destination chirp exp(i pi (x2^2 + y2^2) / (lam z)).  No padding;
    source coordinates x1 = (m - Nx/2) dx, destination x2 = (k - Nx/2) lam z / (Nx dx) (array
    element N/2 is the optical axis on both planes).  The centred DFT is computed as
    fftshift(FFT(ifftshift(.))) with the oracle's own FFT."""
    u1 = _c128(u1)
    ny, nx = u1.shape
    x1 = _centred(nx) * dx
    y1 = _centred(ny) * dy
    pre = np.exp(1j * np.pi * (x1[None, :] ** 2 + y1[:, None] ** 2) / (lam * z))
    g = np.fft.ifftshift(u1 * pre)
    G = np.fft.fftshift(fft2(g, -1))
    x2 = _centred(nx) * lam * z / (nx * dx)
    y2 = _centred(ny) * lam * z / (ny * dy)
    post = np.exp(1j * np.pi * (x2[None, :] ** 2 + y2[:, None] ** 2) / (lam * z))
    return _coeff(dx, dy, lam, z, flags) * post * G


def fresnel_fourier_direct(u1, dx: float, dy: float, lam: float, z: float, flags: int = 0) -> np.ndarray:
    """Eq. fre_fourier3 as a literal double sum over the source samples (tiny grids only)."""
    u1 = _c128(u1)
    ny, nx = u1.shape
    x1 = _centred(nx) * dx
    y1 = _centred(ny) * dy
    x2 = _centred(nx) * lam * z / (nx * dx)
    y2 = _centred(ny) * lam * z / (ny * dy)
    c = _coeff(dx, dy, lam, z, flags)
    out = np.zeros((ny, nx), dtype=np.complex128)
    for l in range(ny):
        for k in range(nx):
            s = 0j
            for n in range(ny):
                for m in range(nx):
                    s += u1[n, m] * np.exp(1j * np.pi * (x1[m] ** 2 + y1[n] ** 2) / (lam * z)) * \
                        np.exp(-2j * np.pi * (x2[k] * x1[m] + y2[l] * y1[n]) / (lam * z))
            out[l, k] = c * np.exp(1j * np.pi * (x2[k] ** 2 + y2[l] ** 2) / (lam * z)) * s
    return out


def shifted_fresnel(u1, dx0: float, dy0: float, dx1: float, dy1: float, lam: float, z: float,
                    ox0: float = 0.0, oy0: float = 0.0, ox1: float = 0.0, oy1: float = 0.0,
                    flags: int = 0) -> np.ndarray:
    """Shifted Fresnel diffraction (Section "Shifted Fresnel diffraction", Eqs. shift_fre1 to
    shift_fre3) with source pitch (dx0, dy0) centred at (ox0, oy0) and destination pitch
    (dx1, dy1) centred at (ox1, oy1): x0 = m0 dx0 + ox0, x1 = m1 dx1 + ox1, m = array index - N/2.
    Expanding x1 x0 with 2 m1 m0 = m1^2 + m0^2 - (m1 - m0)^2 turns the Fresnel sum into a
    linear convolution with h_S[d] = exp(i pi S d^2), S = dx0 dx1 / (lam z):
        u1'[m0] = u1 exp(i pi x0^2 / (lam z)) exp(-2 pi i m0 dx0 ox1 / (lam z)) exp(-i pi S m0^2)
        u2[m1]  = C exp(i pi x1^2 / (lam z)) exp(-2 pi i ox0 x1 / (lam z)) exp(-i pi S m1^2)
                  (u1' * h_S)[m1]
    (per axis, times the y factors), C = exp(i 2 pi z / lam) / (i lam z) dx0 dy0 (LITERAL_SCALE:
    without dx0 dy0).  The convolution is computed by zero padding to 2N and FFTs with the oracle's
    FFT, h_S sampled at d = i (i < N) or i - 2N on the padded axis."""
    u1 = _c128(u1)
    ny, nx = u1.shape
    lz = lam * z
    Sx, Sy = dx0 * dx1 / lz, dy0 * dy1 / lz
    mx, my = _centred(nx), _centred(ny)
    x0, y0 = mx * dx0 + ox0, my * dy0 + oy0
    x1, y1 = mx * dx1 + ox1, my * dy1 + oy1
    fx = np.exp(1j * np.pi * x0 ** 2 / lz) * np.exp(-2j * np.pi * mx * dx0 * ox1 / lz) * np.exp(-1j * np.pi * Sx * mx ** 2)
    fy = np.exp(1j * np.pi * y0 ** 2 / lz) * np.exp(-2j * np.pi * my * dy0 * oy1 / lz) * np.exp(-1j * np.pi * Sy * my ** 2)
    px, py = 2 * nx, 2 * ny
    g = np.zeros((py, px), dtype=np.complex128)
    g[:ny, :nx] = u1 * fy[:, None] * fx[None, :]
    dxs = np.where(np.arange(px) < nx, np.arange(px), np.arange(px) - px)
    dys = np.where(np.arange(py) < ny, np.arange(py), np.arange(py) - py)
    h = np.exp(1j * np.pi * Sy * dys[:, None] ** 2) * np.exp(1j * np.pi * Sx * dxs[None, :] ** 2)
    conv = fft2(fft2(g, -1) * fft2(h, -1), +1)[:ny, :nx] / (px * py)
    qx = np.exp(1j * np.pi * x1 ** 2 / lz) * np.exp(-2j * np.pi * ox0 * x1 / lz) * np.exp(-1j * np.pi * Sx * mx ** 2)
    qy = np.exp(1j * np.pi * y1 ** 2 / lz) * np.exp(-2j * np.pi * oy0 * y1 / lz) * np.exp(-1j * np.pi * Sy * my ** 2)
    c = np.exp(2j * np.pi * np.fmod(z / lam, 1.0)) / (1j * lz)
    if not flags & LITERAL_SCALE:
        c = c * dx0 * dy0
    return c * qy[:, None] * qx[None, :] * conv


def fresnel_sum(u1, dx0: float, dy0: float, dx1: float, dy1: float, lam: float, z: float,
                ox0: float = 0.0, oy0: float = 0.0, ox1: float = 0.0, oy1: float = 0.0) -> np.ndarray:
    """The Fresnel diffraction integral (Eq. fre_conv) as a literal sum over the source samples,
    evaluated at every destination sample (tiny grids only): C dx0 dy0 sum u1 exp(i pi ((x1 - x0)^2
    + (y1 - y0)^2) / (lam z)), coordinates as in shifted_fresnel."""
    u1 = _c128(u1)
    ny, nx = u1.shape
    lz = lam * z
    x0 = _centred(nx) * dx0 + ox0
    y0 = _centred(ny) * dy0 + oy0
    x1 = _centred(nx) * dx1 + ox1
    y1 = _centred(ny) * dy1 + oy1
    c = np.exp(2j * np.pi * np.fmod(z / lam, 1.0)) / (1j * lz) * dx0 * dy0
    out = np.zeros((ny, nx), dtype=np.complex128)
    for l in range(ny):
        for k in range(nx):
            ph = ((x1[k] - x0[None, :]) ** 2 + (y1[l] - y0[:, None]) ** 2) / lz
            out[l, k] = c * np.sum(u1 * np.exp(1j * np.pi * ph))
    return out
