"""Pins for the FP64 oracle: each check compares it with something other than itself --
closed forms, special cases, invariants, brute force on tiny inputs, or physics that the
paper's equations are derived from.  No GPU needed."""
import numpy as np
import pytest

import oracle
from paper_1107_5578_gb300 import synth

LAM = 633e-9
PITCH = 10e-6


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# ------------------------------------------------------------------------------------- DFT/FFT

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16])
def test_dft_delta_gives_ones(n):
    x = np.zeros(n, complex)
    x[0] = 1.0
    assert np.allclose(oracle.dft(x, -1), np.ones(n), atol=1e-14)


@pytest.mark.parametrize("n,m", [(8, 1), (8, 3), (16, 5), (7, 2)])
def test_dft_tone_gives_scaled_delta(n, m):
    # forward sign -1: the tone exp(+2 pi i m j / n) lands on bin m with weight n
    j = np.arange(n)
    x = np.exp(2j * np.pi * m * j / n)
    X = oracle.dft(x, -1)
    want = np.zeros(n, complex)
    want[m] = n
    assert np.allclose(X, want, atol=1e-12)
    # inverse sign +1 sends it to bin n - m
    Xp = oracle.dft(x, +1)
    want = np.zeros(n, complex)
    want[(n - m) % n] = n
    assert np.allclose(Xp, want, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_direct_dft(n, sign):
    x = synth.random_field(n, seed=n + (sign > 0), ny=1)[0]
    assert rel(oracle.fft(x, sign), oracle.dft(x, sign)) < 1e-13


@pytest.mark.parametrize("n", [128, 1024, 4096])
def test_fft_matches_numpy(n):
    x = synth.random_field(n, seed=7, ny=1)[0]
    assert rel(oracle.fft(x, -1), np.fft.fft(x)) < 1e-13
    assert rel(oracle.fft(x, +1), np.fft.ifft(x) * n) < 1e-13


@pytest.mark.parametrize("shape", [(4, 8), (16, 16), (32, 8)])
def test_fft2_matches_numpy(shape):
    x = synth.random_field(shape[1], seed=3, ny=shape[0])
    assert rel(oracle.fft2(x, -1), np.fft.fft2(x)) < 1e-13


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12), -1)


# ------------------------------------------------------------------- brute-force direct sums

@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 8), (4, 16)])
@pytest.mark.parametrize("flags", [0, oracle.ADJOINT, oracle.LITERAL_SCALE])
def test_fresnel_fft_equals_direct_sum(nx, ny, flags):
    u = synth.random_field(nx, seed=11, ny=ny)
    args = (PITCH, 1.5 * PITCH, LAM, 0.02)
    a = oracle.propagate(u, *args, kind=oracle.FRESNEL_CONV, flags=flags)
    b = oracle.propagate_direct(u, *args, kind=oracle.FRESNEL_CONV, flags=flags)
    assert rel(a, b) < 1e-12


@pytest.mark.parametrize("nx,ny,z", [(64, 128, 0.02), (128, 32, -0.05)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_fresnel_is_a_row_then_column_convolution(nx, ny, z, adjoint):
    # the discretised Fresnel integral (Eq. fre_conv) with its separable chirp is
    # u2 = C * Hy @ u1 @ Hx^T, Hx[m2, m1] = exp(i pi ((m2 - m1) dx)^2 / (lambda z)): one linear
    # convolution along every row, then one along every column; the padded 2-D FFT method
    # computes exactly that (adjoint: conj(C) with the conjugate, symmetric chirp matrices)
    dx, dy = PITCH, 0.8 * PITCH
    u = synth.random_field(nx, seed=12, ny=ny)
    mx = np.arange(nx)
    my = np.arange(ny)
    hx = np.exp(1j * np.pi * ((mx[:, None] - mx[None, :]) * dx) ** 2 / (LAM * z))
    hy = np.exp(1j * np.pi * ((my[:, None] - my[None, :]) * dy) ** 2 / (LAM * z))
    c = dx * dy * np.exp(2j * np.pi * z / LAM) / (1j * LAM * z)
    if adjoint:
        want = np.conj(c) * np.conj(hy) @ u @ np.conj(hx).T
    else:
        want = c * hy @ u @ hx.T
    got = oracle.propagate(u, dx, dy, LAM, z, kind=oracle.FRESNEL_CONV, flags=oracle.ADJOINT if adjoint else 0)
    assert rel(got, want) < 1e-10


@pytest.mark.parametrize("nx,ny,dx,dy,z", [
    (8, 8, 1e-6, 1e-6, 1e-4),        # several cycles of phase across the band
    (16, 8, 1e-6, 2e-6, 3e-4),
    (8, 4, 0.4e-6, 0.5e-6, 2e-6),    # pitch below lambda/sqrt(2): evanescent corners
])
@pytest.mark.parametrize("flags", [0, oracle.ADJOINT])
def test_asm_fft_equals_kernel_sum(nx, ny, dx, dy, z, flags):
    u = synth.random_field(nx, seed=5, ny=ny)
    a = oracle.propagate(u, dx, dy, LAM, z, kind=oracle.ANGULAR, flags=flags)
    b = oracle.propagate_direct(u, dx, dy, LAM, z, kind=oracle.ANGULAR, flags=flags)
    assert rel(a, b) < 1e-12


# --------------------------------------------------------------------- special cases / physics

def test_asm_zero_distance_is_identity():
    u = synth.random_field(64, seed=2, ny=32)
    out = oracle.propagate(u, PITCH, PITCH, LAM, 0.0, kind=oracle.ANGULAR)
    assert rel(out, u) < 1e-14


@pytest.mark.parametrize("z", [0.05, 0.2, 1.0])
def test_asm_normal_plane_wave_phase(z):
    # a uniform field is the normally incident plane wave: it picks up exp(i k z), k = 2 pi / lambda
    n = 16
    u = np.ones((n, n), complex)
    out = oracle.propagate(u, PITCH, PITCH, LAM, z, kind=oracle.ANGULAR, flags=oracle.NO_PAD)
    want = np.exp(1j * 2 * np.pi * np.fmod(z / LAM, 1.0))
    assert np.allclose(out, want, atol=1e-9)


@pytest.mark.parametrize("a,b", [(1, 0), (3, -2), (-5, 7)])
def test_asm_oblique_plane_wave_dispersion(a, b):
    # exp(i (kx x + ky y)) is a Helmholtz solution that propagates as exp(i kz z) with
    # kx^2 + ky^2 + kz^2 = k^2; on a circular grid it is an exact eigenvector of the method.
    nx, ny, dx, dy, z = 32, 16, 2e-6, 3e-6, 4e-3
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    u = np.exp(2j * np.pi * (a * x / nx + b * y / ny))
    kx, ky = 2 * np.pi * a / (nx * dx), 2 * np.pi * b / (ny * dy)
    k = 2 * np.pi / LAM
    kz = np.sqrt(k * k - kx * kx - ky * ky)
    out = oracle.propagate(u, dx, dy, LAM, z, kind=oracle.ANGULAR, flags=oracle.NO_PAD)
    assert np.allclose(out, np.exp(1j * kz * z) * u, atol=1e-9)


def test_asm_evanescent_plane_wave_is_removed():
    nx, dx = 16, 0.25e-6             # bin 7: |f| = 7/(16*0.25um) = 1.75/um > 1/lambda = 1.58/um
    x = np.arange(nx)[None, :]
    u = np.exp(2j * np.pi * 7 * x / nx) * np.ones((nx, 1))
    out = oracle.propagate(u, dx, dx, LAM, 1e-6, kind=oracle.ANGULAR, flags=oracle.NO_PAD)
    assert np.max(np.abs(out)) < 1e-13


def test_asm_semigroup():
    # on the circular grid A(z1 + z2) = A(z2) A(z1) exactly (products of exponentials)
    u = synth.random_field(32, seed=9)
    args = (1e-6, 1e-6, LAM)
    ab = oracle.propagate(oracle.propagate(u, *args, 1e-4, flags=oracle.NO_PAD), *args, 2e-4,
                          flags=oracle.NO_PAD)
    c = oracle.propagate(u, *args, 3e-4, flags=oracle.NO_PAD)
    assert rel(ab, c) < 1e-12


def _fresnel_gaussian(r2, w0, z):
    # closed-form Fresnel propagation of exp(-r^2/w0^2) (Gaussian integral of Eq. fre_conv)
    alpha = LAM * z / (np.pi * w0 * w0)
    return np.exp(1j * 2 * np.pi * np.fmod(z / LAM, 1.0)) / (1 + 1j * alpha) * \
        np.exp(-r2 / (w0 * w0 * (1 + 1j * alpha)))


def _grid_r2(n, pitch):
    y, x = np.mgrid[0:n, 0:n].astype(float)
    return ((x - n / 2) * pitch) ** 2 + ((y - n / 2) * pitch) ** 2


def test_fresnel_gaussian_closed_form():
    n, w0, z = 256, 200e-6, 0.1
    u = synth.gaussian_beam(n, PITCH, w0)
    out = oracle.propagate(u, PITCH, PITCH, LAM, z, kind=oracle.FRESNEL_CONV)
    want = _fresnel_gaussian(_grid_r2(n, PITCH), w0, z)
    assert np.max(np.abs(out - want)) < 1e-10
    # the literal-scale reading differs by exactly the area element dx*dy
    lit = oracle.propagate(u, PITCH, PITCH, LAM, z, kind=oracle.FRESNEL_CONV,
                           flags=oracle.LITERAL_SCALE)
    assert rel(lit * PITCH * PITCH, out) < 1e-13


def test_asm_gaussian_matches_paraxial_closed_form():
    # the exact (ASM) and paraxial (Fresnel) Gaussian differ by non-paraxial terms of order
    # (z/lambda) * (lambda/(pi w0))^4 / 8 cycles ~ 1e-7 here
    n, w0, z = 256, 200e-6, 0.1
    u = synth.gaussian_beam(n, PITCH, w0)
    out = oracle.propagate(u, PITCH, PITCH, LAM, z, kind=oracle.ANGULAR)
    want = _fresnel_gaussian(_grid_r2(n, PITCH), w0, z)
    err = np.max(np.abs(out - want))
    assert 1e-10 < err < 2e-6


def _hankel_asm_gaussian(r, w0, z, panels=400, nodes=24):
    # u2(r) = 2 pi int_0^inf A(rho) H(rho) J0(2 pi rho r) rho d rho with the exact angular
    # spectrum A(rho) = pi w0^2 exp(-pi^2 w0^2 rho^2) of exp(-r^2/w0^2)
    from scipy.special import j0, roots_legendre
    rho_max = np.sqrt(800.0) / (np.pi * w0)
    xg, wg = roots_legendre(nodes)
    edges = np.linspace(0.0, rho_max, panels + 1)
    a, b = edges[:-1, None], edges[1:, None]
    rho = (0.5 * (b - a) * xg[None, :] + 0.5 * (a + b)).ravel()
    wt = (0.5 * (b - a) * wg[None, :]).ravel()
    inv = 1.0 / LAM
    # z (sqrt(1/lam^2 - rho^2) - 1/lam), written without cancellation
    dphase = -z * rho * rho / (inv + np.sqrt(inv * inv - rho * rho))
    A = np.pi * w0 * w0 * np.exp(-(np.pi * w0 * rho) ** 2)
    integrand = A * np.exp(2j * np.pi * dphase) * rho * wt
    out = 2 * np.pi * (j0(2 * np.pi * np.outer(r, rho)) @ integrand)
    return np.exp(1j * 2 * np.pi * np.fmod(z / LAM, 1.0)) * out


def test_asm_gaussian_hankel_quadrature():
    n, w0, z = 256, 200e-6, 0.1
    u = synth.gaussian_beam(n, PITCH, w0)
    out = oracle.propagate(u, PITCH, PITCH, LAM, z, kind=oracle.ANGULAR)
    cols = np.array([128, 130, 140, 150, 160, 180, 200])
    r = (cols - n / 2) * PITCH
    want = _hankel_asm_gaussian(r, w0, z)
    assert np.max(np.abs(out[n // 2, cols] - want)) < 1e-10


def test_asm_parseval_full_grid():
    # with no evanescent bins |H| = 1, so the energy on the whole padded grid is conserved
    u = synth.random_field(32, seed=4, ny=16)
    out = oracle.propagate(u, PITCH, PITCH, LAM, 0.3, kind=oracle.ANGULAR,
                           flags=oracle.FULL_OUTPUT)
    assert out.shape == (32, 64)
    e_in, e_out = np.sum(np.abs(u) ** 2), np.sum(np.abs(out) ** 2)
    assert abs(e_out - e_in) / e_in < 1e-13


def test_asm_z_then_minus_z_recovers_input():
    # full padded grid forward by z, then back by -z on that circular grid: H(z) H(-z) = 1
    u = synth.random_field(16, seed=8)
    full = oracle.propagate(u, PITCH, PITCH, LAM, 0.05, flags=oracle.FULL_OUTPUT)
    back = oracle.propagate(full, PITCH, PITCH, LAM, -0.05, flags=oracle.NO_PAD)
    padded = np.zeros((32, 32), complex)
    padded[:16, :16] = u
    assert rel(back, padded) < 1e-13


@pytest.mark.parametrize("kind", [oracle.ANGULAR, oracle.FRESNEL_CONV])
def test_adjoint_dot_product(kind):
    nx, ny = 32, 16
    x = synth.random_field(nx, seed=21, ny=ny)
    y = synth.random_field(nx, seed=22, ny=ny)
    args = (2e-6, 3e-6, LAM, 2e-3)
    Ax = oracle.propagate(x, *args, kind=kind)
    AHy = oracle.propagate(y, *args, kind=kind, flags=oracle.ADJOINT)
    lhs, rhs = np.vdot(y, Ax), np.vdot(AHy, x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13


def test_asm_adjoint_equals_back_propagation():
    u = synth.random_field(16, seed=6)
    a = oracle.propagate(u, PITCH, PITCH, LAM, 0.1, flags=oracle.ADJOINT)
    b = oracle.propagate(u, PITCH, PITCH, LAM, -0.1)
    assert rel(a, b) < 1e-13


def test_hologram_gradient_central_differences():
    g = synth.rng(31)
    h, w, canvas, off = 12, 20, (32, 32), (10, 6)
    phi = g.random((h, w)) * 2 * np.pi
    tgt = g.random((h, w))
    args = (canvas, off, tgt, 4e-6, 520e-9, 2e-3)
    _, grad = oracle.hologram_loss_grad(phi, *args)
    eps = 1e-5
    for (i, j) in [(0, 0), (5, 7), (11, 19), (3, 12)]:
        p, m = phi.copy(), phi.copy()
        p[i, j] += eps
        m[i, j] -= eps
        fd = (oracle.hologram_loss_grad(p, *args)[0] - oracle.hologram_loss_grad(m, *args)[0]) / (2 * eps)
        assert abs(fd - grad[i, j]) <= 1e-7 * max(1.0, abs(fd))


def test_rejects_bad_arguments():
    u = np.ones((8, 8), complex)
    with pytest.raises(ValueError):
        oracle.propagate(u, PITCH, PITCH, LAM, 0.0, kind=oracle.FRESNEL_CONV)
    with pytest.raises(ValueError):
        oracle.propagate(np.ones((8, 12), complex), PITCH, PITCH, LAM, 0.1)
    with pytest.raises(ValueError):
        oracle.propagate(u, -PITCH, PITCH, LAM, 0.1)


# ---------------------------------------------------------------------------------------------
# GS kinoform iteration (Section "GS algorithm")
# ---------------------------------------------------------------------------------------------
def test_gs_zero_distance_is_a_fixed_point():
    # ASM at z = 0 is the identity, so the kinoform is the phase of the initial field, the
    # amplitude and phase constraints leave it unchanged, and the reconstruction is |1|^2
    amp, f0 = synth.gs_problem(32, seed=4)
    kin, inten = oracle.gs_run(amp, f0, 8e-6, 8e-6, 532e-9, 0.0, iterations=3)
    assert np.max(np.abs(kin - np.exp(1j * np.angle(f0)))) < 1e-12
    assert np.max(np.abs(inten - 1.0)) < 1e-12


def test_gs_zero_iterations_is_one_propagation_and_the_phase():
    amp, f0 = synth.gs_problem(32, seed=5)
    kin, inten = oracle.gs_run(amp, f0, 8e-6, 8e-6, 532e-9, 0.01, iterations=0)
    u = np.fft.ifft2(np.fft.fft2(np.pad(f0, ((0, 32), (0, 32)))) *
                     oracle.asm_transfer(64, 64, 8e-6, 8e-6, 532e-9, 0.01))[:32, :32]
    assert np.max(np.abs(kin - u / np.abs(u))) < 1e-10
    r = np.fft.ifft2(np.fft.fft2(np.pad(kin, ((0, 32), (0, 32)))) *
                     oracle.asm_transfer(64, 64, 8e-6, 8e-6, 532e-9, -0.01))[:32, :32]
    assert np.max(np.abs(inten - np.abs(r) ** 2)) < 1e-10


def test_gs_kinoform_has_unit_amplitude():
    amp, f0 = synth.gs_problem(64, seed=6)
    kin, _ = oracle.gs_run(amp, f0, 8e-6, 8e-6, 532e-9, 0.02, iterations=4)
    assert np.max(np.abs(np.abs(kin) - 1.0)) < 1e-13


def test_gs_error_never_increases_on_the_unitary_grid():
    # with circular (unpadded) ASM and no evanescent band the propagation is unitary, and the
    # iteration is an alternating projection: the object-plane amplitude error is non-increasing
    amp, f0 = synth.gs_problem(64, seed=7)
    errs = oracle.gs_amplitude_errors(amp, f0, 8e-6, 8e-6, 532e-9, 0.02, iterations=12, flags=oracle.NO_PAD)
    assert np.all(np.diff(errs) <= 1e-9 * errs[0])
    assert errs[-1] < 0.95 * errs[0]


def test_gs_planted_amplitude_error_is_caught():
    # a mistake planted in the amplitude constraint (squared amplitude instead of amplitude)
    # breaks the fixed point of the z = 0 case
    amp, f0 = synth.gs_problem(32, seed=4)
    wrong_amp = amp ** 2
    _, inten = oracle.gs_run(wrong_amp, f0, 8e-6, 8e-6, 532e-9, 0.0, iterations=1)
    assert np.max(np.abs(inten - 1.0)) < 1e-12        # intensity of a kinoform: still 1 at z = 0
    errs_ok = oracle.gs_amplitude_errors(amp, f0, 8e-6, 8e-6, 532e-9, 0.0, 1)
    errs_bad = oracle.gs_amplitude_errors(wrong_amp, f0, 8e-6, 8e-6, 532e-9, 0.0, 1)
    assert np.all(errs_ok > 0) and not np.allclose(errs_ok, errs_bad)


# ---------------------------------------------------------------------------------------------
# Shifted / band-limited angular spectrum (Section "Shifted angular spectrum method")
# ---------------------------------------------------------------------------------------------
def test_shifted_asm_without_shift_or_window_is_asm():
    u = synth.random_field(32, seed=21, ny=16)
    got = oracle.propagate_shifted(u, 6e-6, 8e-6, 532e-9, 0.01)
    want = oracle.propagate(u, 6e-6, 8e-6, 532e-9, 0.01)
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("mx,my", [(3, 0), (-5, 2), (7, -4)])
def test_shifted_asm_is_a_translation_on_the_circular_grid(mx, my):
    # exp(i 2 pi ox fx) with ox = mx dx on the unpadded N-grid is exactly a circular shift of the
    # ASM result by -mx pixels: u_SA(x) = u_A(x + ox)
    n, dx = 32, 8e-6
    u = synth.random_field(n, seed=22)
    shifted = oracle.propagate_shifted(u, dx, dx, 633e-9, 0.005, ox=mx * dx, oy=my * dx, flags=oracle.NO_PAD)
    plain = oracle.propagate_shifted(u, dx, dx, 633e-9, 0.005, flags=oracle.NO_PAD)
    assert np.max(np.abs(shifted - np.roll(plain, (-my, -mx), axis=(0, 1)))) < 1e-12


def test_window_removes_the_spectrum_outside():
    n, dx = 32, 8e-6
    u = synth.random_field(n, seed=23)
    wx, wy = 1.0 / (4 * dx), 1.0 / (3 * dx)
    cx, cy = 1.0 / (16 * dx), -1.0 / (20 * dx)
    full = oracle.propagate_shifted(u, dx, dx, 633e-9, 0.02, cx=cx, wx=wx, cy=cy, wy=wy, flags=oracle.FULL_OUTPUT)
    spec = np.fft.fft2(full)
    fx = np.fft.fftfreq(2 * n, dx)[None, :]
    fy = np.fft.fftfreq(2 * n, dx)[:, None]
    outside = (np.abs(fx - cx) > wx / 2) | (np.abs(fy - cy) > wy / 2)
    assert outside.sum() > 0
    assert np.max(np.abs(spec[outside])) < 1e-9 * np.max(np.abs(spec))


@pytest.mark.parametrize("n,dx,lam,z", [(256, 10e-6, 633e-9, 0.5), (512, 4e-6, 532e-9, 0.2), (128, 8e-6, 450e-9, 2.0)])
def test_band_limit_is_the_nyquist_rate_of_the_transfer_phase(n, dx, lam, z):
    # at f = u_limit the local "frequency" of the transfer-function phase in the frequency domain,
    # |d(z sqrt(1/lam^2 - f^2)) / df| = z f / sqrt(1/lam^2 - f^2), equals the Nyquist limit
    # 1 / (2 df) of the padded grid's frequency sampling df = 1 / (2 n dx)
    wx, _ = oracle.band_limit(n, n, dx, dx, lam, z)
    u = wx / 2
    df = 1.0 / (2 * n * dx)
    h = 1e-6 * u
    psi = lambda f: z * np.sqrt(1.0 / lam ** 2 - f ** 2)
    slope = abs(psi(u + h) - psi(u - h)) / (2 * h)
    assert abs(slope * 2 * df - 1.0) < 1e-6


# ---------------------------------------------------------------------------------------------
# Fresnel diffraction, Fourier form (Eqs. fre_fourier2, fre_fourier3)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny,z", [(8, 8, 0.02), (16, 8, -0.05), (8, 4, 0.3)])
def test_fresnel_fourier_equals_direct_sum(nx, ny, z):
    u = synth.random_field(nx, seed=41, ny=ny)
    got = oracle.fresnel_fourier(u, 9e-6, 7e-6, 532e-9, z)
    want = oracle.fresnel_fourier_direct(u, 9e-6, 7e-6, 532e-9, z)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_fresnel_fourier_gaussian_closed_form():
    # the same closed form as the convolution form, sampled on the destination grid
    # x2 = (k - N/2) lam z / (N dx)
    n, w0, z = 256, 200e-6, 1.0
    u = synth.gaussian_beam(n, PITCH, w0)
    out = oracle.fresnel_fourier(u, PITCH, PITCH, LAM, z)
    d2 = LAM * z / (n * PITCH)
    want = _fresnel_gaussian(_grid_r2(n, d2), w0, z)
    assert np.max(np.abs(out - want)) < 1e-10
    lit = oracle.fresnel_fourier(u, PITCH, PITCH, LAM, z, flags=oracle.LITERAL_SCALE)
    assert rel(lit * PITCH * PITCH, out) < 1e-13


def test_fresnel_fourier_conserves_energy():
    # with the area element the discrete transform conserves sum |u|^2 dx dy exactly (DFT Parseval)
    nx, ny, dx, dy, z = 64, 32, 6e-6, 9e-6, 0.07
    u = synth.random_field(nx, seed=42, ny=ny)
    out = oracle.fresnel_fourier(u, dx, dy, LAM, z)
    dx2, dy2 = LAM * z / (nx * dx), LAM * z / (ny * dy)
    e1 = np.sum(np.abs(u) ** 2) * dx * dy
    e2 = np.sum(np.abs(out) ** 2) * dx2 * dy2
    assert abs(e2 - e1) < 1e-12 * e1


# ---------------------------------------------------------------------------------------------
# Shifted Fresnel diffraction (Eqs. shift_fre1 to shift_fre3)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny,p1,offs,z", [
    (8, 8, (9e-6, 7e-6), (0, 0, 0, 0), 0.02),
    (16, 8, (4e-6, 12e-6), (30e-6, -20e-6, 150e-6, 40e-6), 0.05),
    (8, 16, (20e-6, 5e-6), (-10e-6, 5e-6, -300e-6, 90e-6), -0.1)])
def test_shifted_fresnel_equals_the_fresnel_sum(nx, ny, p1, offs, z):
    # the Bluestein rewriting plus padded FFT convolution reproduces the literal Fresnel sum at
    # arbitrary destination pitches and off-axis positions
    u = synth.random_field(nx, seed=43, ny=ny)
    got = oracle.shifted_fresnel(u, 8e-6, 6e-6, p1[0], p1[1], 532e-9, z, *offs)
    want = oracle.fresnel_sum(u, 8e-6, 6e-6, p1[0], p1[1], 532e-9, z, *offs)
    assert np.max(np.abs(got - want)) < 1e-11 * np.max(np.abs(want))


def test_shifted_fresnel_reduces_to_the_convolution_form():
    # equal pitches and no offsets: the convolution form (source placed top-left, which only
    # relabels the shared origin)
    u = synth.random_field(32, seed=44, ny=16)
    got = oracle.shifted_fresnel(u, 8e-6, 6e-6, 8e-6, 6e-6, 532e-9, 0.03)
    want = oracle.propagate(u, 8e-6, 6e-6, 532e-9, 0.03, oracle.FRESNEL_CONV)
    assert np.max(np.abs(got - want)) < 1e-11 * np.max(np.abs(want))


def test_shifted_fresnel_gaussian_off_axis():
    # a centred Gaussian observed on a finer, shifted destination grid: the closed form at x1
    n, w0, z = 256, 200e-6, 0.1
    u = synth.gaussian_beam(n, PITCH, w0)
    p1, ox1, oy1 = 3e-6, 120e-6, -80e-6
    out = oracle.shifted_fresnel(u, PITCH, PITCH, p1, p1, LAM, z, 0.0, 0.0, ox1, oy1)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r2 = ((x - n / 2) * p1 + ox1) ** 2 + ((y - n / 2) * p1 + oy1) ** 2
    assert np.max(np.abs(out - _fresnel_gaussian(r2, w0, z))) < 1e-10


def test_oracle_results_do_not_depend_on_the_thread_count():
    """Timing runs the oracle on one thread and on all of them; the arithmetic is the same."""
    u = synth.random_field(64, seed=31)
    cores = oracle.max_threads()
    try:
        oracle.set_threads(1)
        one = oracle.propagate(u, 10e-6, 10e-6, 633e-9, 0.05, oracle.ANGULAR)
        oracle.set_threads(max(2, cores))
        many = oracle.propagate(u, 10e-6, 10e-6, 633e-9, 0.05, oracle.ANGULAR)
    finally:
        oracle.set_threads(cores)
    assert np.array_equal(one, many)
