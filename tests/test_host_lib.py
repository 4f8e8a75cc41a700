"""Host-only checks of libcwo_gb300.so: exports, argument validation, FP64 tables, and the
host emulation of the kernels against the oracle.  No GPU needed."""
import ctypes
import json
import os
import re
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
from paper_1107_5578_gb300 import cwo, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1107_5578_gb300 import build
    build.build()
    return cwo.lib()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(cwo_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_default_constants(lib):
    assert lib.cwo_version() >= 10000
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_defaults.json")))
    assert cwo.DEFAULT_WAVELENGTH == gold["wavelength_m"]
    assert cwo.DEFAULT_PITCH == gold["pitch_m"]
    hdr = open(os.path.join(ROOT, "include", "cwo.h")).read()
    assert re.search(r"#define CWO_DEFAULT_WAVELENGTH 633e-9", hdr)
    assert re.search(r"#define CWO_DEFAULT_PITCH 10e-6", hdr)


@pytest.mark.parametrize("nx,ny,batch", [(16, 16, 1), (2048, 2048, 16), (4096, 1024, 3)])
def test_device_bytes_is_host_only(lib, nx, ny, batch):
    b = cwo.device_bytes(nx, ny, batch)
    assert b >= batch * ny * 2 * nx * 8            # the 2Nx-wide intermediate per field
    assert b < batch * ny * 2 * nx * 8 + (1 << 22)


@pytest.mark.parametrize("args,status", [
    ((12, 16, 1e-5, 1e-5, 633e-9, 0.1, 0, 0), cwo.ERR_INVALID_ARG),       # not a power of two
    ((8192, 16, 1e-5, 1e-5, 633e-9, 0.1, 0, 0), cwo.ERR_INVALID_ARG),     # too large
    ((16, 16, 0.0, 1e-5, 633e-9, 0.1, 0, 0), cwo.ERR_INVALID_ARG),        # zero pitch
    ((16, 16, 1e-5, 1e-5, -1.0, 0.1, 0, 0), cwo.ERR_INVALID_ARG),         # negative wavelength
    ((16, 16, 1e-5, 1e-5, 633e-9, 0.0, 1, 0), cwo.ERR_INVALID_ARG),       # Fresnel at z = 0
    ((16, 16, 1e-5, 1e-5, 633e-9, float("nan"), 0, 0), cwo.ERR_INVALID_ARG),
    ((16, 16, 1e-5, 1e-5, 633e-9, 0.1, 2, 0), cwo.ERR_INVALID_ARG),       # Fourier form needs N >= 32
    ((32, 32, 1e-5, 1e-5, 633e-9, 0.0, 2, 0), cwo.ERR_INVALID_ARG),       # Fourier form at z = 0
    ((32, 32, 1e-5, 1e-5, 633e-9, 0.1, 2, 1), cwo.ERR_INVALID_ARG),       # phase flag on the Fourier form
    ((16, 16, 1e-5, 1e-5, 633e-9, 0.1, 3, 0), cwo.ERR_UNSUPPORTED),       # shifted Fresnel
    ((16, 16, 1e-5, 1e-5, 633e-9, 0.1, 4, 0), cwo.ERR_INVALID_ARG),       # shifted ASM: own constructor
    ((16, 16, 1e-5, 1e-5, 633e-9, 0.1, 9, 0), cwo.ERR_INVALID_ARG),       # unknown type
    ((16, 16, 1e-5, 1e-5, 633e-9, 0.1, 0, 0x80), cwo.ERR_INVALID_ARG),    # unknown flag
    ((16, 16, 1e-5, 1e-5, 633e-9, 0.1, 0, 3), cwo.ERR_INVALID_ARG),       # exclusive flags
    ((16, 16, 1e-5, 1e-5, 633e-9, 0.1, 1, 1), cwo.ERR_INVALID_ARG),       # phase flag on Fresnel
    ((16, 16, 1e-5, 1e-5, 633e-9, 0.1, 0, 4), cwo.ERR_INVALID_ARG),       # literal scale on ASM
    ((16, 16, 1e-5, 1e-5, 633e-9, 0.1, 1, 8), cwo.ERR_INVALID_ARG),       # transfer-function cache on Fresnel
    ((32, 32, 1e-5, 1e-5, 633e-9, 0.1, 2, 8), cwo.ERR_INVALID_ARG),       # ... and on the Fourier form
])
def test_plan_create_rejects_bad_arguments_before_touching_a_device(lib, args, status):
    h = ctypes.c_void_p(123)
    st = lib.cwo_plan_create(*args, ctypes.byref(h))
    assert st == status
    assert not h.value
    assert cwo.last_error()


def test_null_arguments(lib):
    assert lib.cwo_plan_create(16, 16, 1e-5, 1e-5, 633e-9, 0.1, 0, 0, None) == cwo.ERR_INVALID_ARG
    assert lib.cwo_propagate(None, None, None, None) == cwo.ERR_INVALID_ARG
    assert lib.cwo_plan_destroy(None) == cwo.OK
    assert lib.cwo_plan_reserve(None, 1) == cwo.ERR_INVALID_ARG
    assert lib.cwo_plan_device_bytes(16, 16, 1, None) == cwo.ERR_INVALID_ARG


@pytest.mark.parametrize("p", [32, 64, 128, 256, 512, 1024, 2048, 4096, 8192])
def test_axis_bins_are_a_permutation_matching_the_line_fft(lib, p):
    b = cwo.axis_bins(p)
    assert sorted(b.tolist()) == list(range(p))
    x = synth.random_field(p // 2, seed=p, ny=1)[0]
    X = cwo.line_fft(x.astype(np.complex64))
    ref = np.fft.fft(np.concatenate([x, np.zeros(p // 2)]))
    assert np.linalg.norm(X - ref[b]) / np.linalg.norm(ref) < 5e-7
    Y = synth.random_field(p, seed=p + 1, ny=1)[0]
    y = cwo.line_fft(Y[b].astype(np.complex64), inverse=True)
    want = (np.fft.ifft(Y) * p)[: p // 2]
    assert np.linalg.norm(y - want) / np.linalg.norm(want) < 5e-7


@pytest.mark.parametrize("p", [64, 512, 8192])
def test_split_axis_order_and_phase(lib, p):
    # the split order of the column pass at P = 8192 (cached transfer function): the padded
    # p-point DFT of p/2 samples equals the (p/2)-point DFTs of x_n and x_n W_p^n at the even and
    # odd frequencies, and split index h p/2 + idx holds frequency 2 bin(idx) + h
    q = p // 2
    index, w = cwo.split_axis(p)
    assert sorted(index.tolist()) == list(range(p))
    bins_p, bins_q = cwo.axis_bins(p), cwo.axis_bins(q)
    i = np.arange(p)
    assert np.array_equal(bins_p[index], 2 * bins_q[i % q] + i // q)
    n = np.arange(q)
    assert np.max(np.abs(w.astype(np.complex128) - np.exp(-2j * np.pi * n / p))) < 1e-7
    x = synth.random_field(q, seed=p + 7, ny=1)[0]
    X = np.fft.fft(np.concatenate([x, np.zeros(q)]))
    even, odd = np.fft.fft(x), np.fft.fft(x * w.astype(np.complex128))
    split = np.concatenate([even[bins_q], odd[bins_q]])   # the split order
    assert np.linalg.norm(split - X[bins_p[index]]) / np.linalg.norm(X) < 1e-6
    assert lib.cwo_debug_split_axis(32, None, None) == cwo.ERR_INVALID_ARG
    assert lib.cwo_debug_split_axis(96, None, None) == cwo.ERR_INVALID_ARG


@pytest.mark.parametrize("p", [32, 256, 4096, 8192])
def test_twiddle_tables(lib, p):
    tw = cwo.twiddles(p)          # complex64 view: per stage [kp][j] pairs (k = 2kp+1, 2kp+2)
    nst = (p.bit_length() - 1 + 3) // 4
    L, off = p, 0
    for s in range(nst - 1):
        S = L // 16                # thread t uses j = t mod S
        blk = tw[off:off + 16 * S].reshape(8, S, 2)
        j = np.arange(S)[None, :]
        for h in range(2):
            k = (2 * np.arange(8) + 1 + h)[:, None]
            want = np.exp(-2j * np.pi * (j * k % L) / L)
            assert np.max(np.abs(blk[:, :, h] - want)) < 1e-7
        off += 16 * S
        L //= 16
    assert off == len(tw)


@pytest.mark.parametrize("p,pitch,lam,z", [(64, 10e-6, 633e-9, 0.05), (512, 8e-6, 532e-9, -0.3),
                                           (8192, 3.74e-6, 532e-9, 0.011)])
def test_fresnel_axis_dft(lib, p, pitch, lam, z):
    # the sampled chirp (built by a product recurrence) and its radix-4/2 FP64 FFT against numpy
    d = np.where(np.arange(p) < p // 2, np.arange(p), np.arange(p) - p).astype(float)
    h = np.exp(1j * np.pi * (d * pitch) ** 2 / (lam * z))
    assert np.max(np.abs(cwo.fresnel_axis(p, pitch, lam, z) - np.fft.fft(h))) < 1e-9 * p



@pytest.mark.parametrize("p,pitch,lam,z", [(8192, Decimal("3.74e-6"), Decimal("532e-9"), Decimal("1.0")),
                                           (4096, Decimal("10e-6"), Decimal("633e-9"), Decimal("-0.2"))])
def test_asm_axis_phase_reduction_is_exact(lib, p, pitch, lam, z):
    # W = frac(K a/2 + K a^2/8) - frac(K) on x, recomputed with 50-digit decimals
    getcontext().prec = 50
    tab = cwo.asm_axis(p, float(pitch), float(lam), float(z), True)
    bins = cwo.axis_bins(p)
    K = z / lam
    frK = K - (K.to_integral_value(rounding="ROUND_FLOOR"))
    for i in list(range(0, p, p // 64)) + [p - 1]:
        k = int(bins[i])
        kt = k if k < p // 2 else k - p
        a = lam * lam * Decimal(kt * kt) / (Decimal(p) * pitch) ** 2
        ph = K * a / 2 + K * a * a / 8
        W = ph - ph.to_integral_value(rounding="ROUND_FLOOR") - frK
        got = Decimal(float(tab[i, 1]))
        # compare modulo one cycle; float storage of a value in (-1, 1) is good to 6e-8
        diff = (got - W) % 1
        diff = min(diff, 1 - diff)
        assert diff < Decimal("1.2e-7"), (i, kt, got, W)
        assert abs(float(tab[i, 0]) - float(a)) <= 1e-7 * float(a) + 1e-30


@pytest.mark.parametrize("nx,ny,kind,z,pitch", [
    (16, 16, 0, 0.05, 10e-6), (32, 16, 0, 1e-3, 1e-6), (16, 64, 1, 0.02, 10e-6),
    (64, 64, 1, 0.08, 8e-6), (64, 32, 0, 20e-6, 0.4e-6), (128, 128, 0, -0.1, 10e-6),
    (128, 32, 1, -0.3, 6e-6), (256, 16, 1, 0.01, 4e-6),
])
@pytest.mark.parametrize("adjoint", [0, 1])
def test_host_emulation_of_the_kernels_matches_the_oracle(lib, nx, ny, kind, z, pitch, adjoint):
    u = synth.random_field(nx, seed=nx + ny, ny=ny)
    got = cwo.emulate(u.astype(np.complex64), pitch, pitch, 633e-9, z, kind, 0, adjoint)
    want = oracle.propagate(u, pitch, pitch, 633e-9, z, kind, oracle.ADJOINT if adjoint else 0)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-5


@pytest.mark.parametrize("nx,z,pitch,lam", [(16, 0.2, 3.74e-6, 532e-9), (32, 0.05, 10e-6, 633e-9), (16, 1.0, 3.74e-6, 532e-9)])
@pytest.mark.parametrize("adjoint", [0, 1])
def test_host_emulation_of_the_split_column_pass_matches_the_oracle(lib, nx, z, pitch, lam, adjoint):
    # the column pass of a cached transfer function at Py = 8192 (Ny = 4096), emulated on the
    # host with the kernel's own butterflies, tables and split order: the zero-padded column as the
    # 4096-point transforms of x_n and x_n W_8192^n, H read in the split order
    ny = 4096
    u = synth.random_field(nx, seed=nx + 5, ny=ny)
    got = cwo.emulate(u.astype(np.complex64), pitch, pitch, lam, z, 0, cwo.FLAG_CACHE_H, adjoint)
    want = oracle.propagate(u, pitch, pitch, lam, z, 0, oracle.ADJOINT if adjoint else 0)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-5
    plain = cwo.emulate(u.astype(np.complex64), pitch, pitch, lam, z, 0, 0, adjoint)
    assert np.linalg.norm(got - plain) / np.linalg.norm(plain) < 1e-6


@pytest.mark.parametrize("n,dx,lam,z", [(256, 10e-6, 633e-9, 0.5), (512, 4e-6, 532e-9, 0.2), (64, 8e-6, 450e-9, -1.5)])
def test_band_limit_matches_the_oracle(lib, n, dx, lam, z):
    import oracle
    bl = cwo.band_limit(n, n // 2, dx, 1.5 * dx, lam, z)
    wx, wy = oracle.band_limit(n, n // 2, dx, 1.5 * dx, lam, z)
    assert abs(bl.wx - wx) <= 1e-12 * wx and abs(bl.wy - wy) <= 1e-12 * wy
    assert bl.ox == bl.oy == bl.cx == bl.cy == 0.0


def test_shifted_plan_argument_checks_need_no_device(lib):
    empty = cwo.Shift(0.0, 0.0, 1e9, 1.0, 0.0, 0.0)          # window far outside the grid
    with pytest.raises(cwo.CwoError) as e:
        cwo.Plan(64, 64, 8e-6, 8e-6, 532e-9, 0.01, shift=empty)
    assert e.value.status == cwo.ERR_INVALID_ARG
    bad = cwo.Shift(float("nan"), 0.0, 0.0, 0.0, 0.0, 0.0)
    with pytest.raises(cwo.CwoError):
        cwo.Plan(64, 64, 8e-6, 8e-6, 532e-9, 0.01, shift=bad)
    with pytest.raises(cwo.CwoError) as e:
        cwo.Plan(64, 64, 8e-6, 8e-6, 532e-9, 0.01, flags=cwo.FLAG_PHASE_FP32, shift=cwo.Shift())
    assert e.value.status == cwo.ERR_UNSUPPORTED
    with pytest.raises(cwo.CwoError):
        cwo.Plan(64, 64, 8e-6, 8e-6, 532e-9, 0.01, kind=cwo.SHIFTED_ANGULAR)   # needs the shifted constructor


@pytest.mark.parametrize("px,py,dx,lam,z,mode,tol", [
    (4096, 512, 10e-6, 633e-9, 0.05, 0, 1e-6),      # 2048^2 field geometry
    (1024, 1024, 10e-6, 633e-9, -0.1, 0, 1e-6),
    (2048, 256, 3.74e-6, 532e-9, 1.0, 0, 1e-6),     # cross term up to ~12 cycles: float-float
    (512, 512, 0.5e-6, 633e-9, 20e-6, 1, 4e-6),     # s up to 0.8: closed-form tail
    (256, 256, 0.4e-6, 633e-9, 0.01, 2, 1e-7),      # K s^3 large: per-element FP64, evanescent corners
])
def test_asm_transfer_function_phase_against_fp64(lib, px, py, dx, lam, z, mode, tol):
    # H_A = exp(2 pi i (z / lambda) sqrt(1 - lambda^2 (fx^2 + fy^2))), zero where the root is
    # imaginary (Eq. ang2), evaluated directly in FP64 on the padded frequency grid
    got_mode, h = cwo.asm_h(px, py, dx, dx, lam, z)
    assert got_mode == mode
    kx, ky = cwo.axis_bins(px).astype(np.int64), cwo.axis_bins(py).astype(np.int64)
    kx = np.where(kx < px // 2, kx, kx - px)
    ky = np.where(ky < py // 2, ky, ky - py)
    s = lam ** 2 * ((kx[None, :] / (px * dx)) ** 2 + (ky[:, None] / (py * dx)) ** 2)
    prop = s < 1.0 - 1e-6
    psi = (z / lam) * np.sqrt(np.where(prop, 1.0 - s, 0.0))
    ref = np.exp(2j * np.pi * (psi - np.round(psi)))
    err = np.angle(h[prop] * np.conj(ref[prop])) / (2 * np.pi)
    assert np.max(np.abs(err)) < tol, np.max(np.abs(err))
    assert np.max(np.abs(np.abs(h[prop]) - 1.0)) < 1e-6
    assert np.all(h[s > 1.0 + 1e-6] == 0)


@pytest.mark.parametrize("nx,ny,dx0,dy0,lam,z,prm", [
    (64, 64, 8e-6, 8e-6, 532e-9, 0.05, (4e-6, 4e-6, 0.0, 0.0, 100e-6, -60e-6)),
    (128, 64, 6e-6, 9e-6, 633e-9, 0.2, (12e-6, 5e-6, 30e-6, -20e-6, -400e-6, 250e-6)),
    (64, 32, 10e-6, 10e-6, 450e-9, -0.1, (10e-6, 10e-6, 0.0, 0.0, 1e-3, 0.0)),
])
def test_host_emulation_of_shifted_fresnel_matches_the_oracle(lib, nx, ny, dx0, dy0, lam, z, prm):
    # the plan's tables and its two separable passes with per-axis source and destination factors,
    # run on the host, against the oracle's shifted Fresnel; the adjoint by the dot-product test
    u = synth.random_field(nx, seed=75, ny=ny).astype(np.complex64)
    sf = cwo.ShiftedFresnel(*prm)
    got = cwo.emulate_shifted_fresnel(u, dx0, dy0, lam, z, sf)
    want = oracle.shifted_fresnel(u, dx0, dy0, prm[0], prm[1], lam, z, *prm[2:])
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-5
    v = synth.random_field(nx, seed=76, ny=ny).astype(np.complex64)
    ahv = cwo.emulate_shifted_fresnel(v, dx0, dy0, lam, z, sf, adjoint=True)
    lhs = np.vdot(v.astype(np.complex128), got.astype(np.complex128))
    rhs = np.vdot(ahv.astype(np.complex128), u.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(got) * np.linalg.norm(v)


@pytest.mark.parametrize("n,dx,lam,z,shift", [
    (64, 8e-6, 532e-9, 0.01, (200e-6, -120e-6, 0.0, 0.0, 0.0, 0.0)),              # shift only
    (64, 8e-6, 532e-9, 0.05, (0.0, 0.0, 5e3, 2e4, -3e3, 1.5e4)),                   # windows only
    (128, 4e-6, 633e-9, -0.02, (-80e-6, 40e-6, 1e4, 6e4, 0.0, 4e4)),               # both, z < 0
])
@pytest.mark.parametrize("adjoint", [0, 1])
def test_host_emulation_of_shifted_asm_matches_the_oracle(lib, n, dx, lam, z, shift, adjoint):
    # the shifted plan's tables (shift phase folded into W, windows as a = 2) and its three
    # passes, run on the host, against the oracle's shifted ASM
    u = synth.random_field(n, seed=77, ny=n // 2).astype(np.complex64)
    sh = cwo.Shift(*shift)
    got = cwo.emulate_shifted(u, dx, dx, lam, z, sh, adjoint=bool(adjoint))
    want = oracle.propagate_shifted(u, dx, dx, lam, z, *shift, flags=oracle.ADJOINT if adjoint else 0)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-5


def test_ffma_calibration_rejects_bad_arguments_on_the_host(lib):
    for blocks, iters in ((0, 8), (4, 7), (4, 0), (1 << 21, 8)):
        assert lib.cwo_debug_ffma_rate(blocks, iters, None, None) == cwo.ERR_INVALID_ARG
