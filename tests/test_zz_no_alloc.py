"""The allocation-free angular-spectrum entry point against the FP64 oracle and the regular one.

cwo_propagate_asm_noalloc exists for callers that cannot allocate device memory when they
propagate (a host that owns the device's allocator, a real-time loop that must avoid the device
synchronisation an allocation can cause).  It keeps its intermediate and tables in fixed device
arrays of the library and builds the tables on the device, so it is compared with the oracle
directly as well as with the regular entry point, in every transfer-function evaluation mode
(series tail, closed-form tail, per-element FP64), at the smallest and largest sizes it takes,
and with an input off a 16-byte boundary.  This file is collected last so that a run stopping at
the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1107_5578_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 2e-5


@pytest.fixture(scope="module")
def lib(gpu):
    import paper_1107_5578_gb300.cwo as cwo
    L = cwo.lib()
    f = L.cwo_propagate_asm_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                  ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return cwo


def _noalloc(cwo, x, dx, dy, lam, z):
    import torch
    ny, nx = x.shape
    y = torch.empty_like(x)
    st = cwo.lib().cwo_propagate_asm_noalloc(nx, ny, dx, dy, lam, z, x.data_ptr(), y.data_ptr(),
                                             torch.cuda.current_stream().cuda_stream)
    assert st == cwo.OK, cwo.last_error()
    return y


def _regular(cwo, x, dx, dy, lam, z):
    ny, nx = x.shape
    plan = cwo.Plan(nx, ny, dx, dy, lam, z, cwo.ANGULAR)
    y = plan.propagate(x)
    plan.close()
    return y


def _host(a):
    import torch
    torch.cuda.synchronize()
    return a.cpu().numpy().astype(np.complex128)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _field(nx, ny, seed):
    import torch
    u = synth.random_field(nx, seed=seed, ny=ny)
    return u, torch.from_numpy(u.astype(np.complex64)).cuda()


# (ny, nx), dx, dy, wavelength, z, seed.  At 2 um pitch and 532 nm the tail term of the reduced
# phase grows with z: z = 0.5 m selects the closed-form tail, z = 1 m the per-element FP64 phase.
CASES = [
    ((512, 512), 10e-6, 10e-6, 633e-9, 0.05, 1),       # series tail
    ((256, 1024), 8e-6, 6e-6, 532e-9, -0.03, 2),       # rectangular, negative z
    ((128, 128), 2e-6, 2e-6, 532e-9, 0.5, 3),          # closed-form tail
    ((128, 128), 2e-6, 2e-6, 532e-9, 1.0, 4),          # per-element FP64 phase
    ((16, 16), 10e-6, 10e-6, 633e-9, 0.01, 5),         # smallest field
    ((1024, 1024), 10e-6, 10e-6, 633e-9, 0.05, 6),     # the whole fixed scratch
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0][0]}x{c[0][1]}_z{c[4]}" for c in CASES])
def test_noalloc_against_oracle(lib, case):
    (ny, nx), dx, dy, lam, z, seed = case
    u, x = _field(nx, ny, seed)
    want = oracle.propagate(u.astype(np.complex64), dx, dy, lam, z, oracle.ANGULAR)
    assert _rel(_host(_noalloc(lib, x, dx, dy, lam, z)), want) <= TOL


def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row(lib):
    outs = []
    for (ny, nx), dx, dy, lam, z, seed in CASES[:4]:     # calls back to back, different shapes and modes
        _, x = _field(nx, ny, seed)
        outs.append((x, _noalloc(lib, x, dx, dy, lam, z), (dx, dy, lam, z)))
    for x, y, args in outs:
        assert _rel(_host(y), _host(_regular(lib, x, *args))) <= TOL


def test_noalloc_input_off_a_16_byte_boundary(lib):
    import torch
    n = 256
    u = synth.random_field(n, seed=7)
    buf = torch.empty(n * n + 1, dtype=torch.complex64, device="cuda")
    x = buf[1:].view(n, n)                       # 8-byte aligned, not 16
    x.copy_(torch.from_numpy(u.astype(np.complex64)))
    assert x.data_ptr() % 16 == 8
    want = oracle.propagate(u.astype(np.complex64), 10e-6, 10e-6, 633e-9, 0.05, oracle.ANGULAR)
    assert _rel(_host(_noalloc(lib, x, 10e-6, 10e-6, 633e-9, 0.05)), want) <= TOL


def test_noalloc_rejects_fields_above_its_fixed_scratch(lib):
    import torch
    x = torch.zeros(16, 2048, dtype=torch.complex64, device="cuda")
    st = lib.lib().cwo_propagate_asm_noalloc(2048, 16, 10e-6, 10e-6, 633e-9, 0.05, x.data_ptr(),
                                             x.data_ptr(), None)
    assert st == lib.ERR_INVALID_ARG
    assert "1024" in lib.last_error()


def test_noalloc_rejects_short_and_host_buffers(lib):
    """A buffer whose allocation ends before nx * ny complex64 values, or host memory, is refused
    on the host before anything is launched.  The short buffer is a driver allocation of its own
    (the caching allocator could place a tensor inside a larger segment)."""
    import torch
    try:
        cu = ctypes.CDLL("libcuda.so.1")
    except OSError:
        pytest.skip("driver library not loadable")
    n = 1024
    good = torch.zeros(n, n, dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    ptr = ctypes.c_uint64(0)
    short_bytes = n * n * 8 - (2 << 20)          # 2 MiB short of the field
    assert cu.cuMemAlloc_v2(ctypes.byref(ptr), ctypes.c_size_t(short_bytes)) == 0
    try:
        f = lib.lib().cwo_propagate_asm_noalloc
        st = f(n, n, 10e-6, 10e-6, 633e-9, 0.05, ptr.value, good.data_ptr(), None)
        assert st == lib.ERR_INVALID_ARG and "input" in lib.last_error()
        st = f(n, n, 10e-6, 10e-6, 633e-9, 0.05, good.data_ptr(), ptr.value, None)
        assert st == lib.ERR_INVALID_ARG and "output" in lib.last_error()
    finally:
        cu.cuMemFree_v2(ptr)
    host = np.zeros((64, 64), dtype=np.complex64)
    st = lib.lib().cwo_propagate_asm_noalloc(64, 64, 10e-6, 10e-6, 633e-9, 0.05, host.ctypes.data,
                                             good.data_ptr(), None)
    assert st == lib.ERR_INVALID_ARG
    # the entry point still works after the refusals
    _, x = _field(64, 64, 8)
    y = _noalloc(lib, x, 10e-6, 10e-6, 633e-9, 0.05)
    assert _rel(_host(y), _host(_regular(lib, x, 10e-6, 10e-6, 633e-9, 0.05))) <= TOL
