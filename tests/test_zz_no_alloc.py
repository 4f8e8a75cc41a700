"""The allocation-free angular-spectrum entry point against the regular one.

cwo_propagate_asm_noalloc exists for callers that cannot allocate device memory when they
propagate (a host that owns the device's allocator, a real-time loop that must avoid the device
synchronisation an allocation can cause).  It keeps its intermediate and tables in fixed device
arrays of the library.  This file is collected last so that a run stopping at the first failure
has already run every other test."""
import ctypes

import numpy as np
import pytest

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


def _rel(a, b):
    import torch
    torch.cuda.synchronize()
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row(lib):
    import torch
    cases = [((512, 512), 10e-6, 10e-6, 633e-9, 0.05, 1), ((256, 1024), 8e-6, 6e-6, 532e-9, -0.03, 2)]
    outs = []
    for (ny, nx), dx, dy, lam, z, seed in cases:     # two calls back to back, different shapes
        x = torch.from_numpy(synth.random_field(nx, seed=seed, ny=ny).astype(np.complex64)).cuda()
        outs.append((x, _noalloc(lib, x, dx, dy, lam, z), (dx, dy, lam, z)))
    for x, y, args in outs:
        assert _rel(y, _regular(lib, x, *args)) <= TOL


def test_noalloc_rejects_fields_above_its_fixed_scratch(lib):
    import torch
    x = torch.zeros(16, 2048, dtype=torch.complex64, device="cuda")
    st = lib.lib().cwo_propagate_asm_noalloc(2048, 16, 10e-6, 10e-6, 633e-9, 0.05, x.data_ptr(),
                                             x.data_ptr(), None)
    assert st == lib.ERR_INVALID_ARG
    assert "1024" in lib.last_error()
