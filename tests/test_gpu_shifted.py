"""Shifted and band-limited angular spectrum (Section "Shifted angular spectrum method") on the
GPU against the FP64 oracle, at the 2e-5 relative-L2 bar."""
import numpy as np
import pytest

import oracle
from paper_1107_5578_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 2e-5


@pytest.fixture(scope="module")
def cwo(gpu):
    import paper_1107_5578_gb300.cwo as m
    m.lib()
    return m


def _run(cwo, u, dx, dy, lam, z, sh, flags=0, adjoint=False):
    import torch
    ny, nx = u.shape
    plan = cwo.Plan(nx, ny, dx, dy, lam, z, flags=flags, shift=sh)
    x = torch.from_numpy(u.astype(np.complex64)).cuda()
    y = plan.adjoint(x) if adjoint else plan.propagate(x)
    plan.check()
    return y.cpu().numpy().astype(np.complex128)


def _want(u, dx, dy, lam, z, sh, adjoint=False):
    return oracle.propagate_shifted(u.astype(np.complex64), dx, dy, lam, z, sh.ox, sh.oy, sh.cx, sh.wx, sh.cy, sh.wy,
                                    oracle.ADJOINT if adjoint else 0)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [  # (nx, ny, dx, dy, lam, z, shift)
    (128, 64, 8e-6, 6e-6, 532e-9, 0.02, (37.3e-6, -21e-6, 0.0, 0.0, 0.0, 0.0)),
    (64, 64, 10e-6, 10e-6, 633e-9, 0.05, (0.0, 0.0, 1.5e3, 2.0e4, -2.0e3, 3.0e4)),
    (256, 128, 4e-6, 5e-6, 450e-9, 0.01, (120e-6, 80e-6, 2.0e4, 6.0e4, -1.0e4, 5.0e4)),
    (512, 512, 8e-6, 8e-6, 532e-9, -0.03, (-50e-6, 0.0, 0.0, 8.0e4, 0.0, 0.0)),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("adjoint", [False, True])
def test_shifted_against_oracle(cwo, case, adjoint):
    nx, ny, dx, dy, lam, z, s = case
    sh = cwo.Shift(*s)
    u = synth.random_field(nx, seed=31, ny=ny)
    got = _run(cwo, u, dx, dy, lam, z, sh, adjoint=adjoint)
    assert _rel(got, _want(u, dx, dy, lam, z, sh, adjoint)) <= TOL


def test_shifted_fp64_arm(cwo):
    nx, ny, dx, dy, lam, z, s = CASES[2]
    sh = cwo.Shift(*s)
    u = synth.random_field(nx, seed=32, ny=ny)
    got = _run(cwo, u, dx, dy, lam, z, sh, flags=cwo.FLAG_PHASE_FP64)
    assert _rel(got, _want(u, dx, dy, lam, z, sh)) <= TOL


@pytest.mark.parametrize("n,dx,lam,z", [(256, 8e-6, 532e-9, 0.8), (1024, 10e-6, 633e-9, 2.0)])
def test_band_limited_long_distance(cwo, n, dx, lam, z):
    sh = cwo.band_limit(n, n, dx, dx, lam, z)
    u = synth.masked_gaussian(n, seed=33, sigma_px=n / 8)
    got = _run(cwo, u, dx, dx, lam, z, sh)
    assert _rel(got, _want(u, dx, dx, lam, z, sh)) <= TOL


def test_shifted_stack_equals_single_calls(cwo):
    import torch
    sh = cwo.Shift(30e-6, 10e-6, 0.0, 0.0, 0.0, 0.0)
    plan = cwo.Plan(128, 128, 8e-6, 8e-6, 532e-9, 0.02, shift=sh)
    x = torch.from_numpy(synth.random_field(128, seed=34).astype(np.complex64)).cuda()
    stack = plan.propagate_batch(x.unsqueeze(0).expand(3, -1, -1).contiguous())
    one = plan.propagate(x)
    for k in range(3):
        assert torch.equal(stack[k], one)
    with pytest.raises(cwo.CwoError) as e:
        plan.propagate_batch(x.unsqueeze(0).expand(2, -1, -1).contiguous(), z=[0.01, 0.02])
    assert e.value.status == cwo.ERR_UNSUPPORTED
