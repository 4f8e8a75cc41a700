"""Shifted Fresnel diffraction (Eqs. shift_fre1 to shift_fre3) on the GPU against the FP64
oracle (itself pinned to the literal Fresnel sum), at the 2e-5 relative-L2 bar."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# (nx, ny, dx0, dy0, lam, z, (dx1, dy1, ox0, oy0, ox1, oy1))
CASES = [
    (64, 64, 8e-6, 8e-6, 532e-9, 0.05, (4e-6, 4e-6, 0.0, 0.0, 100e-6, -60e-6)),
    (128, 64, 6e-6, 9e-6, 633e-9, 0.2, (12e-6, 5e-6, 30e-6, -20e-6, -400e-6, 250e-6)),
    (256, 256, 10e-6, 10e-6, 450e-9, -0.1, (10e-6, 10e-6, 0.0, 0.0, 1e-3, 0.0)),
    (512, 256, 4e-6, 4e-6, 532e-9, 0.3, (20e-6, 20e-6, -50e-6, 80e-6, 2e-3, -1e-3)),
]


@pytest.mark.parametrize("case", CASES)
def test_shifted_fresnel_against_oracle(cwo, case):
    import torch
    nx, ny, dx0, dy0, lam, z, prm = case
    u = synth.random_field(nx, seed=71, ny=ny)
    plan = cwo.Plan(nx, ny, dx0, dy0, lam, z, shifted_fresnel=cwo.ShiftedFresnel(*prm))
    got = plan.propagate(torch.from_numpy(u.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
    plan.check()
    want = oracle.shifted_fresnel(u.astype(np.complex64), dx0, dy0, prm[0], prm[1], lam, z, *prm[2:])
    assert _rel(got, want) <= TOL
    assert plan.output_pitch == (prm[0], prm[1])


@pytest.mark.parametrize("case", CASES[:2])
def test_shifted_fresnel_adjoint_dot_product(cwo, case):
    import torch
    nx, ny, dx0, dy0, lam, z, prm = case
    plan = cwo.Plan(nx, ny, dx0, dy0, lam, z, shifted_fresnel=cwo.ShiftedFresnel(*prm))
    x = synth.random_field(nx, seed=72, ny=ny)
    y = synth.random_field(nx, seed=73, ny=ny)
    ax = plan.propagate(torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
    ahy = plan.adjoint(torch.from_numpy(y.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(y.astype(np.complex64), ax)
    rhs = np.vdot(ahy, x.astype(np.complex64))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_shifted_fresnel_equal_grids_is_the_convolution_form(cwo):
    import torch
    u = torch.from_numpy(synth.random_field(128, seed=74, ny=64).astype(np.complex64)).cuda()
    sf = cwo.Plan(128, 64, 8e-6, 6e-6, 532e-9, 0.03, shifted_fresnel=cwo.ShiftedFresnel(8e-6, 6e-6, 0, 0, 0, 0))
    conv = cwo.Plan(128, 64, 8e-6, 6e-6, 532e-9, 0.03, cwo.FRESNEL_CONV)
    a, b = sf.propagate(u), conv.propagate(u)
    assert float((a - b).norm() / b.norm()) <= 1e-5


def test_shifted_fresnel_literal_scale_and_rejections(cwo):
    import torch
    prm = cwo.ShiftedFresnel(5e-6, 5e-6, 0.0, 0.0, 1e-4, 0.0)
    u = torch.from_numpy(synth.random_field(64, seed=75).astype(np.complex64)).cuda()
    a = cwo.Plan(64, 64, 8e-6, 8e-6, 532e-9, 0.05, shifted_fresnel=prm).propagate(u)
    b = cwo.Plan(64, 64, 8e-6, 8e-6, 532e-9, 0.05, flags=cwo.FLAG_LITERAL_SCALE, shifted_fresnel=prm).propagate(u)
    assert float((b * 8e-6 * 8e-6 - a).norm() / a.norm()) <= 1e-6
    plan = cwo.Plan(64, 64, 8e-6, 8e-6, 532e-9, 0.05, shifted_fresnel=prm)
    with pytest.raises(cwo.CwoError) as e:
        plan.propagate_batch(u.unsqueeze(0).expand(2, -1, -1).contiguous(), z=[0.04, 0.05])
    assert e.value.status == cwo.ERR_UNSUPPORTED
    with pytest.raises(cwo.CwoError):
        cwo.Plan(64, 64, 8e-6, 8e-6, 532e-9, 0.05, shifted_fresnel=cwo.ShiftedFresnel(0.0, 5e-6, 0, 0, 0, 0))


@pytest.mark.parametrize("case", CASES[1:])
@pytest.mark.parametrize("adjoint", [False, True])
def test_shifted_fresnel_two_passes_equal_three(cwo, case, adjoint):
    # the plan runs two separable line passes (source and destination factors fused per axis);
    # an output off a 16-byte boundary takes the three-pass method: the two agree
    import torch
    nx, ny, dx0, dy0, lam, z, prm = case
    plan = cwo.Plan(nx, ny, dx0, dy0, lam, z, shifted_fresnel=cwo.ShiftedFresnel(*prm))
    assert plan.launches_per_call == 2
    x = torch.from_numpy(synth.random_field(nx, seed=74, ny=ny).astype(np.complex64)).cuda()
    run = plan.adjoint if adjoint else plan.propagate
    a = run(x).cpu().numpy().astype(np.complex128)
    buf = torch.empty(nx * ny + 1, dtype=torch.complex64, device="cuda")
    out = buf[1:].view(ny, nx)
    run(x, out=out)
    b = out.cpu().numpy().astype(np.complex128)
    plan.check()
    plan.close()
    assert _rel(a, b) <= 1e-5


@pytest.mark.slow
def test_shifted_fresnel_large_lines_against_oracle(cwo):
    # rows padded to 4096 and columns to 2048: the pair form of the line pass with the source and
    # destination factors of both axes
    import torch
    nx, ny, dx0, dy0, lam, z = 2048, 1024, 6e-6, 6e-6, 532e-9, 0.25
    prm = (9e-6, 4e-6, 20e-6, -30e-6, 600e-6, -300e-6)
    u = synth.random_field(nx, seed=75, ny=ny)
    plan = cwo.Plan(nx, ny, dx0, dy0, lam, z, shifted_fresnel=cwo.ShiftedFresnel(*prm))
    assert plan.launches_per_call == 2
    got = plan.propagate(torch.from_numpy(u.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
    plan.check()
    plan.close()
    want = oracle.shifted_fresnel(u.astype(np.complex64), dx0, dy0, prm[0], prm[1], lam, z, *prm[2:])
    assert _rel(got, want) <= TOL


@pytest.mark.slow
@pytest.mark.parametrize("adjoint", [False, True])
def test_shifted_fresnel_4096_two_passes_equal_three(cwo, adjoint):
    # 4096^2: the persistent line pass at P = 8192 with both factors against the three-pass method
    # (an output off a 16-byte boundary), whose forward row pass multiplies by the source factors
    # (the cluster kernel at P = 8192) and whose inverse row pass applies the destination factors
    import torch
    n, dx0, lam, z = 4096, 3.74e-6, 532e-9, 0.3
    prm = (5e-6, 5e-6, 0.0, 0.0, 2e-3, -1e-3)
    plan = cwo.Plan(n, n, dx0, dx0, lam, z, shifted_fresnel=cwo.ShiftedFresnel(*prm))
    x = torch.from_numpy(synth.random_field(n, seed=76).astype(np.complex64)).cuda()
    run = plan.adjoint if adjoint else plan.propagate
    a = run(x).cpu().numpy().astype(np.complex128)
    buf = torch.empty(n * n + 1, dtype=torch.complex64, device="cuda")
    out = buf[1:].view(n, n)
    run(x, out=out)
    b = out.cpu().numpy().astype(np.complex128)
    plan.check()
    plan.close()
    assert _rel(a, b) <= 1e-5
