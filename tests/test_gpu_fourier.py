"""Fresnel diffraction in Fourier form (Eqs. fre_fourier2, fre_fourier3) on the GPU against the
FP64 oracle at the 2e-5 relative-L2 bar."""
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


def _gpu(cwo, u, dx, dy, lam, z, flags=0):
    import torch
    ny, nx = u.shape
    plan = cwo.Plan(nx, ny, dx, dy, lam, z, cwo.FRESNEL_FOURIER, flags)
    y = plan.propagate(torch.from_numpy(u.astype(np.complex64)).cuda())
    plan.check()
    return y.cpu().numpy().astype(np.complex128)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nx,ny", [(32, 32), (64, 128), (256, 256), (512, 256), (1024, 1024)])
@pytest.mark.parametrize("z", [0.3, -0.12])
def test_fourier_form_against_oracle(cwo, nx, ny, z):
    u = synth.random_field(nx, seed=51, ny=ny)
    got = _gpu(cwo, u, 8e-6, 6e-6, 532e-9, z)
    want = oracle.fresnel_fourier(u.astype(np.complex64), 8e-6, 6e-6, 532e-9, z)
    assert _rel(got, want) <= TOL


def test_fourier_form_gaussian_and_literal_scale(cwo):
    n, pitch, lam, w0, z = 256, 10e-6, 633e-9, 200e-6, 1.0
    u = synth.gaussian_beam(n, pitch, w0)
    got = _gpu(cwo, u, pitch, pitch, lam, z)
    want = oracle.fresnel_fourier(u.astype(np.complex64), pitch, pitch, lam, z)
    assert _rel(got, want) <= TOL
    lit = _gpu(cwo, u, pitch, pitch, lam, z, flags=cwo.FLAG_LITERAL_SCALE)
    assert _rel(lit * pitch * pitch, got) <= 1e-6


def test_fourier_form_batch_and_rejections(cwo):
    import torch
    plan = cwo.Plan(128, 64, 8e-6, 8e-6, 532e-9, 0.2, cwo.FRESNEL_FOURIER)
    assert plan.launches_per_call == 2
    x = torch.from_numpy(np.stack([synth.random_field(128, seed=60 + k, ny=64) for k in range(3)]).astype(np.complex64)).cuda()
    y = plan.propagate_batch(x)
    for k in range(3):
        assert torch.equal(y[k], plan.propagate(x[k]))
    for call in (lambda: plan.adjoint(x[0]), lambda: plan.propagate_batch(x, z=[0.1, 0.2, 0.3]),
                 lambda: plan.propagate_epilogue(x, cwo.EPI_PHASE)):
        with pytest.raises(cwo.CwoError) as e:
            call()
        assert e.value.status == cwo.ERR_UNSUPPORTED
    dx2, dy2 = plan.output_pitch
    assert abs(dx2 - 532e-9 * 0.2 / (128 * 8e-6)) < 1e-18 and abs(dy2 - 532e-9 * 0.2 / (64 * 8e-6)) < 1e-18


@pytest.mark.slow
def test_fourier_form_4096(cwo):
    u = synth.random_field(4096, seed=52)
    got = _gpu(cwo, u, 3.74e-6, 3.74e-6, 532e-9, 0.5)
    want = oracle.fresnel_fourier(u.astype(np.complex64), 3.74e-6, 3.74e-6, 532e-9, 0.5)
    assert _rel(got, want) <= TOL
