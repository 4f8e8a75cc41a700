"""Differentiation: the autograd.Function over propagate/adjoint, and the phase-only hologram
objective, against the FP64 oracle's gradient and central finite differences of the oracle loss.

Tolerances: the GPU loss and gradient are FP32 end to end (field, FFTs, |U|^2 - T, the mean);
with the propagation at <= 2e-5 relative L2, the residual (|U|^2 - T) carries relative errors up
to ~1e-4 where |U|^2 and T nearly cancel, so gradients are compared at 5e-4 relative L2 (all
pixels, vs the oracle gradient) and at 1e-3 of the largest component (64 pixels, vs FD)."""
import numpy as np
import pytest

import oracle
from paper_1107_5578_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods(gpu):
    import torch
    from paper_1107_5578_gb300 import autograd, cwo, hologram
    cwo.lib()
    return torch, autograd, cwo, hologram


def test_backward_is_the_adjoint(mods):
    # <A x, y> = <x, A^H y> through autograd: vjp of y = A x with cotangent g is A^H g
    torch, autograd, cwo, _ = mods
    plan = cwo.Plan(128, 64, 8e-6, 6e-6, 532e-9, 0.02, cwo.ANGULAR)
    x = torch.from_numpy(synth.random_field(128, seed=1, ny=64).astype(np.complex64)).cuda().requires_grad_(True)
    g = torch.from_numpy(synth.random_field(128, seed=2, ny=64).astype(np.complex64)).cuda()
    y = autograd.propagate(x, plan)
    (gx,) = torch.autograd.grad(y, x, grad_outputs=g)
    want = oracle.propagate(g.detach().cpu().numpy(), 8e-6, 6e-6, 532e-9, 0.02, oracle.ANGULAR, oracle.ADJOINT)
    got = gx.detach().cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 2e-5


def _small(hologram):
    return hologram.HologramProblem(h=96, w=160, canvas=256, pitch=6.4e-6, wavelength=520e-9, z=0.02, seed=3)


def test_hologram_gradient_matches_oracle(mods):
    torch, _, _, hologram = mods
    prob = _small(hologram)
    phi = torch.from_numpy(prob.phi0).float().cuda().requires_grad_(True)
    L = prob.loss(phi)
    L.backward()
    g = phi.grad.detach().cpu().numpy().astype(np.float64)
    loss_o, g_o = oracle.hologram_loss_grad(prob.phi0, (256, 256), (prob.oy, prob.ox), prob.target_np,
                                            6.4e-6, 520e-9, 0.02)
    assert abs(float(L.detach()) - loss_o) / loss_o < 1e-4
    assert np.linalg.norm(g - g_o) / np.linalg.norm(g_o) <= 5e-4


def test_hologram_gradient_central_differences(mods):
    torch, _, _, hologram = mods
    prob = _small(hologram)
    phi = torch.from_numpy(prob.phi0).float().cuda().requires_grad_(True)
    prob.loss(phi).backward()
    g = phi.grad.detach().cpu().numpy().astype(np.float64)
    rng = synth.rng(64)
    pix = [(int(rng.integers(0, 96)), int(rng.integers(0, 160))) for _ in range(64)]
    args = ((256, 256), (prob.oy, prob.ox), prob.target_np, 6.4e-6, 520e-9, 0.02)
    h = 1e-4
    fd = []
    for (i, j) in pix:
        p, m = prob.phi0.copy(), prob.phi0.copy()
        p[i, j] += h
        m[i, j] -= h
        fd.append((oracle.hologram_loss_grad(p, *args)[0] - oracle.hologram_loss_grad(m, *args)[0]) / (2 * h))
    fd = np.array(fd)
    got = np.array([g[i, j] for (i, j) in pix])
    assert np.max(np.abs(got - fd)) <= 1e-3 * np.max(np.abs(fd))


def test_adam_reduces_the_loss(mods):
    torch, _, _, hologram = mods
    prob = _small(hologram)
    _, losses, _ = hologram.optimise(prob, steps=25, lr=0.05)
    assert losses[-1] < 0.5 * losses[0]


@pytest.mark.slow
def test_full_size_hologram_gradient_matches_oracle(mods):
    # 1920 x 1080 phase in a 2048^2 canvas, ASM padded to 4096^2, 520 nm, 6.4 um, z = 0.15 m
    torch, _, _, hologram = mods
    prob = hologram.HologramProblem()
    phi = torch.from_numpy(prob.phi0).float().cuda().requires_grad_(True)
    L = prob.loss(phi)
    L.backward()
    g = phi.grad.detach().cpu().numpy().astype(np.float64)
    loss_o, g_o = oracle.hologram_loss_grad(prob.phi0, (2048, 2048), (prob.oy, prob.ox), prob.target_np,
                                            6.4e-6, 520e-9, 0.15)
    assert abs(float(L.detach()) - loss_o) / loss_o < 1e-4
    assert np.linalg.norm(g - g_o) / np.linalg.norm(g_o) <= 5e-4
