"""GS kinoform iteration on the GPU against the FP64 oracle.

The constraints are nonlinear where |u| ~ 0 (the phase of a vanishing value is ill-conditioned),
so single steps are compared where the phase is defined: the propagated value itself at the
2e-5 relative-L2 bar (it is the plain propagation), the output's unit amplitude to 1e-6, and
its phase where |u| > 1e-3 max|u|.  A short full run is compared on the reconstructed intensity,
which is smooth in the kinoform, at 1e-3 relative L2 (FP32 vs FP64 iterates drift apart only
through the ill-conditioned pixels)."""
import numpy as np
import pytest

import oracle
from paper_1107_5578_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods(gpu):
    import torch
    from paper_1107_5578_gb300 import cwo, gs
    cwo.lib()
    return torch, cwo, gs


def _phase_ok(got, want_u, tol_rad=2e-4):
    m = np.abs(want_u)
    sel = m > 1e-3 * m.max()
    d = np.angle(got[sel] * np.conj(want_u[sel]))
    return np.max(np.abs(d)) <= tol_rad, np.max(np.abs(np.abs(got) - 1.0))


@pytest.mark.parametrize("n", [64, 256, pytest.param(4096, marks=pytest.mark.slow)])
def test_epilogue_steps(mods, n):
    # 4096: the inverse row pass with a thread per pair of rows (P = 8192) and each epilogue
    torch, cwo, _ = mods
    amp, f0 = synth.gs_problem(n, seed=3)
    plan = cwo.Plan(n, n, 8e-6, 8e-6, 532e-9, 0.02, cwo.ANGULAR)
    x = torch.from_numpy(f0.astype(np.complex64)).cuda()
    a = torch.from_numpy(amp.astype(np.float32)).cuda()
    u_fwd = oracle.propagate(f0.astype(np.complex64), 8e-6, 8e-6, 532e-9, 0.02)
    # forward + phase constraint
    ph = plan.propagate_epilogue(x, cwo.EPI_PHASE).cpu().numpy().astype(np.complex128)
    ok, dev = _phase_ok(ph, u_fwd)
    assert ok and dev < 1e-6
    # adjoint (= -z) + amplitude constraint
    u_bwd = oracle.propagate(f0.astype(np.complex64), 8e-6, 8e-6, 532e-9, -0.02)
    am = plan.propagate_epilogue(x, cwo.EPI_AMPLITUDE, amplitude=a, adjoint=True).cpu().numpy().astype(np.complex128)
    m = np.abs(u_bwd)
    sel = m > 1e-3 * m.max()
    assert np.max(np.abs(np.abs(am) - amp.astype(np.float32))) < 1e-6
    assert np.max(np.abs(np.angle(am[sel] * np.conj(u_bwd[sel])))) < 2e-4
    # intensity
    it = plan.propagate_epilogue(x, cwo.EPI_INTENSITY, adjoint=True).cpu().numpy().astype(np.float64)
    want = np.abs(u_bwd) ** 2
    assert np.linalg.norm(it - want) / np.linalg.norm(want) <= 4e-5
    # plain epilogue equals the ordinary call bit for bit
    assert torch.equal(plan.propagate_epilogue(x, cwo.EPI_NONE), plan.propagate(x))
    plan.check()


@pytest.mark.parametrize("n,iters", [(64, 3), (128, 5)])
def test_gs_run_against_oracle(mods, n, iters):
    torch, cwo, gs = mods
    amp, f0 = synth.gs_problem(n, seed=9)
    plan = cwo.Plan(n, n, 10e-6, 10e-6, 633e-9, 0.1, cwo.ANGULAR)
    field = torch.from_numpy(f0.astype(np.complex64)).cuda()
    inten = plan.gs_run(torch.from_numpy(amp.astype(np.float32)).cuda(), field, iters)
    kin_o, int_o = oracle.gs_run(amp.astype(np.float32), f0.astype(np.complex64), 10e-6, 10e-6, 633e-9, 0.1, iters)
    got_k = field.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(np.abs(got_k) - 1.0)) < 1e-6
    got_i = inten.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got_i - int_o) / np.linalg.norm(int_o) <= 1e-3


@pytest.mark.parametrize("n,iters", [(128, 4), (512, 3), pytest.param(1024, 2, marks=pytest.mark.slow)])
def test_gs_each_iteration_against_oracle_step(mods, n, iters):
    """Every GS iterate of the device loop checked against one oracle step taken from it
    (Section "GS algorithm": -z, amplitude constraint, +z, phase constraint).  The two plain
    propagations of each step are compared at the 2e-5 relative-L2 bar; each constraint's output
    has the required amplitude to 1e-6 and the oracle's phase within 2e-4 rad wherever the
    propagated value exceeds 1e-3 of its maximum; and ``cwo_gs_run`` after k + 1 iterations --
    which keeps the field in the intermediate and turns from one propagation to the next in one
    kernel -- equals the step-by-step composition bit for bit, so the bar holds for every
    iterate of the loop itself.  512^2 and 1024^2 are sizes of Table tbl:gs."""
    torch, cwo, _ = mods
    dx, lam, z = 10e-6, 633e-9, 0.1
    amp, f0 = synth.gs_problem(n, seed=21)
    a32 = amp.astype(np.float32)
    plan = cwo.Plan(n, n, dx, dx, lam, z, cwo.ANGULAR)
    a = torch.from_numpy(a32).cuda()
    x0 = torch.from_numpy(f0.astype(np.complex64)).cuda()

    def host(t):
        torch.cuda.synchronize()
        return t.cpu().numpy().astype(np.complex128)

    def rel(g, w):
        return float(np.linalg.norm(g - w) / np.linalg.norm(w))

    def constraint_ok(got, want_prop, amp_want):
        m = np.abs(want_prop)
        sel = m > 1e-3 * m.max()
        dph = np.max(np.abs(np.angle(got[sel] * np.conj(want_prop[sel]))))
        damp = np.max(np.abs(np.abs(got) - amp_want))
        return dph, damp

    # hologram plane: +z and the phase constraint
    fwd0 = host(plan.propagate(x0))
    want0 = oracle.propagate(f0.astype(np.complex64), dx, dx, lam, z)
    assert rel(fwd0, want0) <= 2e-5
    u = plan.propagate_epilogue(x0, cwo.EPI_PHASE)
    dph, damp = constraint_ok(host(u), want0, 1.0)
    assert dph <= 2e-4 and damp <= 1e-6
    f = x0.clone()
    plan.gs_run(a, f, 0, intensity=False)
    assert torch.equal(f, u)
    for k in range(iters):
        uk = host(u)
        # -z (the adjoint of the +z plan) from the device iterate, then the amplitude constraint
        back = host(plan.adjoint(u))
        back_o = oracle.propagate(uk, dx, dx, lam, -z)
        assert rel(back, back_o) <= 2e-5, f"iteration {k}: back-propagation"
        obj = plan.propagate_epilogue(u, cwo.EPI_AMPLITUDE, amplitude=a, adjoint=True)
        dph, damp = constraint_ok(host(obj), back_o, a32.astype(np.float64))
        assert dph <= 2e-4 and damp <= 1e-6, f"iteration {k}: amplitude constraint {dph:.2e} {damp:.2e}"
        # +z from the device object field, then the phase constraint
        fwd = host(plan.propagate(obj))
        fwd_o = oracle.propagate(host(obj), dx, dx, lam, z)
        assert rel(fwd, fwd_o) <= 2e-5, f"iteration {k}: forward propagation"
        u = plan.propagate_epilogue(obj, cwo.EPI_PHASE)
        dph, damp = constraint_ok(host(u), fwd_o, 1.0)
        assert dph <= 2e-4 and damp <= 1e-6, f"iteration {k}: phase constraint {dph:.2e} {damp:.2e}"
        # the fused loop reaches the same iterate
        f = x0.clone()
        plan.gs_run(a, f, k + 1, intensity=False)
        assert torch.equal(f, u), f"iteration {k}: cwo_gs_run differs from the step composition"
    plan.check()
    plan.close()


def test_gs_batch_equals_single_and_error_drops(mods):
    torch, cwo, gs = mods
    prob = gs.GSProblem(n=256, seed=4, batch=3)
    kin, inten = prob.run(10)
    for k in range(3):
        one = cwo.Plan(256, 256, gs.PITCH, gs.PITCH, gs.WAVELENGTH, gs.DISTANCE, cwo.ANGULAR)
        f = prob.field0[k].clone()
        i1 = one.gs_run(prob.amplitude[k], f, 10)
        assert torch.equal(f, kin[k]) and torch.equal(i1, inten[k])
    _, i0 = prob.run(0)
    e0 = gs.amplitude_error(i0, prob.amplitude)
    e10 = gs.amplitude_error(inten, prob.amplitude)
    assert e10 < 0.8 * e0


def test_gs_rejects(mods):
    torch, cwo, _ = mods
    fres = cwo.Plan(64, 64, 8e-6, 8e-6, 532e-9, 0.02, cwo.FRESNEL_CONV)
    f = torch.zeros(64, 64, dtype=torch.complex64, device="cuda")
    a = torch.ones(64, 64, dtype=torch.float32, device="cuda")
    with pytest.raises(cwo.CwoError):
        fres.gs_run(a, f, 2)
    asm = cwo.Plan(64, 64, 8e-6, 8e-6, 532e-9, 0.02, cwo.ANGULAR)
    with pytest.raises(cwo.CwoError):
        asm.gs_run(a, f, -1)
    with pytest.raises(ValueError):
        asm.gs_run(torch.ones(32, 32, dtype=torch.float32, device="cuda"), f, 2)
