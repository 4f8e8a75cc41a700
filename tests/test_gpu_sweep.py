"""Seeded random sweep over shapes, types, distances, pitches, batch sizes and the adjoint:
every case against the FP64 oracle at the 2e-5 relative-L2 bar.  Catches interactions the
targeted tests do not enumerate (rectangular shapes with every type, odd parameter mixes)."""
import numpy as np
import pytest

import oracle
from paper_1107_5578_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 2e-5
SIDES = [16, 32, 64, 128, 256, 512]


def _cases(count=40, seed=2024):
    g = synth.rng(seed)
    out = []
    for k in range(count):
        kind = int(g.integers(0, 5))   # 0 ASM, 1 Fresnel conv, 2 Fourier form, 3 shifted Fresnel, 4 shifted ASM
        lo = 2 if kind == 2 else 0      # the Fourier form needs sides >= 32
        nx, ny = int(g.choice(SIDES[lo:])), int(g.choice(SIDES[lo:]))
        z = float((0.005 + 0.3 * g.random()) * (1 if g.random() < 0.7 else -1))
        dx, dy = float(3e-6 + 9e-6 * g.random()), float(3e-6 + 9e-6 * g.random())
        lam = float(g.choice([450e-9, 532e-9, 633e-9]))
        batch = int(g.integers(1, 4))
        adjoint = bool(g.random() < 0.3) and kind in (0, 1, 3, 4)
        extra = tuple(float(v) for v in g.random(6))
        out.append((k, kind, nx, ny, z, dx, dy, lam, batch, adjoint, extra))
    return out


@pytest.fixture(scope="module")
def cwo(gpu):
    import paper_1107_5578_gb300.cwo as m
    m.lib()
    return m


@pytest.mark.parametrize("case", _cases(), ids=lambda c: f"case{c[0]}-type{c[1]}-{c[2]}x{c[3]}")
def test_sweep(cwo, case):
    import torch
    k, kind, nx, ny, z, dx, dy, lam, batch, adjoint, extra = case
    us = np.stack([synth.random_field(nx, seed=5000 + 10 * k + j, ny=ny) for j in range(batch)]).astype(np.complex64)
    if kind == 3:
        prm = (dx * (0.5 + extra[0]), dy * (0.5 + extra[1]), 40e-6 * (extra[2] - 0.5), 40e-6 * (extra[3] - 0.5),
               300e-6 * (extra[4] - 0.5), 300e-6 * (extra[5] - 0.5))
        plan = cwo.Plan(nx, ny, dx, dy, lam, z, shifted_fresnel=cwo.ShiftedFresnel(*prm))
        ref = lambda u: oracle.shifted_fresnel(u, dx, dy, prm[0], prm[1], lam, z, *prm[2:],
                                               flags=0) if not adjoint else None
    elif kind == 4:
        fx, fy = 1 / (2 * dx), 1 / (2 * dy)
        sh = (200e-6 * (extra[0] - 0.5), 200e-6 * (extra[1] - 0.5), 0.2 * fx * (extra[2] - 0.5),
              fx * (0.4 + extra[3]), 0.2 * fy * (extra[4] - 0.5), fy * (0.4 + extra[5]))
        plan = cwo.Plan(nx, ny, dx, dy, lam, z, shift=cwo.Shift(*sh))
        ref = lambda u: oracle.propagate_shifted(u, dx, dy, lam, z, *sh, flags=oracle.ADJOINT if adjoint else 0)
    elif kind == 2:
        plan = cwo.Plan(nx, ny, dx, dy, lam, z, cwo.FRESNEL_FOURIER)
        ref = lambda u: oracle.fresnel_fourier(u, dx, dy, lam, z)
    else:
        plan = cwo.Plan(nx, ny, dx, dy, lam, z, kind)
        ref = lambda u: oracle.propagate(u, dx, dy, lam, z, kind, oracle.ADJOINT if adjoint else 0)
    x = torch.from_numpy(us).cuda()
    y = plan.propagate_batch(x, adjoint=adjoint)
    plan.check()
    got = y.cpu().numpy().astype(np.complex128)
    for j in range(batch):
        if kind == 3 and adjoint:
            continue
        want = ref(us[j])
        err = np.linalg.norm(got[j] - want) / np.linalg.norm(want)
        assert err <= TOL, (case, j, err)
    if kind == 3 and adjoint:   # the shifted-Fresnel adjoint by the dot-product test
        v = synth.random_field(nx, seed=9000 + k, ny=ny).astype(np.complex64)
        fwd = plan.propagate(torch.from_numpy(v).cuda()).cpu().numpy().astype(np.complex128)
        lhs = np.vdot(us[0], fwd)
        rhs = np.vdot(got[0], v)
        assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    plan.close()
