"""Mixed batches (cwo_propagate_items): every item with its own type, distance, wavelength and
pitches, against the FP64 oracle at the 2e-5 relative-L2 bar; an item's result does not depend on
the batch it rides in (bit for bit); items the mixed path does not take are rejected."""
import numpy as np
import pytest

import oracle
from paper_1107_5578_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 2e-5

# (type, z, wavelength, dx, dy, flags): ASM near and far, negative and zero distance, a pitch
# below lambda/2 (evanescent band), Fresnel with and without the literal scale
ITEMS = [
    (0, 0.02, 532e-9, 8e-6, 6e-6, 0),
    (1, 0.05, 633e-9, 10e-6, 10e-6, 0),
    (0, -0.01, 450e-9, 4e-6, 5e-6, 0),
    (0, 0.0, 633e-9, 10e-6, 10e-6, 0),
    (1, 0.3, 450e-9, 6e-6, 4e-6, 4),
    (0, 2e-5, 633e-9, 0.25e-6, 0.25e-6, 0),
    (0, 1.0, 532e-9, 3e-6, 3e-6, 0),
    (1, -0.1, 532e-9, 8e-6, 8e-6, 0),
    (0, 5e-4, 633e-9, 1.0e-6, 0.8e-6, 0),
]


@pytest.fixture(scope="module")
def cwo(gpu):
    import paper_1107_5578_gb300.cwo as m
    m.lib()
    return m


def _item(t):
    return {"type": t[0], "z": t[1], "wavelength": t[2], "dx": t[3], "dy": t[4], "flags": t[5]}


def _fields(nx, ny, b, seed):
    return np.stack([synth.random_field(nx, seed=seed + k, ny=ny) for k in range(b)])


@pytest.mark.parametrize("nx,ny", [(256, 128), (64, 64), (1024, 1024)])
def test_mixed_batch_against_oracle(cwo, nx, ny):
    import torch
    u = _fields(nx, ny, len(ITEMS), 40)
    plan = cwo.Plan(nx, ny, 10e-6, 10e-6, 633e-9, 0.1, cwo.ANGULAR)
    x = torch.from_numpy(u.astype(np.complex64)).cuda()
    y = plan.propagate_items(x, [_item(t) for t in ITEMS])
    plan.check()
    got = y.cpu().numpy().astype(np.complex128)
    for k, t in enumerate(ITEMS):
        flags = oracle.LITERAL_SCALE if t[5] & 4 else 0
        want = oracle.propagate(u[k], t[3], t[4], t[2], t[1], t[0], flags)
        err = np.linalg.norm(got[k] - want) / np.linalg.norm(want)
        assert err <= TOL, (k, t, err)


def test_item_result_is_independent_of_the_batch(cwo):
    import torch
    u = _fields(128, 128, len(ITEMS), 70)
    plan = cwo.Plan(128, 128, 10e-6, 10e-6, 633e-9, 0.1, cwo.ANGULAR)
    x = torch.from_numpy(u.astype(np.complex64)).cuda()
    whole = plan.propagate_items(x, [_item(t) for t in ITEMS])
    rev = plan.propagate_items(x.flip(0).contiguous(), [_item(t) for t in ITEMS[::-1]])
    for k, t in enumerate(ITEMS):
        alone = plan.propagate_items(x[k:k + 1], [_item(t)])
        assert torch.equal(alone[0], whole[k]), k
        assert torch.equal(rev[len(ITEMS) - 1 - k], whole[k]), k


def test_mixed_item_matches_a_plan_of_its_own(cwo):
    import torch
    u = _fields(256, 256, len(ITEMS), 90)
    host = cwo.Plan(256, 256, 10e-6, 10e-6, 633e-9, 0.1, cwo.ANGULAR)
    x = torch.from_numpy(u.astype(np.complex64)).cuda()
    y = host.propagate_items(x, [_item(t) for t in ITEMS])
    for k, t in enumerate(ITEMS):
        own = cwo.Plan(256, 256, t[3], t[4], t[2], t[1], t[0], t[5])
        r = own.propagate(x[k])
        assert float((r - y[k]).norm() / r.norm()) <= 1e-6, (k, t)
        if t[0] == cwo.FRESNEL_CONV:   # the same two separable line passes as a Fresnel plan
            assert torch.equal(r, y[k]), (k, t)
        own.close()


def test_rejected_items(cwo):
    import torch
    plan = cwo.Plan(64, 64, 10e-6, 10e-6, 633e-9, 0.1, cwo.ANGULAR)
    x = torch.zeros(2, 64, 64, dtype=torch.complex64, device="cuda")
    good = _item(ITEMS[0])
    with pytest.raises(cwo.CwoError):      # Fresnel needs z != 0
        plan.propagate_items(x, [good, {**good, "type": 1, "z": 0.0}])
    with pytest.raises(cwo.CwoError):      # the phase-precision arms are single-plan only
        plan.propagate_items(x, [good, {**good, "flags": cwo.FLAG_PHASE_FP64}])
    with pytest.raises(cwo.CwoError):
        plan.propagate_items(x, [good, {**good, "wavelength": -1.0}])
    with pytest.raises(ValueError):
        plan.propagate_items(x, [good])
    plan.check()


def test_back_to_back_calls_keep_their_own_tables(cwo):
    # per-call tables go through a ring of pinned staging buffers: ten calls enqueued without any
    # synchronisation, each with its own parameters, must each produce its own propagation
    import torch
    n = 128
    u = synth.random_field(n, seed=300)
    x = torch.from_numpy(u.astype(np.complex64)).cuda().unsqueeze(0)
    plan = cwo.Plan(n, n, 10e-6, 10e-6, 633e-9, 0.1, cwo.ANGULAR)
    params = [(k % 2, 0.01 + 0.013 * k, (450e-9, 532e-9, 633e-9)[k % 3], 4e-6 + 5e-7 * k) for k in range(10)]
    outs = [plan.propagate_items(x, [dict(type=t, z=z, wavelength=lam, dx=p)]) for (t, z, lam, p) in params]
    zs = [[0.02 + 0.01 * k, 0.05 + 0.02 * k] for k in range(6)]
    xb = x.expand(2, -1, -1).contiguous()
    zouts = [plan.propagate_batch(xb, z=z) for z in zs]
    torch.cuda.synchronize()
    for (t, z, lam, p), y in zip(params, outs):
        want = oracle.propagate(u.astype(np.complex64), p, p, lam, z, t)
        got = y[0].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= TOL
    for z, y in zip(zs, zouts):
        for k in range(2):
            want = oracle.propagate(u.astype(np.complex64), 10e-6, 10e-6, 633e-9, z[k], oracle.ANGULAR)
            got = y[k].cpu().numpy().astype(np.complex128)
            assert np.linalg.norm(got - want) / np.linalg.norm(want) <= TOL
