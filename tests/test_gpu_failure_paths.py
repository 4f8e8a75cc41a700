"""Failure paths on the GPU without a fault: the bounded mbarrier wait that guards every TMA
load gives up on a barrier that nothing completes, records the timeout in the status word and
returns, leaving the context usable; errors found on the host come back as status codes before
any launch."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cwo(gpu):
    import paper_1107_5578_gb300.cwo as m
    m.lib()
    return m


def test_bounded_wait_gives_up_and_reports(cwo):
    import torch
    assert cwo.debug_bounded_wait(1000, complete=False) == 1
    assert cwo.debug_bounded_wait(1, complete=False) == 1
    assert cwo.debug_bounded_wait(1000, complete=True) == 0
    # the context is still usable: a propagation runs and its own status word is clean
    plan = cwo.Plan(64, 64, 10e-6, 10e-6, 633e-9, 0.05, cwo.ANGULAR)
    x = torch.ones(64, 64, dtype=torch.complex64, device="cuda")
    y = plan.propagate(x)
    plan.check()
    assert torch.isfinite(torch.view_as_real(y)).all()


def test_bounded_wait_rejects_bad_limits(cwo):
    for lim in (0, (1 << 20) + 1):
        with pytest.raises(cwo.CwoError):
            cwo.debug_bounded_wait(lim, complete=False)


def test_host_errors_leave_no_launch(cwo):
    import torch
    plan = cwo.Plan(64, 64, 10e-6, 10e-6, 633e-9, 0.05, cwo.ANGULAR)
    x = torch.zeros(64, 64, dtype=torch.complex64, device="cuda")
    with pytest.raises(cwo.CwoError):
        plan.propagate_batch(x.unsqueeze(0), z=[float("nan")])
    with pytest.raises(cwo.CwoError):
        cwo.Plan(64, 64, 10e-6, 10e-6, 633e-9, 0.0, cwo.FRESNEL_CONV)
    plan.check()
