"""Precision study (4096^2 unit-amplitude random-phase field padded to 8192^2, 532 nm, 3.74 um,
z in {0.05, 0.2, 1.0} m): the default FP64-reduced phase meets the 2e-5 bar at every z; the
literal all-FP32 phase does not once z / lambda is large; the literal FP64 phase agrees with the
default.  A smaller case with the same z / lambda runs in the fast suite."""
import numpy as np
import pytest

import oracle
from paper_1107_5578_gb300 import synth

pytestmark = pytest.mark.gpu
LAM, PITCH = 532e-9, 3.74e-6


@pytest.fixture(scope="module")
def prec(gpu):
    from paper_1107_5578_gb300 import cwo, precision
    cwo.lib()
    return precision


@pytest.mark.parametrize("z", [0.05, 0.2, 1.0])
def test_precision_arms_512(prec, z):
    u = synth.random_phase_field(512, seed=3)
    ref = oracle.propagate(u, PITCH, PITCH, LAM, z, oracle.ANGULAR)
    res = {arm: prec.errors(prec.run_arm(u, PITCH, LAM, z, arm), ref) for arm in prec.ARMS}
    assert res["reduced"]["rel_l2"] <= 2e-5
    assert res["fp64"]["rel_l2"] <= 2e-5
    assert res["fp32"]["rel_l2"] > 10 * res["reduced"]["rel_l2"]


@pytest.mark.slow
@pytest.mark.parametrize("z", [0.05, 0.2, 1.0])
def test_precision_study_4096(prec, z):
    u = synth.random_phase_field(4096, seed=3)
    ref = oracle.propagate(u, PITCH, PITCH, LAM, z, oracle.ANGULAR)
    red = prec.errors(prec.run_arm(u, PITCH, LAM, z, "reduced"), ref)
    f32 = prec.errors(prec.run_arm(u, PITCH, LAM, z, "fp32"), ref)
    print(f"z={z}: reduced {red} fp32 {f32}")
    assert red["rel_l2"] <= 2e-5
    assert f32["rel_l2"] > red["rel_l2"]
