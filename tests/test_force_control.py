"""Body-force adaptation to a target capillary number (Sec. 4.2, Eq.
LB_body_force_adaptation): F <- (Ca*/Ca) F, each change capped at a factor of
two. The controller is host code in the library; these checks need no GPU."""
import math

import pytest


@pytest.fixture(scope="module")
def lbm():
    from paper_2007_12266_gb300 import _build
    _build.build()
    import paper_2007_12266_gb300 as m
    return m


def test_rescale_is_the_ratio_inside_the_cap(lbm):
    F = (1e-5, -2e-5, 3e-5)
    out, g = lbm.force_rescale(F, ca=2e-4, ca_target=3e-4)
    assert g == pytest.approx(1.5, rel=1e-15)
    assert out == pytest.approx(tuple(1.5 * x for x in F), rel=1e-15)
    # the direction of the force is kept
    out, g = lbm.force_rescale(F, ca=4e-4, ca_target=3e-4)
    assert g == pytest.approx(0.75, rel=1e-15)


def test_rescale_is_capped_at_a_factor_of_two(lbm):
    F = (0.0, 0.0, 1e-5)
    out, g = lbm.force_rescale(F, ca=1e-6, ca_target=1e-3)
    assert g == 2.0 and out[2] == 2e-5
    out, g = lbm.force_rescale(F, ca=1e-2, ca_target=1e-5)
    assert g == 0.5 and out[2] == 0.5e-5
    # another cap
    out, g = lbm.force_rescale(F, ca=1e-6, ca_target=1e-3, max_factor=1.25)
    assert g == 1.25


def test_no_flow_raises_the_force_by_the_cap(lbm):
    out, g = lbm.force_rescale((0, 0, 1e-5), ca=0.0, ca_target=1e-4)
    assert g == 2.0 and out[2] == 2e-5


def test_repeated_rescales_reach_the_target_of_a_linear_response(lbm):
    # Darcy regime: Ca proportional to F; the capped iteration doubles the
    # force floor(log2(Ca*/Ca0)) times, then one rescale lands on Ca*
    k = 7.0   # Ca = k |F|
    F = (0.0, 0.0, 1e-6)
    target = 1e-3
    n = 0
    while abs(k * F[2] / target - 1.0) > 1e-12 and n < 20:
        F, _ = lbm.force_rescale(F, ca=k * F[2], ca_target=target)
        n += 1
    assert n == math.floor(math.log2(target / (k * 1e-6))) + 1
    assert k * F[2] == pytest.approx(target, rel=1e-12)


@pytest.mark.parametrize("args", [dict(ca=1e-4, ca_target=0.0), dict(ca=1e-4, ca_target=-1.0),
                                  dict(ca=float("nan"), ca_target=1e-4), dict(ca=1e-4, ca_target=1e-4, max_factor=0.5)])
def test_invalid_arguments_are_rejected(lbm, args):
    with pytest.raises(lbm.LBPMError):
        lbm.force_rescale((0, 0, 1e-5), **args)
