"""FP16-storage form of the step against the FP64 oracle (GPU only).

Populations are stored in fp16 as deviations from a local rest-state
equilibrium (f_q - t_q rho, A_q - w_q (1 + phi)/2, B_q - w_q (1 - phi)/2 of a
reference site);
all arithmetic is fp32. The targets: saturation and Darcy flux within 1e-3
relative of the oracle; one step within fp16 storage precision.
"""
import numpy as np
import pytest

from lbm_cases import T19, W7, pair, random_state, rel_err, set_both
from synthetic import workload_parity32

pytestmark = pytest.mark.gpu

KW = dict(tau_a=0.7, tau_b=0.7, alpha=0.005, beta=0.95, force=(0.0, 0.0, 1e-5))


def test_fp16_one_step_within_storage_precision():
    w = workload_parity32()
    dom, ref = pair(w.labels, w.affinity, w.periodic, precision="fp16", **KW)
    for step in (0, 1):
        st = random_state(ref, seed=5 + step, amp=0.02)
        set_both(dom, ref, st, step)
        # what the fp16 store holds of the loaded state
        f0 = dom.distributions("f").astype(np.float64)
        a0 = dom.distributions("a").astype(np.float64)
        b0 = dom.distributions("b").astype(np.float64)
        ref.set_state(f0, a0, b0, step=step)
        dom.advance(1)
        ref.step(1)
        f, A, B = ref.state()
        # the stored numbers are deviations of at most a few 1e-2 t_q from a
        # local rest state, rounded to 2^-11 relative
        ef = np.abs(dom.distributions("f") - f) / T19[:, None]
        assert ef.max() < 5e-5, ef.max()
        assert rel_err(dom.distributions("a"), A, W7).max() < 2e-3
        assert rel_err(dom.distributions("b"), B, W7).max() < 2e-3


@pytest.mark.parametrize("steps", [200, 1000])
def test_fp16_saturation_and_flux(steps):
    w = workload_parity32()
    dom, ref = pair(w.labels, w.affinity, w.periodic, precision="fp16", **KW)
    dom.init_fluids(w.phi0)
    ref.init_fluids(w.phi0)
    dom.advance(steps)
    ref.step(steps)
    m, mo = dom.measure(), ref.measure()
    e_sw = abs(m["sat_mass"] / mo["sat_mass"] - 1)
    e_q = abs(m["flux"][2] / mo["flux_z"] - 1)
    print(f"fp16 {steps} steps: Sw err {e_sw:.2e}, flux err {e_q:.2e}, "
          f"mass drift {m['mass_a'] + m['mass_b'] - mo['mass_a'] - mo['mass_b']:.2e}")
    assert e_sw <= 1e-3 and e_q <= 1e-3
    # total N = Na + Nb: fp16 rounding only (the fp32 weights' excess over 1,
    # 2^-26 per step, is compensated in the rest populations)
    tot, tot_o = m["mass_a"] + m["mass_b"], mo["mass_a"] + mo["mass_b"]
    assert abs(tot / tot_o - 1) <= 1e-5, tot / tot_o - 1
