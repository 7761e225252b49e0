"""The sum form of lbpm_advance (components carried as per-site fixed-point
sums inside a call of two or more timesteps) against the FP64 oracle, and
against the population form (GPU only).

Tolerances: each fp32 timestep keeps every distribution within 1e-6
max(|o|, w_q) of the oracle's (the one-step bound of the population form);
a call of k steps is held to k times that, the errors of successive steps
adding at most linearly over so few steps. The sum form's component sums are
exact to 2^-28 per received value, finer than an fp32 population, so the
bound of the population form applies unchanged.
"""
import numpy as np
import pytest

from lbm_cases import compare_state, pair, random_state, set_both
from synthetic import random_affinity, sphere_pack, workload_parity32

pytestmark = pytest.mark.gpu

KW = dict(tau_a=0.7, tau_b=0.7, alpha=0.005, beta=0.95, force=(0.0, 0.0, 1e-5))


def _pack(shape, porosity, seed):
    nz, ny, nx = shape
    return sphere_pack((nx, ny, nz), porosity, 2.0, 0.6, seed).labels


CASES = [
    ("spherepack32", (1, 1, 1), dict(KW)),
    ("ragged_walls", (0, 1, 0), dict(tau_a=0.9, tau_b=0.6, alpha=0.02, beta=0.7, force=(2e-5, -1e-5, 3e-5))),
    ("closed_box", (0, 0, 0), dict(tau_a=0.55, tau_b=1.4, alpha=0.01, beta=0.95, force=(0.0, 1e-4, 0.0))),
    ("thin_periodic_column", (1, 1, 1), dict(KW)),
    # reservoir slabs: the reset writes the slab sites' sums inside a call
    ("reservoir_pack", (1, 1, 0), dict(KW, reservoir_z=1, rho_in=1.001, rho_out=0.999)),
]


def _case(name):
    if name == "spherepack32":
        w = workload_parity32()
        return w.labels, w.affinity
    if name == "ragged_walls":
        lab = _pack((7, 9, 13), 0.55, 3)
        return lab, random_affinity(lab, -1, 1, 4)
    if name == "closed_box":
        lab = _pack((6, 11, 5), 0.6, 8)
        return lab, random_affinity(lab, -0.9, 0.9, 9)
    if name == "reservoir_pack":
        lab = _pack((16, 8, 10), 0.55, 17)
        return lab, random_affinity(lab, -0.7, 0.7, 18)
    lab = np.zeros((11, 1, 1), np.uint16)     # x and y neighbours wrap onto the site itself
    return lab, None


@pytest.mark.parametrize("name,periodic,kw", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("start", [0, 1], ids=["even", "odd"])
@pytest.mark.parametrize("k", [2, 3, 5])
def test_sum_form_call_of_k_steps_matches_oracle(name, periodic, kw, start, k):
    lab, aff = _case(name)
    dom, ref = pair(lab, aff, periodic, **kw)
    set_both(dom, ref, random_state(ref, seed=31 + start + 7 * k), start)
    dom.advance(k)                       # first, k - 2 middle and last step of the sum form
    ref.step(k)
    ef, ea, eb = compare_state(dom, ref)
    assert max(ef, ea, eb) <= k * 1e-6, (ef, ea, eb)
    assert dom.step_count == ref.step_count == start + k


def test_sum_form_and_population_form_agree_with_oracle_over_a_run():
    """40 steps of the 32^3 parity workload as one call in each form, both
    against the oracle: the two forms differ only by fp32 rounding of the
    stored component populations."""
    import paper_2007_12266_gb300 as lbm
    w = workload_parity32()
    doms = {}
    for form in ("auto", "populations"):
        d = lbm.Domain(w.labels, w.affinity, periodic=w.periodic, **KW)
        d.set_step_form(form)
        d.init_fluids(w.phi0)
        d.advance(40)
        doms[form] = d
    _, ref = pair(w.labels, w.affinity, w.periodic, **KW)
    ref.init_fluids(w.phi0)
    ref.step(40)
    mo = ref.measure()
    for form, d in doms.items():
        m = d.measure()
        assert abs(m["sat_mass"] / mo["sat_mass"] - 1) <= 1e-5, form
        assert abs(m["flux"][2] / mo["flux_z"] - 1) <= 1e-3, form
        print(form, "per-distribution error after 40 steps", compare_state(d, ref))


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_sum_form_is_deterministic_and_conserves_component_mass(precision):
    """Integer sums do not depend on the order of the atomic additions: two
    runs are bit-identical. Within a call the component masses are conserved
    exactly; only the last step's fp32 (fp16) population store rounds them."""
    import paper_2007_12266_gb300 as lbm
    w = workload_parity32()
    runs = []
    for _ in range(2):
        d = lbm.Domain(w.labels, w.affinity, periodic=w.periodic, precision=precision, **KW)
        d.init_fluids(w.phi0)
        m0 = d.measure()
        d.advance(500)
        m1 = d.measure()
        runs.append((d.distributions("f"), d.distributions("a"), d.distributions("b"), m0, m1))
        d.close()
    for a, b in zip(runs[0][:3], runs[1][:3]):
        assert np.array_equal(a, b)
    m0, m1 = runs[0][3], runs[0][4]
    tol = 1e-7 if precision == "fp32" else 2e-6
    for key in ("mass_a", "mass_b"):
        assert abs(m1[key] / m0[key] - 1) < tol, (key, m1[key] / m0[key] - 1)


def test_population_form_is_selectable_and_rejects_unknown_forms():
    import paper_2007_12266_gb300 as lbm
    from paper_2007_12266_gb300 import _lib
    w = workload_parity32()
    d = lbm.Domain(w.labels, w.affinity, periodic=w.periodic, **KW)
    assert _lib.load().lbpm_set_step_form(d._h, 7) == 1
    d.set_step_form("populations")
    d.init_fluids(w.phi0)
    n0 = d.launch_count
    d.advance(4)
    assert d.launch_count - n0 == 8      # two kernels per step in either form
    d.close()
