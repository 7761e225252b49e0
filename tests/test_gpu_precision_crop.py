"""The displacement protocol of the 1024^3 precision workload on a 128^3 domain
of the same recipe (GPU only): FP32 and FP16 storage against the FP64 oracle
after 500 steps. Spec bound for the FP16 form: saturation and Darcy flux
within 1e-3 relative of the oracle (the 5,000-step 128^3 crop of the full
workload is run by `bench.py --mode precision`)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    import oracle
    from synthetic import workload_precision1024
    w = workload_precision1024(128)
    kw = dict(tau_a=w.tau_a, tau_b=w.tau_b, alpha=w.alpha, beta=w.beta, force=w.force, periodic=w.periodic,
              reservoir_z=1, rho_in=w.rho_in, rho_out=w.rho_out)
    ref = oracle.Oracle(w.labels, w.affinity, w.periodic, **{k: v for k, v in kw.items() if k != "periodic"})
    ref.init_fluids(w.phi0)
    ref.step(500)
    return w, kw, ref.measure()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_displacement_crop_protocol_500_steps(case, precision):
    import paper_2007_12266_gb300 as lbm
    w, kw, mo = case
    d = lbm.Domain(w.labels, w.affinity, precision=precision, **kw)
    d.init_fluids(w.phi0)
    for _ in range(5):
        d.advance(100)                  # five calls: the sum form inside each, populations between
    m = d.measure()
    e_sw = abs(m["sat_mass"] / mo["sat_mass"] - 1)
    e_q = abs(m["flux"][2] / mo["flux_z"] - 1)
    print(f"{precision}: {d.n_sites} sites, 500 steps: Sw {m['sat_mass']:.6f} (err {e_sw:.2e}), "
          f"flux {m['flux'][2]:.4e} (err {e_q:.2e})")
    assert mo["sat_mass"] > 0.005          # fluid A has entered from the inlet
    assert e_sw <= 1e-3 and e_q <= 1e-3
    d.close()
