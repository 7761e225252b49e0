"""The displacement workload at its full size (1024^3 voxels, 214.7 M pore
sites) against the FP64 oracle, sampled (GPU only).

The oracle cannot hold the full domain, so the check samples it: the library
runs the whole domain with the launch configuration of the benchmark for 300
steps, so that fluid A has entered from the inlet reservoir; a 48^3 box next
to the inlet (z from 4, above the reservoir slab) is read back (lbpm_read_box)
before and after each of one even and one odd step; the oracle, restarted
from the box's state as a domain of its own, takes the same step. One step
only reaches two voxels (the phase stencil, then streaming), so every site at
least two voxels inside the box must agree with the oracle within the
one-step tolerance of the storage: FP32 1e-6 max(|o|, w_q) (t_q for f); FP16
twice fp16's half-ulp of the largest stored deviation on f, 2e-3 (floor w_q)
on A and B.
"""
import numpy as np
import pytest

import oracle
from lbm_cases import T19, W7, rel_err
from synthetic import crop, workload_parity32, workload_precision1024

pytestmark = pytest.mark.gpu

BOX_LO, BOX_HI = (488, 488, 4), (536, 536, 52)   # x, y, z bounds
WARM_STEPS = 300
MARGIN = 2


def _box_sites(lab_box):
    """Pore voxels of a [z][y][x] label box in the library's site order."""
    return (lab_box == 0).ravel()


def test_read_box_equals_the_distributions_of_its_sites():
    import paper_2007_12266_gb300 as lbm
    w = workload_parity32()
    dom = lbm.Domain(w.labels, w.affinity, periodic=w.periodic, tau_a=0.7, tau_b=0.7, alpha=0.005,
                     beta=0.95, force=(0.0, 0.0, 1e-5))
    dom.init_fluids(w.phi0)
    dom.advance(3)                               # odd parity: the read map applies
    sv, _ = dom.index()
    nz, ny, nx = w.labels.shape
    lo, hi = (3, 5, 7), (30, 21, 32)
    for which in ("f", "a", "b"):
        full = dom.distributions(which)
        box = dom.read_box(which, lo, hi)
        Q = full.shape[0]
        assert box.shape == (Q, hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0])
        x, y, z = sv % nx, (sv // nx) % ny, sv // (nx * ny)
        inside = (x >= lo[0]) & (x < hi[0]) & (y >= lo[1]) & (y < hi[1]) & (z >= lo[2]) & (z < hi[2])
        got = box[:, z[inside] - lo[2], y[inside] - lo[1], x[inside] - lo[0]]
        assert np.array_equal(got, full[:, inside])
        solid = crop(w.labels, lo, hi) != 0
        assert np.isnan(box[:, solid]).all()
    with pytest.raises(lbm.LBPMError):
        dom.read_box("f", (0, 0, 0), (33, 4, 4))  # outside the image


@pytest.fixture(scope="module")
def displacement1024():
    return workload_precision1024()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_displacement1024_one_step_at_every_site_of_a_box(displacement1024, precision):
    import paper_2007_12266_gb300 as lbm
    w = displacement1024
    kw = dict(tau_a=w.tau_a, tau_b=w.tau_b, alpha=w.alpha, beta=w.beta, force=w.force)
    dom = lbm.Domain(w.labels, w.affinity, periodic=w.periodic, reservoir_z=w.reservoir_z,
                     rho_in=w.rho_in, rho_out=w.rho_out, precision=precision, **kw)
    dom.init_fluids(w.phi0)
    dom.advance(WARM_STEPS)
    lab_b, aff_b = crop(w.labels, BOX_LO, BOX_HI), crop(w.affinity, BOX_LO, BOX_HI)
    pore = _box_sites(lab_b)
    # sites at least MARGIN voxels inside the box, in the box's site order
    inner = np.zeros(lab_b.shape, bool)
    inner[MARGIN:-MARGIN, MARGIN:-MARGIN, MARGIN:-MARGIN] = True
    inner = inner.ravel()[pore]
    assert inner.sum() > 2000
    ref = oracle.Oracle(lab_b, aff_b, (0, 0, 0), **kw)
    for step in (0, 1):
        held = [dom.read_box(k, BOX_LO, BOX_HI).reshape(q, -1)[:, pore].astype(np.float64)
                for k, q in (("f", 19), ("a", 7), ("b", 7))]
        if step == 0:
            Na, Nb = held[1][:, inner].sum(axis=0), held[2][:, inner].sum(axis=0)
            n_if = np.count_nonzero(np.abs((Na - Nb) / (Na + Nb)) < 0.5)
            print(f"{precision}: {inner.sum()} sites compared, {n_if} of them at an interface")
            assert n_if > 20   # interfaces are sampled
        ref.set_state(*held, step=WARM_STEPS + step)
        dom.advance(1)
        ref.step(1)
        f, A, B = (v[:, inner] for v in ref.state())
        g = [dom.read_box(k, BOX_LO, BOX_HI).reshape(q, -1)[:, pore][:, inner]
             for k, q in (("f", 19), ("a", 7), ("b", 7))]
        if precision == "fp32":
            assert rel_err(g[0], f, T19).max() <= 1e-6, step
            assert rel_err(g[1], A, W7).max() <= 1e-6, step
            assert rel_err(g[2], B, W7).max() <= 1e-6, step
        else:
            dev = (np.abs(f - T19[:, None] * f.sum(axis=0)) / T19[:, None]).max()
            ef = np.abs(g[0] - f) / T19[:, None]
            assert ef.max() < 2.0 ** -10 * max(dev, 1e-2), (step, ef.max(), dev)
            assert rel_err(g[1], A, W7).max() < 2e-3, step
            assert rel_err(g[2], B, W7).max() < 2e-3, step
    dom.close()
