"""CUDA path vs the FP64 oracle, through the C ABI (GPU only).

Tolerances (from the arithmetic of an fp32 step, see the design notes):
  * indexer: bit-exact (site numbering and all 18 neighbour lists);
  * one step from an identical state: |g - o| <= 1e-6 max(|o|, w_q) for every
    distribution (t_q for f), at both AA parities;
  * after 200 and 1,000 steps of the 32^3 two-phase case: saturation and
    Darcy flux within 1e-3 relative.
"""
import numpy as np
import pytest

import oracle
from lbm_cases import T19, W7, compare_state, pair, random_state, rel_err, set_both
from synthetic import (phi0_iid, random_affinity, sphere_pack, uniform_affinity,
                       workload_parity32)

pytestmark = pytest.mark.gpu

KW = dict(tau_a=0.7, tau_b=0.7, alpha=0.005, beta=0.95, force=(0.0, 0.0, 1e-5))


def _pack(shape, porosity, seed):
    nz, ny, nx = shape
    sp = sphere_pack((nx, ny, nz), porosity, 2.0, 0.6, seed)
    return sp.labels


INDEX_CASES = [
    ((8, 8, 8), (1, 1, 1)), ((7, 9, 13), (0, 1, 0)), ((5, 6, 7), (0, 0, 0)),
    ((16, 1, 16), (1, 1, 0)), ((1, 1, 11), (1, 1, 1)), ((12, 10, 9), (1, 0, 1)),
]


@pytest.mark.parametrize("shape,periodic", INDEX_CASES)
def test_index_bit_exact(shape, periodic):
    lab = _pack(shape, 0.5, sum(shape))
    dom, ref = pair(lab, None, periodic, **KW)
    sv, nb = dom.index()
    sv_o, nb_o = ref.index()
    assert sv.dtype == np.int64 and nb.dtype == np.int32
    assert np.array_equal(sv, sv_o)
    assert np.array_equal(nb, nb_o)


def test_index_bit_exact_parity_workload():
    w = workload_parity32()
    dom, ref = pair(w.labels, w.affinity, w.periodic, **KW)
    sv, nb = dom.index()
    sv_o, nb_o = ref.index()
    assert dom.n_sites == ref.N == len(sv)
    assert np.array_equal(sv, sv_o) and np.array_equal(nb, nb_o)


def test_init_state_matches_oracle():
    w = workload_parity32()
    dom, ref = pair(w.labels, w.affinity, w.periodic, **KW)
    dom.init_fluids(w.phi0)
    ref.init_fluids(w.phi0)
    ef, ea, eb = compare_state(dom, ref)
    assert max(ef, ea, eb) < 1e-7


STEP_CASES = [
    ("spherepack32", (1, 1, 1), dict(KW)),
    ("ragged_walls", (0, 1, 0), dict(tau_a=0.9, tau_b=0.6, alpha=0.02, beta=0.7,
                                     force=(2e-5, -1e-5, 3e-5))),
    ("closed_box", (0, 0, 0), dict(tau_a=0.55, tau_b=1.4, alpha=0.01, beta=0.95,
                                   force=(0.0, 1e-4, 0.0))),
]


def _case(name, periodic):
    if name == "spherepack32":
        w = workload_parity32()
        return w.labels, w.affinity
    if name == "ragged_walls":
        lab = _pack((7, 9, 13), 0.55, 3)
        return lab, random_affinity(lab, -1, 1, 4)
    lab = _pack((6, 11, 5), 0.6, 8)
    return lab, random_affinity(lab, -0.9, 0.9, 9)


@pytest.mark.parametrize("name,periodic,kw", STEP_CASES, ids=[c[0] for c in STEP_CASES])
@pytest.mark.parametrize("step", [0, 1], ids=["even", "odd"])
def test_one_step_from_identical_state(name, periodic, kw, step):
    lab, aff = _case(name, periodic)
    dom, ref = pair(lab, aff, periodic, **kw)
    state = random_state(ref, seed=11 + step)
    set_both(dom, ref, state, step)
    ef, ea, eb = compare_state(dom, ref)
    assert max(ef, ea, eb) == 0.0          # the loaded state is bit-identical
    dom.advance(1)
    ref.step(1)
    ef, ea, eb = compare_state(dom, ref)
    assert ef <= 1e-6 and ea <= 1e-6 and eb <= 1e-6, (ef, ea, eb)
    assert dom.step_count == ref.step_count == step + 1


def test_parity_workload_200_steps():
    w = workload_parity32()
    dom, ref = pair(w.labels, w.affinity, w.periodic, **KW)
    dom.init_fluids(w.phi0)
    ref.init_fluids(w.phi0)
    dom.advance(1)
    ref.step(1)
    ef, ea, eb = compare_state(dom, ref)
    assert max(ef, ea, eb) <= 1e-6
    dom.advance(199)
    ref.step(199)
    m, mo = dom.measure(), ref.measure()
    assert abs(m["sat_mass"] / mo["sat_mass"] - 1) <= 1e-3
    assert abs(m["flux"][2] / mo["flux_z"] - 1) <= 1e-3
    phi_o, _, _ = ref.fields()
    phi_g = dom.read_field("phi")
    sv, _ = ref.index()
    dphi = np.abs(phi_g.ravel()[sv] - phi_o)
    print(f"200 steps: max |dphi| {dphi.max():.2e}, per-dist err {compare_state(dom, ref)}")


def test_parity_workload_1000_steps():
    w = workload_parity32()
    dom, ref = pair(w.labels, w.affinity, w.periodic, **KW)
    dom.init_fluids(w.phi0)
    ref.init_fluids(w.phi0)
    dom.advance(1000)
    ref.step(1000)
    m, mo = dom.measure(), ref.measure()
    assert m["status"] == 0 and mo["status"] == 0
    assert abs(m["sat_mass"] / mo["sat_mass"] - 1) <= 1e-3
    for a, key in enumerate(("flux_x", "flux_y", "flux_z")):
        scale = max(abs(mo["flux_z"]), 1e-30)
        assert abs(m["flux"][a] - mo[key]) <= 1e-3 * scale, key
    print("1000 steps:", {k: (m[k], mo[k]) for k in ("sat_mass", "sat_count", "ca")})


def test_measures_match_oracle():
    w = workload_parity32()
    dom, ref = pair(w.labels, w.affinity, w.periodic, **KW)
    dom.init_fluids(w.phi0)
    ref.init_fluids(w.phi0)
    dom.advance(50)
    ref.step(50)
    m, mo = dom.measure(), ref.measure()
    assert m["step"] == mo["step"] == 50 and m["n_sites"] == mo["n_sites"]
    # sums of the fp32 state formed to fp64 accuracy: each component is
    # conserved exactly inside a call of the sum form and to unbiased fp32
    # rounding by the population stores of its first and last step, so the
    # component totals agree with the oracle's to about 1e-9 relative (measured
    # 5e-11 on Sw, 9e-10 on the masses; gate 1e-8). The momentum populations'
    # total Sum rho carries the fp32 rounding of every collision (measured
    # 1.7e-8 after 50 steps; gate 1e-7), and so do the pressures of the two
    # regions phi > 0 / phi < 0 (same gate, as long as the regions hold the
    # same sites).
    for k, tol in (("sat_mass", 1e-8), ("mass_a", 1e-8), ("mass_b", 1e-8), ("mass_total", 1e-7),
                   ("p_a", 1e-7), ("p_b", 1e-7)):
        print(k, abs(m[k] / mo[k] - 1))
        assert abs(m[k] - mo[k]) <= tol * abs(mo[k]), k
    for k in ("sat_count", "vol_a", "vol_b"):
        assert abs(m[k] - mo[k]) <= 1e-3 * abs(mo[k]) + 2, k
    for k in ("flux", "flux_a", "flux_b", "mom_a", "mom_b"):
        for a, ax in enumerate("xyz"):
            ref_v = mo[f"{k}_{ax}"]
            scale = max(abs(mo[f"{k}_z"]), 1e-12)
            assert abs(m[k][a] - ref_v) <= 2e-3 * scale, (k, ax)
    assert abs(m["ca"] - mo["ca"]) <= 2e-3 * mo["ca"]


def test_read_fields_match_oracle():
    w = workload_parity32()
    dom, ref = pair(w.labels, w.affinity, w.periodic, **KW)
    dom.init_fluids(w.phi0)
    ref.init_fluids(w.phi0)
    dom.advance(3)
    ref.step(3)
    phi, p, u = ref.fields()
    sv, _ = ref.index()
    pore = np.zeros(w.labels.size, bool)
    pore[sv] = True
    for name, val, tol in (("phi", phi, 2e-6), ("pressure", p, 1e-6 * p.max()), ("ux", u[0], 2e-7),
                           ("uy", u[1], 2e-7), ("uz", u[2], 2e-7)):
        g = dom.read_field(name).ravel()
        assert np.isnan(g[~pore]).all()
        assert np.abs(g[sv] - val).max() <= tol, name


def test_mass_conservation_fp32():
    w = workload_parity32()
    dom, _ = pair(w.labels, w.affinity, w.periodic, **KW)
    dom.init_fluids(w.phi0)
    m0 = dom.measure()
    dom.advance(1000)
    m1 = dom.measure()
    for k in ("mass_a", "mass_b", "mass_total"):
        assert abs(m1[k] / m0[k] - 1) < 2e-6, k


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_reservoir_slabs_parity(precision):
    sp = sphere_pack((12, 10, 24), 0.55, 2.0, 0.5, 17)
    lab = sp.labels
    aff = uniform_affinity(lab, -0.7)
    kw = dict(KW, reservoir_z=1, rho_in=1.001, rho_out=0.999)
    per = (1, 1, 0)
    dom, ref = pair(lab, aff, per, precision=precision, **kw)
    phi0 = np.full(lab.shape, -1.0, np.float32)
    dom.init_fluids(phi0)
    ref.init_fluids(phi0)
    if precision == "fp32":
        assert max(compare_state(dom, ref)) < 1e-7
        for _ in range(3):
            dom.advance(1)
            ref.step(1)
            assert max(compare_state(dom, ref)) <= 1e-6
    else:
        # one step from what the fp16 store holds, at both parities, within
        # the storage bounds of the fp16 one-step test (the slab reset writes
        # its rest state through the same component references)
        ef, ea, eb = compare_state(dom, ref)
        assert ef < 5e-5 and max(ea, eb) < 2e-3
        for step in range(3):
            held = [dom.distributions(k).astype(np.float64) for k in ("f", "a", "b")]
            ref.set_state(*held, step=step)
            dom.advance(1)
            ref.step(1)
            f, A, B = ref.state()
            assert (np.abs(dom.distributions("f") - f) / T19[:, None]).max() < 5e-5, step
            assert rel_err(dom.distributions("a"), A, W7).max() < 2e-3, step
            assert rel_err(dom.distributions("b"), B, W7).max() < 2e-3, step
    dom.advance(197)
    ref.step(197)
    m, mo = dom.measure(), ref.measure()
    assert abs(m["sat_mass"] / mo["sat_mass"] - 1) <= 1e-3
    assert mo["sat_mass"] > 0.05     # fluid A entered from the inlet


@pytest.mark.parametrize("precision,mode", [("fp32", 2), ("fp16", 2), ("fp32", 3), ("fp16", 3)])
def test_pressure_faces_parity(precision, mode):
    """Pressure boundary at the z faces (reservoir_z = 2) and flux inlet
    (reservoir_z = 3) against the oracle: every distribution over the first
    steps (fp32), then saturation and the Darcy flux after 200 steps."""
    sp = sphere_pack((12, 10, 24), 0.55, 2.0, 0.5, 19)
    lab = sp.labels
    aff = uniform_affinity(lab, -0.7)
    kw = dict(KW, reservoir_z=mode, rho_in=1.002, rho_out=0.998, flux_in=0.2)
    per = (1, 1, 0)
    dom, ref = pair(lab, aff, per, precision=precision, **kw)
    phi0 = np.full(lab.shape, -1.0, np.float32)
    dom.init_fluids(phi0)
    ref.init_fluids(phi0)
    tol = 1e-6 if precision == "fp32" else 2e-3
    if precision == "fp32":
        assert max(compare_state(dom, ref)) < 1e-7
        for _ in range(3):
            dom.advance(1)
            ref.step(1)
            assert max(compare_state(dom, ref)) <= tol
        dom.advance(197)
        ref.step(197)
    else:
        dom.advance(200)
        ref.step(200)
    m, mo = dom.measure(), ref.measure()
    assert abs(m["sat_mass"] / mo["sat_mass"] - 1) <= 1e-3
    assert abs(m["flux"][2] / mo["flux_z"] - 1) <= 1e-3
    # fluid A entered at the inlet (the pack is B-wet, phi_s = -0.7: capillary
    # pressure, not the small face pressure difference, sets the early flux)
    assert mo["sat_mass"] > 0.02


def test_snapshot_restore_is_bit_exact():
    w = workload_parity32()
    import paper_2007_12266_gb300 as lbm
    dom = lbm.Domain(w.labels, w.affinity, periodic=w.periodic, **KW)
    dom.init_fluids(w.phi0)
    dom.advance(11)
    snap = dom.snapshot()
    dom.advance(7)
    f1 = dom.distributions("f")
    a1 = dom.distributions("a")
    dom.restore(snap)
    assert dom.step_count == 11
    dom.advance(7)
    assert np.array_equal(dom.distributions("f"), f1)
    assert np.array_equal(dom.distributions("a"), a1)


def test_unstable_state_is_reported():
    """Host-side fault injection: a NaN written into the state is caught by the
    measure pass, and advance refuses to continue until re-initialised."""
    import paper_2007_12266_gb300 as lbm
    lab = _pack((8, 8, 8), 0.6, 2)
    dom = lbm.Domain(lab, None, **KW)
    dom.init_fluids(np.ones(lab.shape, np.float32))
    f = dom.distributions("f")
    f[3, 5] = np.nan
    dom.write_distributions("f", f)
    m = dom.measure()
    assert m["status"] & 1
    with pytest.raises(lbm.LBPMError):
        dom.advance(1)
    dom.init_fluids(np.ones(lab.shape, np.float32))
    dom.advance(2)
    assert dom.measure()["status"] == 0


def test_edge_cases():
    import paper_2007_12266_gb300 as lbm
    # a single pore voxel: every link bounces back
    lab = np.ones((3, 3, 3), np.uint16)
    lab[1, 1, 1] = 0
    dom, ref = pair(lab, uniform_affinity(lab, 0.3), (0, 0, 0), **KW)
    assert dom.n_sites == 1
    phi0 = np.zeros(lab.shape, np.float32)
    dom.init_fluids(phi0)
    ref.init_fluids(phi0)
    for _ in range(4):
        dom.advance(1)
        ref.step(1)
        assert max(compare_state(dom, ref)) <= 1e-6
    # an all-pore periodic box of odd sizes (N not a multiple of the block)
    lab = np.zeros((5, 3, 7), np.uint16)
    dom, ref = pair(lab, None, (1, 1, 1), **KW)
    assert dom.n_sites == 105
    st = random_state(ref, 3)
    set_both(dom, ref, st, 0)
    dom.advance(2)
    ref.step(2)
    assert max(compare_state(dom, ref)) <= 1e-6
    # no pore voxel, bad parameters, mismatched inputs
    with pytest.raises(lbm.LBPMError) as e:
        lbm.Domain(np.ones((4, 4, 4), np.uint16))
    assert e.value.status == 1
    for bad in (dict(tau_a=0.5), dict(alpha=-1.0), dict(beta=-0.1), dict(force=(np.nan, 0, 0))):
        kw = dict(KW)
        kw.update(bad)
        with pytest.raises(lbm.LBPMError):
            lbm.Domain(np.zeros((4, 4, 4), np.uint16), **kw)
    with pytest.raises(lbm.LBPMError):
        lbm.Domain(np.zeros((4, 4, 4), np.uint16), periodic=(1, 1, 1), reservoir_z=1, **KW)
    dom = lbm.Domain(np.zeros((4, 4, 4), np.uint16), **KW)
    with pytest.raises(lbm.LBPMError):
        dom.advance(1)                               # no fluids yet
    with pytest.raises(lbm.LBPMError):
        dom.restore(b"\0" * 40)                      # corrupt snapshot


DEGENERATE = [
    ("thin_periodic_column", (11, 1, 1), (1, 1, 1)),   # x and y neighbours wrap onto the site itself
    ("two_voxel_slab", (9, 1, 2), (1, 1, 0)),          # z walls, x of width 2, y of width 1
    ("single_pore", (3, 3, 3), (0, 0, 0)),             # every link bounces back
]


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("name,shape,periodic", DEGENERATE, ids=[c[0] for c in DEGENERATE])
def test_degenerate_domains_one_step(name, shape, periodic, precision):
    """One even and one odd step on domains whose neighbours are the site
    itself or solid on most links, from the same state on both sides: FP32
    within 1e-6 max(|o|, w_q); FP16 from the state its store holds, within
    the bounds of the fp16 one-step test."""
    lab = np.zeros(shape, np.uint16)
    if name == "single_pore":
        lab[:] = 1
        lab[1, 1, 1] = 0
    aff = uniform_affinity(lab, 0.3)
    dom, ref = pair(lab, aff, periodic, precision=precision, **KW)
    for step in (0, 1):
        st = random_state(ref, seed=11 + step, amp=0.02)
        set_both(dom, ref, st, step)
        if precision == "fp16":
            held = [dom.distributions(k).astype(np.float64) for k in ("f", "a", "b")]
            ref.set_state(*held, step=step)
        dom.advance(1)
        ref.step(1)
        if precision == "fp32":
            assert max(compare_state(dom, ref)) <= 1e-6, step
        else:
            f, A, B = ref.state()
            assert (np.abs(dom.distributions("f") - f) / T19[:, None]).max() < 5e-5, step
            assert rel_err(dom.distributions("a"), A, W7).max() < 2e-3, step
            assert rel_err(dom.distributions("b"), B, W7).max() < 2e-3, step


def test_full_size_steady256_two_steps():
    """The bench workload (256^3 pack, 3.6 M sites) at full size: bit-exact
    index, then one even and one odd step against the oracle at every site."""
    from synthetic import workload_steady256
    w = workload_steady256()
    dom, ref = pair(w.labels, w.affinity, w.periodic, tau_a=w.tau_a, tau_b=w.tau_b,
                    alpha=w.alpha, beta=w.beta, force=w.force)
    sv, nb = dom.index()
    sv_o, nb_o = ref.index()
    assert np.array_equal(sv, sv_o) and np.array_equal(nb, nb_o)
    del nb, nb_o
    dom.init_fluids(w.phi0)
    ref.init_fluids(w.phi0)
    for _ in range(2):
        dom.advance(1)
        ref.step(1)
        ef, ea, eb = compare_state(dom, ref)
        assert max(ef, ea, eb) <= 1e-6, (ef, ea, eb)


def test_full_size_steady256_fp16_two_steps():
    """The bench workload with fp16 storage: after init and after each of one
    even and one odd step, the oracle restarts from what the fp16 store holds
    and one step of both must agree at every site within the storage
    precision. fp16 rounds a stored deviation to 2^-11 of itself; the first
    steps from the sharp blob interfaces leave deviations f_q - t_q rho of up
    to 0.17 t_q, so f is held to 2^-10 times the largest deviation of the
    step's result (twice the half-ulp, for the rounding of the inputs carried
    through one collision); A and B to the 2e-3 (floor w_q) of the 32^3 test."""
    from synthetic import workload_steady256
    w = workload_steady256()
    dom, ref = pair(w.labels, w.affinity, w.periodic, tau_a=w.tau_a, tau_b=w.tau_b,
                    alpha=w.alpha, beta=w.beta, force=w.force, precision="fp16")
    dom.init_fluids(w.phi0)
    for step in (0, 1):
        held = [dom.distributions(k).astype(np.float64) for k in ("f", "a", "b")]
        ref.set_state(*held, step=step)
        dom.advance(1)
        ref.step(1)
        f, A, B = ref.state()
        dev = (np.abs(f - T19[:, None] * f.sum(axis=0)) / T19[:, None]).max()
        ef = np.abs(dom.distributions("f") - f) / T19[:, None]
        print(f"fp16 full size, step {step}: max |f - o| / t_q = {ef.max():.3e}, bound {2.0 ** -10 * dev:.3e}")
        assert ef.max() < 2.0 ** -10 * dev, (step, ef.max(), dev)
        assert rel_err(dom.distributions("a"), A, W7).max() < 2e-3, step
        assert rel_err(dom.distributions("b"), B, W7).max() < 2e-3, step


def test_graph_bundles_match_plain_launches():
    """advance() replays captured step bundles; with kernel timing on it
    launches every kernel on its own. Both orders of work are the same, so the
    states must be bit-identical, from an even and from an odd start."""
    import paper_2007_12266_gb300 as lbm
    w = workload_parity32()
    doms = []
    for timing in (False, True):
        d = lbm.Domain(w.labels, w.affinity, periodic=w.periodic, **KW)
        d.enable_kernel_timing(timing)
        d.init_fluids(w.phi0)
        d.advance(1)
        d.advance(37)
        d.advance(18)
        doms.append(d)
    for which in ("f", "a", "b"):
        assert np.array_equal(doms[0].distributions(which), doms[1].distributions(which))
    assert doms[0].step_count == doms[1].step_count == 56
