"""Batched form: several jobs in one persistent launch per phase (GPU only).

Each site runs the same device functions whether its domain is advanced
alone or inside a batch; the batched and single-domain kernels are compiled
in separate translation units, where the compiler may contract a*b + c into
fused multiply-adds differently, so the two agree to fp32 round-off rather
than bit for bit (two runs through the batch kernels are bit-identical, see
the serving tests). The batched fp64 measures sum in another order.
"""
import numpy as np
import pytest

from lbm_cases import T19, W7

from synthetic import phi0_blob, phi0_iid, random_affinity, sphere_pack, uniform_affinity

pytestmark = pytest.mark.gpu


def _jobs():
    """Uneven jobs: sizes, periodicities, wetting, tau, force and a reservoir job."""
    specs = []
    for j, (L, por, per, kw) in enumerate([
            ((24, 20, 28), 0.35, (1, 1, 1), dict(tau_a=0.7, tau_b=0.7, force=(0, 0, 1e-5))),
            ((16, 16, 16), 0.45, (0, 0, 1), dict(tau_a=0.9, tau_b=0.6, force=(0, 1e-5, 2e-5))),
            ((40, 12, 20), 0.30, (1, 0, 1), dict(tau_a=0.8, tau_b=0.8, force=(3e-5, 0, 0))),
            ((12, 14, 30), 0.50, (1, 1, 0), dict(tau_a=0.7, tau_b=0.7, force=(0, 0, 2e-5),
                                                 reservoir_z=1, rho_in=1.001, rho_out=0.999))]):
        sp = sphere_pack(L, por, 2.5, 0.8, 40 + j)
        lab = sp.labels
        aff = random_affinity(lab, -0.8, 0.8, 60 + j)
        phi0 = phi0_blob(lab, 0.45, 70 + j, sigma=2.0) if j % 2 else phi0_iid(lab, 0.5, 80 + j)
        kw = dict(kw, alpha=0.005, beta=0.95)
        specs.append((lab, aff, phi0, per, kw))
    return specs


def _make(spec, precision):
    import paper_2007_12266_gb300 as lbm
    lab, aff, phi0, per, kw = spec
    d = lbm.Domain(lab, aff, periodic=per, precision=precision, **kw)
    d.init_fluids(phi0)
    return d


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_batch_matches_alone(precision):
    import paper_2007_12266_gb300 as lbm
    specs = _jobs()
    alone = [_make(s, precision) for s in specs]
    batched = [_make(s, precision) for s in specs]
    b = lbm.Batch()
    for d in batched:
        b.add(d)
    b.advance(10)
    b.advance(14)
    for d in alone:
        # the same calls: a call boundary stores the components as populations
        # (fp16 rounding in FP16 storage), the steps inside a call carry sums
        d.advance(10)
        d.advance(14)
    for da, db in zip(alone, batched):
        assert db.step_count == 24
        for which, floor in (("f", T19), ("a", W7), ("b", W7)):
            ga, gb = da.distributions(which).astype(np.float64), db.distributions(which).astype(np.float64)
            err = np.abs(ga - gb) / np.maximum(np.abs(ga), floor[:, None])
            assert err.max() <= 1e-5, (which, err.max())
    # measures: batched fp64 reduction vs per-job reduction
    mb = b.measure()
    for d, m in zip(alone, mb):
        mo = d.measure()
        for k in ("sat_mass", "mass_a", "mass_b", "mass_total", "p_a", "p_b"):
            assert abs(m[k] - mo[k]) <= 1e-6 * max(abs(mo[k]), 1e-30), k
        assert abs(m["vol_a"] - mo["vol_a"]) <= 2
        for k in ("flux", "mom_a", "mom_b"):
            scale = max(np.abs(mo[k]).max(), 1e-30)
            assert np.abs(np.array(m[k]) - np.array(mo[k])).max() <= 1e-4 * scale, k
    b.close()


@pytest.mark.parametrize("mode", ["launches", "fused"])
@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_batched_jobs_match_the_oracle(precision, mode):
    """Every job of the uneven set (three periodicities, two viscosity pairs,
    a reservoir job) advanced in one batch against its own FP64 oracle: one
    even plus one odd step per distribution (FP32: 2 x 1e-6 max(|o|, w_q),
    one-step bound per step; FP16: from what its store holds, twice the
    storage bounds of the FP16 one-step test), then saturation and Darcy flux
    within 1e-3 after 200 steps; in FP16 saturation only: these jobs hold 1.8 k
    to 7 k pore sites, too few for the fp16 rounding of each site's velocity
    (about 2^-11 of the populations' deviations from the rest state) to
    average out of the Darcy flux (measured 1.3e-3 to 2.9e-3 relative after 200
    and 1,000 steps). The FP16 flux bound is checked on jobs of the batched
    workload's size below."""
    import oracle
    import paper_2007_12266_gb300 as lbm
    specs = _jobs()
    doms = [_make(s, precision) for s in specs]
    refs = []
    for (lab, aff, phi0, per, kw), d in zip(specs, doms):
        o = oracle.Oracle(lab, aff, per, **kw)
        if precision == "fp32":
            o.init_fluids(phi0)
        else:
            o.set_state(*[d.distributions(k).astype(np.float64) for k in ("f", "a", "b")], step=0)
        refs.append(o)
    b = lbm.Batch()
    for d in doms:
        b.add(d)
    if mode == "fused":
        b.set_launch(256, -2, -2)
    b.advance(2)
    for j, (d, o) in enumerate(zip(doms, refs)):
        o.step(2)
        f, A, B = o.state()
        if precision == "fp32":
            for which, ref, floor in (("f", f, T19), ("a", A, W7), ("b", B, W7)):
                g = d.distributions(which).astype(np.float64)
                err = np.abs(g - ref) / np.maximum(np.abs(ref), floor[:, None])
                assert err.max() <= 2e-6, (j, which, err.max())
        else:
            ef = np.abs(d.distributions("f") - f) / T19[:, None]
            assert ef.max() < 2 * 5e-5, (j, ef.max())
            for which, ref in (("a", A), ("b", B)):
                g = d.distributions(which).astype(np.float64)
                assert (np.abs(g - ref) / np.maximum(np.abs(ref), W7[:, None])).max() < 2 * 2e-3, (j, which)
    b.advance(198)
    for j, (m, o) in enumerate(zip(b.measure(), refs)):
        o.step(198)
        mo = o.measure()
        assert m["step"] == mo["step"] == 200
        assert abs(m["sat_mass"] / mo["sat_mass"] - 1) <= 1e-3, (j, m["sat_mass"], mo["sat_mass"])
        if precision == "fp16":
            continue
        # the flux along each job's drive (z, or x for the job driven along x)
        a = int(np.argmax(np.abs(specs[j][4]["force"]))) if j != 3 else 2
        key = "flux_" + "xyz"[a]
        assert abs(m["flux"][a] - mo[key]) <= 1e-3 * abs(mo[key]), (j, m["flux"][a], mo[key])
    b.close()


def test_batched_fp16_jobs_of_the_batched_workload_match_the_oracle():
    """FP16 storage, batched: three jobs of the 64-job batched workload (its
    64^3 class: sphere packs of porosity 0.15-0.35, x/y walls, own affinity,
    saturation and force) in one batch, 1,000 steps, against the FP64 oracle:
    saturation and Darcy flux within 1e-3 (the benchmark spec's bound of the FP16
    form)."""
    import oracle
    import paper_2007_12266_gb300 as lbm
    from synthetic import workload_batched_job
    ws = [workload_batched_job(j) for j in (7, 8, 12)]
    doms, refs = [], []
    b = lbm.Batch()
    for w in ws:
        kw = dict(tau_a=w.tau_a, tau_b=w.tau_b, alpha=w.alpha, beta=w.beta, force=w.force)
        d = lbm.Domain(w.labels, w.affinity, periodic=w.periodic, precision="fp16", **kw)
        d.init_fluids(w.phi0)
        o = oracle.Oracle(w.labels, w.affinity, w.periodic, **kw)
        o.init_fluids(w.phi0)
        b.add(d)
        doms.append(d)
        refs.append(o)
    b.advance(1000)
    for j, (m, o) in enumerate(zip(b.measure(), refs)):
        o.step(1000)
        mo = o.measure()
        e_sw, e_q = abs(m["sat_mass"] / mo["sat_mass"] - 1), abs(m["flux"][2] / mo["flux_z"] - 1)
        print(f"job {j}: {doms[j].n_sites} sites, Sw err {e_sw:.2e}, flux err {e_q:.2e}")
        assert e_sw <= 1e-3 and e_q <= 1e-3, (j, e_sw, e_q)
    b.close()


def test_batch_membership_and_tuner():
    import paper_2007_12266_gb300 as lbm
    specs = _jobs()[:3]
    alone = [_make(s, "fp32") for s in specs]
    batched = [_make(s, "fp32") for s in specs]
    b = lbm.Batch()
    for d in batched[:2]:
        b.add(d)
    b.advance(6)
    b.add(batched[2])              # joins at step 0 while the others are at 6
    threads, p, c = b.tune(steps_per_candidate=2)
    assert threads in (128, 192, 256, 512) and (p in (-1, -2) or p >= 1) and (c in (-1, -2) or c >= 1)
    b.remove(batched[0])
    b.advance(4)
    batched[0].advance(8)          # continues alone
    steps = [d.step_count for d in batched]
    for d, n in zip(alone, steps):
        d.advance(n)
    for da, db in zip(alone, batched):
        for which, floor in (("f", T19), ("b", W7)):
            ga, gb = da.distributions(which).astype(np.float64), db.distributions(which).astype(np.float64)
            err = np.abs(ga - gb) / np.maximum(np.abs(ga), floor[:, None])
            assert err.max() <= 1e-5, (which, err.max())
    b.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_launch_shapes_give_identical_results(precision):
    """Every launch shape the tuner may pick computes the same thing: persistent
    grids of any size and one block per tile, at 128, 192, 256 or 512 threads."""
    import paper_2007_12266_gb300 as lbm
    specs = _jobs()
    results = []
    for threads, bps in ((256, 0), (256, -1), (128, 1), (192, -1), (192, 2), (512, -1)):
        doms = [_make(s, precision) for s in specs]
        b = lbm.Batch()
        for d in doms:
            b.add(d)
        b.set_launch(threads, bps, bps)
        b.advance(8)
        results.append([d.distributions("f").copy() for d in doms])
        b.close()
        for d in doms:
            d.close()
    for other in results[1:]:
        for a, o in zip(results[0], other):
            assert np.array_equal(a, o)


def test_more_jobs_than_one_launch_table():
    """A batch larger than one launch's job table (128 jobs) runs as several
    launches per kernel; every job still matches its own run."""
    import paper_2007_12266_gb300 as lbm
    rng = np.random.default_rng(9)
    jobs = []
    for j in range(131):
        L = (6 + j % 3, 7, 5 + j % 4)
        lab = np.where(rng.uniform(size=L[::-1]) < 0.2, 1, 0).astype(np.uint16)
        aff = uniform_affinity(lab, -0.3)
        phi0 = phi0_iid(lab, 0.5, 300 + j)
        jobs.append((lab, aff, phi0))
    kw = dict(periodic=(1, 1, 1), tau_a=0.7, tau_b=0.7, alpha=0.005, beta=0.95, force=(0, 0, 1e-5))
    doms, alone = [], []
    for lab, aff, phi0 in jobs:
        for lst in (doms, alone):
            d = lbm.Domain(lab, aff, **kw)
            d.init_fluids(phi0)
            lst.append(d)
    b = lbm.Batch()
    for d in doms:
        b.add(d)
    b.set_launch(256, -1, -1)
    b.advance(6)
    for da, db in zip(alone, doms):
        da.advance(6)
        ga, gb = da.distributions("f").astype(np.float64), db.distributions("f").astype(np.float64)
        err = np.abs(ga - gb) / np.maximum(np.abs(ga), T19[:, None])
        assert err.max() <= 1e-5
    b.close()
    for d in doms + alone:
        d.close()


def test_batch_rejects_bad_jobs():
    import paper_2007_12266_gb300 as lbm
    specs = _jobs()
    b = lbm.Batch()
    d32 = _make(specs[0], "fp32")
    d16 = _make(specs[1], "fp16")
    b.add(d32)
    with pytest.raises(lbm.LBPMError):
        b.add(d16)                 # another precision
    odd = _make(specs[2], "fp32")
    odd.advance(1)
    with pytest.raises(lbm.LBPMError):
        b.add(odd)                 # odd step
    with pytest.raises(lbm.LBPMError):
        b.advance(3)               # bundles are even
    b.close()


@pytest.mark.parametrize("form", ["auto", "populations"])
@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_fused_kernel_matches_separate_launches(precision, form):
    """The fused persistent kernel (one cooperative launch per bundle: phase
    pass, collision and reservoir reset of every job, grid barriers between the
    passes) against the separate launches, on the uneven set with its reservoir
    job, in both step forms and at 128, 192 and 256 threads: the same device
    functions compiled into another kernel, so agreement to fp32 round-off
    (1e-5 per distribution after 24 steps, as for batched against alone)."""
    import paper_2007_12266_gb300 as lbm
    specs = _jobs()
    results = {}
    for shape in ((256, -1), (256, -2), (192, -2), (128, -2)):
        doms = [_make(s, precision) for s in specs]
        for d in doms:
            d.set_step_form(form)
        b = lbm.Batch()
        for d in doms:
            b.add(d)
        b.set_launch(shape[0], shape[1], shape[1])
        n0 = b.launch_count
        b.advance(10)
        b.advance(14)
        if shape[1] == -2:
            # one launch per two steps; the sum form launches the first and the
            # last step of each call alone: (1 + 4 + 1) + (1 + 6 + 1)
            assert b.launch_count - n0 == (14 if form == "auto" else 12), b.launch_count - n0
        assert all(m["status"] == 0 for m in b.measure())
        results[shape] = [[d.distributions(k).astype(np.float64) for k in ("f", "a", "b")] for d in doms]
        b.close()
        for d in doms:
            d.close()
    base = results[(256, -1)]
    for shape in ((256, -2), (192, -2), (128, -2)):
        for j, (ga, gb) in enumerate(zip(base, results[shape])):
            for which, x, y, floor in zip("fab", ga, gb, (T19, W7, W7)):
                err = np.abs(x - y) / np.maximum(np.abs(x), floor[:, None])
                assert err.max() <= 1e-5, (shape, j, which, err.max())


def test_fused_barrier_wait_is_bounded():
    """The fused kernel's grid barrier gives up after its limit: a barrier
    that expects one arrival more than there are blocks (a flag nothing sets)
    ends with LBPM_E_TIMEOUT after the limit, and the GPU stays usable."""
    import time

    import paper_2007_12266_gb300 as lbm
    b = lbm.Batch()
    assert b.check_barrier(0, 0.5) is True          # every block arrives: completes
    t0 = time.perf_counter()
    assert b.check_barrier(1, 0.05) is False        # one arrival never comes: the wait runs out
    assert time.perf_counter() - t0 < 5.0
    assert b.check_barrier(0, 0.5) is True          # the context still works
    specs = _jobs()[:2]
    doms = [_make(s, "fp32") for s in specs]
    for d in doms:
        b.add(d)
    b.set_launch(256, -2, -2)
    b.advance(4)
    assert all(m["status"] == 0 for m in b.measure())
    b.close()
