"""The synthetic inputs follow their stated recipe (CPU only): the sphere-pack
porosity target, the lognormal radius law with the stated mean and sd,
seeded determinism, walls on the named planes, affinity ranges, the target
saturation of the initial phases, and the parameters of the workloads."""
import numpy as np
import pytest

from synthetic import (add_walls, phi0_blob, phi0_iid, phi0_reservoir, random_affinity, serving_job,
                       sphere_pack, uniform_affinity, workload_batched_job, workload_parity32,
                       workload_steady256)
from synthetic.spherepack import _lognormal_params


@pytest.mark.parametrize("mean,sd", [(4.0, 1.0), (10.0, 3.0), (8.0, 2.0)])
def test_lognormal_radius_law_has_the_stated_mean_and_sd(mean, sd):
    mu, sig = _lognormal_params(mean, sd)
    # closed forms of the lognormal moments
    assert np.exp(mu + sig ** 2 / 2) == pytest.approx(mean, rel=1e-12)
    assert np.sqrt((np.exp(sig ** 2) - 1) * np.exp(2 * mu + sig ** 2)) == pytest.approx(sd, rel=1e-12)


@pytest.mark.parametrize("L,porosity,r", [(32, 0.35, (4.0, 1.0)), (48, 0.22, (6.0, 2.0)), ((40, 24, 16), 0.3, (3.0, 1.0))])
def test_sphere_pack_reaches_the_porosity_target(L, porosity, r):
    sp = sphere_pack(L, porosity, r[0], r[1], seed=11)
    measured = np.count_nonzero(sp.labels == 0) / sp.labels.size
    assert sp.porosity == pytest.approx(measured, abs=1e-12)   # recorded truthfully
    assert measured <= porosity                                 # spheres are added until it is reached
    assert measured > porosity - 0.03                           # the last sphere overshoots a little
    again = sphere_pack(L, porosity, r[0], r[1], seed=11)
    assert np.array_equal(sp.labels, again.labels)              # seeded
    other = sphere_pack(L, porosity, r[0], r[1], seed=12)
    assert not np.array_equal(sp.labels, other.labels)


def test_walls_affinities_and_phases():
    sp = sphere_pack(24, 0.4, 3.0, 1.0, seed=3)
    lab = add_walls(sp.labels, ("x", "y"))
    assert (lab[:, :, 0] != 0).all() and (lab[:, :, -1] != 0).all()
    assert (lab[:, 0, :] != 0).all() and (lab[:, -1, :] != 0).all()
    assert np.array_equal(lab[:, 1:-1, 1:-1], sp.labels[:, 1:-1, 1:-1])
    solid, pore = lab != 0, lab == 0
    aff = random_affinity(lab, -0.3, 0.3, seed=4)
    assert (aff[pore] == 0).all() and aff[solid].min() >= -0.3 and aff[solid].max() <= 0.3
    assert aff[solid].std() > 0.1
    assert (uniform_affinity(lab, -0.7)[solid] == np.float32(-0.7)).all()
    blob = phi0_blob(lab, 0.4, seed=5)
    assert set(np.unique(blob[pore])) <= {-1.0, 1.0} and (blob[solid] == 0).all()
    assert np.count_nonzero(blob[pore] > 0) / pore.sum() == pytest.approx(0.4, abs=2.0 / pore.sum())
    iid = phi0_iid(lab, 0.5, seed=6)
    assert np.count_nonzero(iid[pore] > 0) / pore.sum() == pytest.approx(0.5, abs=0.05)
    res = phi0_reservoir(lab, -1.0)
    assert (res[pore] == -1.0).all() and (res[solid] == 0).all()


def test_workload_parameters():
    w = workload_parity32()
    assert w.labels.shape == (32, 32, 32) and w.periodic == (1, 1, 1)
    assert 0.33 < w.porosity <= 0.35 and (w.affinity[w.labels != 0] == np.float32(-0.5)).all()
    assert (w.tau_a, w.tau_b, w.alpha, w.beta, w.force) == (0.7, 0.7, 0.005, 0.95, (0.0, 0.0, 1e-5))
    s = workload_steady256(L=64)
    assert s.periodic == (0, 0, 1) and (s.labels[:, :, 0] != 0).all() and (s.labels[:, 0, :] != 0).all()
    pore = s.labels == 0
    assert np.count_nonzero(s.phi0[pore] > 0) / pore.sum() == pytest.approx(0.4, abs=1e-3)
    b = workload_batched_job(3)
    assert b.labels.shape[0] in (64, 96, 128, 160, 192) and b.periodic == (0, 0, 1)
    assert 1e-5 <= b.force[2] <= 1e-4
    kinds = {serving_job(i, L_choices=(64,)).meta["kind"] for i in range(12)}
    assert kinds <= {"steady", "unsteady", "centrifuge"} and len(kinds) >= 2
