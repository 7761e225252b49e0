"""Pins of the oracle's full timestep: conservation and brute force.

* Per-component mass: sum_q w_q = 1 and sum_q w_q xi_q = 0 make the recolored
  distributions keep Na and Nb at every site (Eqs. LBE-mass-a/b); streaming
  moves every value to exactly one slot and halfway bounce-back returns it to
  its own site, so on a closed or periodic domain sum Na and sum Nb are
  constant. Over 1,000 steps the fp64 drift must stay at round-off (1e-12).
* Fluid momentum: sum rho u grows by exactly F per pore site per step on a
  fully periodic domain with no solids (no wall to take momentum).
* Brute force: an independent dense np.roll implementation agrees to
  round-off on small lattices with solids, walls, mixed tau and a force.
"""
import numpy as np
import pytest

import oracle
from oracle.dense import DenseLBM
from synthetic import phi0_iid, random_affinity, sphere_pack


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 1), (0, 0, 0)])
def test_mass_conservation_1000_steps(periodic):
    sp = sphere_pack(16, 0.45, 2.5, 0.8, 21)
    aff = random_affinity(sp.labels, -0.9, 0.9, 22)
    o = oracle.Oracle(sp.labels, aff, periodic, tau_a=0.8, tau_b=0.6, alpha=0.005,
                      beta=0.95, force=(2e-5, 0, 1e-5))
    o.init_fluids(phi0_iid(sp.labels, 0.5, 23))
    m0 = o.measure()
    o.step(1000)
    m1 = o.measure()
    assert m1["status"] == 0
    for k in ("mass_a", "mass_b", "mass_total"):
        assert abs(m1[k] - m0[k]) <= 1e-12 * m0[k], k


def test_momentum_grows_by_force_without_walls():
    lab = np.zeros((6, 5, 4), np.uint16)
    F = np.array([1e-5, -2e-5, 3e-5])
    o = oracle.Oracle(lab, None, (1, 1, 1), alpha=0.0, force=F)
    phi0 = np.ones(lab.shape, np.float32)
    o.init_fluids(phi0)
    o.step(10)
    f, _, _ = o.state()
    xi = oracle.lattice_tables()[0]
    j = xi.T @ f.sum(axis=1)
    assert np.allclose(j, 10 * o.N * F, rtol=1e-12, atol=1e-17)


def test_rest_state_is_steady():
    """A single phase at rest with uniform affinity = phi is a fixed point."""
    sp = sphere_pack(12, 0.5, 2.0, 0.5, 31)
    aff = np.where(sp.labels != 0, 1.0, 0.0).astype(np.float32)
    o = oracle.Oracle(sp.labels, aff, (1, 1, 1), alpha=0.005, beta=0.95)
    o.init_fluids(np.ones(sp.labels.shape, np.float32))
    f0, A0, B0 = o.state()
    o.step(20)
    f1, A1, B1 = o.state()
    assert np.abs(f1 - f0).max() < 1e-15
    assert np.abs(A1 - A0).max() < 1e-15 and np.abs(B1).max() == 0


def test_single_link_pulse_streams_and_reflects():
    """Component B is a tracer with beta = 0 and u = 0: its D3Q7 populations
    leave each site as w_q Nb. A tube one voxel wide along x (walls in y, z)
    bounces everything except the x links back in place."""
    nx = 6
    lab = np.ones((3, 3, nx), np.uint16)
    lab[1, 1, :] = 0
    o = oracle.Oracle(lab, np.zeros(lab.shape, np.float32), (1, 0, 0), alpha=0.0, beta=0.0)
    f = np.outer(oracle.lattice_tables()[1], np.ones(o.N))
    w = oracle.lattice_tables()[2]
    A = np.outer(w, np.ones(o.N))
    B = np.zeros((7, o.N))
    B[:, 2] = w            # Nb = 1 at x = 2
    A[:, 2] = 0.0
    o.set_state(f, A, B)
    o.step(1)
    _, _, B1 = o.state()
    Nb = B1.sum(0)
    assert np.allclose(Nb, [0, 1 / 9, 7 / 9, 1 / 9, 0, 0], atol=1e-16)
    assert abs(B1[1, 3] - 1 / 9) < 1e-16 and abs(B1[2, 1] - 1 / 9) < 1e-16
    # y and z links bounce back: direction 3 (+y) returns as direction 4 (-y)
    assert abs(B1[4, 2] - 1 / 9) < 1e-16 and abs(B1[3, 2] - 1 / 9) < 1e-16


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 1, 1), (1, 0, 0), (0, 0, 0)])
def test_brute_force_dense_8cubed(periodic):
    sp = sphere_pack(8, 0.5, 1.5, 0.5, 7)
    lab = sp.labels
    aff = random_affinity(lab, -0.8, 0.8, 8)
    phi0 = phi0_iid(lab, 0.5, 9)
    args = dict(tau_a=0.8, tau_b=0.6, alpha=0.01, beta=0.9, force=(1e-4, -2e-4, 3e-4))
    o = oracle.Oracle(lab, aff, periodic, **args)
    o.init_fluids(phi0)
    d = DenseLBM(lab, aff, periodic, args["tau_a"], args["tau_b"], args["alpha"],
                 args["beta"], args["force"])
    d.init_fluids(phi0)
    for _ in range(6):
        o.step(1)
        d.step()
    f, A, B = o.state()
    assert np.abs(f - d.site_values(d.f)).max() < 1e-13
    assert np.abs(A - d.site_values(d.A)).max() < 1e-13
    assert np.abs(B - d.site_values(d.B)).max() < 1e-13


def test_brute_force_dense_random_state_anisotropic_box():
    rng = np.random.default_rng(41)
    lab = (rng.uniform(size=(5, 6, 7)) < 0.3).astype(np.uint16)
    aff = rng.uniform(-1, 1, size=lab.shape).astype(np.float32)
    o = oracle.Oracle(lab, aff, (1, 0, 1), tau_a=0.9, tau_b=0.55, alpha=0.02, beta=0.7,
                      force=(0, 1e-4, 0))
    phi0 = rng.uniform(-1, 1, size=lab.shape).astype(np.float32)
    o.init_fluids(phi0)
    d = DenseLBM(lab, aff, (1, 0, 1), 0.9, 0.55, 0.02, 0.7, (0, 1e-4, 0))
    d.init_fluids(phi0)
    for _ in range(4):
        o.step(1)
        d.step()
    f, A, B = o.state()
    assert np.abs(f - d.site_values(d.f)).max() < 1e-13
    assert np.abs(A - d.site_values(d.A)).max() < 1e-13
