"""Pins of the oracle's basic analysis (Sec. 4 basic analysis, Sec. 3.4 table
of integral measures, Eq. capillary_number), through configurations whose
measures have closed forms:

* uniform flow of pure A: the Darcy flux is the porosity times the reported
  velocity (j + F/2)/rho0, every per-phase quantity belongs to A, and the
  capillary number reduces to eps_a mu_a |u| / sigma with sigma = 6 alpha;
* A and B on alternating sites with different densities, velocities and
  viscosities: each phase's volume, mass, momentum, mean pressure and its
  term of the capillary number separately;
* a uniform mixture Na = 0.6, Nb = 0.4: the mass saturation and the phase
  fluxes split 0.6 / 0.4 (weights Na/N and Nb/N);
* the instability flags: a non-finite value, a component density below
  -1e-2.
"""
import numpy as np
import pytest

import oracle

_, T19, W7, _, _ = oracle.lattice_tables()
XI = oracle.lattice_tables()[0]
TAU_A, TAU_B, ALPHA = 0.8, 0.6, 0.004
F = np.array([2e-5, -1e-5, 3e-5])


def _box():
    """6 x 5 x 4 voxels (x, y, z), a few solid voxels, all axes periodic."""
    lab = np.zeros((4, 5, 6), np.uint16)
    lab[1, 2, 3] = lab[2, 0, 0] = lab[3, 4, 5] = 1
    o = oracle.Oracle(lab, np.zeros(lab.shape, np.float32), (1, 1, 1), tau_a=TAU_A, tau_b=TAU_B,
                      alpha=ALPHA, beta=0.95, force=tuple(F))
    return o, lab


def _state(rho, j, Na, Nb):
    """Populations with the given density, momentum and component densities
    per site: f_q = t_q (rho + 3 xi_q . j), A_q = w_q Na, B_q = w_q Nb."""
    f = T19[:, None] * (rho[None, :] + 3.0 * (XI @ j.T))
    return f, W7[:, None] * Na[None, :], W7[:, None] * Nb[None, :]


def test_uniform_flow_of_pure_a():
    o, lab = _box()
    N, V = o.N, lab.size
    u0 = np.array([1e-3, -2e-3, 4e-3])
    f, A, B = _state(np.full(N, 1.02), np.tile(u0, (N, 1)), np.ones(N), np.zeros(N))
    o.set_state(f, A, B, 0)
    m = o.measure()
    u = u0 + 0.5 * F                       # reported velocity, rho0 = 1
    assert m["sat_mass"] == 1.0 and m["sat_count"] == 1.0
    assert m["vol_a"] == N and m["vol_b"] == 0
    for a, c in enumerate("xyz"):
        assert m[f"flux_{c}"] == pytest.approx(u[a] * N / V, rel=1e-12)
        assert m[f"flux_a_{c}"] == pytest.approx(u[a] * N / V, rel=1e-12)
        assert abs(m[f"flux_b_{c}"]) < 1e-18
        assert m[f"mom_a_{c}"] == pytest.approx(1.02 * u[a] * N, rel=1e-12)
    assert m["mass_a"] == pytest.approx(N, rel=1e-14) and abs(m["mass_b"]) < 1e-15
    assert m["mass_total"] == pytest.approx(1.02 * N, rel=1e-14)
    assert m["p_a"] == pytest.approx(1.02 / 3.0, rel=1e-14)
    assert m["ke_a"] == pytest.approx(1.02 * (u @ u) * N, rel=1e-12)
    mu_a = (TAU_A - 0.5) / 3.0
    assert m["ca"] == pytest.approx((N / V) * mu_a * np.linalg.norm(u) / (6.0 * ALPHA), rel=1e-12)
    assert m["status"] == 0


def test_two_phases_on_alternating_sites():
    o, lab = _box()
    N, V = o.N, lab.size
    is_a = (np.arange(N) % 2) == 0
    na, nb = int(is_a.sum()), int((~is_a).sum())
    ua, ub = np.array([2e-3, 0.0, 1e-3]), np.array([-1e-3, 3e-3, 0.0])
    rho = np.where(is_a, 1.01, 0.97)
    j = np.where(is_a[:, None], ua, ub)
    f, A, B = _state(rho, j, is_a.astype(float), (~is_a).astype(float))
    o.set_state(f, A, B, 0)
    m = o.measure()
    ra, rb = ua + 0.5 * F, ub + 0.5 * F       # reported velocities
    assert m["vol_a"] == na and m["vol_b"] == nb and m["sat_count"] == pytest.approx(na / N, rel=1e-14)
    assert m["sat_mass"] == pytest.approx(na / N, rel=1e-14)
    for a, c in enumerate("xyz"):
        assert m[f"mom_a_{c}"] == pytest.approx(1.01 * ra[a] * na, rel=1e-12, abs=1e-18)
        assert m[f"mom_b_{c}"] == pytest.approx(0.97 * rb[a] * nb, rel=1e-12, abs=1e-18)
        assert m[f"flux_a_{c}"] == pytest.approx(ra[a] * na / V, rel=1e-12, abs=1e-18)
        assert m[f"flux_b_{c}"] == pytest.approx(rb[a] * nb / V, rel=1e-12, abs=1e-18)
    assert m["p_a"] == pytest.approx(1.01 / 3.0, rel=1e-14)
    assert m["p_b"] == pytest.approx(0.97 / 3.0, rel=1e-14)
    mu_a, mu_b = (TAU_A - 0.5) / 3.0, (TAU_B - 0.5) / 3.0
    # <u>_alpha = |P_alpha| / M_alpha, eps_alpha = V_alpha / V
    ca = ((na / V) * mu_a * np.linalg.norm(ra) + (nb / V) * mu_b * np.linalg.norm(rb)) / (6.0 * ALPHA)
    assert m["ca"] == pytest.approx(ca, rel=1e-12)


def test_uniform_mixture_splits_by_component_fraction():
    o, lab = _box()
    N, V = o.N, lab.size
    u0 = np.array([0.0, 0.0, 2e-3])
    f, A, B = _state(np.ones(N), np.tile(u0, (N, 1)), np.full(N, 0.6), np.full(N, 0.4))
    o.set_state(f, A, B, 0)
    m = o.measure()
    u = u0 + 0.5 * F
    assert m["sat_mass"] == pytest.approx(0.6, rel=1e-14)
    assert m["sat_count"] == 1.0                     # phi = 0.2 > 0 at every site
    for a, c in enumerate("xyz"):
        assert m[f"flux_a_{c}"] == pytest.approx(0.6 * u[a] * N / V, rel=1e-12)
        assert m[f"flux_b_{c}"] == pytest.approx(0.4 * u[a] * N / V, rel=1e-12)


def test_instability_flags():
    o, lab = _box()
    N = o.N
    f, A, B = _state(np.ones(N), np.zeros((N, 3)), np.full(N, 0.5), np.full(N, 0.5))
    f[3, 7] = np.nan
    o.set_state(f, A, B, 0)
    assert int(o.measure()["status"]) & 1
    f, A, B = _state(np.ones(N), np.zeros((N, 3)), np.full(N, 0.5), np.full(N, 0.5))
    A[:, 5] = W7 * -0.05                             # Na = -0.05 < -1e-2
    o.set_state(f, A, B, 0)
    assert int(o.measure()["status"]) & 2
    A[:, 5] = W7 * -0.005                            # small negative values are legitimate
    o.set_state(f, A, B, 0)
    assert int(o.measure()["status"]) == 0
