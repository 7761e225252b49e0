"""Checks of the oracle's reservoir slabs (reservoir_z = 1; the reading of
Sec. 4.1's inlet and outlet reservoirs: after streaming, the first four z
layers hold fluid A at rest at rho_in and the last four fluid B at rest at
rho_out).

What is fixed:
* Construction: after every step each slab site holds exactly the reset
  state, f_q = t_q rho, A_q = w_q (inlet) or B_q = w_q (outlet), the other
  component zero.
* Sanity of the displacement they drive: with the body force pushing A from
  the inlet into a duct filled with B, the saturation of A never decreases
  and the displacement front moves down the duct.
* The steady state they drive, in closed form: with both reservoirs at one
  density, no force, alpha = beta = 0, rest at that density everywhere and
  component densities exactly linear along the duct between the slabs.
(The pressure-driven flow between reservoirs at different densities has an
entrance region of the order of the duct width and no closed form; it uses
the same reset with each side's density, pinned here, and the momentum
solver pinned by the duct series.)
"""
import numpy as np

import oracle

RIN, ROUT = 1.002, 0.998


def _duct(a=6, nz=40, force=1e-4):
    n = a + 2
    lab = np.ones((nz, n, n), np.uint16)
    lab[:, 1:-1, 1:-1] = 0
    aff = np.zeros(lab.shape, np.float32)        # neutral walls
    o = oracle.Oracle(lab, aff, (0, 0, 0), tau_a=0.7, tau_b=0.7, alpha=0.005, beta=0.95,
                      force=(0.0, 0.0, force), reservoir_z=1, rho_in=RIN, rho_out=ROUT)
    o.init_fluids(-np.ones(lab.shape, np.float32))   # B everywhere; the inlet slab resets to A
    return o, lab


def _z_of_sites(o, lab):
    sv, _ = o.index()
    return sv // (lab.shape[1] * lab.shape[2])


def test_slab_sites_hold_the_reset_state_after_every_step():
    o, lab = _duct()
    z = _z_of_sites(o, lab)
    nz = lab.shape[0]
    _, t19, w7, _, _ = oracle.lattice_tables()
    for _ in range(3):
        o.step(1)
        f, A, B = o.state()
        for sel, rho, a_full in ((z < 4, RIN, True), (z >= nz - 4, ROUT, False)):
            assert sel.any()
            assert np.abs(f[:, sel] - t19[:, None] * rho).max() < 1e-15
            full, empty = (A, B) if a_full else (B, A)
            assert np.abs(full[:, sel] - w7[:, None]).max() < 1e-15
            assert np.abs(empty[:, sel]).max() == 0.0


def test_injection_raises_saturation_and_advances_the_front():
    o, lab = _duct()
    z = _z_of_sites(o, lab)
    interior = (z >= 4) & (z < lab.shape[0] - 4)
    sat, front = [], []
    for _ in range(10):
        o.step(150)
        sat.append(o.measure()["sat_mass"])
        _, A, B = o.state()
        Na, Nb = A.sum(axis=0), B.sum(axis=0)
        phi = (Na - Nb) / (Na + Nb)
        # front: the A volume in the interior, as a length along the duct
        front.append(np.count_nonzero(phi[interior] > 0) / np.count_nonzero(z == 4))
    assert all(b >= a - 1e-12 for a, b in zip(sat, sat[1:])), sat
    assert sat[-1] > sat[0]
    assert front[-1] > front[0] + 1.0, front


def test_equal_reservoirs_reach_rest_and_a_linear_component_profile():
    """Closed-form steady state of the slabs: both reservoirs at the same
    density rho_r, no body force, alpha = 0 and beta = 0. The momentum
    lattice's only steady state is then rest at rho_r (f_q = t_q rho_r at every
    site), and with u = 0 and beta = 0 the recoloring gives A*_q = w_q Na, so
    each component performs a lattice random walk: along the walled duct (the
    walls reflect, so every cross-section stays uniform) Na'(z) = (w_0 + 4 w_1)
    Na(z) + w_1 (Na(z - 1) + Na(z + 1)), whose steady state between the last
    inlet layer (z = 3, Na = 1) and the first outlet layer (z = nz - 4, Na = 0)
    is exactly linear: Na(z) = (nz - 4 - z) / (nz - 7), Nb = 1 - Na. Started
    from rest at rho = 1 filled with B, the oracle must reach both to
    round-off; the slowest component mode decays by 1 - w_1 pi^2 / (nz - 7)^2
    per step (1/263 at nz = 24), so 9,000 steps leave under 1e-13."""
    rho_r, nz, a = 1.01, 24, 4
    n = a + 2
    lab = np.ones((nz, n, n), np.uint16)
    lab[:, 1:-1, 1:-1] = 0
    aff = np.zeros(lab.shape, np.float32)
    o = oracle.Oracle(lab, aff, (0, 0, 0), tau_a=0.8, tau_b=0.8, alpha=0.0, beta=0.0,
                      force=(0.0, 0.0, 0.0), reservoir_z=1, rho_in=rho_r, rho_out=rho_r)
    o.init_fluids(-np.ones(lab.shape, np.float32))
    o.step(9000)
    f, A, B = o.state()
    _, t19, _, _, _ = oracle.lattice_tables()
    z = _z_of_sites(o, lab)
    assert np.abs(f - t19[:, None] * rho_r).max() < 1e-13
    Na, Nb = A.sum(axis=0), B.sum(axis=0)
    zc = np.clip(z, 3, nz - 4)
    exact = (nz - 4 - zc) / (nz - 7)
    assert np.abs(Na - exact).max() < 1e-12, np.abs(Na - exact).max()
    assert np.abs(Nb - (1.0 - exact)).max() < 1e-12
