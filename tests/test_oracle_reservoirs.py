"""Checks of the oracle's reservoir slabs (reservoir_z = 1; the reading of
Sec. 4.1's inlet and outlet reservoirs: after streaming, the first four z
layers hold fluid A at rest at rho_in and the last four fluid B at rest at
rho_out).

The slabs have no closed form to pin their effect on the flow against (their
parity stays unpinned beyond agreement with the CUDA path); what is fixed:
* Construction: after every step each slab site holds exactly the reset
  state, f_q = t_q rho, A_q = w_q (inlet) or B_q = w_q (outlet), the other
  component zero.
* Sanity of the displacement they drive: with the body force pushing A from
  the inlet into a duct filled with B, the saturation of A never decreases
  and the displacement front moves down the duct.
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
