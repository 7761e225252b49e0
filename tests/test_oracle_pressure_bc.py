"""Pins of the oracle's pressure boundary at the z faces (reservoir_z = 2;
Sec. 4.1 cites Zou and He's constant-pressure scheme) and of the flux inlet
(reservoir_z = 3; Sec. 4.1's flux condition: a total volumetric flow rate).

* Construction: after every step each face site holds exactly the face
  density and no tangential momentum.
* Physics: single-phase flow in a square duct driven only by the pressure
  difference between the two faces matches the body-force-driven duct series
  with F = -dp/dz = (rho_in - rho_out) / (3 (nz - 1)), at mid length, within
  0.3 % (measured 0.09 %; the rest is the lattice fluid's compressibility),
  and carries the same mass flux through every cross-section.
* The entering component population: a duct driven by a body force between
  two faces held at the same density rho_f, started at rest at rho_f, has no
  pressure drop, so the momentum density stays rho_f; the total component
  density N = Na + Nb, which the faces feed, must then stay rho_f at every
  site too (an advected and diffused density with the same value at both
  ends), and the components must carry the momentum lattice's mass flux.
"""
import numpy as np
import pytest

import oracle
from test_oracle_physics import duct_series

def _duct(a, nz, rin, rout, tau=0.7, mode=2, flux=0.0):
    n = a + 2
    lab = np.ones((nz, n, n), np.uint16)
    lab[:, 1:-1, 1:-1] = 0
    aff = np.zeros(lab.shape, np.float32)
    # alpha = 0 and tau_a = tau_b: the momentum equation is single phase
    # whatever the two components do
    o = oracle.Oracle(lab, aff, (0, 0, 0), tau_a=tau, tau_b=tau, alpha=0.0, beta=0.95, force=(0, 0, 0),
                      reservoir_z=mode, rho_in=rin, rho_out=rout, flux_in=flux)
    o.init_fluids(np.ones(lab.shape, np.float32))
    return o, lab


def test_face_sites_hold_the_face_density_and_no_tangential_momentum():
    o, lab = _duct(6, 10, 1.004, 0.996)
    o.step(7)
    f, _, _ = o.state()                # canonical (19, N)
    sv, _ = o.index()
    z = sv // (lab.shape[1] * lab.shape[2])
    xi = oracle.lattice_tables()[0]
    for zz, rho in ((0, 1.004), (lab.shape[0] - 1, 0.996)):
        sel = z == zz
        assert sel.any()
        assert np.abs(f[:, sel].sum(axis=0) - rho).max() < 1e-14
        for a in (0, 1):
            assert np.abs(xi[:, a] @ f[:, sel]).max() < 1e-14


def test_pressure_driven_duct_matches_the_body_force_series():
    a, nz = 16, 48
    rin, rout = 1.0 + 6e-4, 1.0 - 6e-4
    o, lab = _duct(a, nz, rin, rout)
    o.step(4000)
    _, _, u = o.fields()
    uz = o.dense(u[2])
    F = (rin - rout) / 3.0 / (nz - 1)
    n = a + 2
    c = np.arange(1, n - 1) - (n - 1) / 2
    yy, xx = np.meshgrid(c, c, indexing="ij")
    exact = duct_series(a, F, (0.7 - 0.5) / 3, xx, yy)
    mid = uz[nz // 2, 1:-1, 1:-1]
    assert abs(mid.mean() / exact.mean() - 1) < 3e-3
    assert np.abs(mid - exact).max() < 3e-3 * exact.max()
    # steady mass flux rho u_z: the same through every cross-section
    _, p, _ = o.fields()
    rho = 3.0 * o.dense(p)
    flux = np.nansum((rho * uz)[:, 1:-1, 1:-1], axis=(1, 2))
    assert np.abs(flux / flux[nz // 2] - 1).max() < 2e-3


def test_flux_inlet_carries_exactly_the_prescribed_flux():
    a, nz, Q = 6, 12, 0.3
    o, lab = _duct(a, nz, 1.0, 0.999, mode=3, flux=Q)
    xi = oracle.lattice_tables()[0]
    sv, _ = o.index()
    inlet = sv // (lab.shape[1] * lab.shape[2]) == 0
    for _ in range(5):
        o.step(3)
        f, _, _ = o.state()
        rho = f[:, inlet].sum(axis=0)
        uz = (xi[:, 2] @ f[:, inlet]) / rho
        assert abs(uz.sum() - Q) < 1e-12
        assert np.abs(rho - rho[0]).max() < 1e-14        # one uniform inlet density
        assert np.abs(xi[:, 0] @ f[:, inlet]).max() < 1e-14


def test_flux_driven_duct_has_the_poiseuille_profile_and_flux():
    a, nz, Q = 16, 48, 0.4
    o, lab = _duct(a, nz, 1.0, 1.0, mode=3, flux=Q)
    o.step(4000)
    _, p, u = o.fields()
    uz = o.dense(u[2])
    rho = 3.0 * o.dense(p)
    mid = uz[nz // 2, 1:-1, 1:-1]
    # the steady mass flux of every section is the inlet's: rho_in Q
    flux = np.nansum((rho * uz)[:, 1:-1, 1:-1], axis=(1, 2))
    assert np.abs(flux / flux[nz // 2] - 1).max() < 2e-3
    assert abs(mid.sum() / Q - 1) < 5e-3
    # the profile is the duct series, scaled to the same total
    n = a + 2
    c = np.arange(1, n - 1) - (n - 1) / 2
    yy, xx = np.meshgrid(c, c, indexing="ij")
    shape = duct_series(a, 1.0, 1.0, xx, yy)
    shape *= mid.sum() / shape.sum()
    assert np.abs(mid - shape).max() < 3e-3 * shape.max()


def test_entering_component_population_keeps_the_face_density():
    # Closed form: uniform N = rho_f. The A fed at the inlet and the B fed at
    # the outlet fill the duct from both ends; only their sum is fixed.
    a, nz, rf, Fz = 4, 10, 1.01, 1e-4
    n = a + 2
    lab = np.ones((nz, n, n), np.uint16)
    lab[:, 1:-1, 1:-1] = 0
    o = oracle.Oracle(lab, np.zeros(lab.shape, np.float32), (0, 0, 0), tau_a=0.7, tau_b=0.7, alpha=0.0,
                      beta=0.95, force=(0, 0, Fz), reservoir_z=2, rho_in=rf, rho_out=rf)
    xi, t, w = oracle.lattice_tables()[:3]
    sv, _ = o.index()
    ones = np.ones((1, len(sv)))
    o.set_state(t[:, None] * rf * ones, w[:, None] * rf * ones, np.zeros((7, len(sv))))
    o.step(1000)
    f, A, B = o.state()
    rho, Nt, jz = f.sum(axis=0), A.sum(axis=0) + B.sum(axis=0), xi[:, 2] @ f
    assert B.sum(axis=0).max() > 0.5 * rf            # B entered from the outlet face
    u_mean = jz.mean() / rf
    assert u_mean > 5e-4                              # the force drives a real flow
    assert np.abs(rho - rf).max() < 2e-5             # no pressure drop (measured 1e-5)
    # measured 3.7e-5; a face that fed its fluid at the wrong velocity sign
    # or at density 1 instead of rho_f gives 8e-3 and 1e-2
    assert np.abs(Nt - rf).max() < 0.2 * u_mean
    # component flux through each cross-section z | z + 1 (post-collision
    # D3Q7 totals w N (1 + 4.5 j.xi), moved along +z and -z) against the
    # momentum lattice's mass flux at the face density
    Nd, Jd = o.dense(Nt)[:, 1:-1, 1:-1], o.dense(jz)[:, 1:-1, 1:-1]
    wf = w[1]
    for k in range(nz - 1):
        flux = (wf * Nd[k] * (1 + 4.5 * Jd[k]) - wf * Nd[k + 1] * (1 - 4.5 * Jd[k + 1])).sum()
        mass = 0.5 * rf * (Jd[k].sum() + Jd[k + 1].sum())
        assert abs(flux / mass - 1) < 2e-3
