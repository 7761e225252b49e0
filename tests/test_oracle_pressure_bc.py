"""Pins of the oracle's pressure boundary at the z faces (reservoir_z = 2;
Sec. 4.1 cites Zou and He's constant-pressure scheme).

* Construction: after every step each face site holds exactly the face
  density and no tangential momentum.
* Physics: single-phase flow in a square duct driven only by the pressure
  difference between the two faces matches the body-force-driven duct series
  with F = -dp/dz = (rho_in - rho_out) / (3 (nz - 1)), at mid length, within
  0.3 % (measured 0.09 %; the rest is the lattice fluid's compressibility),
  and carries the same mass flux through every cross-section.
"""
import numpy as np
import pytest

import oracle
from test_oracle_physics import duct_series

def _duct(a, nz, rin, rout, tau=0.7):
    n = a + 2
    lab = np.ones((nz, n, n), np.uint16)
    lab[:, 1:-1, 1:-1] = 0
    aff = np.zeros(lab.shape, np.float32)
    # alpha = 0 and tau_a = tau_b: the momentum equation is single phase
    # whatever the two components do
    o = oracle.Oracle(lab, aff, (0, 0, 0), tau_a=tau, tau_b=tau, alpha=0.0, beta=0.95, force=(0, 0, 0),
                      reservoir_z=2, rho_in=rin, rho_out=rout)
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
