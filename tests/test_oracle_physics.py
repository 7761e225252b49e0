"""Physics pins of the oracle: what the paper's model must reproduce.

* Square-duct Poiseuille flow (single phase, C = 0): textbook series solution
  of the Stokes equation with halfway bounce-back walls.
* Flat interface (Sec. 3.2, Eq. lb-dist; Sec. 3.3, Eq. lb-dist-to-phase):
  the relaxed profile is phi = tanh(beta (x - x0)).
* Normal-stress balance across a flat interface (Sec. 3.1 equilibria): the
  alpha terms put (alpha|C|/2)(n n - I/3) into the equilibrium momentum flux
  and -alpha|C| into the energy moment m1, which is -alpha|C|/19 in the trace;
  with p = rho/3 a static flat interface must carry a density dip of
  3 alpha |C| (1/3 - 1/57). This pins the m1 and m9 alpha terms.
* Laplace law (sigma_ab = 6 alpha, Sec. 3.1): cylinders in each coordinate
  plane (dp = sigma / R; pins m9, m11, m13, m14, m15) and a sphere
  (dp = 2 sigma / R).
* Contact angle (Sec. 3.2, Eq. phi_s): cos(theta) = phi_s on a flat plate,
  phi_s = +1 water-wet (fluid A, phi > 0, wets). The angle depends on the
  strength of the alpha|C| stress terms relative to the colour segregation:
  converged drops at phi_s = 0.5 give 58.2, 56.7, 53.0, 47.3, 41.4 degrees for
  alpha = 0.00083, 0.00125, 0.0025, 0.005, 0.01. The paper's two statements on
  the colour gradient (C = grad phi, and sigma = 6 alpha with the printed
  alpha|C|/2 terms) fix that strength differently: the stencil C = 6 grad phi
  taken here makes sigma = 6 alpha hold (the Laplace pins) and gives
  cos(theta) ~ 1.35 phi_s at alpha = 0.005; the stress scale of C = grad phi is
  the same model at alpha / 6, where cos(theta) = phi_s holds within 2 degrees.
  The pins check the neutral angle, the A/B antisymmetry, the sign convention
  and the angle within 15 degrees at the paper's alpha, and the closed form
  cos(theta) = phi_s within 3 degrees at the stress scale of C = grad phi.
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CONST = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
SIGMA_OVER_ALPHA = CONST["interfacial_tension"]["sigma_over_alpha"]


def duct_series(a, F, mu, y, z, nterms=201):
    """Stokes flow in a square duct of side a (centre at 0): White, Viscous
    Fluid Flow, rectangular duct series with half-width b = a/2."""
    b = a / 2
    u = np.zeros_like(y, dtype=float)
    for n in range(1, nterms, 2):
        u += ((-1) ** ((n - 1) // 2) / n ** 3
              * (1 - np.cosh(n * np.pi * z / a) / np.cosh(n * np.pi / 2))
              * np.cos(n * np.pi * y / a))
    return 16 * b * b * F / (mu * np.pi ** 3) * u


@pytest.mark.parametrize("a,tau,steps,tol", [(16, 0.7, 3000, 3e-3), (32, 1.0, 4500, 3e-3)])
def test_square_duct_poiseuille(a, tau, steps, tol):
    n = a + 2
    lab = np.ones((1, n, n), np.uint16)
    lab[0, 1:-1, 1:-1] = 0
    aff = np.where(lab != 0, 1.0, 0.0).astype(np.float32)
    F = 1e-6
    o = oracle.Oracle(lab, aff, (0, 0, 1), tau_a=tau, tau_b=tau, alpha=0.005, beta=0.95,
                      force=(0, 0, F))
    o.init_fluids(np.ones(lab.shape, np.float32))
    o.step(steps)
    _, _, u = o.fields()
    uz = o.dense(u[2])[0, 1:-1, 1:-1]
    c = np.arange(1, n - 1) - (n - 1) / 2
    yy, xx = np.meshgrid(c, c, indexing="ij")
    exact = duct_series(a, F, (tau - 0.5) / 3, xx, yy)
    assert np.abs(uz - exact).max() <= tol * exact.max()
    assert abs(uz.mean() / exact.mean() - 1) <= tol
    # no cross flow
    assert np.abs(u[:2]).max() < 1e-6 * exact.max()


def _slab(L, axis):
    shape = [1, 1, 1]
    shape[2 - axis] = L
    lab = np.zeros(shape, np.uint16)
    c = np.arange(L).reshape(shape)
    phi0 = np.where((c >= L // 4) & (c < 3 * L // 4), 1.0, -1.0).astype(np.float32)
    return lab, phi0


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_flat_interface_tanh_profile(axis):
    L = 64
    lab, phi0 = _slab(L, axis)
    beta = CONST["interface_profile"]["beta"]
    o = oracle.Oracle(lab, None, (1, 1, 1), alpha=0.005, beta=beta)
    o.init_fluids(phi0)
    o.step(5000)
    phi, _, _ = o.fields()
    x = np.arange(L)
    sel = (np.abs(phi) < 0.95) & (x < L // 2)
    k, b = np.polyfit(x[sel], np.arctanh(phi[sel]), 1)
    assert abs(k / beta - 1) < 0.01
    assert abs(-b / k - (L // 4 - 0.5)) < 1e-6
    # about 5 voxels of interface (|phi| < 0.95), as the paper states for beta = 0.95
    assert 4 <= np.count_nonzero(np.abs(phi[: L // 2]) < 0.95) <= 6


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_flat_interface_normal_stress_balance(axis):
    L = 64
    lab, phi0 = _slab(L, axis)
    alpha = 0.005
    o = oracle.Oracle(lab, None, (1, 1, 1), alpha=alpha, beta=0.95)
    o.init_fluids(phi0)
    o.step(5000)
    phi, p, u = o.fields()
    _, C = o.phase_gradient()
    cmag = np.sqrt((C ** 2).sum(0))
    rho = 3 * p
    rho_bulk = rho[np.abs(phi) > 0.99999].mean()
    predicted = 3 * alpha * cmag * (1 / 3 - 1 / 57)
    sel = cmag > 0.05 * cmag.max()
    ratio = (rho_bulk - rho[sel]) / predicted[sel]
    assert np.abs(ratio - 1).max() < 2e-3
    assert np.abs(u).max() < 1e-7


def _cylinder_dp(plane, L, R, steps=3000):
    shape = {"xz": (L, 1, L), "xy": (1, L, L), "yz": (L, L, 1)}[plane]
    lab = np.zeros(shape, np.uint16)
    z, y, x = np.meshgrid(*[np.arange(n) + 0.5 for n in shape], indexing="ij")
    a, b = {"xz": (x, z), "xy": (x, y), "yz": (y, z)}[plane]
    d = np.sqrt((a - L / 2) ** 2 + (b - L / 2) ** 2)
    phi0 = np.where(d < R, -1.0, 1.0).astype(np.float32)
    o = oracle.Oracle(lab, None, (1, 1, 1), alpha=0.005, beta=0.95)
    o.init_fluids(phi0)
    o.step(steps)
    phi, p, _ = o.fields()
    dd = d.ravel()
    dp = p[dd < R - 4].mean() - p[dd > R + 5].mean()
    r_eff = np.sqrt(((1 - phi) / 2).sum() / np.pi)
    return dp, r_eff


def test_laplace_law_cylinders_slope():
    alpha = 0.005
    sigma = SIGMA_OVER_ALPHA * alpha
    res = [_cylinder_dp("xz", 64, R) for R in (8, 12, 16)]
    inv_r = np.array([1 / r for _, r in res])
    dp = np.array([d for d, _ in res])
    for d, r in res:
        assert abs(d * r / sigma - 1) < 0.05
    slope, icpt = np.polyfit(inv_r, dp, 1)
    assert abs(slope / sigma - 1) < 0.10
    assert abs(icpt) < 0.10 * dp.min()


@pytest.mark.parametrize("plane", ["xy", "yz"])
def test_laplace_law_cylinders_other_planes(plane):
    sigma = SIGMA_OVER_ALPHA * 0.005
    dp, r = _cylinder_dp(plane, 48, 12)
    assert abs(dp * r / sigma - 1) < 0.05


def test_laplace_law_sphere():
    L, R = 28, 7
    lab = np.zeros((L, L, L), np.uint16)
    z, y, x = np.meshgrid(*[np.arange(L) + 0.5] * 3, indexing="ij")
    d = np.sqrt((x - L / 2) ** 2 + (y - L / 2) ** 2 + (z - L / 2) ** 2)
    o = oracle.Oracle(lab, None, (1, 1, 1), alpha=0.005, beta=0.95)
    o.init_fluids(np.where(d < R, -1.0, 1.0).astype(np.float32))
    o.step(1500)
    phi, p, _ = o.fields()
    dd = d.ravel()
    dp = p[dd < R - 4].mean() - p[dd > R + 5].mean()
    r_eff = (3 * ((1 - phi) / 2).sum() / (4 * np.pi)) ** (1 / 3)
    sigma = SIGMA_OVER_ALPHA * 0.005
    assert abs(dp * r_eff / (2 * sigma) - 1) < 0.10


def _interface_points(ph, zmin):
    pts = []
    nz, nx = ph.shape
    for x in range(nx):
        col = ph[:, x]
        for z in range(zmin, nz - 1):
            a, b = col[z], col[z + 1]
            if a * b < 0:
                pts.append((x, z + a / (a - b)))
    for z in range(zmin, nz):
        row = ph[z]
        for x in range(nx - 1):
            a, b = row[x], row[x + 1]
            if a * b < 0:
                pts.append((x + a / (a - b), z))
    return np.array(pts)


def _contact_angle(phis, nx=96, nz=48, R0=14, steps=8000, alpha=0.005):
    lab = np.zeros((nz, 1, nx), np.uint16)
    lab[0] = 1
    aff = np.where(lab != 0, phis, 0).astype(np.float32)
    z, x = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    d = np.sqrt((x - nx / 2) ** 2 + (z - 0.5) ** 2)
    phi0 = np.where(d < R0, 1.0, -1.0).astype(np.float32).reshape(nz, 1, nx)
    o = oracle.Oracle(lab, aff, (1, 1, 0), tau_a=0.7, tau_b=0.7, alpha=alpha, beta=0.95)
    o.init_fluids(phi0)
    o.step(steps)
    phi, _, _ = o.fields()
    pts = _interface_points(o.dense(phi)[:, 0, :], 4)
    # algebraic circle fit
    A = np.vstack([pts[:, 0], pts[:, 1], np.ones(len(pts))]).T
    c = np.linalg.lstsq(A, pts[:, 0] ** 2 + pts[:, 1] ** 2, rcond=None)[0]
    xc, zc = c[0] / 2, c[1] / 2
    R = np.sqrt(c[2] + xc ** 2 + zc ** 2)
    wall = 0.5                       # halfway bounce-back: wall between z = 0 and 1
    return np.degrees(np.arccos(np.clip((wall - zc) / R, -1, 1)))


def test_contact_angle_against_affinity():
    th = {ps: _contact_angle(ps) for ps in (-0.5, 0.0, 0.5)}
    assert abs(th[0.0] - 90) < 3
    assert abs(th[0.5] + th[-0.5] - 180) < 2          # A/B antisymmetry
    assert th[0.5] < th[0.0] < th[-0.5]               # phi_s = +1 water-wet (A wets)
    for ps, t in th.items():
        assert abs(t - np.degrees(np.arccos(ps))) < 15, (ps, t)


def test_contact_angle_is_acos_phis_at_the_stress_scale_of_the_plain_gradient():
    """cos(theta) = phi_s (Sec. 3.2) with the interfacial stress at the scale of
    C = grad(phi): the same model with alpha / 6 (alpha enters only as
    alpha|C|). A wetting drop (phi_s = 0.5, radius of curvature 23 voxels,
    five interface widths) converges to 58.2 degrees; the gate is 3 degrees."""
    th = _contact_angle(0.5, steps=32000, alpha=0.005 / 6)
    assert abs(th - 60.0) < 3.0, th
