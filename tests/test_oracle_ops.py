"""Pins of the oracle's single-site operators (Sec. 3.1).

collision   : fixed point at the second-order equilibrium, BGK special case,
              exact mass/momentum bookkeeping with the body force
recoloring  : per-component conservation, cancellation of the beta terms in
              A + B, A/B symmetry under phi -> -phi, n -> -n
gradient    : exact on linear and quadratic phase fields; phi_s enters at a
              solid neighbour with the face/edge weights of the stencil
"""
import numpy as np
import pytest

import oracle

XI, T, W, _, _ = oracle.lattice_tables()


def feq_poly(rho, j):
    """Second-order incompressible equilibrium t_q [rho + 3 xi.j + 4.5 (xi.j)^2 - 1.5 j.j]
    (rho0 = 1), written independently of the moment basis."""
    cu = XI @ j
    return T * (rho + 3 * cu + 4.5 * cu * cu - 1.5 * (j @ j))


def test_collision_fixed_point_at_equilibrium():
    rng = np.random.default_rng(0)
    for _ in range(20):
        rho = 1 + 0.05 * rng.standard_normal()
        j = 0.02 * rng.standard_normal(3)
        f = feq_poly(rho, j)
        for tau in (0.55, 0.7, 1.3):
            out = oracle.collide_site(f, np.zeros(3), tau, 0.0, np.zeros(3))
            assert np.abs(out - f).max() < 1e-15


def test_collision_mrt_equals_bgk_when_rates_equal():
    rng = np.random.default_rng(1)
    for _ in range(20):
        f = T * (1 + 0.1 * rng.standard_normal(19))
        F = 1e-4 * rng.standard_normal(3)
        tau = float(rng.uniform(0.52, 1.8))
        rho = f.sum()
        j = XI.T @ f
        bgk = f - (f - feq_poly(rho, j)) / tau + 3 * T * (XI @ F)
        out = oracle.collide_site(f, np.zeros(3), tau, 0.0, F, rate_mode=1)
        assert np.abs(out - bgk).max() < 1e-15


def test_collision_conserves_mass_and_adds_force():
    rng = np.random.default_rng(2)
    for _ in range(20):
        f = T * (1 + 0.2 * rng.standard_normal(19))
        C = rng.standard_normal(3)
        F = 1e-3 * rng.standard_normal(3)
        out = oracle.collide_site(f, C, 0.7, 0.01, F)
        assert abs(out.sum() - f.sum()) < 1e-14
        assert np.abs(XI.T @ out - (XI.T @ f + F)).max() < 1e-14


def test_collision_relaxes_toward_equilibrium_with_dhumieres_rates():
    """Non-equilibrium parts decay: the stress moments with s_nu = 1/tau, the
    energy flux with s_m = 8(2 - s_nu)/(8 - s_nu)."""
    _, _, _, M, _ = oracle.lattice_tables()
    rng = np.random.default_rng(3)
    f = T * (1 + 0.1 * rng.standard_normal(19))
    tau = 0.8
    neq = M @ (f - feq_poly(f.sum(), XI.T @ f))
    out = oracle.collide_site(f, np.zeros(3), tau, 0.0, np.zeros(3))
    neq_out = M @ (out - feq_poly(out.sum(), XI.T @ out))
    s_nu = 1 / tau
    s_m = 8 * (2 - s_nu) / (8 - s_nu)
    for k in (1, 2, 9, 10, 11, 12, 13, 14, 15):
        assert abs(neq_out[k] - (1 - s_nu) * neq[k]) < 1e-14
    for k in (4, 6, 8, 16, 17, 18):
        assert abs(neq_out[k] - (1 - s_m) * neq[k]) < 1e-14


def test_recolor_conserves_each_component():
    rng = np.random.default_rng(4)
    for _ in range(50):
        Na, Nb = rng.uniform(0, 1, 2)
        u = 0.01 * rng.standard_normal(3)
        C = rng.standard_normal(3)
        A, B = oracle.recolor_site(Na, Nb, u, C, 0.95)
        assert abs(A.sum() - Na) < 1e-15 and abs(B.sum() - Nb) < 1e-15


def test_recolor_beta_terms_cancel_in_total():
    rng = np.random.default_rng(5)
    for _ in range(20):
        Na, Nb = rng.uniform(0, 1, 2)
        u = 0.01 * rng.standard_normal(3)
        C = rng.standard_normal(3)
        A1, B1 = oracle.recolor_site(Na, Nb, u, C, 0.95)
        A0, B0 = oracle.recolor_site(Na, Nb, u, C, 0.0)
        assert np.abs((A1 + B1) - (A0 + B0)).max() < 1e-15
        # total follows the D3Q7 equilibrium of N with velocity u (c_s^2 = 2/9)
        N = Na + Nb
        assert np.abs((A1 + B1) - W * N * (1 + 4.5 * (XI[:7] @ u))).max() < 1e-15


def test_recolor_symmetry_under_phase_swap():
    rng = np.random.default_rng(6)
    for _ in range(20):
        Na, Nb = rng.uniform(0, 1, 2)
        u = 0.01 * rng.standard_normal(3)
        C = rng.standard_normal(3)
        A, B = oracle.recolor_site(Na, Nb, u, C, 0.9)
        A2, B2 = oracle.recolor_site(Nb, Na, u, -C, 0.9)
        assert np.abs(A - B2).max() < 1e-15 and np.abs(B - A2).max() < 1e-15


def test_recolor_pushes_a_along_normal():
    """With u = 0 the A flux is (2/9) beta Na Nb/N n: it points up the gradient."""
    A, B = oracle.recolor_site(0.5, 0.5, np.zeros(3), np.array([1.0, 0, 0]), 0.95)
    flux_a = XI[:7].T @ A
    assert np.allclose(flux_a, [2 / 9 * 0.95 * 0.25, 0, 0], rtol=1e-14, atol=1e-17)
    assert np.allclose(XI[:7].T @ B, -flux_a, rtol=1e-14)


def _state_from_phi(phi_sites):
    N = phi_sites.size
    Na = 0.5 * (1 + phi_sites)
    Nb = 0.5 * (1 - phi_sites)
    f = np.outer(T, np.ones(N))
    return f, np.outer(W, Na), np.outer(W, Nb)


@pytest.mark.parametrize("kind", ["linear", "quadratic"])
def test_gradient_exact_on_polynomials(kind):
    """The stencil is 18 sum_q t_q xi_q phi(x+xi_q) = 6 grad(phi): exact for
    linear and quadratic phi (second-order terms cancel by symmetry)."""
    nz, ny, nx = 6, 7, 8
    lab = np.zeros((nz, ny, nx), np.uint16)
    o = oracle.Oracle(lab, None, (0, 0, 0))
    sv, _ = o.index()
    x = sv % nx
    y = (sv // nx) % ny
    z = sv // (nx * ny)
    g = np.array([0.021, -0.013, 0.017])
    xc, yc, zc = x - 3.5, y - 3.0, z - 2.5
    phi = 0.1 + g[0] * xc + g[1] * yc + g[2] * zc
    grad = np.vstack([np.full_like(xc, g[0]), np.full_like(yc, g[1]), np.full_like(zc, g[2])])
    if kind == "quadratic":
        H = np.array([[0.004, 0.002, -0.001], [0.002, -0.003, 0.0015], [-0.001, 0.0015, 0.002]])
        P = np.vstack([xc, yc, zc])
        phi = phi + 0.5 * np.einsum("an,ab,bn->n", P, H, P)
        grad = grad + H @ P
    o.set_state(*_state_from_phi(phi))
    phi_o, C = o.phase_gradient()
    assert np.abs(phi_o - phi).max() < 1e-15
    interior = (x > 0) & (x < nx - 1) & (y > 0) & (y < ny - 1) & (z > 0) & (z < nz - 1)
    assert np.abs(C[:, interior] - 6 * grad[:, interior]).max() < 1e-14


def test_gradient_sees_affinity_of_solid_neighbour():
    """One solid voxel with affinity phi_s in a uniform phase c: a face neighbour
    sees (phi_s - c) with weight 1, an edge neighbour with weight 1/2."""
    n = 5
    lab = np.zeros((n, n, n), np.uint16)
    lab[2, 2, 2] = 1
    aff = np.zeros(lab.shape, np.float32)
    aff[2, 2, 2] = -0.5
    o = oracle.Oracle(lab, aff, (1, 1, 1))
    c = 0.3
    o.set_state(*_state_from_phi(np.full(o.N, c)))
    _, C = o.phase_gradient()
    dense = np.stack([o.dense(C[a]) for a in range(3)])
    ps = float(np.float32(-0.5))
    # face neighbour at x-1: the solid lies along +x
    assert np.allclose(dense[:, 2, 2, 1], [(ps - c), 0, 0], atol=1e-15)
    # edge neighbour at (x-1, y-1): the solid lies along (+1, +1, 0)
    assert np.allclose(dense[:, 2, 1, 1], [0.5 * (ps - c), 0.5 * (ps - c), 0], atol=1e-15)
    # far voxel: uniform field, no gradient
    assert np.abs(dense[:, 0, 0, 0]).max() < 1e-15


def test_gradient_wall_outside_non_periodic_face_is_zero_phase():
    n = 4
    lab = np.zeros((n, n, n), np.uint16)
    o = oracle.Oracle(lab, None, (0, 1, 1))
    o.set_state(*_state_from_phi(np.full(o.N, 0.8)))
    _, C = o.phase_gradient()
    dense = np.stack([o.dense(C[a]) for a in range(3)])
    # at x = 0 the outside (x = -1) contributes phi = 0 with weights 1 + 4 * 1/2
    assert np.allclose(dense[0, :, :, 0], 3 * 0.8, atol=1e-14)
    assert np.allclose(dense[0, :, :, n - 1], -3 * 0.8, atol=1e-14)
    assert np.abs(dense[1:]).max() < 1e-14
