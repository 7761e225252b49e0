"""Pins of the oracle's lattice tables against closed forms and printed values.

Sec. 3.1 (Eq. d3q19 and the weights given with the LBEs) fixes the velocity
groups and weights; d'Humieres et al. (2002), cited there for M, fixes the
moment basis (its squared row norms are stored under tests/golden).
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def test_velocity_groups_match_paper():
    xi, t, w, M, Minv = oracle.lattice_tables()
    g = _load("paper_constants.json")["d3q19_groups"]
    assert np.all(xi[0] == 0)
    for key, axes in (("x_faces", [0]), ("y_faces", [1]), ("z_faces", [2]),
                      ("xy_edges", [0, 1]), ("xz_edges", [0, 2]), ("yz_edges", [1, 2])):
        qs = g[key]
        vecs = {tuple(int(v) for v in xi[q]) for q in qs}
        expect = set()
        for signs in itertools.product((-1, 1), repeat=len(axes)):
            v = [0, 0, 0]
            for a, s in zip(axes, signs):
                v[a] = s
            expect.add(tuple(v))
        assert vecs == expect, key
    # opposite pairs are adjacent: (1,2), (3,4), ...
    for q in range(1, 19, 2):
        assert np.all(xi[q] == -xi[q + 1])


def test_weights_match_paper():
    xi, t, w, M, Minv = oracle.lattice_tables()
    g = _load("paper_constants.json")
    fr = lambda p: p[0] / p[1]
    assert abs(t[0] - fr(g["d3q19_weights"]["t0"])) < 1e-16
    assert np.allclose(t[1:7], fr(g["d3q19_weights"]["t_face"]), atol=0, rtol=1e-15)
    assert np.allclose(t[7:], fr(g["d3q19_weights"]["t_edge"]), atol=0, rtol=1e-15)
    assert abs(w[0] - fr(g["d3q7_weights"]["w0"])) < 1e-16
    assert np.allclose(w[1:], fr(g["d3q7_weights"]["w_face"]), atol=0, rtol=1e-15)


def test_isotropy_d3q19():
    xi, t, _, _, _ = oracle.lattice_tables()
    assert abs(t.sum() - 1) < 1e-15
    assert np.abs(t @ xi).max() < 1e-16
    second = np.einsum("q,qa,qb->ab", t, xi, xi)
    assert np.abs(second - np.eye(3) / 3).max() < 1e-15          # c_s^2 = 1/3
    third = np.einsum("q,qa,qb,qc->abc", t, xi, xi, xi)
    assert np.abs(third).max() < 1e-16
    fourth = np.einsum("q,qa,qb,qc,qd->abcd", t, xi, xi, xi, xi)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.abs(fourth - iso).max() < 1e-15


def test_isotropy_d3q7():
    xi, _, w, _, _ = oracle.lattice_tables()
    x7 = xi[:7]
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ x7).max() < 1e-16
    second = np.einsum("q,qa,qb->ab", w, x7, x7)
    cs2 = _load("paper_constants.json")["d3q7_weights"]["cs2"]
    assert np.abs(second - np.eye(3) * cs2[0] / cs2[1]).max() < 1e-15   # c_s^2 = 2/9


def test_moment_basis_norms_and_orthogonality():
    _, _, _, M, Minv = oracle.lattice_tables()
    norms = _load("dhumieres_d3q19_norms.json")["norms"]
    G = M @ M.T
    assert np.abs(np.diag(G) - np.array(norms, float)).max() < 1e-12
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-12
    assert oracle.lattice_check() < 1e-14
    assert np.abs(M @ Minv - np.eye(19)).max() < 1e-14
    # integer entries: each row is an integer polynomial of xi
    assert np.all(M == np.round(M))


def test_moment_rows_named_by_paper_equilibria():
    """m13, m14, m15 are p_xy, p_yz, p_xz (the paper pairs them with n_x n_y,
    n_y n_z, n_x n_z); m9 and m11 are 3p_xx and p_ww."""
    xi, _, _, M, _ = oracle.lattice_tables()
    x, y, z = xi.T
    assert np.all(M[13] == x * y) and np.all(M[14] == y * z) and np.all(M[15] == x * z)
    assert np.all(M[9] == 3 * x * x - (x * x + y * y + z * z))
    assert np.all(M[11] == y * y - z * z)
    assert np.all(M[3] == x) and np.all(M[5] == y) and np.all(M[7] == z)


def test_exact_fractions_of_weights():
    _, t, w, _, _ = oracle.lattice_tables()
    assert Fraction(t[1]).limit_denominator(100) == Fraction(1, 18)
    assert Fraction(t[7]).limit_denominator(100) == Fraction(1, 36)
    assert Fraction(w[1]).limit_denominator(100) == Fraction(1, 9)
