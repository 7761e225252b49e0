"""Pins of the shell-aggregation oracle (Sec. 3.3): the distance map built from
Eq. lb-dist and its far-field rule, and the new phase of Eq.
lb-dist-to-phase."""
import numpy as np
import pytest

import oracle
from oracle import morph

BETA = 0.95
W7 = morph.W7
T19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _oracle_with_phase(shape, periodic, phi_of_xyz, n_of_xyz=None):
    """Oracle at rest with phase phi and total component density N (default 1)."""
    nz, ny, nx = shape
    lab = np.zeros(shape, np.uint16)
    o = oracle.Oracle(lab, np.zeros(shape, np.float32), periodic, tau_a=0.7, tau_b=0.7, alpha=0.005,
                      beta=BETA, force=(0, 0, 0))
    o.init_fluids(np.zeros(shape, np.float32))
    sv, _ = o.index()
    z, r = np.divmod(sv, ny * nx)
    y, x = np.divmod(r, nx)
    phi = phi_of_xyz(x.astype(float), y.astype(float), z.astype(float))
    N = np.ones_like(phi) if n_of_xyz is None else n_of_xyz(x.astype(float), y.astype(float), z.astype(float))
    A = W7[:, None] * (0.5 * N * (1 + phi))[None, :]
    B = W7[:, None] * (0.5 * N * (1 - phi))[None, :]
    f = np.repeat(T19[:, None], o.N, axis=1)
    o.set_state(f, A, B, 0)
    return o, x, y, z, phi


def test_flat_equilibrium_interface_moves_by_delta():
    x0, delta = 12.3, 0.7
    # a non-uniform total density: the re-initialised sites must keep theirs
    n_of = lambda x, y, z: 1.0 + 0.03 * np.sin(0.7 * x + 0.3 * y)
    o, x, y, z, phi = _oracle_with_phase((4, 4, 24), (0, 1, 1), lambda x, y, z: np.tanh(BETA * (x0 - x)), n_of)
    before, after = morph.morph(o, delta, BETA, (0, 1, 1))
    _, A, B = o.state()
    phin = (A.sum(0) - B.sum(0)) / (A.sum(0) + B.sum(0))
    d = np.abs(x - x0)
    band = d < 3.0
    # nearest band voxel of a non-band site, along the normal
    xb = x[band]
    reach = band | np.array([np.min(np.abs(xb - xi)) <= 4 for xi in x])
    want = np.where(reach, np.tanh(BETA * (x0 + delta - x)), phi)
    assert np.abs(phin - want).max() < 1e-12
    assert np.abs(A.sum(0) + B.sum(0) - n_of(x, y, z)).max() < 1e-14      # N kept at every site


def test_one_voxel_of_dilation_adds_one_plane():
    x0 = 11.5 + 0.25
    o, x, _, _, _ = _oracle_with_phase((5, 6, 24), (0, 1, 1), lambda x, y, z: np.tanh(BETA * (x0 - x)))
    before, after = morph.morph(o, 1.0, BETA, (0, 1, 1), apply=False)
    assert before == np.count_nonzero(x < x0)
    assert after - before == 5 * 6
    before, after = morph.morph(o, -1.0, BETA, (0, 1, 1), apply=False)
    assert before - after == 5 * 6


@pytest.mark.parametrize("delta", [1.0, -1.5, 2.25])
def test_relaxed_drop_grows_by_a_shell(delta):
    R0, c = 6.0, 11.5
    shape = (24, 24, 24)
    r = lambda x, y, z: np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    o, x, y, z, _ = _oracle_with_phase(shape, (1, 1, 1), lambda x, y, z: np.tanh(BETA * (R0 - r(x, y, z))))
    before, after = morph.morph(o, delta, BETA, (1, 1, 1), apply=False)
    rr = r(x, y, z)
    # inside the band the distance map is exact, so the new drop is r < R0 + delta
    assert before == np.count_nonzero(rr < R0)
    assert after == np.count_nonzero(rr < R0 + delta)
