"""Oracle of the shell-aggregation morphological step (test infrastructure only).

Sec. 3.3 (shell aggregation protocol) moves the fluid-fluid interface of fluid
a by a distance delta through the distance map Phi_a (< 0 inside fluid a) and
re-initialises the component densities from the new phase field. Readings
(the same as the CUDA path's):

* Phi_a near the interface is Eq. lb-dist solved for the distance,
  Phi = -atanh(phi) / beta, on the band |phi| < tanh(3 beta);
* further out it is min over band voxels y within R = 4 voxels of
  |x - y| + |Phi(y)| with the sign of -phi(x); voxels with no band voxel
  within R keep their phase;
* phi' = -tanh(beta (Phi - delta)) (Eq. lb-dist-to-phase);
* the changed sites get A_q = w_q N (1 + phi')/2, B_q = w_q N (1 - phi')/2 at
  rest, N = Na + Nb of the site; the momentum populations are unchanged.

numpy, fp64, whole-array shifts over the ball offsets. Pins in
tests/test_oracle_morph.py: a flat equilibrium interface moves by exactly
delta, one voxel of dilation adds exactly one voxel plane, a relaxed drop grows
by the volume of a shell, N is conserved per site.
"""
from __future__ import annotations

import numpy as np

RADIUS = 4
W7 = np.array([1 / 3] + [1 / 9] * 6)


def ball(R: int = RADIUS):
    return [(x, y, z) for z in range(-R, R + 1) for y in range(-R, R + 1) for x in range(-R, R + 1)
            if 0 < x * x + y * y + z * z <= R * R]


def _shifted(grid: np.ndarray, o, periodic, fill) -> np.ndarray:
    """out[x] = grid[x + o] on a (nz, ny, nx) grid; `fill` outside non-periodic axes."""
    res = grid
    for comp, (d, per) in enumerate(zip(o, periodic)):
        if d == 0:
            continue
        ax = 2 - comp
        if per:
            res = np.roll(res, -d, axis=ax)
        else:
            n = res.shape[ax]
            out = np.full_like(res, fill)
            src = [slice(None)] * 3
            dst = [slice(None)] * 3
            if d > 0:
                src[ax], dst[ax] = slice(d, n), slice(0, n - d)
            else:
                src[ax], dst[ax] = slice(0, n + d), slice(-d, n)
            out[tuple(dst)] = res[tuple(src)]
            res = out
    return res


def new_phase(phi: np.ndarray, site_vox: np.ndarray, shape, periodic, beta: float, delta: float):
    """phi per site -> (phi' per site, changed mask): the distance map and Eq.
    lb-dist-to-phase. shape = (nz, ny, nx); site_vox = linear voxel index."""
    phi = np.asarray(phi, np.float64)
    band = np.abs(phi) < np.tanh(3.0 * beta)
    dist = np.full(int(np.prod(shape)), np.inf)
    dist[site_vox[band]] = np.abs(np.arctanh(phi[band])) / beta
    dist = dist.reshape(shape)
    best = np.full(shape, np.inf)
    for o in ball():
        best = np.minimum(best, np.sqrt(o[0] ** 2 + o[1] ** 2 + o[2] ** 2) + _shifted(dist, o, periodic, np.inf))
    best = best.ravel()[site_vox]
    Phi = np.where(band, -np.arctanh(np.where(band, phi, 0.0)) / beta,
                   np.where(phi > 0, -best, best))
    changed = band | np.isfinite(best)
    phin = np.where(changed, -np.tanh(beta * (Phi - delta)), phi)
    return phin, changed


def morph(o, delta: float, beta: float, periodic, apply: bool = True):
    """One morphological step on an oracle.Oracle; returns (A sites before,
    after). With apply the oracle's state is updated."""
    f, A, B = o.state()
    Na, Nb = A.sum(axis=0), B.sum(axis=0)
    N = Na + Nb
    phi = np.where(N > 0, (Na - Nb) / np.where(N > 0, N, 1.0), 0.0)
    sv, _ = o.index()
    phin, changed = new_phase(phi, sv, o.shape, periodic, beta, delta)
    before = int(np.count_nonzero(phi > 0))
    after = int(np.count_nonzero(phin > 0))
    if apply:
        A, B = A.copy(), B.copy()
        na, nb = 0.5 * N * (1 + phin), 0.5 * N * (1 - phin)
        A[:, changed] = W7[:, None] * na[changed]
        B[:, changed] = W7[:, None] * nb[changed]
        o.set_state(f, A, B, o.step_count)
    return before, after
