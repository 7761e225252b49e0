"""Pins of the oracle's sparse pore-site indexer.

The labelled image (Sec. 3.3: one integer label per voxel; here 0 = pore)
is compacted lexicographically (x fastest). For each site and direction
q = 1..18 the neighbour table holds the site id of voxel + xi_q, wrapped on
periodic axes, or -1 where that voxel is solid or outside a non-periodic face.
The pins: an independent NumPy re-derivation and neighbour symmetry.
"""
import numpy as np
import pytest

import oracle
from synthetic import sphere_pack

XI = oracle.lattice_tables()[0].astype(int)
OPP = np.array([0] + [q + 1 if q % 2 else q - 1 for q in range(1, 19)])


def brute_index(labels, periodic):
    nz, ny, nx = labels.shape
    flat = labels.ravel()
    site_vox = np.flatnonzero(flat == 0).astype(np.int64)
    vox_site = -np.ones(flat.size, np.int64)
    vox_site[site_vox] = np.arange(site_vox.size)
    x = site_vox % nx
    y = (site_vox // nx) % ny
    z = site_vox // (nx * ny)
    nbr = np.empty((18, site_vox.size), np.int32)
    for q in range(1, 19):
        c = [x + XI[q, 0], y + XI[q, 1], z + XI[q, 2]]
        ok = np.ones(site_vox.size, bool)
        for a, L in enumerate((nx, ny, nz)):
            if periodic[a]:
                c[a] = np.mod(c[a], L)
            else:
                ok &= (c[a] >= 0) & (c[a] < L)
                c[a] = np.clip(c[a], 0, L - 1)
        t = vox_site[c[0] + nx * (c[1] + ny * c[2])]
        nbr[q - 1] = np.where(ok, t, -1)
    return site_vox, nbr


@pytest.mark.parametrize("shape,periodic", [
    ((8, 8, 8), (1, 1, 1)), ((5, 7, 9), (0, 1, 1)), ((9, 4, 6), (1, 0, 0)),
    ((6, 6, 6), (0, 0, 0)), ((1, 1, 7), (1, 1, 1)), ((3, 1, 5), (0, 1, 0))])
def test_index_matches_brute_force(shape, periodic):
    nz, ny, nx = shape
    rng = np.random.default_rng(sum(shape))
    lab = (rng.uniform(size=shape) < 0.4).astype(np.uint16)
    o = oracle.Oracle(lab, None, periodic)
    sv, nb = o.index()
    sv2, nb2 = brute_index(lab, periodic)
    assert np.array_equal(sv, sv2)
    assert np.array_equal(nb, nb2)


def test_index_symmetry_on_sphere_pack():
    sp = sphere_pack(24, 0.35, 3.0, 1.0, 11)
    for per in ((1, 1, 1), (0, 0, 1)):
        o = oracle.Oracle(sp.labels, None, per)
        sv, nb = o.index()
        n = np.arange(o.N)
        for q in range(1, 19):
            t = nb[q - 1]
            ok = t >= 0
            assert np.array_equal(nb[OPP[q] - 1][t[ok]], n[ok])


def test_index_empty_and_full():
    full = np.ones((4, 4, 4), np.uint16)
    o = oracle.Oracle(full, None, (1, 1, 1))
    assert o.N == 0
    empty = np.zeros((3, 3, 3), np.uint16)
    o = oracle.Oracle(empty, None, (1, 1, 1))
    sv, nb = o.index()
    assert o.N == 27 and np.array_equal(sv, np.arange(27))
    assert (nb >= 0).all()
