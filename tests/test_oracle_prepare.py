"""Pins of the image-preparation oracle (mixing region, mixed-wet relabel)."""
import numpy as np
import pytest

from oracle import prepare


def test_ball_sizes_are_lattice_point_counts():
    # lattice points with 0 < |o|^2 <= r^2: shells of 6, 12, 8, 6 points
    assert len(prepare.ball_offsets(1.0)) == 6
    assert len(prepare.ball_offsets(np.sqrt(2.0))) == 18
    assert len(prepare.ball_offsets(1.7321)) == 26     # just above sqrt(3)
    assert len(prepare.ball_offsets(2.0)) == 32


def test_single_oil_voxel_relabels_a_ball():
    lab = np.ones((9, 9, 9), np.uint16)
    oil = np.zeros_like(lab, dtype=bool)
    oil[4, 4, 4] = True
    lab[4, 4, 4] = 0                       # the oil sits in a pore voxel
    out = prepare.mixed_wet_relabel(lab, oil, (0, 0, 0), 2.0, 7)
    assert np.count_nonzero(out == 7) == 32
    z, y, x = np.nonzero(out == 7)
    d2 = (z - 4) ** 2 + (y - 4) ** 2 + (x - 4) ** 2
    assert d2.max() == 4 and d2.min() == 1
    assert out[4, 4, 4] == 0               # pores are never relabelled


def test_relabel_matches_scipy_distance_transform():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    lab = np.where(rng.uniform(size=(13, 11, 17)) < 0.5, 3, 0).astype(np.uint16)
    oil = (rng.uniform(size=lab.shape) < 0.03) & (lab == 0)
    for r in (1.0, 1.5, 2.0, 2.5, 3.0):
        out = prepare.mixed_wet_relabel(lab, oil, (0, 0, 0), r, 9)
        dist = ndi.distance_transform_edt(~oil)       # distance to the nearest oil voxel
        want = np.where((lab != 0) & (dist <= r), 9, lab)
        assert np.array_equal(out, want), r


def test_relabel_wraps_on_periodic_axes():
    lab = np.ones((6, 6, 6), np.uint16)
    oil = np.zeros(lab.shape, bool)
    oil[0, 0, 0] = True
    lab[0, 0, 0] = 0
    per = prepare.mixed_wet_relabel(lab, oil, (1, 1, 1), 2.0, 5)
    non = prepare.mixed_wet_relabel(lab, oil, (0, 0, 0), 2.0, 5)
    assert np.count_nonzero(per == 5) == 32          # the whole ball, through the faces
    assert per[5, 5, 5] == 5 and non[5, 5, 5] == 1    # (-1, -1, -1) wraps to the far corner
    # without wrap only the ball's points in the non-negative octant remain:
    # (1,0,0) x3, (1,1,0) x3, (1,1,1), (2,0,0) x3
    assert np.count_nonzero(non == 5) == 10


def _img():
    # 4 x 3 x 6 image (nz, ny, nx); z is the flow axis
    lab = np.ones((6, 3, 4), np.uint16)
    lab[0, 1, 2] = 0      # inlet face pores
    lab[0, 2, 0] = 0
    lab[5, 0, 1] = 0      # outlet face pores
    lab[5, 2, 0] = 0
    return lab


def test_mixing_layer_by_hand():
    lab = _img()
    out = prepare.mixing_layer(lab, axis=2, n_mix=2)
    # inlet layers z = 0, 1: cleared where the outlet face is pore, (x, y) = (1, 0) and (0, 2)
    for z in (0, 1):
        assert out[z, 0, 1] == 0 and out[z, 2, 0] == 0
    # outlet layers z = 4, 5: cleared where the inlet face is pore, (2, 1) and (0, 2)
    for z in (4, 5):
        assert out[z, 1, 2] == 0 and out[z, 2, 0] == 0
    # the middle is untouched, no pore turns solid, nothing else changes
    assert np.array_equal(out[2:4], lab[2:4])
    assert not np.any((lab == 0) & (out != 0))
    changed = np.argwhere(out != lab)
    # two columns in each of the four layers, minus the face voxels (0, 2) of
    # z = 0 and z = 5 that were pore already
    assert len(changed) == 4 * 2 - 2
    # other axes: the same rule on the transposed image
    outx = prepare.mixing_layer(np.transpose(lab, (2, 1, 0)).copy(), axis=0, n_mix=2)
    assert np.array_equal(np.transpose(outx, (2, 1, 0)), out)


def test_mixing_layer_keeps_the_wetting_labels():
    lab = _img() * 4
    lab[3, 1, 1] = 9
    out = prepare.mixing_layer(lab, axis=2, n_mix=1)
    kept = (out != 0)
    assert np.array_equal(out[kept], lab[kept])
