"""Oracle of the image-preparation steps (test infrastructure only).

Plain numpy restatements of two image operations of the paper, written from
their description and sharing nothing with the CUDA kernels:

* mixing region (Sec. 4.2): within n_mix voxels of the inlet and the outlet
  of the flow axis, solid voxels that block the pore structure of the other
  face are removed - inlet layers use the pore space of the outlet face,
  outlet layers the pore space of the inlet face (reading: the face is the
  last / first voxel layer, applied voxel by voxel along lines parallel to
  the axis);
* mixed-wet relabel (Sec. 3.3): after a distance transform of the oil phase,
  solid voxels within 2 voxel units of the oil get a new label (reading:
  Euclidean distance between voxel centres, <= the radius, minimum image on
  periodic axes).

Pins (tests/test_oracle_prepare.py): the exact relabel counts around a single
oil voxel (lattice points of a ball), scipy's Euclidean distance transform on
non-periodic images, wrap-around on periodic axes, and hand-built images for
the mixing region.
"""
from __future__ import annotations

import numpy as np

AXIS_OF = {0: 2, 1: 1, 2: 0}   # x, y, z -> numpy axis of a (nz, ny, nx) array


def mixing_layer(labels: np.ndarray, axis: int, n_mix: int) -> np.ndarray:
    """Sec. 4.2 mixing region; `axis` counts x = 0, y = 1, z = 2."""
    lab = np.asarray(labels)
    out = lab.copy()
    ax = AXIS_OF[axis]
    L = lab.shape[ax]
    inlet_face = np.take(lab, [0], axis=ax)          # first layer, kept as a 1-thick slab
    outlet_face = np.take(lab, [L - 1], axis=ax)
    for a in range(L):
        layer = np.take(lab, [a], axis=ax)
        new = np.take(out, [a], axis=ax)
        if a < n_mix:
            new = np.where((layer != 0) & (outlet_face == 0), 0, new)
        if a >= L - n_mix:
            new = np.where((layer != 0) & (inlet_face == 0), 0, new)
        idx = [slice(None)] * 3
        idx[ax] = slice(a, a + 1)
        out[tuple(idx)] = new
    return out


def ball_offsets(radius: float):
    """Integer offsets o != 0 with |o| <= radius."""
    R = int(np.floor(radius))
    return [(x, y, z) for z in range(-R, R + 1) for y in range(-R, R + 1) for x in range(-R, R + 1)
            if (x, y, z) != (0, 0, 0) and x * x + y * y + z * z <= radius * radius]


def _shift(mask: np.ndarray, o, periodic) -> np.ndarray:
    """out[v] = mask[v + o] (False outside non-periodic axes)."""
    res = mask.copy()
    for c, (d, per) in enumerate(zip(o, periodic)):
        ax = AXIS_OF[c]
        if d == 0:
            continue
        if per:
            res = np.roll(res, -d, axis=ax)
        else:
            n = res.shape[ax]
            shifted = np.zeros_like(res)
            src = [slice(None)] * 3
            dst = [slice(None)] * 3
            if d > 0:
                src[ax], dst[ax] = slice(d, n), slice(0, n - d)
            else:
                src[ax], dst[ax] = slice(0, n + d), slice(-d, n)
            shifted[tuple(dst)] = res[tuple(src)]
            res = shifted
    return res


def mixed_wet_relabel(labels: np.ndarray, oil: np.ndarray, periodic, radius: float, new_label: int) -> np.ndarray:
    """Sec. 3.3 relabel: solid voxels within `radius` of an oil voxel."""
    lab = np.asarray(labels)
    o = np.asarray(oil) != 0
    near = np.zeros(lab.shape, dtype=bool)
    for off in ball_offsets(radius):
        near |= _shift(o, off, periodic)
    out = lab.copy()
    out[(lab != 0) & near] = new_label
    return out
