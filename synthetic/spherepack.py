"""Seeded sphere-pack images, wetting maps and initial phase fields.

The paper's workloads are segmented micro-CT images of sandstone (Section 5:
a 900x900x1600 Bentheimer sub-volume at porosity 0.235). That dataset is not
available here, so these generators stand in for it with random overlapping
spheres at the porosities and sphere sizes of the named workloads.

Recipe (also stated in the design notes):
  * solid = union of overlapping spheres; centres uniform in [0, L)^3 with the
    periodic minimum image; radius lognormal with the given mean m and sd s of
    r (sigma_l^2 = ln(1 + s^2/m^2), mu_l = ln m - sigma_l^2/2);
  * a voxel (centre at i+1/2, j+1/2, k+1/2) is solid when it lies within r of a
    centre; spheres are added one at a time until porosity <= target;
  * wall-bounded axes get solid planes at index 0 and L-1;
  * affinity (phi_s) is drawn per solid voxel after the geometry;
  * labels: 0 = pore, 1 = solid (the per-voxel affinity map is separate);
  * initial phi: i.i.d. +-1, or "blob" (Gaussian-smoothed white noise,
    sigma = 3 voxels, periodic, thresholded at the pore quantile that gives
    the target saturation Sw of fluid A, phi = +1).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


@dataclasses.dataclass
class SpherePack:
    labels: np.ndarray          # uint16 (nz, ny, nx); 0 = pore
    porosity: float             # realised porosity
    n_spheres: int
    seed: int


def _lognormal_params(mean: float, sd: float):
    s2 = np.log1p((sd / mean) ** 2)
    return np.log(mean) - 0.5 * s2, np.sqrt(s2)


def sphere_pack(L, porosity: float, r_mean: float, r_sd: float, seed: int,
                max_spheres: int = 10_000_000) -> SpherePack:
    """Overlapping-sphere solid in a periodic box of edge L (int or (nx,ny,nz))."""
    if np.isscalar(L):
        nx = ny = nz = int(L)
    else:
        nx, ny, nz = (int(v) for v in L)
    rng = np.random.default_rng(seed)
    mu_l, sig_l = _lognormal_params(r_mean, r_sd)
    solid = np.zeros((nz, ny, nx), dtype=bool)
    V = nx * ny * nz
    n_solid = 0
    target_solid = (1.0 - porosity) * V
    n = 0
    while n_solid < target_solid and n < max_spheres:
        c = rng.uniform(0.0, 1.0, size=3) * np.array([nx, ny, nz])
        r = float(rng.lognormal(mu_l, sig_l))
        r = min(r, 0.49 * min(nx, ny, nz))
        n += 1
        lo = np.floor(c - r - 0.5).astype(np.int64)
        hi = np.ceil(c + r - 0.5).astype(np.int64)
        ix = np.arange(lo[0], hi[0] + 1)
        iy = np.arange(lo[1], hi[1] + 1)
        iz = np.arange(lo[2], hi[2] + 1)
        dx = (ix + 0.5 - c[0]) ** 2
        dy = (iy + 0.5 - c[1]) ** 2
        dz = (iz + 0.5 - c[2]) ** 2
        ball = (dz[:, None, None] + dy[None, :, None] + dx[None, None, :]) <= r * r
        sub = np.ix_(iz % nz, iy % ny, ix % nx)
        before = solid[sub]
        n_solid += int(np.count_nonzero(ball & ~before))
        solid[sub] = before | ball
    labels = solid.astype(np.uint16)
    return SpherePack(labels=labels, porosity=1.0 - n_solid / V, n_spheres=n, seed=seed)


def add_walls(labels: np.ndarray, axes=("x", "y")) -> np.ndarray:
    """Solid planes at index 0 and L-1 on each named axis (returns a copy)."""
    lab = labels.copy()
    for a in axes:
        if a == "x":
            lab[:, :, 0] = 1
            lab[:, :, -1] = 1
        elif a == "y":
            lab[:, 0, :] = 1
            lab[:, -1, :] = 1
        elif a == "z":
            lab[0, :, :] = 1
            lab[-1, :, :] = 1
        else:
            raise ValueError(a)
    return lab


def uniform_affinity(labels: np.ndarray, value: float) -> np.ndarray:
    """Per-voxel affinity map: `value` on every solid voxel, 0 on pores."""
    aff = np.zeros(labels.shape, dtype=np.float32)
    aff[labels != 0] = value
    return aff


def random_affinity(labels: np.ndarray, lo: float, hi: float, seed: int) -> np.ndarray:
    """Per-voxel affinity map drawn i.i.d. U[lo, hi] on solid voxels."""
    rng = np.random.default_rng(seed)
    aff = np.zeros(labels.shape, dtype=np.float32)
    mask = labels != 0
    aff[mask] = rng.uniform(lo, hi, size=int(mask.sum())).astype(np.float32)
    return aff


def phi0_iid(labels: np.ndarray, sw: float, seed: int) -> np.ndarray:
    """phi = +1 with probability sw, else -1, i.i.d. per pore voxel (0 on solid)."""
    rng = np.random.default_rng(seed)
    phi = np.where(rng.uniform(size=labels.shape) < sw, 1.0, -1.0).astype(np.float32)
    phi[labels != 0] = 0.0
    return phi


def _gauss_smooth_periodic(x: np.ndarray, sigma: float) -> np.ndarray:
    out = np.fft.rfftn(x)
    shape = x.shape
    k = [np.fft.fftfreq(n) for n in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    g = np.ones(out.shape)
    for ax, kk in enumerate(k):
        s = [1] * len(shape)
        s[ax] = kk.size
        g = g * np.exp(-2.0 * (np.pi * sigma * kk.reshape(s)) ** 2)
    return np.fft.irfftn(out * g, s=shape, axes=tuple(range(len(shape))))


def phi0_blob(labels: np.ndarray, sw: float, seed: int, sigma: float = 3.0) -> np.ndarray:
    """Random blobs: smoothed noise thresholded so a fraction sw of pores is A."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(labels.shape)
    sm = _gauss_smooth_periodic(noise, sigma)
    pore = labels == 0
    vals = sm[pore]
    thr = np.quantile(vals, 1.0 - sw) if vals.size else 0.0
    phi = np.where(sm > thr, 1.0, -1.0).astype(np.float32)
    phi[~pore] = 0.0
    return phi


def phi0_reservoir(labels: np.ndarray, value: float = -1.0) -> np.ndarray:
    """Uniform interior phase (for displacement runs whose reservoirs set the rest)."""
    phi = np.full(labels.shape, value, dtype=np.float32)
    phi[labels != 0] = 0.0
    return phi


def crop(a: np.ndarray, lo, hi) -> np.ndarray:
    """Sub-volume [lo, hi) given as (x, y, z) triples."""
    return np.ascontiguousarray(a[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]])


@dataclasses.dataclass
class Workload:
    """One synthetic simulation case: image, wetting map, phi0 and parameters."""
    name: str
    labels: np.ndarray
    affinity: np.ndarray
    phi0: np.ndarray
    periodic: tuple
    tau_a: float = 0.7
    tau_b: float = 0.7
    alpha: float = 0.005
    beta: float = 0.95
    force: tuple = (0.0, 0.0, 1e-5)
    steps: int = 200
    reservoir_z: int = 0
    rho_in: float = 1.0
    rho_out: float = 1.0
    porosity: float = 0.0
    meta: Optional[dict] = None

    @property
    def shape_xyz(self):
        nz, ny, nx = self.labels.shape
        return nx, ny, nz

    @property
    def n_pore(self) -> int:
        return int(np.count_nonzero(self.labels == 0))


def workload_parity32(seed: int = 1, phi_seed: int = 2) -> Workload:
    """32^3 periodic pack, r ~ LN(4, 1), porosity 0.35, phi_s = -0.5, i.i.d. phi0."""
    sp = sphere_pack(32, 0.35, 4.0, 1.0, seed)
    return Workload(
        name="spherepack32_parity", labels=sp.labels,
        affinity=uniform_affinity(sp.labels, -0.5),
        phi0=phi0_iid(sp.labels, 0.5, phi_seed), periodic=(1, 1, 1),
        steps=200, porosity=sp.porosity)


def workload_steady256(L: int = 256, seed: int = 3) -> Workload:
    """256^3 steady-state pack: r ~ LN(10, 3), porosity 0.22, z periodic, x/y walls,
    phi_s ~ U[-0.3, 0.3] per solid voxel, blob phi0 at Sw = 0.4, 20k steps."""
    sp = sphere_pack(L, 0.22, 10.0, 3.0, seed)
    lab = add_walls(sp.labels, ("x", "y"))
    return Workload(
        name=f"spherepack{L}_steady", labels=lab,
        affinity=random_affinity(lab, -0.3, 0.3, seed + 1000),
        phi0=phi0_blob(lab, 0.4, seed + 2000), periodic=(0, 0, 1),
        steps=20000, porosity=float(np.count_nonzero(lab == 0) / lab.size))


def workload_precision1024(L: int = 1024, seed: int = 4) -> Workload:
    """Unsteady displacement pack: r ~ LN(10, 3), porosity 0.20, periodic x/y,
    reservoir slabs in z (A inlet at z=0, B outlet at z=L-1), phi0 = -1, phi_s = -0.7."""
    sp = sphere_pack(L, 0.20, 10.0, 3.0, seed)
    return Workload(
        name=f"spherepack{L}_displacement", labels=sp.labels,
        affinity=uniform_affinity(sp.labels, -0.7),
        phi0=phi0_reservoir(sp.labels, -1.0), periodic=(1, 1, 0),
        steps=5000, reservoir_z=1, porosity=sp.porosity)


def workload_batched_job(j: int) -> Workload:
    """Job j of the batched set: L in {64..192}, porosity U[0.15, 0.35], r ~ LN(8, 2),
    periodic z + x/y walls, phi_s ~ U[-0.9, 0.9] per job, blob phi0 at Sw ~ U[0.2, 0.8],
    F_z ~ U[1e-5, 1e-4]."""
    rng = np.random.default_rng(100 + j)
    L = int(rng.choice([64, 96, 128, 160, 192]))
    por = float(rng.uniform(0.15, 0.35))
    aff = float(rng.uniform(-0.9, 0.9))
    sw = float(rng.uniform(0.2, 0.8))
    fz = float(rng.uniform(1e-5, 1e-4))
    sp = sphere_pack(L, por, 8.0, 2.0, 100 + j)
    lab = add_walls(sp.labels, ("x", "y"))
    return Workload(
        name=f"batched_job{j}_L{L}", labels=lab,
        affinity=uniform_affinity(lab, aff),
        phi0=phi0_blob(lab, sw, 5000 + j), periodic=(0, 0, 1),
        force=(0.0, 0.0, fz), steps=2000,
        porosity=float(np.count_nonzero(lab == 0) / lab.size))


def serving_job(i: int, seed: int = 5, L_choices=(64, 96, 128, 160, 192, 224, 256, 288, 320, 352, 384)) -> Workload:
    """Job i of a serving trace: L uniform on L_choices, porosity U[0.15, 0.35],
    r ~ LN(8, 2); kind mix 50 % steady state (x/y walls, z periodic, blob phi0,
    F_z = 1e-5), 30 % unsteady displacement (reservoirs in z, interior phi0 = -1,
    phi_s = -0.7, F_z = 1e-5) and 20 % centrifuge-like (reservoirs, F_z from 1e-5
    doubled at each saturation plateau up to 1.6e-4)."""
    rng = np.random.default_rng(seed * 100003 + i)
    L = int(rng.choice(list(L_choices)))
    por = float(rng.uniform(0.15, 0.35))
    u = float(rng.uniform())
    kind = "steady" if u < 0.5 else ("unsteady" if u < 0.8 else "centrifuge")
    sp = sphere_pack(L, por, 8.0, 2.0, seed * 7919 + i)
    if kind == "steady":
        lab = add_walls(sp.labels, ("x", "y"))
        w = Workload(name=f"serve{i}_steady_L{L}", labels=lab,
                     affinity=random_affinity(lab, -0.3, 0.3, seed * 31 + i),
                     phi0=phi0_blob(lab, float(rng.uniform(0.2, 0.8)), seed * 37 + i),
                     periodic=(0, 0, 1), force=(0.0, 0.0, 1e-5), steps=10000)
    else:
        lab = sp.labels
        w = Workload(name=f"serve{i}_{kind}_L{L}", labels=lab, affinity=uniform_affinity(lab, -0.7),
                     phi0=phi0_reservoir(lab, -1.0), periodic=(1, 1, 0), force=(0.0, 0.0, 1e-5),
                     reservoir_z=1, steps=10000)
    w.meta = {"kind": kind, "L": L}
    w.porosity = float(np.count_nonzero(lab == 0) / lab.size)
    return w
