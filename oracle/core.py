"""ctypes binding of the C oracle (``lbpm_oracle.c``). Test infrastructure only."""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional

import numpy as np

from .build import build, OUT

_lib = None

MEASURE_FIELDS = (
    "step", "sat_mass", "sat_count", "mass_a", "mass_b", "mass_total",
    "mom_a_x", "mom_a_y", "mom_a_z", "mom_b_x", "mom_b_y", "mom_b_z",
    "flux_x", "flux_y", "flux_z", "flux_a_x", "flux_a_y", "flux_a_z",
    "flux_b_x", "flux_b_y", "flux_b_z", "ke_a", "ke_b", "p_a", "p_b",
    "vol_a", "vol_b", "ca", "n_sites", "status")

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_fp = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_u16p = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def load_library():
    global _lib
    if _lib is not None:
        return _lib
    # LBPM_ORACLE_LIB: another build of the oracle (the tests that plant
    # mistakes in a copy of the source load it in a subprocess)
    path = os.environ.get("LBPM_ORACLE_LIB")
    if not path:
        path = OUT if os.path.exists(OUT) else build()
        if os.path.getmtime(path) < os.path.getmtime(path.replace("liboracle.so", "lbpm_oracle.c")):
            path = build()
    lib = ct.CDLL(path)
    lib.orc_lattice_check.restype = ct.c_double
    lib.orc_tables.argtypes = [_dp, _dp, _dp, _dp, _dp]
    lib.orc_set_threads.argtypes = [ct.c_int]
    lib.orc_get_threads.restype = ct.c_int
    lib.orc_have_openmp.restype = ct.c_int
    lib.orc_collide_site.argtypes = [_dp, _dp, ct.c_double, ct.c_double, _dp, ct.c_int, _dp]
    lib.orc_recolor_site.argtypes = [ct.c_double, ct.c_double, _dp, _dp, ct.c_double, _dp, _dp]
    lib.orc_create.restype = ct.c_void_p
    lib.orc_create.argtypes = [ct.c_int, ct.c_int, ct.c_int, _u16p, ct.c_void_p, _i32p]
    lib.orc_destroy.argtypes = [ct.c_void_p]
    lib.orc_num_sites.restype = ct.c_longlong
    lib.orc_num_sites.argtypes = [ct.c_void_p]
    lib.orc_step_count.restype = ct.c_longlong
    lib.orc_step_count.argtypes = [ct.c_void_p]
    lib.orc_get_index.argtypes = [ct.c_void_p, _i64p, _i32p]
    lib.orc_set_params.argtypes = [ct.c_void_p, ct.c_double, ct.c_double, ct.c_double,
                                   ct.c_double, _dp, ct.c_int, ct.c_double, ct.c_double, ct.c_double]
    lib.orc_set_rate_mode.argtypes = [ct.c_void_p, ct.c_int]
    lib.orc_init_fluids.argtypes = [ct.c_void_p, _fp]
    lib.orc_set_state.argtypes = [ct.c_void_p, _dp, _dp, _dp, ct.c_longlong]
    lib.orc_get_state.argtypes = [ct.c_void_p, _dp, _dp, _dp]
    lib.orc_step.argtypes = [ct.c_void_p, ct.c_int]
    lib.orc_phase_gradient.argtypes = [ct.c_void_p, _dp, _dp]
    lib.orc_fields.argtypes = [ct.c_void_p, _dp, _dp, _dp]
    lib.orc_measure.argtypes = [ct.c_void_p, _dp]
    _lib = lib
    return lib


def set_threads(n: int) -> None:
    load_library().orc_set_threads(int(n))


def get_threads() -> int:
    return int(load_library().orc_get_threads())


def have_openmp() -> bool:
    return bool(load_library().orc_have_openmp())


def lattice_check() -> float:
    return float(load_library().orc_lattice_check())


def lattice_tables():
    """(xi [19,3], t [19], w [7], M [19,19] (row k = moment k), Minv [19,19])."""
    lib = load_library()
    xi = np.zeros(57)
    t = np.zeros(19)
    w = np.zeros(7)
    m = np.zeros(361)
    mi = np.zeros(361)
    lib.orc_tables(xi, t, w, m, mi)
    return xi.reshape(19, 3), t, w, m.reshape(19, 19), mi.reshape(19, 19)


def collide_site(f, C, tau, alpha, F, rate_mode: int = 0) -> np.ndarray:
    out = np.zeros(19)
    load_library().orc_collide_site(np.ascontiguousarray(f, np.float64),
                                    np.ascontiguousarray(C, np.float64), float(tau),
                                    float(alpha), np.ascontiguousarray(F, np.float64),
                                    int(rate_mode), out)
    return out


def recolor_site(Na, Nb, u, C, beta):
    A = np.zeros(7)
    B = np.zeros(7)
    load_library().orc_recolor_site(float(Na), float(Nb), np.ascontiguousarray(u, np.float64),
                                    np.ascontiguousarray(C, np.float64), float(beta), A, B)
    return A, B


class Oracle:
    """One simulated domain held by the C oracle.

    labels: uint16 (nz, ny, nx), 0 = pore; affinity: float32 (nz, ny, nx) phi_s of
    solid voxels; periodic: (px, py, pz).
    """

    def __init__(self, labels: np.ndarray, affinity: Optional[np.ndarray], periodic,
                 tau_a=0.7, tau_b=0.7, alpha=0.005, beta=0.95, force=(0.0, 0.0, 0.0),
                 reservoir_z=0, rho_in=1.0, rho_out=1.0, flux_in=0.0):
        self._lib = load_library()
        labels = np.ascontiguousarray(labels, dtype=np.uint16)
        nz, ny, nx = labels.shape
        self.shape = (nz, ny, nx)
        self.V = nx * ny * nz
        self._aff = None
        aff_ptr = None
        if affinity is not None:
            self._aff = np.ascontiguousarray(affinity, dtype=np.float32)
            aff_ptr = self._aff.ctypes.data
        per = np.ascontiguousarray(periodic, dtype=np.int32)
        self._h = self._lib.orc_create(nx, ny, nz, labels, aff_ptr, per)
        self.N = int(self._lib.orc_num_sites(self._h))
        self.set_params(tau_a, tau_b, alpha, beta, force, reservoir_z, rho_in, rho_out, flux_in)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, tau_a, tau_b, alpha, beta, force, reservoir_z=0, rho_in=1.0,
                   rho_out=1.0, flux_in=0.0):
        self.params = dict(tau_a=tau_a, tau_b=tau_b, alpha=alpha, beta=beta,
                           force=tuple(force), reservoir_z=reservoir_z,
                           rho_in=rho_in, rho_out=rho_out, flux_in=flux_in)
        self._lib.orc_set_params(self._h, float(tau_a), float(tau_b), float(alpha),
                                 float(beta), np.ascontiguousarray(force, np.float64),
                                 int(reservoir_z), float(rho_in), float(rho_out), float(flux_in))

    def set_rate_mode(self, mode: int):
        self._lib.orc_set_rate_mode(self._h, int(mode))

    def init_fluids(self, phi0: np.ndarray):
        self._lib.orc_init_fluids(self._h, np.ascontiguousarray(phi0, np.float32).ravel())

    def index(self):
        sv = np.zeros(self.N, np.int64)
        nb = np.zeros(18 * self.N, np.int32)
        self._lib.orc_get_index(self._h, sv, nb)
        return sv, nb.reshape(18, self.N)

    def state(self):
        f = np.zeros(19 * self.N)
        A = np.zeros(7 * self.N)
        B = np.zeros(7 * self.N)
        self._lib.orc_get_state(self._h, f, A, B)
        return f.reshape(19, self.N), A.reshape(7, self.N), B.reshape(7, self.N)

    def set_state(self, f, A, B, step=0):
        self._lib.orc_set_state(self._h, np.ascontiguousarray(f, np.float64).ravel(),
                                np.ascontiguousarray(A, np.float64).ravel(),
                                np.ascontiguousarray(B, np.float64).ravel(), int(step))

    @property
    def step_count(self) -> int:
        return int(self._lib.orc_step_count(self._h))

    def step(self, n: int = 1):
        self._lib.orc_step(self._h, int(n))

    def phase_gradient(self):
        phi = np.zeros(self.N)
        C = np.zeros(3 * self.N)
        self._lib.orc_phase_gradient(self._h, phi, C)
        return phi, C.reshape(3, self.N)

    def fields(self):
        """(phi [N], p [N], u [3, N]) of the current state, in site order."""
        phi = np.zeros(self.N)
        p = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        self._lib.orc_fields(self._h, phi, p, u)
        return phi, p, u.reshape(3, self.N)

    def dense(self, site_values: np.ndarray, fill=np.nan) -> np.ndarray:
        sv, _ = self.index()
        out = np.full(self.V, fill, dtype=np.float64)
        out[sv] = site_values
        return out.reshape(self.shape)

    def measure(self) -> dict:
        out = np.zeros(len(MEASURE_FIELDS))
        self._lib.orc_measure(self._h, out)
        return dict(zip(MEASURE_FIELDS, out.tolist()))
