"""GB300-native color-gradient lattice Boltzmann (LBPM two-fluid model).

Python binding of the CUDA library ``libcolorlbm.so`` (C ABI in
``include/lbpm.h``). This layer only marshals arguments: image loading,
indexing, time stepping, measures and exports all run in the library's CUDA
kernels on sm_103a. PyTorch supplies the device memory (its caching
allocator) and the CUDA stream.

Model: Sec. 3.1 of the LBPM paper (arXiv 2007.12266) - D3Q19 MRT momentum
LBE with the color-gradient interfacial-tension terms, two D3Q7 component
LBEs with recoloring, wetting affinity phi_s at solid voxels (Sec. 3.2).
"""
from __future__ import annotations

import atexit
import ctypes as ct
import json
import weakref
from typing import Optional

import numpy as np

from . import _lib
from ._lib import JobSpec, JobStatus, LBPMError, Measures, Params

__all__ = ["Domain", "Batch", "Server", "trace_run", "TRACE_FIELDS", "JOB_KINDS", "JOB_STATES", "LBPMError", "FIELDS", "DISTS", "STEP_FORMS", "library_path",
           "version", "force_rescale", "mixing_layer", "mixed_wet_relabel"]

STEP_FORMS = {"auto": 0, "populations": 1}
FIELDS = {"phi": 0, "pressure": 1, "ux": 2, "uy": 3, "uz": 4, "na": 5, "nb": 6, "rho": 7}
DISTS = {"f": (0, 19), "a": (1, 7), "b": (2, 7)}
PRECISION = {"fp32": 0, "fp16": 1}
JOB_KINDS = {"steady": 0, "unsteady": 1, "centrifuge": 2}
JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


def library_path() -> str:
    return _lib.library_path()


def version() -> str:
    return _lib.load().lbpm_version().decode()


def force_rescale(force, ca: float, ca_target: float, max_factor: float = 2.0):
    """Body force rescaled toward a target capillary number (library call
    lbpm_force_rescale): returns (new_force, factor)."""
    L = _lib.load()
    f = (ct.c_double * 3)(*[float(x) for x in force])
    out = (ct.c_double * 3)()
    g = ct.c_double()
    st = L.lbpm_force_rescale(f, float(ca), float(ca_target), float(max_factor), out, ct.byref(g))
    if st != 0:
        raise LBPMError(st, "invalid force rescale arguments")
    return tuple(out), g.value


_LIVE = weakref.WeakSet()


@atexit.register
def _close_all():
    # release device memory through the allocator callbacks while torch is alive
    for d in list(_LIVE):
        try:
            d.close()
        except Exception:
            pass


def _params(tau_a, tau_b, alpha, beta, force, precision, periodic, reservoir_z, rho_in, rho_out,
            flux_in=0.0) -> Params:
    p = Params()
    p.tau_a, p.tau_b, p.alpha, p.beta = float(tau_a), float(tau_b), float(alpha), float(beta)
    for a in range(3):
        p.force[a] = float(force[a])
        p.periodic[a] = int(periodic[a])
    p.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    p.reservoir_z = int(reservoir_z)
    p.rho_in, p.rho_out = float(rho_in), float(rho_out)
    p.flux_in = float(flux_in)
    return p


def _measures_dict(m: Measures) -> dict:
    out = {}
    for name, _ in Measures._fields_:
        v = getattr(m, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    return out


TRACE_FIELDS = ("step", "sat_mass", "sat_count", "flux", "flux_a", "flux_b", "ca", "mass_drift", "status")


def trace_run(sim, steps: int, interval: int, path: Optional[str] = None) -> list:
    """Advance `sim` (a Domain) by `steps` timesteps in chunks of `interval`,
    taking the basic analysis (Sec. 4) before the first chunk and after each:
    one row per analysis with the step, both saturations, the Darcy and phase
    fluxes, the capillary number, the drift of the total component mass
    (Na + Nb summed over the sites) relative to the first row, and the status.
    With `path`, the rows are appended to that file as JSON lines. Stops early
    (after writing the row) when a measure reports an unstable state."""
    if interval <= 0 or steps < 0:
        raise ValueError("interval must be > 0 and steps >= 0")
    rows = []
    m0 = None
    done = 0
    fh = open(path, "a") if path else None
    try:
        while True:
            m = sim.measure()
            if m0 is None:
                m0 = m
            total0 = m0["mass_a"] + m0["mass_b"]
            row = {"step": int(m["step"]), "sat_mass": m["sat_mass"], "sat_count": m["sat_count"],
                   "flux": list(m["flux"]), "flux_a": list(m["flux_a"]), "flux_b": list(m["flux_b"]),
                   "ca": m["ca"],
                   "mass_drift": (m["mass_a"] + m["mass_b"]) / total0 - 1.0 if total0 else 0.0,
                   "status": int(m["status"])}
            rows.append(row)
            if fh:
                fh.write(json.dumps(row) + "\n")
                fh.flush()
            if row["status"] != 0 or done >= steps:
                return rows
            n = min(interval, steps - done)
            sim.advance(n)
            done += n
    finally:
        if fh:
            fh.close()


def _torch_allocator(torch, device, stream):
    def _alloc(nbytes, strm, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), device, stream))
        except Exception:
            return None

    def _free(ptr, user):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    return _lib.ALLOC_FN(_alloc), _lib.FREE_FN(_free)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the color-LBM library runs on the GPU only")
    return torch


def mixing_layer(labels: np.ndarray, n_mix: int, axis: int = 2, device: int = 0) -> np.ndarray:
    """Mixing region at the inlet/outlet faces of `axis` (library call
    lbpm_mixing_layer, runs on the GPU). labels: (nz, ny, nx); axis counts
    x = 0, y = 1, z = 2. Returns the new label image."""
    _torch()
    lab = np.array(labels, dtype=np.uint16, order="C", copy=True)
    nz, ny, nx = lab.shape
    st = _lib.load().lbpm_mixing_layer(int(device), lab.ctypes.data, nx, ny, nz, int(axis), int(n_mix))
    if st != 0:
        raise LBPMError(st, "lbpm_mixing_layer failed")
    return lab


def mixed_wet_relabel(labels: np.ndarray, oil: np.ndarray, radius: float = 2.0, new_label: int = 2,
                      periodic=(1, 1, 1), device: int = 0) -> np.ndarray:
    """Relabel the solid within `radius` voxels of the oil phase (library call
    lbpm_mixed_wet_relabel, runs on the GPU). oil: boolean (nz, ny, nx)."""
    _torch()
    lab = np.array(labels, dtype=np.uint16, order="C", copy=True)
    o = np.ascontiguousarray(oil, dtype=np.uint8)
    if o.shape != lab.shape:
        raise ValueError("oil mask must match the image shape")
    nz, ny, nx = lab.shape
    per = (ct.c_int * 3)(*[int(p) for p in periodic])
    st = _lib.load().lbpm_mixed_wet_relabel(int(device), lab.ctypes.data, o.ctypes.data, nx, ny, nz, per,
                                           float(radius), int(new_label))
    if st != 0:
        raise LBPMError(st, "lbpm_mixed_wet_relabel failed")
    return lab


class Domain:
    """One simulated domain (one library context) on one GPU.

    labels   : uint16 array (nz, ny, nx), 0 = pore, k >= 1 = solid of wetting class k
    affinity : optional float32 (nz, ny, nx) per-voxel phi_s (solid voxels read)
    periodic : (px, py, pz) flags; non-periodic faces are solid walls
    precision: "fp32" or "fp16" storage of the distributions
    """

    def __init__(self, labels: np.ndarray, affinity: Optional[np.ndarray] = None, *,
                 periodic=(1, 1, 1), tau_a=0.7, tau_b=0.7, alpha=0.005, beta=0.95,
                 force=(0.0, 0.0, 0.0), precision="fp32", reservoir_z=0, rho_in=1.0,
                 rho_out=1.0, flux_in=0.0, device: int = 0, stream=None, use_torch_allocator: bool = True):
        torch = _torch()
        self._L = _lib.load()
        self.device = int(device)
        with torch.cuda.device(self.device):
            self._stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ct.c_void_p()
        st = self._L.lbpm_create(ct.byref(h), self.device, ct.c_void_p(self._stream.cuda_stream))
        if st != 0:
            raise LBPMError(st, self._L.lbpm_last_error(None).decode())
        self._h = h
        _LIVE.add(self)
        self._callbacks = None
        if use_torch_allocator:
            self._callbacks = _torch_allocator(torch, self.device, self._stream)
            self._check(self._L.lbpm_set_allocator(self._h, self._callbacks[0], self._callbacks[1], None))
        self.set_params(tau_a=tau_a, tau_b=tau_b, alpha=alpha, beta=beta, force=force,
                        precision=precision, periodic=periodic, reservoir_z=reservoir_z,
                        rho_in=rho_in, rho_out=rho_out, flux_in=flux_in)
        self.load_image(labels)
        if affinity is not None:
            self.set_affinity_map(affinity)

    # -- plumbing --------------------------------------------------------
    def _check(self, status: int):
        if status != 0:
            raise LBPMError(status, self._L.lbpm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.lbpm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- setup -----------------------------------------------------------
    def load_image(self, labels: np.ndarray):
        """(Re)load the labelled image and rebuild the pore-site index; the
        fluid state must then be initialised again."""
        labels = np.ascontiguousarray(labels, dtype=np.uint16)
        if labels.ndim != 3:
            raise ValueError("labels must be a 3-D (nz, ny, nx) array")
        nz, ny, nx = labels.shape
        self._check(self._L.lbpm_load_image(self._h, labels.ctypes.data, nx, ny, nz))
        self.shape = labels.shape

    def set_params(self, *, tau_a, tau_b, alpha, beta, force, precision="fp32",
                   periodic=(1, 1, 1), reservoir_z=0, rho_in=1.0, rho_out=1.0, flux_in=0.0):
        p = _params(tau_a, tau_b, alpha, beta, force, precision, periodic, reservoir_z, rho_in, rho_out, flux_in)
        self._check(self._L.lbpm_set_params(self._h, ct.byref(p)))
        self.params = dict(tau_a=tau_a, tau_b=tau_b, alpha=alpha, beta=beta, force=tuple(force),
                           precision=precision, periodic=tuple(periodic), reservoir_z=reservoir_z,
                           rho_in=rho_in, rho_out=rho_out, flux_in=flux_in)

    def update_params(self, **kw):
        p = dict(self.params)
        p.update(kw)
        self.set_params(**p)

    def set_affinity_map(self, affinity: np.ndarray):
        a = np.ascontiguousarray(affinity, dtype=np.float32)
        if a.shape != self.shape:
            raise ValueError("affinity map must match the image shape")
        self._check(self._L.lbpm_set_affinity_map(self._h, a.ctypes.data))

    def set_affinity_table(self, table):
        t = np.ascontiguousarray(table, dtype=np.float32)
        self._check(self._L.lbpm_set_affinity_table(self._h, t.ctypes.data, int(t.size)))

    def init_fluids(self, phi0: np.ndarray):
        p = np.ascontiguousarray(phi0, dtype=np.float32)
        if p.shape != self.shape:
            raise ValueError("phi0 must match the image shape")
        self._check(self._L.lbpm_init_fluids(self._h, p.ctypes.data))

    # -- running ---------------------------------------------------------
    def advance(self, nsteps: int):
        self._check(self._L.lbpm_advance(self._h, int(nsteps)))

    def set_step_form(self, form: str):
        """How advance() carries the component distributions between the steps
        of one call: "auto" (per-site component sums inside a call of two or
        more steps, the default) or "populations" (lbpm_set_step_form)."""
        self._check(self._L.lbpm_set_step_form(self._h, STEP_FORMS[form]))

    def run_with_trace(self, steps: int, interval: int, path: Optional[str] = None) -> list:
        """Advance with the basic analysis every `interval` steps (see trace_run)."""
        return trace_run(self, steps, interval, path)

    def sync(self):
        self._check(self._L.lbpm_sync(self._h))

    # -- shell aggregation (morphological steps on fluid A) ----------------
    def morph(self, delta: float, apply: bool = True):
        """Move the interface of fluid A by delta voxels (library call
        lbpm_morph); returns (A sites before, A sites after)."""
        b, a = ct.c_longlong(), ct.c_longlong()
        self._check(self._L.lbpm_morph(self._h, float(delta), int(bool(apply)), ct.byref(b), ct.byref(a)))
        return b.value, a.value

    def shell_aggregation(self, target_ratio: float, relax_steps: int = 1000, max_rounds: int = 8):
        """Change the volume of fluid A by target_ratio (lbpm_shell_aggregation);
        returns (achieved ratio, rounds)."""
        r, n = ct.c_double(), ct.c_int()
        self._check(self._L.lbpm_shell_aggregation(self._h, float(target_ratio), int(relax_steps), int(max_rounds),
                                                    ct.byref(r), ct.byref(n)))
        return r.value, n.value

    def measure(self, raise_unstable: bool = False) -> dict:
        m = Measures()
        st = self._L.lbpm_measure(self._h, ct.byref(m))
        if st != 0 and (st != 5 or raise_unstable):
            self._check(st)
        return _measures_dict(m)

    # -- results ---------------------------------------------------------
    @property
    def n_sites(self) -> int:
        n = ct.c_longlong()
        self._check(self._L.lbpm_num_sites(self._h, ct.byref(n)))
        return n.value

    @property
    def step_count(self) -> int:
        n = ct.c_longlong()
        self._check(self._L.lbpm_step_count(self._h, ct.byref(n)))
        return n.value

    @property
    def launch_count(self) -> int:
        n = ct.c_longlong()
        self._check(self._L.lbpm_launch_count(self._h, ct.byref(n)))
        return n.value

    def read_field(self, name: str) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float32)
        self._check(self._L.lbpm_read_field(self._h, FIELDS[name], out.ctypes.data))
        return out

    def read_field_noalloc(self, name: str) -> np.ndarray:
        """Same as read_field, without any device allocation: the library stages
        the field in a fixed static device buffer (images up to
        LBPM_NOALLOC_FIELD_MAX_VOXELS voxels), for callers that must not let it
        allocate after set-up. Concurrent calls on one GPU race on that buffer."""
        out = np.empty(self.shape, dtype=np.float32)
        self._check(self._L.lbpm_read_field_noalloc(self._h, FIELDS[name], out.ctypes.data))
        return out

    def distributions(self, which: str) -> np.ndarray:
        code, Q = DISTS[which]
        out = np.empty((Q, self.n_sites), dtype=np.float32)
        self._check(self._L.lbpm_read_distributions(self._h, code, out.ctypes.data))
        return out

    def read_box(self, which: str, lo, hi) -> np.ndarray:
        """Distributions (canonical order) at the voxels of the box [lo, hi)
        given as (x, y, z) bounds: array [Q][bz][by][bx], NaN at solids."""
        code, Q = DISTS[which]
        l = np.ascontiguousarray(lo, dtype=np.int32)
        h = np.ascontiguousarray(hi, dtype=np.int32)
        if l.shape != (3,) or h.shape != (3,):
            raise ValueError("lo and hi take three voxel bounds (x, y, z)")
        ext = h - l
        out = np.empty((Q, int(ext[2]), int(ext[1]), int(ext[0])) if (ext > 0).all() else (Q, 0, 0, 0),
                       dtype=np.float32)
        self._check(self._L.lbpm_read_box(self._h, code, l.ctypes.data, h.ctypes.data, out.ctypes.data))
        return out

    def write_distributions(self, which: str, values: np.ndarray):
        code, Q = DISTS[which]
        v = np.ascontiguousarray(values, dtype=np.float32)
        if v.shape != (Q, self.n_sites):
            raise ValueError(f"expected shape {(Q, self.n_sites)}")
        self._check(self._L.lbpm_write_distributions(self._h, code, v.ctypes.data))

    def index(self):
        N = self.n_sites
        sv = np.empty(N, dtype=np.int64)
        nb = np.empty((18, N), dtype=np.int32)
        self._check(self._L.lbpm_get_index(self._h, sv.ctypes.data, nb.ctypes.data))
        return sv, nb

    def snapshot(self) -> bytes:
        n = ct.c_size_t(0)
        self._check(self._L.lbpm_snapshot(self._h, None, ct.byref(n)))
        buf = ct.create_string_buffer(n.value)
        self._check(self._L.lbpm_snapshot(self._h, buf, ct.byref(n)))
        return buf.raw[: n.value]

    def restore(self, snap: bytes):
        buf = ct.create_string_buffer(snap, len(snap))
        self._check(self._L.lbpm_restore(self._h, buf, len(snap)))

    # -- timing ----------------------------------------------------------
    def enable_kernel_timing(self, on: bool = True):
        self._check(self._L.lbpm_enable_kernel_timing(self._h, int(bool(on))))

    def kernel_timing(self) -> dict:
        mc, nc, mp, np_ = ct.c_double(), ct.c_longlong(), ct.c_double(), ct.c_longlong()
        self._check(self._L.lbpm_kernel_timing(self._h, ct.byref(mc), ct.byref(nc), ct.byref(mp),
                                               ct.byref(np_)))
        return {"collide_ms": mc.value, "collide_launches": nc.value,
                "phase_ms": mp.value, "phase_launches": np_.value}


class Batch:
    """Several Domains (same GPU, same storage precision) advanced together by
    one launch per pass over all their sites, or one fused cooperative launch
    per bundle of steps (lbpm_batch_* ABI).
    Results agree with advancing each domain alone to fp32 rounding (the
    batched kernels are compiled separately, so multiply-add contraction may
    differ); two batched runs of the same jobs are bit-identical."""

    def __init__(self, device: int = 0, stream=None, use_torch_allocator: bool = True):
        torch = _torch()
        self._L = _lib.load()
        self.device = int(device)
        with torch.cuda.device(self.device):
            self._stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ct.c_void_p()
        st = self._L.lbpm_batch_create(ct.byref(h), self.device, ct.c_void_p(self._stream.cuda_stream))
        if st != 0:
            raise LBPMError(st, "lbpm_batch_create failed")
        self._h = h
        _LIVE.add(self)
        self._callbacks = None
        if use_torch_allocator:
            self._callbacks = _torch_allocator(torch, self.device, self._stream)
            self._check(self._L.lbpm_batch_set_allocator(self._h, self._callbacks[0], self._callbacks[1], None))
        self.jobs = []

    def _check(self, status: int):
        if status != 0:
            raise LBPMError(status, self._L.lbpm_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.lbpm_batch_destroy(self._h)
            self._h = None
            self.jobs = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, dom: "Domain"):
        self._check(self._L.lbpm_batch_add(self._h, dom._h))
        self.jobs.append(dom)

    def remove(self, dom: "Domain"):
        self._check(self._L.lbpm_batch_remove(self._h, dom._h))
        self.jobs.remove(dom)

    def refresh(self):
        self._check(self._L.lbpm_batch_refresh(self._h))

    def advance(self, nsteps: int):
        self._check(self._L.lbpm_batch_advance(self._h, int(nsteps)))

    def measure(self) -> list:
        arr = (Measures * max(len(self.jobs), 1))()
        st = self._L.lbpm_batch_measure(self._h, arr)
        if st not in (0, 5):
            self._check(st)
        return [_measures_dict(arr[j]) for j in range(len(self.jobs))]

    def check_barrier(self, missing: int = 0, limit_s: float = 0.05):
        """Self-test of the fused kernel's bounded grid barrier
        (lbpm_batch_check_barrier): True if it completed, False if its wait ran
        out (as it must when `missing` arrivals never come)."""
        st = self._L.lbpm_batch_check_barrier(self._h, int(missing), float(limit_s))
        if st == 6:
            return False
        self._check(st)
        return True

    def set_launch(self, threads: int, blocks_per_sm_phase: int = 0, blocks_per_sm_collide: int = 0):
        self._check(self._L.lbpm_batch_set_launch(self._h, int(threads), int(blocks_per_sm_phase),
                                                  int(blocks_per_sm_collide)))

    def tune(self, steps_per_candidate: int = 20):
        """Time every candidate launch shape over one advance call of
        steps_per_candidate steps (see lbpm_batch_tune) and keep the fastest."""
        t, p, c = ct.c_int(), ct.c_int(), ct.c_int()
        self._check(self._L.lbpm_batch_tune(self._h, int(steps_per_candidate), ct.byref(t), ct.byref(p),
                                            ct.byref(c)))
        return t.value, p.value, c.value

    @property
    def n_sites(self) -> int:
        n, s = ct.c_int(), ct.c_longlong()
        self._check(self._L.lbpm_batch_size(self._h, ct.byref(n), ct.byref(s)))
        return s.value

    @property
    def launch_count(self) -> int:
        n = ct.c_longlong()
        self._check(self._L.lbpm_batch_launch_count(self._h, ct.byref(n)))
        return n.value


class _JobView:
    """Read-only access to a served job's device state (fields, distributions)."""

    def __init__(self, server: "Server", handle, shape):
        self._L = server._L
        self._h = handle
        self.shape = shape
        self._server = server

    _check = Domain._check
    read_field = Domain.read_field
    distributions = Domain.distributions
    measure = Domain.measure
    n_sites = Domain.n_sites
    step_count = Domain.step_count


class Server:
    """Continuous-batching request loop (lbpm_server_* ABI): submit jobs, then
    call run() repeatedly; each call admits queued jobs while slots and the
    memory budget allow, advances all running jobs one check interval in one
    batched launch sequence, and retires the finished ones."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, max_jobs: int = 64, check_interval: int = 500,
                 stream=None, use_torch_allocator: bool = True):
        torch = _torch()
        self._L = _lib.load()
        self.device = int(device)
        with torch.cuda.device(self.device):
            self._stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ct.c_void_p()
        st = self._L.lbpm_server_create(ct.byref(h), self.device, ct.c_void_p(self._stream.cuda_stream),
                                        int(budget_bytes), int(max_jobs), int(check_interval))
        if st != 0:
            raise LBPMError(st, "lbpm_server_create failed")
        self._h = h
        _LIVE.add(self)
        self._callbacks = None
        if use_torch_allocator:
            self._callbacks = _torch_allocator(torch, self.device, self._stream)
            self._check(self._L.lbpm_server_set_allocator(self._h, self._callbacks[0], self._callbacks[1], None))
        self._shapes = {}

    def _check(self, status: int):
        if status != 0:
            raise LBPMError(status, self._L.lbpm_server_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.lbpm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, labels, phi0, affinity=None, *, kind="steady", max_steps=10000, flux_tol=1e-4,
               sw_tol=1e-4, force_factor=2.0, force_cap=1.6e-4, tau_a=0.7, tau_b=0.7, alpha=0.005,
               beta=0.95, force=(0.0, 0.0, 0.0), precision="fp32", periodic=(1, 1, 1), reservoir_z=0,
               rho_in=1.0, rho_out=1.0, flux_in=0.0, ca_target=0.0, relax_steps=0, ca_tol=0.05) -> int:
        lab = np.ascontiguousarray(labels, dtype=np.uint16)
        ph = np.ascontiguousarray(phi0, dtype=np.float32)
        aff = None if affinity is None else np.ascontiguousarray(affinity, dtype=np.float32)
        nz, ny, nx = lab.shape
        sp = JobSpec()
        sp.labels, sp.nx, sp.ny, sp.nz = lab.ctypes.data, nx, ny, nz
        sp.affinity = aff.ctypes.data if aff is not None else None
        sp.phi0 = ph.ctypes.data
        sp.params = _params(tau_a, tau_b, alpha, beta, force, precision, periodic, reservoir_z, rho_in, rho_out,
                            flux_in)
        sp.kind = JOB_KINDS[kind] if isinstance(kind, str) else int(kind)
        sp.max_steps = int(max_steps)
        sp.flux_tol, sp.sw_tol = float(flux_tol), float(sw_tol)
        sp.force_factor, sp.force_cap = float(force_factor), float(force_cap)
        sp.ca_target, sp.relax_steps, sp.ca_tol = float(ca_target), int(relax_steps), float(ca_tol)
        t = ct.c_longlong()
        self._check(self._L.lbpm_server_submit(self._h, ct.byref(sp), ct.byref(t)))
        self._shapes[t.value] = lab.shape
        return t.value

    def run(self):
        r, q, f = ct.c_int(), ct.c_int(), ct.c_int()
        self._check(self._L.lbpm_server_run(self._h, ct.byref(r), ct.byref(q), ct.byref(f)))
        return r.value, q.value, f.value

    def poll(self, ticket: int) -> dict:
        st = JobStatus()
        self._check(self._L.lbpm_server_poll(self._h, int(ticket), ct.byref(st)))
        return {"state": JOB_STATES[st.state], "steps": st.steps, "n_sites": st.n_sites,
                "footprint": st.footprint, "t_submit": st.t_submit, "t_admit": st.t_admit,
                "t_done": st.t_done, "force_raises": st.force_raises, "last": _measures_dict(st.last),
                "force": tuple(st.force)}

    def job(self, ticket: int) -> _JobView:
        h = ct.c_void_p()
        self._check(self._L.lbpm_server_job_ctx(self._h, int(ticket), ct.byref(h)))
        if not h.value:
            raise LBPMError(4, "the job has no device state")
        return _JobView(self, h, self._shapes[ticket])

    def cancel(self, ticket: int):
        self._check(self._L.lbpm_server_cancel(self._h, int(ticket)))

    def release(self, ticket: int):
        self._check(self._L.lbpm_server_release(self._h, int(ticket)))

    def stats(self) -> dict:
        su, used, budget = ct.c_longlong(), ct.c_size_t(), ct.c_size_t()
        self._check(self._L.lbpm_server_stats(self._h, ct.byref(su), ct.byref(used), ct.byref(budget)))
        return {"site_updates": su.value, "used_bytes": used.value, "budget_bytes": budget.value}
