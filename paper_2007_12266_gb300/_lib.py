"""ctypes declarations of the C ABI in ``include/lbpm.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library. If the library has not been built this module raises; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as ct
import os

from ._build import LIB, up_to_date

c_ctx_p = ct.c_void_p


class Params(ct.Structure):
    _fields_ = [
        ("tau_a", ct.c_double), ("tau_b", ct.c_double),
        ("alpha", ct.c_double), ("beta", ct.c_double),
        ("force", ct.c_double * 3),
        ("precision", ct.c_int),
        ("periodic", ct.c_int * 3),
        ("reservoir_z", ct.c_int),
        ("rho_in", ct.c_double), ("rho_out", ct.c_double),
        ("flux_in", ct.c_double),
    ]


class Measures(ct.Structure):
    _fields_ = [
        ("step", ct.c_longlong),
        ("sat_mass", ct.c_double), ("sat_count", ct.c_double),
        ("mass_a", ct.c_double), ("mass_b", ct.c_double), ("mass_total", ct.c_double),
        ("mom_a", ct.c_double * 3), ("mom_b", ct.c_double * 3),
        ("flux", ct.c_double * 3), ("flux_a", ct.c_double * 3), ("flux_b", ct.c_double * 3),
        ("ke_a", ct.c_double), ("ke_b", ct.c_double),
        ("p_a", ct.c_double), ("p_b", ct.c_double),
        ("vol_a", ct.c_double), ("vol_b", ct.c_double),
        ("ca", ct.c_double),
        ("n_sites", ct.c_longlong),
        ("status", ct.c_int),
    ]


class JobSpec(ct.Structure):
    _fields_ = [
        ("labels", ct.c_void_p), ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
        ("affinity", ct.c_void_p), ("phi0", ct.c_void_p),
        ("params", Params),
        ("kind", ct.c_int),
        ("max_steps", ct.c_longlong),
        ("flux_tol", ct.c_double), ("sw_tol", ct.c_double),
        ("force_factor", ct.c_double), ("force_cap", ct.c_double),
        ("ca_target", ct.c_double), ("relax_steps", ct.c_longlong), ("ca_tol", ct.c_double),
    ]


class JobStatus(ct.Structure):
    _fields_ = [
        ("state", ct.c_int), ("steps", ct.c_longlong), ("n_sites", ct.c_longlong),
        ("footprint", ct.c_size_t),
        ("t_submit", ct.c_double), ("t_admit", ct.c_double), ("t_done", ct.c_double),
        ("force_raises", ct.c_int),
        ("last", Measures),
        ("force", ct.c_double * 3),
    ]


ALLOC_FN = ct.CFUNCTYPE(ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_void_p)
FREE_FN = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_void_p)

STATUS = {0: "LBPM_OK", 1: "LBPM_E_INVALID", 2: "LBPM_E_OOM", 3: "LBPM_E_CUDA",
          4: "LBPM_E_STATE", 5: "LBPM_E_UNSTABLE", 6: "LBPM_E_TIMEOUT"}

# name -> (restype, argtypes) for every entry point of include/lbpm.h
SIGNATURES = {
    "lbpm_version": (ct.c_char_p, []),
    "lbpm_create": (ct.c_int, [ct.POINTER(c_ctx_p), ct.c_int, ct.c_void_p]),
    "lbpm_destroy": (ct.c_int, [c_ctx_p]),
    "lbpm_set_allocator": (ct.c_int, [c_ctx_p, ALLOC_FN, FREE_FN, ct.c_void_p]),
    "lbpm_last_error": (ct.c_char_p, [c_ctx_p]),
    "lbpm_load_image": (ct.c_int, [c_ctx_p, ct.c_void_p, ct.c_int, ct.c_int, ct.c_int]),
    "lbpm_set_affinity_table": (ct.c_int, [c_ctx_p, ct.c_void_p, ct.c_int]),
    "lbpm_set_affinity_map": (ct.c_int, [c_ctx_p, ct.c_void_p]),
    "lbpm_set_params": (ct.c_int, [c_ctx_p, ct.POINTER(Params)]),
    "lbpm_init_fluids": (ct.c_int, [c_ctx_p, ct.c_void_p]),
    "lbpm_advance": (ct.c_int, [c_ctx_p, ct.c_longlong]),
    "lbpm_set_step_form": (ct.c_int, [c_ctx_p, ct.c_int]),
    "lbpm_morph": (ct.c_int, [c_ctx_p, ct.c_double, ct.c_int, ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_longlong)]),
    "lbpm_shell_aggregation": (ct.c_int, [c_ctx_p, ct.c_double, ct.c_longlong, ct.c_int, ct.POINTER(ct.c_double),
                                          ct.POINTER(ct.c_int)]),
    "lbpm_sync": (ct.c_int, [c_ctx_p]),
    "lbpm_measure": (ct.c_int, [c_ctx_p, ct.POINTER(Measures)]),
    "lbpm_read_field": (ct.c_int, [c_ctx_p, ct.c_int, ct.c_void_p]),
    "lbpm_read_field_noalloc": (ct.c_int, [c_ctx_p, ct.c_int, ct.c_void_p]),
    "lbpm_read_distributions": (ct.c_int, [c_ctx_p, ct.c_int, ct.c_void_p]),
    "lbpm_read_box": (ct.c_int, [c_ctx_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "lbpm_write_distributions": (ct.c_int, [c_ctx_p, ct.c_int, ct.c_void_p]),
    "lbpm_num_sites": (ct.c_int, [c_ctx_p, ct.POINTER(ct.c_longlong)]),
    "lbpm_step_count": (ct.c_int, [c_ctx_p, ct.POINTER(ct.c_longlong)]),
    "lbpm_get_index": (ct.c_int, [c_ctx_p, ct.c_void_p, ct.c_void_p]),
    "lbpm_snapshot": (ct.c_int, [c_ctx_p, ct.c_void_p, ct.POINTER(ct.c_size_t)]),
    "lbpm_restore": (ct.c_int, [c_ctx_p, ct.c_void_p, ct.c_size_t]),
    "lbpm_enable_kernel_timing": (ct.c_int, [c_ctx_p, ct.c_int]),
    "lbpm_kernel_timing": (ct.c_int, [c_ctx_p, ct.POINTER(ct.c_double), ct.POINTER(ct.c_longlong),
                                      ct.POINTER(ct.c_double), ct.POINTER(ct.c_longlong)]),
    "lbpm_launch_count": (ct.c_int, [c_ctx_p, ct.POINTER(ct.c_longlong)]),
    "lbpm_force_rescale": (ct.c_int, [ct.POINTER(ct.c_double), ct.c_double, ct.c_double, ct.c_double,
                                      ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]),
    "lbpm_mixing_layer": (ct.c_int, [ct.c_int, ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int]),
    "lbpm_mixed_wet_relabel": (ct.c_int, [ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_int, ct.c_int,
                                          ct.POINTER(ct.c_int), ct.c_double, ct.c_int]),
    "lbpm_batch_create": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int, ct.c_void_p]),
    "lbpm_batch_destroy": (ct.c_int, [ct.c_void_p]),
    "lbpm_batch_set_allocator": (ct.c_int, [ct.c_void_p, ALLOC_FN, FREE_FN, ct.c_void_p]),
    "lbpm_batch_last_error": (ct.c_char_p, [ct.c_void_p]),
    "lbpm_batch_add": (ct.c_int, [ct.c_void_p, c_ctx_p]),
    "lbpm_batch_remove": (ct.c_int, [ct.c_void_p, c_ctx_p]),
    "lbpm_batch_refresh": (ct.c_int, [ct.c_void_p]),
    "lbpm_batch_size": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int), ct.POINTER(ct.c_longlong)]),
    "lbpm_batch_advance": (ct.c_int, [ct.c_void_p, ct.c_longlong]),
    "lbpm_batch_measure": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "lbpm_batch_set_launch": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int]),
    "lbpm_batch_tune": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                   ct.POINTER(ct.c_int)]),
    "lbpm_batch_launch_count": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_longlong)]),
    "lbpm_batch_check_barrier": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_double]),
    "lbpm_server_create": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int, ct.c_void_p, ct.c_size_t, ct.c_int,
                                      ct.c_int]),
    "lbpm_server_destroy": (ct.c_int, [ct.c_void_p]),
    "lbpm_server_set_allocator": (ct.c_int, [ct.c_void_p, ALLOC_FN, FREE_FN, ct.c_void_p]),
    "lbpm_server_last_error": (ct.c_char_p, [ct.c_void_p]),
    "lbpm_server_submit": (ct.c_int, [ct.c_void_p, ct.POINTER(JobSpec), ct.POINTER(ct.c_longlong)]),
    "lbpm_server_run": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "lbpm_server_poll": (ct.c_int, [ct.c_void_p, ct.c_longlong, ct.POINTER(JobStatus)]),
    "lbpm_server_job_ctx": (ct.c_int, [ct.c_void_p, ct.c_longlong, ct.POINTER(ct.c_void_p)]),
    "lbpm_server_cancel": (ct.c_int, [ct.c_void_p, ct.c_longlong]),
    "lbpm_server_release": (ct.c_int, [ct.c_void_p, ct.c_longlong]),
    "lbpm_server_stats": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_size_t),
                                     ct.POINTER(ct.c_size_t)]),
}

_lib = None


class LBPMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return LIB


def load():
    """Load ``libcolorlbm.so`` (raises if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(
            f"CUDA library {LIB} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    if not up_to_date():
        raise RuntimeError(f"CUDA library {LIB} is older than its sources; rebuild it")
    lib = ct.CDLL(LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
