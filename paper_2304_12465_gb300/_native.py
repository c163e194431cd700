"""ctypes declarations of the C ABI in include/krr.h.

Loading builds the sm_103a library first if it is missing or stale; there is
no CPU implementation to fall back to, so a missing CUDA toolkit or library is
an error.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

KRR_OK, KRR_EINVAL, KRR_ENOMEM, KRR_ECUDA, KRR_ECHOL, KRR_EBREAKDOWN, KRR_ENOCONV, \
    KRR_ETIMEOUT = range(8)
STATUS_NAMES = {0: "KRR_OK", 1: "KRR_EINVAL", 2: "KRR_ENOMEM", 3: "KRR_ECUDA",
                4: "KRR_ECHOL", 5: "KRR_EBREAKDOWN", 6: "KRR_ENOCONV", 7: "KRR_ETIMEOUT"}

GAUSSIAN, LAPLACE_L1, MATERN52 = 0, 1, 2
PREC_FP64, PREC_MIXED, PREC_FLOAT_FLOAT = 0, 1, 2
PIVOT_RPCHOLESKY, PIVOT_UNIFORM, PIVOT_GREEDY = 0, 1, 2
# float32 product path (krr_set_product_path)
PRODUCT_TENSOR, PRODUCT_FMA, PRODUCT_MMA_SYNC = 0, 1, 2


class KrrInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer_refinements", C.c_int), ("rank", C.c_int),
                ("escalated", C.c_int), ("rel_residual", C.c_double),
                ("kernel_entries", C.c_double), ("t_build_s", C.c_double),
                ("t_solve_s", C.c_double), ("kmv_ms", C.c_double),
                ("kmv_launches", C.c_int), ("kmv64_launches", C.c_int),
                ("kmv64_ms", C.c_double), ("kmvff_ms", C.c_double),
                ("kmvff_launches", C.c_int), ("graph_replays", C.c_int),
                ("host_checks", C.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_
                if not name.startswith("reserved")}


class ServerConfig(C.Structure):
    _fields_ = [("max_slots", C.c_int), ("iters_per_step", C.c_int), ("use_graph", C.c_int),
                ("build_threads", C.c_int), ("hbm_budget_bytes", C.c_double)]


class RequestResult(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int), ("iters", C.c_int),
                ("outer_refinements", C.c_int), ("rank", C.c_int), ("m", C.c_int),
                ("escalated", C.c_int), ("reserved", C.c_int), ("rel_residual", C.c_double), ("kernel_entries", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_built", C.c_double),
                ("t_done", C.c_double), ("error", C.c_char * 160)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["error"] = d["error"].decode(errors="replace")
        return d


class RequestProgress(C.Structure):
    _fields_ = [("id", C.c_int64), ("state", C.c_int), ("iters", C.c_int),
                ("outer_refinements", C.c_int), ("reserved", C.c_int),
                ("rel_residual", C.c_double)]

    STATES = ("queued", "building", "iterating", "escalated", "finishing", "parked", "done")

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}
        d["state_name"] = self.STATES[self.state]
        return d


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("queued", C.c_int64),
                ("admitted", C.c_int64), ("steps", C.c_int64), ("step_kernels", C.c_int64),
                ("max_concurrent", C.c_int), ("reserved", C.c_int),
                ("reserved_bytes", C.c_double), ("peak_reserved_bytes", C.c_double),
                ("budget_bytes", C.c_double), ("kernel_entries", C.c_double),
                ("step_ms", C.c_double), ("build_s", C.c_double), ("escalate_s", C.c_double),
                ("escalations", C.c_int64), ("phase_ms", C.c_double * 12)]

    PHASES = ("product", "reduce", "alpha", "update", "resid", "ft_r", "ft_r_reduce", "w_t",
              "wt_u", "z", "beta", "direction")

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}
        d["phase_ms"] = dict(zip(self.PHASES, list(self.phase_ms)))
        return d


class KrrError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


# Every function the header declares, with its ctypes signature.
_vp = C.c_void_p
_i64, _u64, _int, _dbl = C.c_int64, C.c_uint64, C.c_int, C.c_double
SIGNATURES = {
    "krr_kmatvec": (_int, [_vp, _i64, _int, _int, _dbl, _dbl, _vp, _int, _vp, _int, _vp]),
    "krr_kmatvec_f64_noalloc": (_int, [_vp, _i64, _int, _int, _dbl, _dbl, _vp, _int, _vp,
                                       _vp]),
    "krr_kmatvec_batched": (_int, [_vp, _i64, _int, _int, _vp, _vp, _int, _vp, _vp, _vp, _vp]),
    "krr_predict": (_int, [_vp, _i64, _int, _int, _dbl, _vp, _int, _vp, _i64, _vp, _int, _vp]),
    "krr_rpc_sample": (_int, [_vp, _i64, _dbl, _u64, _u64, _int, _vp, C.POINTER(_int), _vp]),
    "krr_rpcholesky": (_int, [_vp, _i64, _int, _int, _dbl, _int, _int, _u64, _vp,
                              C.POINTER(_vp)]),
    "krr_pivoted_cholesky": (_int, [_vp, _i64, _int, _int, _dbl, _int, _int, _u64, _int, _vp,
                                    C.POINTER(_vp)]),
    "krr_factor_info": (_int, [_vp, C.POINTER(_i64), C.POINTER(_int), C.POINTER(_int)]),
    "krr_factor_export": (_int, [_vp, _vp, _vp, _vp]),
    "krr_factor_free": (None, [_vp]),
    "krr_precond_apply": (_int, [_vp, _dbl, _vp, _int, _vp, _int, _vp]),
    "krr_pcg_solve": (_int, [_vp, _i64, _int, _int, _dbl, _vp, _int, _dbl, _vp, _dbl, _int,
                             _int, _vp, _vp, C.POINTER(KrrInfo)]),
    "krr_pcg_solve_batched": (_int, [_vp, _i64, _int, _int, _vp, _vp, _vp, _int, _vp, _vp, _dbl,
                                     _int, _vp, _vp, C.POINTER(KrrInfo)]),
    "krr_sparse_sign": (_int, [_i64, _int, _int, _u64, _vp, _vp, _vp]),
    "krill_build": (_int, [_vp, _i64, _int, _int, _dbl, _vp, _int, _dbl, _int, _int, _u64, _vp,
                           C.POINTER(_vp)]),
    "krill_export": (_int, [_vp, _vp, _vp, _vp, _vp, C.POINTER(_int)]),
    "krill_solve": (_int, [_vp, _vp, _int, _dbl, _int, _vp, _vp, C.POINTER(KrrInfo)]),
    "krill_free": (None, [_vp]),
    "krr_server_footprint": (_int, [_i64, _int, _int, _int, C.POINTER(_dbl)]),
    "krr_server_create": (_int, [C.POINTER(ServerConfig), C.POINTER(_vp)]),
    "krr_server_submit": (_int, [_vp, _vp, _i64, _int, _int, _dbl, _vp, _int, _dbl, _int, _u64,
                                 _dbl, _int, _vp, C.POINTER(_i64)]),
    "krr_server_step": (_int, [_vp, C.POINTER(_i64)]),
    "krr_server_poll": (_int, [_vp, C.POINTER(RequestResult), _int, C.POINTER(_int)]),
    "krr_server_get_stats": (_int, [_vp, C.POINTER(ServerStats)]),
    "krr_server_clock": (_dbl, [_vp]),
    "krr_server_progress": (_int, [_vp, _i64, C.POINTER(RequestProgress)]),
    "krr_server_evict": (_int, [_vp, _i64]),
    "krr_server_resume": (_int, [_vp, _i64]),
    "krr_server_export": (_int, [_vp, _i64, _vp, C.POINTER(C.c_size_t)]),
    "krr_server_import": (_int, [_vp, _vp, C.c_size_t, _vp, _vp, _vp, C.POINTER(_i64)]),
    "krr_server_destroy": (None, [_vp]),
    "krr_set_autotune": (None, [_int]),
    "krr_set_pcg_graphs": (None, [_int]),
    "krr_check_bounded_wait": (_int, [_i64, _vp]),
    "krr_autotune_choice": (_int, [_int, _int, _int, _i64, C.POINTER(_int)]),
    "krr_set_product_path": (_int, [_int]),
    "krr_set_product_variant": (_int, [_int]),
    "krr_profile_collect": (_int, [_int, C.POINTER(C.c_double), C.POINTER(_int)]),
    "krr_autotune_variant": (_int, [_int, _int, _int, _i64, C.POINTER(_int),
                                    C.POINTER(C.c_float)]),
    "krr_set_profiling": (None, [_int]),
    "krr_last_error": (C.c_char_p, []),
    "krr_version": (C.c_char_p, []),
    "krr_launch_count": (C.c_uint64, []),
}

_LIB = None


def library_path() -> str:
    return _build.LIB


def load(auto_build: bool = True):
    """Load libkrr_gb300.so (building it first when allowed)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if auto_build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libkrr_gb300.so not found at {path}; build it with "
                           "paper_2304_12465_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(status: int, where: str, allow=()) -> int:
    if status != KRR_OK and status not in allow:
        msg = _LIB.krr_last_error().decode() if _LIB is not None else ""
        raise KrrError(status, where, msg)
    return status
