"""Python binding of the C ABI: the same call names, argument marshalling only.

Arrays may be numpy arrays (host memory; the library stages them) or torch
tensors (host or CUDA; CUDA tensors are passed by pointer on the current
stream).  Layouts follow include/krr.h: X is (N, d) float64 row-major, a
right-hand-side block is (m, N) float64 (N x m column-major), a factor is
returned as (rank, N).  Outputs match the container of the right-hand side:
torch CUDA in, torch CUDA out; numpy in, numpy out.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Tuple

import numpy as np

from . import _native as N_
from ._native import KrrInfo, check, load

try:  # torch is optional for host-only use
    import torch
except Exception:  # pragma: no cover
    torch = None

_KERNELS = {"gaussian": N_.GAUSSIAN, "laplace": N_.LAPLACE_L1, "laplace_l1": N_.LAPLACE_L1,
            "matern52": N_.MATERN52, "matern": N_.MATERN52}
_PRECS = {"fp64": N_.PREC_FP64, "mixed": N_.PREC_MIXED, "ff": N_.PREC_FLOAT_FLOAT}


def _kern(k) -> int:
    return _KERNELS[k] if isinstance(k, str) else int(k)


def _prec(p) -> int:
    return _PRECS[p] if isinstance(p, str) else int(p)


def _is_torch(a) -> bool:
    return torch is not None and isinstance(a, torch.Tensor)


def _is_cuda(a) -> bool:
    return _is_torch(a) and a.is_cuda


def _arr(a, dtype=np.float64):
    """(keep-alive object, c_void_p) for an input array."""
    if _is_torch(a):
        tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            a = a.to(tdt).contiguous()
        return a, C.c_void_p(a.data_ptr())
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, C.c_void_p(a.ctypes.data)


def _empty_like_container(ref, shape, dtype=np.float64):
    if _is_cuda(ref):
        tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype]
        t = torch.empty(shape, dtype=tdt, device=ref.device)
        return t, C.c_void_p(t.data_ptr())
    out = np.empty(shape, dtype=dtype)
    return out, C.c_void_p(out.ctypes.data)


def _stream(stream, *refs):
    if stream is not None:
        return C.c_void_p(int(stream))
    if any(_is_cuda(r) for r in refs):
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(0)


def _shape2(a):
    return tuple(a.shape) if a.ndim == 2 else (1, a.shape[0])


# --------------------------------------------------------------- product
def krr_kmatvec(X, kern, sigma: float, lam: float, V, prec="fp64", stream=None):
    """(A + lam I) V; V is (m, N)."""
    lib = load()
    Xk, Xp = _arr(X)
    Vk, Vp = _arr(V)
    Nn, d = Xk.shape
    m = _shape2(Vk)[0]
    Y, Yp = _empty_like_container(V, (m, Nn))
    check(lib.krr_kmatvec(Xp, Nn, d, _kern(kern), float(sigma), float(lam), Vp, m, Yp,
                          _prec(prec), _stream(stream, X, V)), "krr_kmatvec")
    return Y


def krr_kmatvec_batched(X, kerns, sigmas, lambdas, V, stream=None):
    """Batched product: settings s (kerns[s], sigmas[s]) with ms = len(V) // S
    columns each; V (S*ms, N), lambdas (S*ms,).  Returns Y like V."""
    lib = load()
    Xk, Xp = _arr(X)
    Vk, Vp = _arr(V)
    Nn, d = Xk.shape
    S = len(kerns)
    mt = _shape2(Vk)[0]
    ms = mt // S
    assert ms * S == mt
    kk = np.ascontiguousarray([_kern(k) for k in kerns], dtype=np.int32)
    ss = np.ascontiguousarray(sigmas, dtype=np.float64)
    ll = np.ascontiguousarray(lambdas, dtype=np.float64)
    Y, Yp = _empty_like_container(V, (mt, Nn))
    check(lib.krr_kmatvec_batched(Xp, Nn, d, S, C.c_void_p(kk.ctypes.data),
                                  C.c_void_p(ss.ctypes.data), ms, C.c_void_p(ll.ctypes.data),
                                  Vp, Yp, _stream(stream, X, V)), "krr_kmatvec_batched")
    return Y


def krr_predict(Xtrain, kern, sigma: float, alpha, Xtest, prec="fp64", stream=None):
    """Predictions K(Xtest, Xtrain) alpha, alpha (m, N) -> (m, Nt)."""
    lib = load()
    Xk, Xp = _arr(Xtrain)
    Ak, Ap = _arr(alpha)
    Tk, Tp = _arr(Xtest)
    Nn, d = Xk.shape
    Nt = Tk.shape[0]
    m = _shape2(Ak)[0]
    out, Op = _empty_like_container(alpha, (m, Nt))
    check(lib.krr_predict(Xp, Nn, d, _kern(kern), float(sigma), Ap, m, Tp, Nt, Op, _prec(prec),
                          _stream(stream, Xtrain, alpha, Xtest)), "krr_predict")
    return out


def krr_rpc_sample(dres, seed: int, t: int, ndraw: int, dfloor: float = 0.0,
                   stream=None) -> np.ndarray:
    lib = load()
    Dk, Dp = _arr(dres)
    out = np.empty(ndraw, dtype=np.int64)
    got = C.c_int(0)
    check(lib.krr_rpc_sample(Dp, Dk.shape[0], float(dfloor), seed, t, ndraw,
                             C.c_void_p(out.ctypes.data), C.byref(got), _stream(stream, dres)),
          "krr_rpc_sample")
    return out[:got.value]


# ------------------------------------------------------------ RPCholesky
class Factor:
    """Owner of a krr_factor handle (Alg. 3 output)."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle

    @property
    def handle(self):
        if not self._h:
            raise ValueError("factor already freed")
        return self._h

    def info(self) -> Tuple[int, int, int]:
        lib = load()
        n, r, b = C.c_int64(), C.c_int(), C.c_int()
        check(lib.krr_factor_info(self.handle, C.byref(n), C.byref(r), C.byref(b)),
              "krr_factor_info")
        return n.value, r.value, b.value

    @property
    def rank(self) -> int:
        return self.info()[1]

    @property
    def nblocks(self) -> int:
        return self.info()[2]

    def export(self):
        """(F as (rank, N), pivots int64[rank], dres float64[N]) on the host."""
        lib = load()
        n, r, _ = self.info()
        F = np.empty((r, n))
        S = np.empty(r, dtype=np.int64)
        D = np.empty(n)
        check(lib.krr_factor_export(self.handle, C.c_void_p(F.ctypes.data),
                                    C.c_void_p(S.ctypes.data), C.c_void_p(D.ctypes.data)),
              "krr_factor_export")
        return F, S, D

    def free(self):
        if self._h:
            load().krr_factor_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()


def krr_rpcholesky(X, kern, sigma: float, k: int, block: int = 0, seed: int = 0,
                   stream=None) -> Factor:
    lib = load()
    Xk, Xp = _arr(X)
    Nn, d = Xk.shape
    h = C.c_void_p()
    check(lib.krr_rpcholesky(Xp, Nn, d, _kern(kern), float(sigma), int(k), int(block), seed,
                             _stream(stream, X), C.byref(h)), "krr_rpcholesky")
    return Factor(h)


_PIVOTS = {"rpcholesky": N_.PIVOT_RPCHOLESKY, "uniform": N_.PIVOT_UNIFORM,
           "greedy": N_.PIVOT_GREEDY}


def krr_pivoted_cholesky(X, kern, sigma: float, k: int, block: int = 0, seed: int = 0,
                         rule="rpcholesky", stream=None) -> Factor:
    """Partial Cholesky with the pivot rule 'rpcholesky', 'uniform' or 'greedy'."""
    lib = load()
    Xk, Xp = _arr(X)
    Nn, d = Xk.shape
    h = C.c_void_p()
    r = _PIVOTS[rule] if isinstance(rule, str) else int(rule)
    check(lib.krr_pivoted_cholesky(Xp, Nn, d, _kern(kern), float(sigma), int(k), int(block),
                                   int(seed), r, _stream(stream, X), C.byref(h)),
          "krr_pivoted_cholesky")
    return Factor(h)


def krr_precond_apply(F: Factor, mu: float, R, prec="fp64", stream=None):
    lib = load()
    Rk, Rp = _arr(R)
    m, Nn = _shape2(Rk)
    Z, Zp = _empty_like_container(R, (m, Nn))
    check(lib.krr_precond_apply(F.handle, float(mu), Rp, m, Zp, _prec(prec),
                                _stream(stream, R)), "krr_precond_apply")
    return Z


def krr_pcg_solve(X, kern, sigma: float, Y, mu: float, F: Optional[Factor], tol: float,
                  maxit: int = 0, prec="mixed", stream=None, out=None, raise_on_noconv=False):
    """Alg. 1 PCG.  Returns (alpha (m, N), info dict with 'status')."""
    lib = load()
    Xk, Xp = _arr(X)
    Yk, Yp = _arr(Y)
    Nn, d = Xk.shape
    m = _shape2(Yk)[0]
    if out is None:
        A, Ap = _empty_like_container(Y, (m, Nn))
    else:
        A, Ap = out, C.c_void_p(out.data_ptr() if _is_torch(out) else out.ctypes.data)
    info = KrrInfo()
    allow = () if raise_on_noconv else (N_.KRR_ENOCONV,)
    st = check(lib.krr_pcg_solve(Xp, Nn, d, _kern(kern), float(sigma), Yp, m, float(mu),
                                 F.handle if F is not None else None, float(tol), int(maxit),
                                 _prec(prec), Ap, _stream(stream, X, Y), C.byref(info)),
               "krr_pcg_solve", allow)
    res = info.as_dict()
    res["status"] = N_.STATUS_NAMES[st]
    return A, res


def krr_pcg_solve_batched(X, kerns, sigmas, factors, mus, Y, tol: float, maxit: int = 0,
                          stream=None, out=None, raise_on_noconv=False):
    """Batched Alg. 1 PCG: settings (kerns[q], sigmas[q], factors[q]) x
    regularisations mus; Y (S*len(mus), N), column q*ms + c.  Returns
    (alpha like Y, info dict)."""
    lib = load()
    Xk, Xp = _arr(X)
    Yk, Yp = _arr(Y)
    Nn, d = Xk.shape
    S, ms = len(kerns), len(mus)
    mt = S * ms
    assert _shape2(Yk)[0] == mt
    kk = np.ascontiguousarray([_kern(k) for k in kerns], dtype=np.int32)
    ss = np.ascontiguousarray(sigmas, dtype=np.float64)
    mm = np.ascontiguousarray(mus, dtype=np.float64)
    handles = (C.c_void_p * S)(*[(f.handle if f is not None else None) for f in factors]) \
        if factors is not None else None
    if out is None:
        A, Ap = _empty_like_container(Y, (mt, Nn))
    else:
        A, Ap = out, C.c_void_p(out.data_ptr() if _is_torch(out) else out.ctypes.data)
    info = KrrInfo()
    allow = () if raise_on_noconv else (N_.KRR_ENOCONV,)
    st = check(lib.krr_pcg_solve_batched(Xp, Nn, d, S, C.c_void_p(kk.ctypes.data),
                                         C.c_void_p(ss.ctypes.data),
                                         C.cast(handles, C.c_void_p) if handles else None, ms,
                                         C.c_void_p(mm.ctypes.data), Yp, float(tol), int(maxit),
                                         Ap, _stream(stream, X, Y), C.byref(info)),
               "krr_pcg_solve_batched", allow)
    res = info.as_dict()
    res["status"] = N_.STATUS_NAMES[st]
    return A, res


# ------------------------------------------------------------------ KRILL
def krr_sparse_sign(N: int, s: int, zeta: int, seed: int, stream=None):
    """(rows int32 (N, zeta), vals float64 (N, zeta)) on the host."""
    lib = load()
    rows = np.empty((N, zeta), dtype=np.int32)
    vals = np.empty((N, zeta))
    check(lib.krr_sparse_sign(N, s, zeta, seed, C.c_void_p(rows.ctypes.data),
                              C.c_void_p(vals.ctypes.data), _stream(stream)), "krr_sparse_sign")
    return rows, vals


class KrillPreconditioner:
    def __init__(self, handle, k: int):
        self._h = handle
        self.k = k

    @property
    def handle(self):
        if not self._h:
            raise ValueError("preconditioner already freed")
        return self._h

    def export(self):
        """dict of H, P, Cu (k x k) and Bsk (s x k) as host arrays."""
        lib = load()
        k = self.k
        s = C.c_int()
        check(lib.krill_export(self.handle, None, None, None, None, C.byref(s)), "krill_export")
        H = np.empty((k, k), order="F")
        P = np.empty((k, k), order="F")
        Cu = np.empty((k, k), order="F")
        B = np.empty((s.value, k), order="F")
        check(lib.krill_export(self.handle, C.c_void_p(H.ctypes.data), C.c_void_p(B.ctypes.data),
                               C.c_void_p(P.ctypes.data), C.c_void_p(Cu.ctypes.data), C.byref(s)),
              "krill_export")
        return {"H": H, "Bsk": B, "P": P, "Cu": Cu, "s": s.value}

    def free(self):
        if self._h:
            load().krill_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def krill_build(X, kern, sigma: float, centers, mu: float, sketch_rows: int = 0, zeta: int = 0,
                seed: int = 0, stream=None) -> KrillPreconditioner:
    lib = load()
    Xk, Xp = _arr(X)
    Ck, Cp = _arr(centers, np.int64)
    Nn, d = Xk.shape
    k = int(Ck.shape[0])
    h = C.c_void_p()
    check(lib.krill_build(Xp, Nn, d, _kern(kern), float(sigma), Cp, k, float(mu),
                          int(sketch_rows), int(zeta), seed, _stream(stream, X), C.byref(h)),
          "krill_build")
    return KrillPreconditioner(h, k)


def krill_solve(P: KrillPreconditioner, Y, tol: float, maxit: int = 0, stream=None,
                raise_on_noconv=False):
    """Alg. 2 PCG.  Returns (beta (m, k), info dict)."""
    lib = load()
    Yk, Yp = _arr(Y)
    m = _shape2(Yk)[0]
    B, Bp = _empty_like_container(Y, (m, P.k))
    info = KrrInfo()
    allow = () if raise_on_noconv else (N_.KRR_ENOCONV,)
    st = check(lib.krill_solve(P.handle, Yp, m, float(tol), int(maxit), Bp, _stream(stream, Y),
                               C.byref(info)), "krill_solve", allow)
    res = info.as_dict()
    res["status"] = N_.STATUS_NAMES[st]
    return B, res


def krr_set_autotune(on: bool) -> None:
    load().krr_set_autotune(1 if on else 0)


def krr_set_pcg_graphs(on: bool) -> None:
    """CUDA-graph replay of the PCG iterations (on by default)."""
    load().krr_set_pcg_graphs(1 if on else 0)


def krr_check_bounded_wait(budget_cycles: int = 1_000_000, stream=None) -> str:
    """Runs a device-side bounded wait that cannot complete; returns the
    status name ('KRR_ETIMEOUT' when the timeout path worked)."""
    st = load().krr_check_bounded_wait(int(budget_cycles), _stream(stream))
    if st not in (N_.KRR_OK, N_.KRR_ETIMEOUT):
        check(st, "krr_check_bounded_wait")
    return N_.STATUS_NAMES[st]


def krr_autotune_choice(kern, d: int, m: int, N: int) -> int:
    """Split count the autotuner chose for a float32 product shape (0: none)."""
    v = C.c_int()
    check(load().krr_autotune_choice(_kern(kern), int(d), int(m), int(N), C.byref(v)),
          "krr_autotune_choice")
    return v.value


def krr_set_product_path(path) -> None:
    """Path of the float32 product for the Gaussian and Matern kernels:
    "tensor" (inner products on the tcgen05 tensor cores, the default),
    "fma", or "mma_sync" (the register-operand tensor path)."""
    code = {"tensor": 0, "fma": 1, "mma_sync": 2}.get(path, path)
    check(load().krr_set_product_path(int(code)), "krr_set_product_path")


# Epilogue variants of the tcgen05 product (KRR_PRODUCT_VARIANTS in krr.h).
PRODUCT_VARIANTS = 11


def krr_set_product_variant(variant: int) -> None:
    """Epilogue variant of the tcgen05 product (0: autotuned / default)."""
    check(load().krr_set_product_variant(int(variant)), "krr_set_product_variant")


def krr_autotune_variant(kern, d: int, m: int, N: int):
    """(chosen variant or 0, per-variant launch times in ms) for a shape."""
    v = C.c_int()
    ms = (C.c_float * PRODUCT_VARIANTS)()
    check(load().krr_autotune_variant(_kern(kern), int(d), int(m), int(N), C.byref(v), ms),
          "krr_autotune_variant")
    return v.value, [float(x) for x in ms]


def krr_profile_collect(which: int = 0):
    """(summed ms, launches) of the recorded product launches of one kind
    (0 float32, 1 float64, 2 float-float) since profiling was switched on."""
    ms, n = C.c_double(), C.c_int()
    check(load().krr_profile_collect(int(which), C.byref(ms), C.byref(n)),
          "krr_profile_collect")
    return ms.value, n.value


def krr_set_profiling(on: bool) -> None:
    load().krr_set_profiling(1 if on else 0)


def krr_version() -> str:
    return load().krr_version().decode()


def krr_launch_count() -> int:
    return int(load().krr_launch_count())


# --------------------------------------------------------------- serving
def krr_server_footprint(N: int, d: int, m: int, k: int) -> float:
    """Estimated peak device bytes of one served request (host-only)."""
    b = C.c_double()
    check(load().krr_server_footprint(int(N), int(d), int(m), int(k), C.byref(b)),
          "krr_server_footprint")
    return b.value


class KrrServer:
    """The krr_server_* calls: continuous batching of Alg. 1 solves.

    submit() queues a request and returns its id; step() advances the engine
    once; poll() returns finished requests as dicts holding the result fields
    of krr_request_result plus 'alpha' (m, N) and the status name.  The
    binding keeps each request's arrays alive until poll() reports it.
    """

    def __init__(self, max_slots: int = 16, iters_per_step: int = 4, use_graph: bool = True,
                 hbm_budget_bytes: float = 0.0, build_threads: int = 0):
        lib = load()
        cfg = N_.ServerConfig(int(max_slots), int(iters_per_step), 1 if use_graph else 0,
                              int(build_threads), float(hbm_budget_bytes))
        h = C.c_void_p()
        check(lib.krr_server_create(C.byref(cfg), C.byref(h)), "krr_server_create")
        self._h = h
        self._keep = {}

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("server destroyed")
        return self._h

    def submit(self, X, kern, sigma: float, Y, mu: float, k: int, tol: float = 1e-6,
               maxit: int = 1000, seed: int = 0, out=None) -> int:
        lib = load()
        Xk, Xp = _arr(X)
        Yk, Yp = _arr(Y)
        Nn, d = Xk.shape
        m = _shape2(Yk)[0]
        if out is None:
            A, Ap = _empty_like_container(Y, (m, Nn))
        else:
            A, Ap = out, C.c_void_p(out.data_ptr() if _is_torch(out) else out.ctypes.data)
        rid = C.c_int64()
        check(lib.krr_server_submit(self.handle, Xp, Nn, d, _kern(kern), float(sigma), Yp, m,
                                    float(mu), int(k), int(seed), float(tol), int(maxit), Ap,
                                    C.byref(rid)), "krr_server_submit")
        self._keep[rid.value] = (Xk, Yk, A)
        return rid.value

    def step(self) -> int:
        """One engine step; returns the number of unfinished requests."""
        n = C.c_int64()
        check(load().krr_server_step(self.handle, C.byref(n)), "krr_server_step")
        return n.value

    def poll(self):
        lib = load()
        out = []
        buf = (N_.RequestResult * 64)()
        while True:
            n = C.c_int()
            check(lib.krr_server_poll(self.handle, buf, 64, C.byref(n)), "krr_server_poll")
            for i in range(n.value):
                r = buf[i].as_dict()
                r["status_name"] = N_.STATUS_NAMES[r["status"]]
                r["alpha"] = self._keep.pop(r["id"])[2]
                out.append(r)
            if n.value < 64:
                return out

    def drain(self):
        """Steps until every submitted request has finished; returns them."""
        done = []
        while True:
            left = self.step()
            done += self.poll()
            if left == 0:
                return done + self.poll()

    def stats(self) -> dict:
        st = N_.ServerStats()
        check(load().krr_server_get_stats(self.handle, C.byref(st)), "krr_server_get_stats")
        return st.as_dict()

    def clock(self) -> float:
        return float(load().krr_server_clock(self.handle))

    def progress(self, rid: int) -> dict:
        pr = N_.RequestProgress()
        check(load().krr_server_progress(self.handle, int(rid), C.byref(pr)),
              "krr_server_progress")
        return pr.as_dict()

    def evict(self, rid: int) -> None:
        check(load().krr_server_evict(self.handle, int(rid)), "krr_server_evict")

    def resume(self, rid: int) -> None:
        check(load().krr_server_resume(self.handle, int(rid)), "krr_server_resume")

    def export(self, rid: int) -> bytes:
        """Checkpoint of a parked request; the request leaves this server."""
        lib = load()
        n = C.c_size_t(0)
        check(lib.krr_server_export(self.handle, int(rid), None, C.byref(n)), "krr_server_export")
        buf = C.create_string_buffer(n.value)
        check(lib.krr_server_export(self.handle, int(rid), buf, C.byref(n)), "krr_server_export")
        self._keep.pop(int(rid), None)
        return buf.raw[:n.value]

    def import_(self, blob: bytes, X, Y, out=None) -> int:
        """Queues a request from a checkpoint with the original X and Y."""
        lib = load()
        Xk, Xp = _arr(X)
        Yk, Yp = _arr(Y)
        Nn = Xk.shape[0]
        m = _shape2(Yk)[0]
        if out is None:
            A, Ap = _empty_like_container(Y, (m, Nn))
        else:
            A, Ap = out, C.c_void_p(out.data_ptr() if _is_torch(out) else out.ctypes.data)
        raw = C.create_string_buffer(bytes(blob), len(blob))
        rid = C.c_int64()
        check(lib.krr_server_import(self.handle, raw, len(blob), Xp, Yp, Ap, C.byref(rid)),
              "krr_server_import")
        self._keep[rid.value] = (Xk, Yk, A)
        return rid.value

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().krr_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
