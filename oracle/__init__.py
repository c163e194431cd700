"""CPU oracle for the RPCholesky-PCG and KRILL hot path -- TEST INFRASTRUCTURE.

Plain, slow, float64 statements of what the paper's method computes.  The
heavy loops (kernel evaluation, products, Alg. 3, the sparse sign embedding
and its sketch) are plain C in ``krr_oracle.c``; the dense linear algebra
steps (economy SVD, Cholesky, triangular solves) are numpy/scipy library
calls.  Only the tests, the package smoke check and the benchmark's CPU
baseline may use this package; the library never does, and the oracle never
imports the library.

Arrays: X is (N, d) float64; right-hand-side blocks are (m, N) float64, i.e.
N x m column-major; the factor F is returned as (rank, N), i.e. N x rank
column-major.  ``mu`` is per data point; the shift is lambda = mu * N.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np

from .build import build_oracle

_LIB = None

GAUSSIAN, LAPLACE_L1, MATERN52 = 0, 1, 2
EPS_MACH = 2.0 ** -52


def lib():
    global _LIB
    if _LIB is None:
        _LIB = C.CDLL(build_oracle())
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int64)
        L = _LIB
        L.orc_kappa.restype = C.c_double
        L.orc_kappa.argtypes = [dp, dp, C.c_int, C.c_int, C.c_double]
        L.orc_kernel_block.argtypes = [dp, C.c_int64, C.c_int, C.c_int, C.c_double,
                                       ip, C.c_int64, ip, C.c_int64, dp]
        L.orc_kmatvec.argtypes = [dp, C.c_int64, C.c_int, C.c_int, C.c_double,
                                  C.c_double, dp, C.c_int, ip, C.c_int64, dp]
        L.orc_kcross_matvec.argtypes = [dp, C.c_int64, dp, C.c_int64, C.c_int, C.c_int,
                                        C.c_double, dp, C.c_int, dp]
        L.orc_kcols_matvec.argtypes = [dp, C.c_int64, C.c_int, C.c_int, C.c_double,
                                       ip, C.c_int, dp, C.c_int, dp]
        L.orc_krows_matvec.argtypes = [dp, C.c_int64, C.c_int, C.c_int, C.c_double,
                                       ip, C.c_int, dp, C.c_int, dp]
        L.orc_philox4x64.argtypes = [C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                     C.POINTER(C.c_uint64)]
        L.orc_fixed_point_bits.restype = C.c_int
        L.orc_fixed_point_bits.argtypes = [C.c_int64]
        L.orc_fixed_point_weight.restype = C.c_uint64
        L.orc_fixed_point_weight.argtypes = [C.c_double, C.c_double, C.c_int]
        L.orc_rpc_sample.restype = C.c_int
        L.orc_rpc_sample.argtypes = [dp, C.c_int64, C.c_double, C.c_uint64, C.c_uint64,
                                     C.c_int, ip]
        L.orc_uniform_pivots.restype = C.c_int
        L.orc_uniform_pivots.argtypes = [C.c_int64, C.c_int, C.c_uint64, ip]
        L.orc_greedy_pick.restype = C.c_int
        L.orc_greedy_pick.argtypes = [dp, C.c_int64, C.c_double, C.c_int, ip]
        L.orc_pivoted_cholesky.restype = C.c_int
        L.orc_pivoted_cholesky.argtypes = [dp, C.c_int64, C.c_int, C.c_int, C.c_double,
                                           C.c_int, C.c_int, C.c_uint64, C.c_int, dp, ip, dp,
                                           ip, dp]
        L.orc_rpcholesky.restype = C.c_int
        L.orc_rpcholesky.argtypes = [dp, C.c_int64, C.c_int, C.c_int, C.c_double,
                                     C.c_int, C.c_int, C.c_uint64, dp, ip, dp, ip, dp]
        L.orc_sparse_sign.argtypes = [C.c_int64, C.c_int, C.c_int, C.c_uint64,
                                      C.POINTER(C.c_int32), dp]
        L.orc_krill_sketch.argtypes = [dp, C.c_int64, C.c_int, C.c_int, C.c_double,
                                       ip, C.c_int, C.POINTER(C.c_int32), dp,
                                       C.c_int, C.c_int, dp]
    return _LIB


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a) -> Optional[np.ndarray]:
    return None if a is None else np.ascontiguousarray(a, dtype=np.int64)


# --------------------------------------------------------------------------
# Kernel matrix and the matrix-free product (Sec. 2.1, Alg. 1 "Product")
# --------------------------------------------------------------------------
def kappa(x: np.ndarray, y: np.ndarray, kern: int, sigma: float) -> float:
    x, y = _f64(x), _f64(y)
    return lib().orc_kappa(_d(x), _d(y), x.shape[0], kern, sigma)


def kernel_block(X, kern: int, sigma: float, rows=None, cols=None) -> np.ndarray:
    """A(rows, cols) with A_ij = kappa(x_i, x_j)."""
    X = _f64(X)
    N, d = X.shape
    rows, cols = _i64(rows), _i64(cols)
    nr = N if rows is None else rows.shape[0]
    nc = N if cols is None else cols.shape[0]
    out = np.empty((nr, nc))
    lib().orc_kernel_block(_d(X), N, d, kern, sigma, _i(rows), nr, _i(cols), nc, _d(out))
    return out


def kmatvec(X, kern: int, sigma: float, lam: float, V, rows=None) -> np.ndarray:
    """(A + lam I) V restricted to the requested output rows; V is (m, N)."""
    X = _f64(X)
    V = _f64(np.atleast_2d(V))
    N, d = X.shape
    m = V.shape[0]
    assert V.shape[1] == N
    rows = _i64(rows)
    nr = N if rows is None else rows.shape[0]
    Y = np.empty((m, nr))
    lib().orc_kmatvec(_d(X), N, d, kern, sigma, lam, _d(V), m, _i(rows), nr, _d(Y))
    return Y


def predict(X, kern, sigma, alpha, T) -> np.ndarray:
    """f(t) = sum_n alpha_n kappa(x_n, t) for every test point (Sec. 2.1);
    alpha (m, N) -> (m, Nt)."""
    X, T, alpha = _f64(X), _f64(T), _f64(np.atleast_2d(alpha))
    N, d = X.shape
    Nt = T.shape[0]
    m = alpha.shape[0]
    out = np.empty((m, Nt))
    lib().orc_kcross_matvec(_d(X), N, _d(T), Nt, d, kern, sigma, _d(alpha), m, _d(out))
    return out


def kcols_matvec(X, kern, sigma, S, beta) -> np.ndarray:
    """A(:, S) beta, beta (m, k) -> (m, N)."""
    X, beta, S = _f64(X), _f64(np.atleast_2d(beta)), _i64(S)
    N, d = X.shape
    m, k = beta.shape
    u = np.empty((m, N))
    lib().orc_kcols_matvec(_d(X), N, d, kern, sigma, _i(S), k, _d(beta), m, _d(u))
    return u


def krows_matvec(X, kern, sigma, S, u) -> np.ndarray:
    """A(S, :) u, u (m, N) -> (m, k)."""
    X, u, S = _f64(X), _f64(np.atleast_2d(u)), _i64(S)
    N, d = X.shape
    m = u.shape[0]
    k = S.shape[0]
    out = np.empty((m, k))
    lib().orc_krows_matvec(_d(X), N, d, kern, sigma, _i(S), k, _d(u), m, _d(out))
    return out


# --------------------------------------------------------------------------
# Counter-based generator and the pivot sampler of Alg. 3
# --------------------------------------------------------------------------
def philox4x64(ctr, key) -> np.ndarray:
    c = (C.c_uint64 * 4)(*[int(v) for v in ctr])
    k = (C.c_uint64 * 2)(*[int(v) for v in key])
    o = (C.c_uint64 * 4)()
    lib().orc_philox4x64(c, k, o)
    return np.array(list(o), dtype=np.uint64)


def fixed_point_bits(N: int) -> int:
    return lib().orc_fixed_point_bits(N)


def fixed_point_weight(dres: float, fbits: int, dfloor: float = 0.0) -> int:
    return int(lib().orc_fixed_point_weight(dres, dfloor, fbits))


def drop_threshold(N: int, maxdiag: float = 1.0) -> float:
    """N eps max_i A_ii: drop threshold of the block Cholesky and floor of the
    sampling weights."""
    return N * EPS_MACH * maxdiag


def rpc_sample(dres, seed: int, t: int, ndraw: int, dfloor: float = 0.0) -> np.ndarray:
    """Draws of block t of Alg. 3 (empty if every weight is zero); residuals
    at or below dfloor carry no weight."""
    dres = _f64(dres)
    out = np.empty(ndraw, dtype=np.int64)
    got = lib().orc_rpc_sample(_d(dres), dres.shape[0], dfloor, seed, t, ndraw, _i(out))
    return out[:got]


@dataclass
class RPCholeskyResult:
    F: np.ndarray          # (rank, N): N x rank column-major
    S: np.ndarray          # int64[rank], pivots in column order
    dres: np.ndarray       # final residual diagonal
    rank: int
    nblocks: int
    trace_hist: np.ndarray  # Sum(d) before the first block and after each block


def default_block(k: int) -> int:
    """Alg. 1: B = min(100, ceil(r / 10))."""
    return min(100, -(-k // 10))


PIVOT_RPCHOLESKY, PIVOT_UNIFORM, PIVOT_GREEDY = 0, 1, 2


def uniform_pivots(N: int, k: int, seed: int) -> np.ndarray:
    """The uniform pivot rule of Sec. 4: a uniformly random k-subset of the
    N columns, in draw order (reading in krr_oracle.c)."""
    out = np.empty(min(k, N), dtype=np.int64)
    got = lib().orc_uniform_pivots(N, k, seed, _i(out))
    return out[:got]


def greedy_pick(dres, npick: int, dfloor: float = 0.0) -> np.ndarray:
    """The npick largest residuals above dfloor, descending (ties: smallest
    index) -- the greedy pivot rule of Sec. 4."""
    dres = _f64(dres)
    out = np.empty(npick, dtype=np.int64)
    got = lib().orc_greedy_pick(_d(dres), dres.shape[0], dfloor, npick, _i(out))
    return out[:got]


def pivoted_cholesky(X, kern: int, sigma: float, k: int, B: int = 0, seed: int = 0,
                     rule: int = PIVOT_RPCHOLESKY) -> RPCholeskyResult:
    """Alg. 3 with the pivots of each block chosen by `rule`: RPCholesky
    sampling, uniform sampling or greedy selection (Sec. 4).  B = 0 selects
    Alg. 1's default block size for RPCholesky and uniform, and 1 (one pivot
    at a time, the paper's greedy rule) for greedy.  With the uniform rule
    k counts the pivots used, kept or dropped, so the rank can be below k."""
    X = _f64(X)
    N, d = X.shape
    k = min(k, N)
    B = B or (1 if rule == PIVOT_GREEDY else default_block(k))
    F = np.zeros((k, N))
    S = np.zeros(k, dtype=np.int64)
    dres = np.empty(N)
    nb = np.zeros(1, dtype=np.int64)
    hist = np.zeros(k + N + 1)
    rank = lib().orc_pivoted_cholesky(_d(X), N, d, kern, sigma, k, B, seed, rule, _d(F), _i(S),
                                      _d(dres), _i(nb), _d(hist))
    return RPCholeskyResult(F[:rank].copy(), S[:rank].copy(), dres, rank, int(nb[0]),
                            hist[:int(nb[0]) + 1].copy())


def rpcholesky(X, kern: int, sigma: float, k: int, B: int = 0,
               seed: int = 0) -> RPCholeskyResult:
    """Alg. 3, blocked RPCholesky, with the sampler reading described in
    krr_oracle.c.  B = 0 selects Alg. 1's default block size."""
    return pivoted_cholesky(X, kern, sigma, k, B, seed, PIVOT_RPCHOLESKY)


# --------------------------------------------------------------------------
# Alg. 1 preconditioner in the paper's SVD form
# --------------------------------------------------------------------------
@dataclass
class NystromPreconditioner:
    U: np.ndarray     # (N, r)
    sig2: np.ndarray  # (r,) squared singular values of F
    lam: float

    def apply(self, v: np.ndarray) -> np.ndarray:
        """v -> U[(Sigma^2 + lam I)^{-1} - lam^{-1} I] U^T v + lam^{-1} v."""
        w = self.U.T @ v
        w = (1.0 / (self.sig2 + self.lam) - 1.0 / self.lam)[:, None] * w \
            if v.ndim == 2 else (1.0 / (self.sig2 + self.lam) - 1.0 / self.lam) * w
        return self.U @ w + v / self.lam


def nystrom_preconditioner(F_rows: np.ndarray, lam: float) -> NystromPreconditioner:
    """(U, Sigma, ~) = EconomySizeSVD(F) of Alg. 1; F_rows is F^T, (r, N)."""
    F = F_rows.T
    if F.shape[1] == 0:
        return NystromPreconditioner(np.zeros((F.shape[0], 0)), np.zeros(0), lam)
    U, s, _ = np.linalg.svd(F, full_matrices=False)
    return NystromPreconditioner(U, s * s, lam)


# --------------------------------------------------------------------------
# PCG (Sec. 3: standard PCG, zero initial iterate, stop on the relative
# residual; Saad, Iterative Methods for Sparse Linear Systems, Alg. 9.1)
# --------------------------------------------------------------------------
@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    relres: float          # recursive residual at exit
    status: str            # "ok", "maxit", "breakdown"


def pcg(product: Callable[[np.ndarray], np.ndarray], b: np.ndarray,
        precond: Callable[[np.ndarray], np.ndarray], tol: float,
        maxit: int = 1000) -> PCGResult:
    """One right-hand side b (1-D)."""
    x = np.zeros_like(b)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return PCGResult(x, 0, 0.0, "ok")
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < maxit:
        q = product(p)
        pq = float(p @ q)
        if not (pq > 0.0):
            return PCGResult(x, it, float(np.linalg.norm(r)) / bnorm, "breakdown")
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rel = float(np.linalg.norm(r)) / bnorm
        if rel <= tol:
            return PCGResult(x, it, rel, "ok")
        z = precond(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return PCGResult(x, it, float(np.linalg.norm(r)) / bnorm, "maxit")


@dataclass
class SolveResult:
    alpha: np.ndarray      # (m, N)
    iters: list
    relres_true: list      # ||y - (A + lam I) alpha|| / ||y|| per column
    status: list


def true_relres(X, kern, sigma, lam, Y, alpha) -> np.ndarray:
    """Float64 relative residual ||y - (A + lam I) alpha|| / ||y|| per column."""
    Y = np.atleast_2d(Y)
    R = Y - kmatvec(X, kern, sigma, lam, alpha)
    ny = np.linalg.norm(Y, axis=1)
    nr = np.linalg.norm(R, axis=1)
    return np.where(ny > 0, nr / np.where(ny > 0, ny, 1.0), nr)


def krr_pcg_solve(X, kern: int, sigma: float, Y, mu: float, F_rows: np.ndarray,
                  tol: float, maxit: int = 1000) -> SolveResult:
    """Alg. 1: PCG on (A + lam I) alpha = y with the RPCholesky preconditioner,
    lam = mu * N; each column of Y runs its own PCG."""
    X = _f64(X)
    Y = _f64(np.atleast_2d(Y))
    N = X.shape[0]
    lam = mu * N
    P = nystrom_preconditioner(F_rows, lam)
    product = lambda v: kmatvec(X, kern, sigma, lam, v[None, :])[0]
    out = np.zeros_like(Y)
    its, sts = [], []
    for c in range(Y.shape[0]):
        res = pcg(product, Y[c].copy(), P.apply, tol, maxit)
        out[c] = res.x
        its.append(res.iters)
        sts.append(res.status)
    rr = true_relres(X, kern, sigma, lam, Y, out)
    return SolveResult(out, its, list(rr), sts)


# --------------------------------------------------------------------------
# KRILL (Alg. 2)
# --------------------------------------------------------------------------
def default_zeta(k: int) -> int:
    """zeta = ceil(log(k + 1)), natural logarithm."""
    return int(math.ceil(math.log(k + 1)))


def sparse_sign(N: int, s: int, zeta: int, seed: int):
    """Sparse sign embedding Phi (s x N) as per-column row indices (N, zeta)
    and values (N, zeta); reading in krr_oracle.c."""
    rows = np.empty((N, zeta), dtype=np.int32)
    vals = np.empty((N, zeta))
    lib().orc_sparse_sign(N, s, zeta, seed, rows.ctypes.data_as(C.POINTER(C.c_int32)),
                          _d(vals))
    return rows, vals


def sparse_sign_dense(N: int, s: int, zeta: int, seed: int) -> np.ndarray:
    rows, vals = sparse_sign(N, s, zeta, seed)
    Phi = np.zeros((s, N))
    for n in range(N):
        Phi[rows[n], n] = vals[n]
    return Phi


def krill_sketch(X, kern, sigma, S, rows, vals, s) -> np.ndarray:
    X, S = _f64(X), _i64(S)
    N, d = X.shape
    k = S.shape[0]
    zeta = rows.shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    vals = _f64(vals)
    Bsk = np.empty((s, k))
    lib().orc_krill_sketch(_d(X), N, d, kern, sigma, _i(S), k,
                           rows.ctypes.data_as(C.POINTER(C.c_int32)), _d(vals), zeta, s,
                           _d(Bsk))
    return Bsk


@dataclass
class KrillPreconditioner:
    H: np.ndarray     # lam A(S,S) + N eps tr(A(S,S)) I
    Bsk: np.ndarray   # Phi A(:, S), (s, k)
    P: np.ndarray     # Bsk^T Bsk + H
    Cu: np.ndarray    # upper Cholesky factor, P = Cu^T Cu
    lam: float
    s: int
    zeta: int


def krill_build(X, kern: int, sigma: float, S, mu: float, s: int = 0,
                zeta: int = 0, seed: int = 0) -> KrillPreconditioner:
    X = _f64(X)
    N = X.shape[0]
    S = _i64(S)
    k = S.shape[0]
    lam = mu * N
    s = s or 2 * k
    zeta = zeta or default_zeta(k)
    ASS = kernel_block(X, kern, sigma, S, S)
    H = lam * ASS
    H = H + N * EPS_MACH * np.trace(ASS) * np.eye(k)
    rows, vals = sparse_sign(N, s, zeta, seed)
    Bsk = krill_sketch(X, kern, sigma, S, rows, vals, s)
    P = Bsk.T @ Bsk + H
    L = np.linalg.cholesky(P)
    return KrillPreconditioner(H, Bsk, P, L.T.copy(), lam, s, zeta)


def krill_product(X, kern, sigma, S, H, beta) -> np.ndarray:
    """beta -> A(S,:)(A(:,S) beta) + H beta, beta (m, k)."""
    beta = np.atleast_2d(beta)
    u = kcols_matvec(X, kern, sigma, S, beta)
    return krows_matvec(X, kern, sigma, S, u) + (H @ beta.T).T


def krill_solve(X, kern: int, sigma: float, S, P: KrillPreconditioner, Y,
                tol: float, maxit: int = 1000) -> SolveResult:
    """Alg. 2: PCG on [A(S,:)A(:,S) + H] beta = A(S,:) y with the preconditioner
    beta -> C^{-1}(C^{-T} beta)."""
    import scipy.linalg as sla
    X = _f64(X)
    Y = _f64(np.atleast_2d(Y))
    S = _i64(S)
    rhs = krows_matvec(X, kern, sigma, S, Y)
    product = lambda v: krill_product(X, kern, sigma, S, P.H, v[None, :])[0]

    def precond(v):
        w = sla.solve_triangular(P.Cu, v, trans="T", lower=False)
        return sla.solve_triangular(P.Cu, w, lower=False)

    out = np.zeros((Y.shape[0], S.shape[0]))
    its, sts = [], []
    for c in range(Y.shape[0]):
        res = pcg(product, rhs[c].copy(), precond, tol, maxit)
        out[c] = res.x
        its.append(res.iters)
        sts.append(res.status)
    R = rhs - krill_product(X, kern, sigma, S, P.H, out)
    rr = np.linalg.norm(R, axis=1) / np.linalg.norm(rhs, axis=1)
    return SolveResult(out, its, list(rr), sts)
