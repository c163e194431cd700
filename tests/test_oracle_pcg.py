"""Pins for the oracle's Alg. 1 preconditioner and PCG (Sec. 3).

* the PCG solution against a dense Cholesky solve (scipy / LAPACK);
* P^{-1}(P v) = v for the SVD-form preconditioner, P = F F^T + lam I;
* the spectrum of P^{-1/2}(A + lam I)P^{-1/2} lies in [1, 1 + tr(A - F F^T)/lam]
  (Sec. 6.1, proof of the RPCholesky guarantee);
* the energy-norm error obeys the PCG rate bound of Sec. 3;
* special cases: rank 0 is lam^{-1} I, an exact factor converges in one step,
  a zero right-hand side returns zero.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from inputs import make_c1_plain_fp64, make_c2_mixed


@pytest.fixture(scope="module")
def c1():
    w = make_c1_plain_fp64(n=1024)
    A = O.kernel_block(w.X, w.kernel, w.sigma)
    r = O.rpcholesky(w.X, w.kernel, w.sigma, 100, 10, seed=0)
    return w, A, r


def test_solution_matches_dense_cholesky(c1):
    w, A, r = c1
    lam = w.lam
    res = O.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, r.F, tol=1e-12)
    ref = sla.cho_solve(sla.cho_factor(A + lam * np.eye(w.N)), w.Y[0])
    assert res.status == ["ok"]
    assert res.relres_true[0] < 1e-11
    assert np.linalg.norm(res.alpha[0] - ref) / np.linalg.norm(ref) < 1e-8


def test_preconditioner_inverts_P(c1):
    w, A, r = c1
    lam = w.lam
    P = r.F.T @ r.F + lam * np.eye(w.N)
    pre = O.nystrom_preconditioner(r.F, lam)
    v = np.random.default_rng(0).standard_normal(w.N)
    np.testing.assert_allclose(pre.apply(P @ v), v, rtol=1e-9, atol=1e-9)


def test_condition_bound(c1):
    w, A, r = c1
    lam = w.lam
    P = r.F.T @ r.F + lam * np.eye(w.N)
    ev = sla.eigh(A + lam * np.eye(w.N), P, eigvals_only=True)
    bound = 1.0 + np.trace(A - r.F.T @ r.F) / lam
    assert ev.min() > 1.0 - 1e-8
    assert ev.max() < bound * (1 + 1e-8)


def test_pcg_rate_bound(c1):
    w, A, r = c1
    lam = w.lam
    M = A + lam * np.eye(w.N)
    P = r.F.T @ r.F + lam * np.eye(w.N)
    ev = sla.eigh(M, P, eigvals_only=True)
    kappa = ev.max() / ev.min()
    rho = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    xs = sla.cho_solve(sla.cho_factor(M), w.Y[0])
    pre = O.nystrom_preconditioner(r.F, lam)
    en = lambda e: np.sqrt(e @ M @ e)
    for t in (1, 3, 8, 15):
        res = O.pcg(lambda v: M @ v, w.Y[0].copy(), pre.apply, tol=0.0, maxit=t)
        assert res.iters == t
        assert en(res.x - xs) / en(xs) <= 2 * rho ** t * (1 + 1e-6)


def test_rank_zero_is_scaled_identity(c1):
    w, A, r = c1
    pre = O.nystrom_preconditioner(np.zeros((0, w.N)), 0.5)
    v = np.arange(w.N, dtype=float)
    np.testing.assert_array_equal(pre.apply(v), v / 0.5)


def test_exact_factor_converges_in_one_step():
    rng = np.random.default_rng(1)
    X = 3 * rng.standard_normal((60, 2))
    r = O.rpcholesky(X, O.GAUSSIAN, 0.7, 60, 1, seed=2)
    assert r.rank == 60
    y = rng.standard_normal((1, 60))
    res = O.krr_pcg_solve(X, O.GAUSSIAN, 0.7, y, 1e-3, r.F, tol=1e-10)
    assert res.iters == [1]
    assert res.relres_true[0] < 1e-10


def test_multiple_rhs_are_independent():
    w = make_c2_mixed(n=800, m=3, k=80)
    r = O.rpcholesky(w.X, w.kernel, w.sigma, 80, 10, seed=1)
    res = O.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, r.F, tol=1e-8)
    for c in range(3):
        one = O.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y[c:c + 1], w.mu, r.F, tol=1e-8)
        np.testing.assert_array_equal(one.alpha[0], res.alpha[c])
        assert one.iters[0] == res.iters[c]
    assert max(res.relres_true) < 1e-7


def test_zero_rhs(c1):
    w, A, r = c1
    res = O.krr_pcg_solve(w.X, w.kernel, w.sigma, np.zeros((1, w.N)), w.mu, r.F, tol=1e-10)
    assert res.iters == [0]
    assert not res.alpha.any()


def test_breakdown_reported():
    res = O.pcg(lambda v: -v, np.ones(4), lambda v: v, tol=1e-10)
    assert res.status == "breakdown"
