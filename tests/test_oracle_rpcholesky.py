"""Pins for the oracle's blocked RPCholesky (Alg. 3).

* brute force on tiny inputs: Alg. 3 restated in numpy/scipy with the
  independent sampler restatement gives the same pivots and factor;
* k = N, B = 1 on distinct points reproduces A (F F^T = A);
* the column Nystrom identity F F^T = A(:,S) A(S,S)^{-1} A(S,:) (Sec. 3.1);
* A - F F^T is psd, the residual diagonal is its diagonal, is >= 0, is zero
  at the pivots, and its trace never increases from block to block;
* a numerically singular block (exact twins) drops the repeated point.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from inputs import make_c1_plain_fp64, make_c2_mixed
from test_oracle_sampler import independent_sample


def brute_rpcholesky(A, k, B, seed):
    N = A.shape[0]
    F = np.zeros((N, 0))
    S = []
    d = np.diag(A).copy()
    t = 0
    while F.shape[1] < k:
        nd = min(B, k - F.shape[1])
        draws = independent_sample(d, seed, t, nd, N * 2.0 ** -52)
        t += 1
        if len(draws) == 0:
            break
        Sp = list(dict.fromkeys(int(v) for v in draws))
        G = A[:, Sp] - F @ F[Sp, :].T
        R = np.linalg.cholesky(G[Sp, :]).T
        Fn = sla.solve_triangular(R, G.T, trans="T", lower=False).T
        F = np.hstack([F, Fn])
        S += Sp
        d = d - (Fn ** 2).sum(axis=1)
        d[Sp] = 0.0
    return F, np.array(S)


@pytest.mark.parametrize("N,k,B,seed", [(8, 8, 1, 0), (30, 12, 4, 1), (64, 40, 7, 2),
                                         (64, 20, 20, 3)])
def test_brute_force_tiny(N, k, B, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, 3))
    A = O.kernel_block(X, O.GAUSSIAN, 0.8)
    r = O.rpcholesky(X, O.GAUSSIAN, 0.8, k, B, seed)
    F, S = brute_rpcholesky(A, k, B, seed)
    np.testing.assert_array_equal(r.S, S)
    np.testing.assert_allclose(r.F.T, F, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("kern", [O.GAUSSIAN, O.LAPLACE_L1, O.MATERN52])
def test_full_rank_reproduces_A(kern):
    rng = np.random.default_rng(10 + kern)
    X = 3.0 * rng.standard_normal((40, 2))
    A = O.kernel_block(X, kern, 0.5)
    r = O.rpcholesky(X, kern, 0.5, 40, 1, seed=4)
    assert r.rank == 40
    np.testing.assert_allclose(r.F.T @ r.F, A, atol=1e-12)
    assert sorted(r.S.tolist()) == list(range(40))


@pytest.mark.parametrize("kern", [O.GAUSSIAN, O.LAPLACE_L1, O.MATERN52])
def test_column_nystrom_identity_and_invariants(kern):
    w = make_c1_plain_fp64(n=400)
    r = O.rpcholesky(w.X, kern, w.sigma, 60, 10, seed=7)
    A = O.kernel_block(w.X, kern, w.sigma)
    S = r.S
    FFt = r.F.T @ r.F
    nys = A[:, S] @ np.linalg.solve(A[np.ix_(S, S)], A[S, :])
    np.testing.assert_allclose(FFt, nys, atol=1e-9)
    E = A - FFt
    assert np.linalg.eigvalsh(E).min() > -1e-10
    assert r.dres.min() > -1e-14
    # pivots are zeroed when drawn and only decrease afterwards, so their
    # fixed-point weight stays zero and they are never drawn again
    assert np.all(r.dres[S] <= 0.0)
    assert np.all(r.dres[S] > -1e-20)
    keep = np.ones(w.N, bool)
    keep[S] = False
    np.testing.assert_allclose(r.dres[keep], np.diag(E)[keep], atol=1e-12)
    assert np.all(np.diff(r.trace_hist) <= 1e-12)
    assert r.trace_hist[0] == pytest.approx(w.N)
    assert len(set(S.tolist())) == len(S)


def test_block_size_rule():
    assert O.default_block(200) == 20
    assert O.default_block(1000) == 100
    assert O.default_block(2000) == 100
    assert O.default_block(5) == 1


def test_twins_are_dropped():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((20, 2)) * 4
    X = np.vstack([X, X[:5]])                 # exact duplicates of rows 0..4
    r = O.rpcholesky(X, O.GAUSSIAN, 0.5, 25, 25, seed=0)
    A = O.kernel_block(X, O.GAUSSIAN, 0.5)
    # each pair contributes one column at most
    assert r.rank <= 20
    for a in range(5):
        assert not (a in r.S and a + 20 in r.S)
    assert np.linalg.eigvalsh(A - r.F.T @ r.F).min() > -1e-10
    assert np.all(np.isfinite(r.F))


def test_zero_weight_stops_early():
    X = np.zeros((6, 2))                     # every point identical: rank one
    r = O.rpcholesky(X, O.GAUSSIAN, 1.0, 6, 2, seed=1)
    assert r.rank == 1
    np.testing.assert_allclose(r.F.T @ r.F, np.ones((6, 6)), atol=1e-15)


def test_deterministic_and_seeded():
    w = make_c2_mixed(n=2000, m=1, k=100)
    a = O.rpcholesky(w.X, w.kernel, w.sigma, 100, 10, seed=3)
    b = O.rpcholesky(w.X, w.kernel, w.sigma, 100, 10, seed=3)
    c = O.rpcholesky(w.X, w.kernel, w.sigma, 100, 10, seed=4)
    np.testing.assert_array_equal(a.S, b.S)
    np.testing.assert_array_equal(a.F, b.F)
    assert not np.array_equal(a.S, c.S)
