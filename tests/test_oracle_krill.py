"""Pins for the oracle's KRILL path (Alg. 2, Sec. 2.2).

* the sparse sign embedding has zeta distinct rows per column, entries
  +-zeta^{-1/2}, unit column norms, E[Phi^T Phi] = I, and matches an
  independent restatement of the sampling reading with numpy's Philox;
* the sketch equals Phi A(:,S) formed with a dense matrix product;
* the KRILL solution matches a direct solve of the restricted equations
  (Sec. 2.2) with the Alg. 2 shift, and an exact Gram matrix in place of the
  sketch converges in one iteration;
* soft check: the preconditioned condition number is near the 2k x k Gaussian
  model of Sec. 2.2.3, (1 + 2^{-1/2})^2 / (1 - 2^{-1/2})^2 ~ 34.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from inputs import make_c4_krill
from test_oracle_sampler import numpy_philox_block

TAG_ROWS = 0x53534531524f5753
TAG_SIGNS = 0x535345325349474e


def independent_sparse_sign(N, s, zeta, seed):
    rows = np.zeros((N, zeta), dtype=np.int64)
    vals = np.zeros((N, zeta))
    for n in range(N):
        kept = []
        q = 0
        while len(kept) < zeta:
            for u in numpy_philox_block((n, q, 0, 0), (seed, TAG_ROWS)):
                r = (int(u) * s) >> 64
                if r not in kept and len(kept) < zeta:
                    kept.append(r)
            q += 1
        rows[n] = kept
        b = int(numpy_philox_block((n, 0, 0, 0), (seed, TAG_SIGNS))[0])
        vals[n] = [(-1 if (b >> t) & 1 else 1) / math.sqrt(zeta) for t in range(zeta)]
    return rows, vals


def test_zeta_rule():
    assert O.default_zeta(2000) == 8          # ceil(ln 2001)
    assert O.default_zeta(1000) == 7
    assert O.default_zeta(1) == 1


@pytest.mark.parametrize("N,s,zeta,seed", [(50, 8, 3, 0), (300, 40, 4, 1), (20, 5, 5, 2)])
def test_sparse_sign_structure_and_restatement(N, s, zeta, seed):
    rows, vals = O.sparse_sign(N, s, zeta, seed)
    for n in range(N):
        assert len(set(rows[n].tolist())) == zeta
    assert rows.min() >= 0 and rows.max() < s
    np.testing.assert_array_equal(np.abs(vals), 1 / math.sqrt(zeta))
    Phi = O.sparse_sign_dense(N, s, zeta, seed)
    np.testing.assert_allclose(np.linalg.norm(Phi, axis=0), 1.0, rtol=1e-15)
    r2, v2 = independent_sparse_sign(N, s, zeta, seed)
    np.testing.assert_array_equal(rows, r2)
    np.testing.assert_array_equal(vals, v2)


def test_sparse_sign_isotropic():
    N, s, zeta = 12, 6, 2
    acc = np.zeros((N, N))
    T = 3000
    for seed in range(T):
        Phi = O.sparse_sign_dense(N, s, zeta, seed)
        acc += Phi.T @ Phi
    acc /= T
    np.testing.assert_allclose(np.diag(acc), 1.0, rtol=1e-12)
    off = acc - np.diag(np.diag(acc))
    # off-diagonal entries are means of T bounded, zero-mean variables
    assert np.abs(off).max() < 5 * math.sqrt(1.0 / T)


@pytest.fixture(scope="module")
def small_krill():
    w = make_c4_krill(n=3000, k=120)
    P = O.krill_build(w.X, w.kernel, w.sigma, w.centers, w.mu, seed=5)
    return w, P


def test_sketch_equals_dense_product(small_krill):
    w, P = small_krill
    Phi = O.sparse_sign_dense(w.N, P.s, P.zeta, 5)
    ref = Phi @ O.kernel_block(w.X, w.kernel, w.sigma, None, w.centers)
    np.testing.assert_allclose(P.Bsk, ref, rtol=1e-11, atol=1e-12)


def test_build_composition(small_krill):
    w, P = small_krill
    ASS = O.kernel_block(w.X, w.kernel, w.sigma, w.centers, w.centers)
    shift = w.N * 2.0 ** -52 * np.trace(ASS)
    np.testing.assert_allclose(P.H - w.lam * ASS, shift * np.eye(w.k), atol=1e-15)
    np.testing.assert_allclose(P.Cu.T @ P.Cu, P.Bsk.T @ P.Bsk + P.H, rtol=1e-12, atol=1e-9)
    assert P.s == 2 * w.k and P.zeta == math.ceil(math.log(w.k + 1))


def test_solution_matches_direct_solve(small_krill):
    w, P = small_krill
    AnS = O.kernel_block(w.X, w.kernel, w.sigma, None, w.centers)
    M = AnS.T @ AnS + P.H
    rhs = AnS.T @ w.Y[0]
    ref = sla.solve(M, rhs, assume_a="pos")
    res = O.krill_solve(w.X, w.kernel, w.sigma, w.centers, P, w.Y, tol=1e-12)
    assert res.status == ["ok"]
    assert res.relres_true[0] < 1e-10
    # relative error within cond(M) x tolerance
    cond = np.linalg.cond(M)
    assert np.linalg.norm(res.alpha[0] - ref) / np.linalg.norm(ref) < max(1e-6, cond * 1e-12)


def test_exact_gram_converges_in_one_step(small_krill):
    w, P = small_krill
    AnS = O.kernel_block(w.X, w.kernel, w.sigma, None, w.centers)
    Pex = O.KrillPreconditioner(P.H, AnS, AnS.T @ AnS + P.H,
                                np.linalg.cholesky(AnS.T @ AnS + P.H).T.copy(),
                                P.lam, w.N, 0)
    res = O.krill_solve(w.X, w.kernel, w.sigma, w.centers, Pex, w.Y, tol=1e-9)
    assert res.iters == [1]


def test_preconditioned_condition_number_soft(small_krill):
    w, P = small_krill
    AnS = O.kernel_block(w.X, w.kernel, w.sigma, None, w.centers)
    M = AnS.T @ AnS + P.H
    ev = sla.eigh(M, P.P, eigvals_only=True)
    kappa = ev.max() / ev.min()
    assert 3 < kappa < 34 * 3
