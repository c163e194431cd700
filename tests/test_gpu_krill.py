"""GPU parity of KRILL (Alg. 2).

The sparse sign embedding is integer work: bit-identical rows and signs.  H
is float64 (rtol 1e-13).  The sketch B uses float32 kernel entries and
float32 partial sums: |B_gpu - B| <= 2e-5 |Phi| A(:,S).  The solve must meet
the tolerance in the float64 residual recomputed by the oracle (within a 2x
margin for the float32 product) and agree with the direct solve of the
restricted equations to cond(M) x tol.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from inputs import make_c4_krill
from gpu_common import rel_err, require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    return require_gpu()


@pytest.mark.parametrize("N,s,zeta,seed", [(1, 4, 2, 0), (1000, 40, 4, 1), (5000, 4000, 8, 3),
                                           (33, 8, 8, 5)])
def test_sparse_sign_bit_exact(K, N, s, zeta, seed):
    rows, vals = K.krr_sparse_sign(N, s, zeta, seed)
    r2, v2 = O.sparse_sign(N, s, zeta, seed)
    np.testing.assert_array_equal(rows, r2)
    np.testing.assert_array_equal(vals, v2)


@pytest.fixture(scope="module")
def small(K):
    w = make_c4_krill(n=4000, k=150)
    ref = O.krill_build(w.X, w.kernel, w.sigma, w.centers, w.mu, seed=11)
    P = K.krill_build(w.X, w.kernel, w.sigma, w.centers, w.mu, seed=11)
    return w, ref, P


def test_build_matches_oracle(K, small):
    w, ref, P = small
    ex = P.export()
    assert ex["s"] == 2 * w.k
    np.testing.assert_allclose(ex["H"], ref.H, rtol=1e-13, atol=1e-15)
    Phi = O.sparse_sign_dense(w.N, ref.s, ref.zeta, 11)
    bound = np.abs(Phi) @ O.kernel_block(w.X, w.kernel, w.sigma, None, w.centers)
    assert np.all(np.abs(ex["Bsk"] - ref.Bsk) <= 2e-5 * bound + 1e-30)
    Pgpu = ex["Bsk"].T @ ex["Bsk"] + ex["H"]
    np.testing.assert_allclose(ex["P"], Pgpu, rtol=1e-12, atol=1e-12 * np.abs(Pgpu).max())
    np.testing.assert_allclose(ex["Cu"].T @ ex["Cu"], ex["P"], rtol=1e-10,
                               atol=1e-12 * np.abs(Pgpu).max())


def test_solve_matches_direct(K, small):
    w, ref, P = small
    beta, info = K.krill_solve(P, w.Y, tol=1e-6)
    assert info["status"] == "KRR_OK"
    AnS = O.kernel_block(w.X, w.kernel, w.sigma, None, w.centers)
    M = AnS.T @ AnS + ref.H
    rhs = AnS.T @ w.Y[0]
    direct = sla.solve(M, rhs, assume_a="pos")
    res = np.linalg.norm(M @ beta[0] - rhs) / np.linalg.norm(rhs)
    assert res <= 2e-6
    assert rel_err(beta[0], direct) <= np.linalg.cond(M) * 4e-6
    assert info["iters"] <= 60          # summed over the refinement steps


def test_multi_rhs_and_device_arrays(K, small):
    w, ref, P = small
    Y = np.vstack([w.Y, 2.0 * w.Y, np.cos(w.X[:, 0])[None, :]])
    beta, info = K.krill_solve(P, to_dev(Y), tol=1e-6)
    beta = beta.cpu().numpy()
    AnS = O.kernel_block(w.X, w.kernel, w.sigma, None, w.centers)
    M = AnS.T @ AnS + ref.H
    for c in range(3):
        rhs = AnS.T @ Y[c]
        assert np.linalg.norm(M @ beta[c] - rhs) / np.linalg.norm(rhs) <= 2e-6


def test_full_size_restricted(K):
    """2,000,000 points, d = 20, 2000 centers, s = 4000, zeta = 8: build and
    solve to 1e-6; the oracle recomputes, in float64, the residual of the
    restricted normal equations of Alg. 2, A(S,:)(A(:,S) beta) + H beta -
    A(S,:) y, over all 2000 center rows (12e9 kernel evaluations), with H =
    lambda A(S,S) + N eps tr(A(S,S)) I from the oracle's own definition."""
    w = make_c4_krill()
    P = K.krill_build(to_dev(w.X), w.kernel, w.sigma, w.centers, w.mu, seed=7)
    beta, info = K.krill_solve(P, to_dev(w.Y), tol=w.tol)
    assert info["status"] == "KRR_OK", info
    assert info["iters"] <= 60
    b = beta.cpu().numpy()
    assert np.all(np.isfinite(b))
    assert math.ceil(math.log(w.k + 1)) == 8
    lam = w.mu * w.N
    ASS = O.kernel_block(w.X, w.kernel, w.sigma, w.centers, w.centers)
    H = lam * ASS + w.N * O.EPS_MACH * np.trace(ASS) * np.eye(w.k)
    u = O.kcols_matvec(w.X, w.kernel, w.sigma, w.centers, b)
    lhs = O.krows_matvec(w.X, w.kernel, w.sigma, w.centers, u) + (H @ b.T).T
    rhs = O.krows_matvec(w.X, w.kernel, w.sigma, w.centers, w.Y)
    res = np.linalg.norm(lhs - rhs, axis=1) / np.linalg.norm(rhs, axis=1)
    assert np.all(res <= 2 * w.tol), res
