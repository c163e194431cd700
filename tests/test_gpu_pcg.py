"""GPU parity of the Alg. 1 preconditioner and PCG, float64 and mixed paths.

float64 path: the same pivots give the same preconditioner, so the GPU and
oracle iterates track each other: at equal iteration counts alpha matches the
oracle's to relative error 1e-10; at tol 1e-10 the float64 residual meets the
tolerance and alpha matches the dense solve within cond(A + lambda I) x tol.
At the solution the 1e-10 bar holds where it is attainable: a solution whose
true relative residual is rho satisfies |alpha - alpha*| / |alpha*| <=
cond(A + lambda I) rho, so two solutions to tolerance tol differ by at most
2 cond tol; on a well-conditioned shift (cond x tol <= 1e-11, checked in the
test) the GPU and oracle solutions and the dense solve agree to 1e-10.
Mixed path: alpha must match the float64 oracle
to relative error 1e-6 when solved to a residual where alpha is pinned
(cond(A + lambda I) x tol << 1e-6), and at the working tolerance the float64
residual, recomputed by the oracle, must be <= tol.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from inputs import make_c1_plain_fp64, make_c2_mixed
from gpu_common import rel_err, require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    return require_gpu()


@pytest.fixture(scope="module")
def c1(K):
    w = make_c1_plain_fp64()
    ref_f = O.rpcholesky(w.X, w.kernel, w.sigma, w.k, w.block, 0)
    f = K.krr_rpcholesky(w.X, w.kernel, w.sigma, w.k, w.block, 0)
    return w, ref_f, f


def test_precond_apply(K, c1):
    w, ref_f, f = c1
    R = np.random.default_rng(0).standard_normal((3, w.N))
    pre = O.nystrom_preconditioner(ref_f.F, w.lam)
    ref = np.stack([pre.apply(r) for r in R])
    got = K.krr_precond_apply(f, w.mu, R, prec="fp64")
    assert rel_err(got, ref) < 1e-10
    got32 = K.krr_precond_apply(f, w.mu, R, prec="mixed")
    assert rel_err(got32, ref) < 1e-4


def test_fp64_solve_matches_oracle(K, c1):
    w, ref_f, f = c1
    # equal iteration counts: the float64 iterates agree to rounding (CG
    # amplifies rounding differences over many iterations, so compare early)
    ref30 = O.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, ref_f.F, tol=1e-300, maxit=30)
    a30, i30 = K.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, f, tol=1e-300, maxit=30,
                               prec="fp64")
    assert i30["status"] == "KRR_ENOCONV" and i30["iters"] == 30
    assert rel_err(a30, ref30.alpha) < 1e-10
    # to the tolerance: same stopping iteration up to rounding of the
    # recursive residual near the threshold, float64 residual below tol
    ref = O.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, ref_f.F, tol=w.tol)
    alpha, info = K.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, f, tol=w.tol, prec="fp64")
    assert info["status"] == "KRR_OK"
    assert abs(info["iters"] - ref.iters[0]) <= 5
    assert info["rel_residual"] < 2 * w.tol
    rr = O.true_relres(w.X, w.kernel, w.sigma, w.lam, w.Y, alpha)
    assert rr.max() < 2 * w.tol
    # pinned to the dense Cholesky solve: error <= cond(A + lam I) x residual
    A = O.kernel_block(w.X, w.kernel, w.sigma)
    M = A + w.lam * np.eye(w.N)
    dense = sla.cho_solve(sla.cho_factor(M), w.Y[0])
    cond = np.linalg.cond(M)
    assert rel_err(alpha[0], dense) < max(1e-9, 2 * cond * w.tol)
    assert rel_err(alpha[0], ref.alpha[0]) < max(1e-9, 4 * cond * w.tol)


def test_fp64_solve_matches_oracle_at_1e10_when_attainable(K):
    """float64 solve at tol 1e-12 on a shift where cond(A + lambda I) x tol
    <= 1e-11: alpha agrees with the oracle's alpha and with the dense solve to
    relative 1e-10 (the bound 2 cond tol of the module docstring)."""
    w = make_c1_plain_fp64(n=2048)
    mu, tol = 3e-2, 1e-12   # cond(A + lambda I) = 4.4 at this shift
    lam = mu * w.N
    A = O.kernel_block(w.X, w.kernel, w.sigma)
    M = A + lam * np.eye(w.N)
    ev = np.linalg.eigvalsh(M)
    cond = ev[-1] / ev[0]
    assert cond * tol <= 1e-11, cond
    ref_f = O.rpcholesky(w.X, w.kernel, w.sigma, 100, 10, 3)
    f = K.krr_rpcholesky(w.X, w.kernel, w.sigma, 100, 10, 3)
    ref = O.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, mu, ref_f.F, tol=tol)
    alpha, info = K.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, mu, f, tol=tol, prec="fp64")
    f.free()
    assert info["status"] == "KRR_OK"
    rr = O.true_relres(w.X, w.kernel, w.sigma, lam, w.Y, alpha)
    assert rr.max() < 2 * tol
    dense = sla.cho_solve(sla.cho_factor(M), w.Y[0])
    assert rel_err(alpha[0], dense) < 1e-10
    assert rel_err(alpha[0], ref.alpha[0]) < 1e-10


def test_float_float_solve_tracks_fp64(K, c1):
    """float64 PCG with the float-float product (entries within about 2^-46)
    follows the float64-product iterates: equal to 1e-9 after 30 iterations,
    and both reach tol 1e-10 within a few iterations of each other."""
    w, ref_f, f = c1
    a64, _ = K.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, f, tol=1e-300, maxit=30,
                             prec="fp64")
    aff, iff = K.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, f, tol=1e-300, maxit=30,
                               prec="ff")
    assert iff["iters"] == 30
    assert rel_err(aff, a64) < 1e-9
    _, i64 = K.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, f, tol=w.tol, prec="fp64")
    aff, iff = K.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, f, tol=w.tol, prec="ff")
    assert iff["status"] == "KRR_OK" and abs(iff["iters"] - i64["iters"]) <= 3
    rr = O.true_relres(w.X, w.kernel, w.sigma, w.lam, w.Y, aff)
    assert rr.max() < 2 * w.tol


def test_mixed_solve_matches_oracle(K, c1):
    w, ref_f, f = c1
    ref = O.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, ref_f.F, tol=1e-12)
    alpha, info = K.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, f, tol=1e-10, prec="mixed")
    assert info["status"] == "KRR_OK"
    assert rel_err(alpha, ref.alpha) < 1e-6
    alpha6, info6 = K.krr_pcg_solve(w.X, w.kernel, w.sigma, w.Y, w.mu, f, tol=1e-6, prec="mixed")
    assert info6["status"] == "KRR_OK"
    rr = O.true_relres(w.X, w.kernel, w.sigma, w.lam, w.Y, alpha6)
    assert rr.max() <= 1e-6
    assert abs(rr.max() - info6["rel_residual"]) < 1e-9


def test_no_preconditioner_and_zero_rhs(K):
    w = make_c1_plain_fp64(n=600)
    Y = np.vstack([w.Y, np.zeros((1, w.N))])
    alpha, info = K.krr_pcg_solve(w.X, w.kernel, w.sigma, Y, 1e-3, None, tol=1e-10, prec="fp64")
    assert info["status"] == "KRR_OK"
    assert not alpha[1].any()
    A = O.kernel_block(w.X, w.kernel, w.sigma)
    dense = np.linalg.solve(A + 1e-3 * w.N * np.eye(w.N), w.Y[0])
    assert rel_err(alpha[0], dense) < 1e-8


@pytest.mark.parametrize("kern", [O.LAPLACE_L1, O.MATERN52])
def test_other_kernels_mixed(K, kern):
    w = make_c2_mixed(n=6000, m=2, k=300)
    f = K.krr_rpcholesky(w.X, kern, 1.0, w.k, 30, 3)
    alpha, info = K.krr_pcg_solve(w.X, kern, 1.0, w.Y, 1e-6, f, tol=1e-6, prec="mixed")
    assert info["status"] == "KRR_OK"
    rr = O.true_relres(w.X, kern, 1.0, 1e-6 * w.N, w.Y, alpha)
    assert rr.max() <= 1e-6


def test_ill_conditioned_mixed_scaled(K):
    """The near-duplicate workload at 20000 points, 4 right-hand sides."""
    w = make_c2_mixed(n=20_000, k=400)
    f = K.krr_rpcholesky(w.X, w.kernel, w.sigma, w.k, 40, 1)
    alpha, info = K.krr_pcg_solve(to_dev(w.X), w.kernel, w.sigma, to_dev(w.Y), w.mu, f,
                                  tol=w.tol, prec="mixed")
    assert info["status"] == "KRR_OK"
    rr = O.true_relres(w.X, w.kernel, w.sigma, w.lam, w.Y, alpha.cpu().numpy())
    assert rr.max() <= w.tol


def test_full_size_mixed_solve(K):
    """100000 points, d = 16, rank 1000, 4 right-hand sides, tol 1e-6: the
    float64 residual recomputed by the oracle meets the tolerance."""
    w = make_c2_mixed()
    f = K.krr_rpcholesky(to_dev(w.X), w.kernel, w.sigma, w.k, w.block, w.seed)
    alpha, info = K.krr_pcg_solve(to_dev(w.X), w.kernel, w.sigma, to_dev(w.Y), w.mu, f,
                                  tol=w.tol, prec="mixed")
    assert info["status"] == "KRR_OK", info
    rr = O.true_relres(w.X, w.kernel, w.sigma, w.lam, w.Y, alpha.cpu().numpy())
    assert rr.max() <= w.tol * 1.001


def test_batched_settings_solve(K):
    """Four (kernel, sigma) settings x two mu values on mixture data: every
    one of the 8 systems meets the tolerance in the float64 residual the
    oracle recomputes, and matches the single-setting solve."""
    from inputs import make_c3_batched
    w = make_c3_batched(n=4000, k=200)
    settings = [(O.MATERN52, 1.0), (O.MATERN52, 2.0), (O.LAPLACE_L1, 1.0), (O.LAPLACE_L1, 4.0)]
    mus = [1e-4, 1e-6]
    kerns = [k for k, _ in settings]
    sigmas = [s for _, s in settings]
    factors = [K.krr_rpcholesky(w.X, k, s, w.k, 20, seed=q) for q, (k, s) in enumerate(settings)]
    Y = np.repeat(w.Y, len(settings) * len(mus), axis=0)
    alpha, info = K.krr_pcg_solve_batched(w.X, kerns, sigmas, factors, mus, Y, tol=1e-8)
    assert info["status"] == "KRR_OK", info
    for q, (k, sg) in enumerate(settings):
        for c, mu in enumerate(mus):
            col = q * len(mus) + c
            rr = O.true_relres(w.X, k, sg, mu * w.N, Y[col:col + 1], alpha[col:col + 1])
            assert rr.max() <= 1e-8, (q, c, rr)
    one, _ = K.krr_pcg_solve(w.X, kerns[1], sigmas[1], Y[2:3], mus[0], factors[1], tol=1e-8)
    assert rel_err(alpha[2], one[0]) < 1e-5


def smooth_tiny_mu_problem(seed):
    """x ~ N(0, I_4), a wide Gaussian (sigma = 3) and mu = 1e-8: lambda = 3e-5
    is far below the float32 product's rounding (about 1e-7 of sum_j a_ij |v_j|),
    so float32 inner iterations cannot converge."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((3000, 4))
    Y = np.stack([np.sin(X @ rng.standard_normal(4)) for _ in range(2)])
    return X, Y


def test_mixed_solve_escalates_when_float32_stalls(K):
    """The mixed path hands a stalled float32 refinement to the float64-vector,
    float-float continuation and still meets the tolerance (oracle residual)."""
    X, Y = smooth_tiny_mu_problem(5)
    f = K.krr_rpcholesky(X, O.GAUSSIAN, 3.0, 300, seed=1)
    a, info = K.krr_pcg_solve(X, O.GAUSSIAN, 3.0, Y, 1e-8, f, tol=1e-6, maxit=2000,
                              prec="mixed")
    f.free()
    assert info["status"] == "KRR_OK", info
    assert info["escalated"] == 1
    R = Y - O.kmatvec(X, O.GAUSSIAN, 3.0, 1e-8 * 3000, a)
    rel = np.linalg.norm(R, axis=1) / np.linalg.norm(Y, axis=1)
    assert rel.max() <= 1e-6 * 1.001, rel
    assert abs(info["rel_residual"] - rel.max()) <= 1e-9
