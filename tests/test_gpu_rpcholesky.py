"""GPU parity of the pivot sampler and of blocked RPCholesky (Alg. 3).

The sampler is integer work on fixed-point weights: given the same residual
diagonal and seed, the draws must be bit-identical to the oracle's.  The
factor is float64: pivots must be identical, F and the residual diagonal
agree to rounding (atol 1e-10 on entries of size <= 1).
"""
import numpy as np
import pytest

import oracle as O
from inputs import make_c1_plain_fp64, make_c2_mixed
from gpu_common import require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    return require_gpu()


@pytest.mark.parametrize("N", [1, 2, 7, 2048, 2049, 100_000, 500_000, 3_000_000])
def test_sampler_bit_exact(K, N):
    rng = np.random.default_rng(N)
    dres = rng.random(N)
    dres[rng.random(N) < 0.25] = 0.0
    dres[rng.random(N) < 0.01] = -1e-18
    if N > 10:
        dres[rng.integers(0, N, 5)] = 1.0
    for t in (0, 1, 17):
        nd = 100 if N > 1 else 3
        got = K.krr_rpc_sample(dres, 1234, t, nd)
        ref = O.rpc_sample(dres, 1234, t, nd)
        np.testing.assert_array_equal(got, ref)
    fl = O.drop_threshold(N) if N > 100 else 0.3
    np.testing.assert_array_equal(K.krr_rpc_sample(dres, 7, 3, 64, fl),
                                  O.rpc_sample(dres, 7, 3, 64, fl))


def test_sampler_zero_weights(K):
    assert K.krr_rpc_sample(np.zeros(5000), 1, 0, 10).size == 0
    d = np.zeros(5000)
    d[4321] = 1e-9
    assert set(K.krr_rpc_sample(d, 1, 0, 50).tolist()) == {4321}


def test_sampler_device_input(K):
    d = np.random.default_rng(3).random(10_000)
    np.testing.assert_array_equal(K.krr_rpc_sample(to_dev(d), 9, 2, 64), O.rpc_sample(d, 9, 2, 64))


def compare_factor(K, X, kern, sigma, k, B, seed, atol=1e-10):
    ref = O.rpcholesky(X, kern, sigma, k, B, seed)
    f = K.krr_rpcholesky(X, kern, sigma, k, B, seed)
    F, S, D = f.export()
    assert f.rank == ref.rank
    assert f.nblocks == ref.nblocks
    np.testing.assert_array_equal(S, ref.S)
    np.testing.assert_allclose(F, ref.F, atol=atol, rtol=0)
    np.testing.assert_allclose(D, ref.dres, atol=atol, rtol=0)
    f.free()


@pytest.mark.parametrize("kern", [O.GAUSSIAN, O.LAPLACE_L1, O.MATERN52])
def test_small_factor(K, kern):
    rng = np.random.default_rng(kern)
    X = rng.standard_normal((333, 5))
    compare_factor(K, X, kern, 1.2, 57, 8, seed=kern + 1)


def test_plain_workload_factor(K):
    """4096 points, d = 8, Gaussian sigma = 1.5, rank 200, B = 20."""
    w = make_c1_plain_fp64()
    compare_factor(K, w.X, w.kernel, w.sigma, w.k, w.block, seed=0)


def test_full_rank_and_twins(K):
    rng = np.random.default_rng(5)
    X = 3.0 * rng.standard_normal((40, 2))
    compare_factor(K, X, O.GAUSSIAN, 0.5, 40, 1, seed=4, atol=1e-9)
    Xt = np.vstack([X, X[:6]])           # exact twins are dropped
    compare_factor(K, Xt, O.GAUSSIAN, 0.5, 46, 46, seed=0, atol=1e-9)


def test_single_point_and_rank_one(K):
    compare_factor(K, np.zeros((1, 3)), O.GAUSSIAN, 1.0, 1, 1, seed=0)
    compare_factor(K, np.zeros((9, 2)), O.LAPLACE_L1, 1.0, 9, 3, seed=1)


def test_full_size_ill_conditioned(K):
    """100000 points with 5% near-duplicates, rank 1000, B = 100: identical
    pivots and F to rounding."""
    w = make_c2_mixed()
    compare_factor(K, w.X, w.kernel, w.sigma, w.k, w.block, seed=w.seed, atol=1e-8)


def compare_rule(K, X, kern, sigma, k, B, seed, rule, atol=1e-10):
    ref = O.pivoted_cholesky(X, kern, sigma, k, B, seed, rule=rule)
    name = {O.PIVOT_UNIFORM: "uniform", O.PIVOT_GREEDY: "greedy"}[rule]
    f = K.krr_pivoted_cholesky(X, kern, sigma, k, B, seed, rule=name)
    F, S, D = f.export()
    assert f.rank == ref.rank
    assert f.nblocks == ref.nblocks
    np.testing.assert_array_equal(S, ref.S)
    np.testing.assert_allclose(F, ref.F, atol=atol, rtol=0)
    np.testing.assert_allclose(D, ref.dres, atol=atol, rtol=0)
    f.free()


@pytest.mark.parametrize("rule", [O.PIVOT_UNIFORM, O.PIVOT_GREEDY])
@pytest.mark.parametrize("kern,N,k,B", [(O.GAUSSIAN, 333, 57, 0), (O.LAPLACE_L1, 1000, 80, 8),
                                        (O.MATERN52, 2500, 120, 0)])
def test_pivot_rules(K, rule, kern, N, k, B):
    """The comparison pivot rules of Sec. 4 (uniform, greedy one at a time or
    in blocks): identical pivots and blocks, F to rounding."""
    rng = np.random.default_rng(N + kern)
    X = rng.standard_normal((N, 5))
    compare_rule(K, X, kern, 1.2, k, B, seed=kern + 3, rule=rule)


def test_uniform_rule_counts_dropped_pivots(K):
    """Sec. 4's two-block example: two uniform pivots usually land in the
    large block, the second is dropped and the rank stays 1."""
    X = np.zeros((512, 2))
    X[504:] = 60.0
    for seed in range(4):
        compare_rule(K, X, O.GAUSSIAN, 1.0, 2, 1, seed, O.PIVOT_UNIFORM)


def test_greedy_full_size(K):
    """100000 points with 5% near-duplicates, rank 200 greedy one at a time."""
    w = make_c2_mixed()
    compare_rule(K, w.X, w.kernel, w.sigma, 200, 0, 0, O.PIVOT_GREEDY, atol=1e-8)
