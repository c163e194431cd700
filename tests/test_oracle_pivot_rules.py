"""Pins for the two pivot rules the paper compares RPCholesky with (Sec. 4):
greedy selection (largest residual diagonal entry) and uniform sampling (a
uniformly random set of columns).

Greedy one pivot at a time is Cholesky with complete (diagonal) pivoting, so
its pivot order is LAPACK's dpstrf order.  The uniform pivots are restated
with numpy's independent Philox and checked for uniformity; the paper's
two-block example shows the failure mode it describes for uniform sampling.
"""
import numpy as np
import pytest
import scipy.linalg.lapack as lapack
import scipy.stats as st

import oracle as O
from test_oracle_sampler import TAG_PIVOTS, numpy_philox_block


def test_greedy_is_complete_pivoting_cholesky():
    """Greedy pivots (B = 1) = the pivot order of LAPACK dpstrf, which picks
    the largest diagonal entry of the Schur complement at every step (first
    occurrence on ties, like the greedy rule)."""
    rng = np.random.default_rng(0)
    for kern, sigma in [(O.GAUSSIAN, 1.3), (O.LAPLACE_L1, 2.0), (O.MATERN52, 1.0)]:
        X = rng.standard_normal((150, 3))
        A = O.kernel_block(X, kern, sigma)
        _, piv, _, info = lapack.dpstrf(A, tol=1e-13)
        assert info >= 0
        r = O.pivoted_cholesky(X, kern, sigma, 40, rule=O.PIVOT_GREEDY)
        assert r.rank == 40 and r.nblocks == 40
        np.testing.assert_array_equal(r.S, piv[:40] - 1)


def test_greedy_pick_order():
    rng = np.random.default_rng(1)
    d = rng.random(50)
    d[[3, 7]] = d.max()          # a tie: the smaller index comes first
    d[10] = -1.0                 # never eligible
    d[11] = 1e-20                # below the floor
    got = O.greedy_pick(d, 6, dfloor=1e-15)
    eligible = [i for i in range(50) if d[i] > 1e-15]
    ref = sorted(eligible, key=lambda i: (-d[i], i))[:6]
    np.testing.assert_array_equal(got, ref)
    assert O.greedy_pick(np.zeros(5), 3).size == 0


def independent_uniform_pivots(N, k, seed):
    seen, out, q = set(), [], 0
    while len(out) < min(k, N):
        u = int(numpy_philox_block((q, 0, 1, 0), (seed, TAG_PIVOTS))[0])
        i = (u * N) >> 64
        q += 1
        if i not in seen:
            seen.add(i)
            out.append(i)
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("N,k,seed", [(10, 10, 1), (1000, 5, 2), (97, 30, 2**63 + 5)])
def test_uniform_pivots_restated(N, k, seed):
    np.testing.assert_array_equal(O.uniform_pivots(N, k, seed),
                                  independent_uniform_pivots(N, k, seed))


def test_uniform_pivots_are_uniform_subsets():
    """Every index is in the k-subset with probability k/N (chi-squared over
    seeds), and each subset has k distinct indices."""
    N, k, trials = 12, 3, 20000
    counts = np.zeros(N)
    for seed in range(trials):
        S = O.uniform_pivots(N, k, seed)
        assert len(set(S.tolist())) == k
        counts[S] += 1
    expected = np.full(N, trials * k / N)
    _, p = st.chisquare(counts, expected)
    assert p > 1e-4


def two_clusters(N):
    """Points whose Gaussian kernel matrix is the Sec. 4 example for uniform
    sampling: a block of ones of size N - N^(1/3), a block of ones of size
    N^(1/3), and zeros between (identical points, clusters 60 apart)."""
    small = round(N ** (1 / 3))
    X = np.zeros((N, 2))
    X[N - small:] = 60.0
    return X, small


def test_uniform_sampling_failure_example():
    """Rank 2 is exact for RPCholesky with two pivots, for every seed; two
    uniform pivots usually both land in the large block, so the factor has
    rank 1 and misses the small block (residual trace N^(1/3))."""
    N = 512
    X, small = two_clusters(N)
    misses = 0
    for seed in range(10):
        rp = O.pivoted_cholesky(X, O.GAUSSIAN, 1.0, 2, B=1, seed=seed)
        assert rp.rank == 2 and rp.trace_hist[-1] == pytest.approx(0.0, abs=1e-9)
        un = O.pivoted_cholesky(X, O.GAUSSIAN, 1.0, 2, B=1, seed=seed, rule=O.PIVOT_UNIFORM)
        assert un.nblocks == 2
        if un.rank == 1:
            misses += 1
            assert un.trace_hist[-1] == pytest.approx(small, rel=1e-12)
    assert misses >= 8     # P(both in the large block) = (504/512)(503/511) ~ 0.97


@pytest.mark.parametrize("rule", [O.PIVOT_UNIFORM, O.PIVOT_GREEDY])
def test_column_nystrom_identity(rule):
    """For any pivot rule the factor is the column Nystrom approximation of
    its kept pivots, A - FF^T is PSD and its diagonal is the residual."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((120, 4))
    r = O.pivoted_cholesky(X, O.MATERN52, 1.4, 25, seed=9, rule=rule)
    A = O.kernel_block(X, O.MATERN52, 1.4)
    S = r.S
    FF = r.F.T @ r.F
    ref = A[:, S] @ np.linalg.solve(A[np.ix_(S, S)], A[S, :])
    np.testing.assert_allclose(FF, ref, atol=1e-9)
    assert np.linalg.eigvalsh(A - FF).min() > -1e-9
    np.testing.assert_allclose(np.diag(A - FF), r.dres, atol=1e-10)
    assert np.all(np.diff(r.trace_hist) <= 1e-12)


def test_rpcholesky_is_rule_zero():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((90, 3))
    a = O.rpcholesky(X, O.GAUSSIAN, 1.0, 20, seed=5)
    b = O.pivoted_cholesky(X, O.GAUSSIAN, 1.0, 20, seed=5, rule=O.PIVOT_RPCHOLESKY)
    np.testing.assert_array_equal(a.S, b.S)
    np.testing.assert_array_equal(a.F, b.F)
