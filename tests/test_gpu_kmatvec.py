"""GPU parity of the fused product (A + lambda I) V against the oracle.

float64 path: direct differences and float64 exp, compared entrywise with
rtol 1e-12.  float32 path: errors are bounded by the float32 unit roundoff
times the condition of the sum; each entry must satisfy
|Y32 - Y| <= 2e-5 (A|V| + lambda|V|) -- the kernel value carries ~1e-6
relative error from the argument and ex2, the accumulation a few 1e-6.
float-float path (the refinement residual): about 48-bit entries and sums,
|Yff - Y| <= 5e-13 (A|V| + lambda|V|) at these sizes (the oracle's own
sequential float64 sums contribute up to N x 2^-53 of the same scale).
"""
import numpy as np
import pytest

import oracle as O
from inputs import make_c1_plain_fp64, make_c2_mixed
from gpu_common import f32_product_bound, require_gpu, to_dev

pytestmark = pytest.mark.gpu

KERNS = [O.GAUSSIAN, O.LAPLACE_L1, O.MATERN52]


@pytest.fixture(scope="module")
def K():
    return require_gpu()


@pytest.mark.parametrize("kern", KERNS)
@pytest.mark.parametrize("N,d,m", [(1, 1, 1), (65, 3, 1), (700, 8, 4), (1500, 16, 3),
                                   (1029, 20, 16), (513, 32, 2), (300, 5, 9)])
def test_fp64_product(K, kern, N, d, m):
    rng = np.random.default_rng(N * 7 + d + kern)
    X = rng.standard_normal((N, d))
    V = rng.standard_normal((m, N))
    ref = O.kmatvec(X, kern, 1.3, 0.25, V)
    got = K.krr_kmatvec(X, kern, 1.3, 0.25, V, prec="fp64")
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("kern", KERNS)
@pytest.mark.parametrize("N,d,m", [(1, 1, 1), (65, 3, 1), (700, 8, 4), (3000, 16, 4),
                                   (1029, 20, 16), (513, 32, 2), (2000, 12, 8)])
def test_fp32_product(K, kern, N, d, m):
    rng = np.random.default_rng(N * 11 + d + kern)
    X = rng.standard_normal((N, d))
    V = rng.standard_normal((m, N))
    ref = O.kmatvec(X, kern, 1.1, 0.5, V)
    bound = f32_product_bound(X, kern, 1.1, 0.5, V)
    got = K.krr_kmatvec(X, kern, 1.1, 0.5, V, prec="mixed")
    assert np.all(np.abs(got - ref) <= 2e-5 * bound)


@pytest.mark.parametrize("kern", KERNS)
@pytest.mark.parametrize("N,d,m", [(1, 1, 1), (130, 16, 11), (1031, 16, 4), (777, 24, 8),
                                   (2049, 5, 2)])
def test_fp32_product_paths(K, kern, N, d, m):
    """Both float32 product paths (inner products on the tensor cores from
    the two-half split, or every entry on the FMA pipe) meet the float32
    bound; the Gaussian and Matern results differ between the paths (the
    tensor path ran), the Laplace results do not (it has no tensor path)."""
    rng = np.random.default_rng(N * 17 + d + kern)
    X = rng.standard_normal((N, d))
    V = rng.standard_normal((m, N))
    ref = O.kmatvec(X, kern, 0.9, 0.5, V)
    bound = f32_product_bound(X, kern, 0.9, 0.5, V)
    try:
        K.krr_set_product_path("fma")
        fma = K.krr_kmatvec(X, kern, 0.9, 0.5, V, prec="mixed")
    finally:
        K.krr_set_product_path("tensor")
    tc = K.krr_kmatvec(X, kern, 0.9, 0.5, V, prec="mixed")
    assert np.all(np.abs(fma - ref) <= 2e-5 * bound)
    assert np.all(np.abs(tc - ref) <= 2e-5 * bound)
    if kern == O.LAPLACE_L1:
        np.testing.assert_array_equal(tc, fma)
    elif N > 1:
        assert not np.array_equal(tc, fma)


def test_fp32_product_large_coordinates(K):
    """Centred, scaled coordinates beyond the half split's range (|x| / sigma
    ~ 1e5) take the FMA path: the result equals the FMA path bit for bit."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((500, 6)) * 1e3
    V = rng.standard_normal((2, 500))
    try:
        K.krr_set_product_path("fma")
        fma = K.krr_kmatvec(X, O.GAUSSIAN, 0.02, 0.5, V, prec="mixed")
    finally:
        K.krr_set_product_path("tensor")
    tc = K.krr_kmatvec(X, O.GAUSSIAN, 0.02, 0.5, V, prec="mixed")
    np.testing.assert_array_equal(tc, fma)
    with pytest.raises(K.KrrError):
        K.krr_set_product_path(3)


@pytest.mark.parametrize("kern", KERNS)
@pytest.mark.parametrize("N,d,m", [(1, 1, 1), (65, 3, 1), (700, 8, 4), (2500, 16, 4),
                                   (1029, 20, 16), (513, 32, 2), (300, 5, 9)])
def test_float_float_product(K, kern, N, d, m):
    rng = np.random.default_rng(N * 13 + d + kern)
    X = rng.standard_normal((N, d))
    V = rng.standard_normal((m, N))
    ref = O.kmatvec(X, kern, 0.9, 0.3, V)
    bound = f32_product_bound(X, kern, 0.9, 0.3, V)
    got = K.krr_kmatvec(X, kern, 0.9, 0.3, V, prec="ff")
    assert np.all(np.abs(got - ref) <= 5e-13 * bound)


def ff_error_bound(X, kern, sigma, lam, V):
    """Entrywise error model of the float-float product.  Each centred,
    scaled coordinate is held to 2^-48 |x|, so a difference d_k carries
    2^-48 (|x_ik| + |x_jk|) and the exponent (S/2, S or q) carries about
    eps_ij = 2^-46 sum_k (|x_ik| + |x_jk|)(1 + |d_k|) + 2^-44; the row error
    is at most a few times sum_j kappa_ij |v_j| eps_ij, plus the oracle's own
    float64 rounding."""
    scale = {O.GAUSSIAN: 1.0 / sigma, O.LAPLACE_L1: 1.0 / sigma,
             O.MATERN52: np.sqrt(5.0) / sigma}[kern]
    Xs = (X - X.mean(axis=0)) * scale
    A = O.kernel_block(X, kern, sigma)
    ax = np.abs(Xs)
    D = np.abs(Xs[:, None, :] - Xs[None, :, :])
    eps = 2.0 ** -46 * ((ax[:, None, :] + ax[None, :, :]) * (1.0 + D)).sum(axis=2) + 2.0 ** -44
    return 8.0 * ((A * eps) @ np.abs(V).T).T + 5e-14 * f32_product_bound(X, kern, sigma, lam, V)


@pytest.mark.parametrize("kern", KERNS)
@pytest.mark.parametrize("N,d,m", [(20077, 16, 4), (15500, 20, 3), (16500, 8, 1)])
def test_float_float_symmetric_product(K, kern, N, d, m):
    """Square float-float products large enough for the symmetric kernel (each
    off-diagonal pair of point tiles evaluated once for both tiles' rows, the
    column sums reduced per pair): ragged N, 256-point (d <= 16) and
    128-point (d > 16) tiles, rows at tile edges and at random against the
    oracle."""
    rng = np.random.default_rng(N + d + m + kern)
    X = rng.standard_normal((N, d)) * 0.5
    V = rng.standard_normal((m, N))
    got = K.krr_kmatvec(to_dev(X), kern, 0.9, 0.1, to_dev(V), prec="ff").cpu().numpy()
    edges = np.array([0, 1, 127, 128, 255, 256, 511, 512, N // 2, N - 257, N - 256, N - 129,
                      N - 128, N - 1])
    rows = np.unique(np.concatenate([edges, rng.choice(N, 40, replace=False)]))
    ref = O.kmatvec(X, kern, 0.9, 0.1, V, rows)
    bound = f32_product_bound(X, kern, 0.9, 0.1, V, rows)
    assert np.all(np.abs(got[:, rows] - ref) <= 2e-12 * bound)


def test_float_float_near_duplicates_and_far_points(K):
    """Twins at 1e-7 and a far cluster (coordinates ~16 after scaling) whose
    cross entries underflow, against the float-float error model."""
    rng = np.random.default_rng(3)
    X = rng.random((800, 16))
    X[400:] = X[:400] + 1e-7 * rng.standard_normal((400, 16))
    X[:50] += 8.0
    V = rng.standard_normal((2, 800))
    for kern in KERNS:
        ref = O.kmatvec(X, kern, 0.5, 0.01, V)
        got = K.krr_kmatvec(X, kern, 0.5, 0.01, V, prec="ff")
        assert np.all(np.abs(got - ref) <= ff_error_bound(X, kern, 0.5, 0.01, V)), kern
        # standardised-scale rows (all but the far cluster) stay at 5e-13
        bound = f32_product_bound(X, kern, 0.5, 0.01, V)
        assert np.all(np.abs(got - ref)[:, 50:] <= 5e-13 * bound[:, 50:]), kern


def test_device_and_host_pointers_agree(K):
    w = make_c1_plain_fp64(n=777)
    V = np.random.default_rng(0).standard_normal((2, w.N))
    host = K.krr_kmatvec(w.X, w.kernel, w.sigma, w.lam, V, prec="fp64")
    dev = K.krr_kmatvec(to_dev(w.X), w.kernel, w.sigma, w.lam, to_dev(V), prec="fp64")
    np.testing.assert_array_equal(host, dev.cpu().numpy())


def test_deterministic(K):
    w = make_c1_plain_fp64(n=4096)
    V = np.random.default_rng(1).standard_normal((1, w.N))
    a = K.krr_kmatvec(w.X, w.kernel, w.sigma, w.lam, V, prec="mixed")
    b = K.krr_kmatvec(w.X, w.kernel, w.sigma, w.lam, V, prec="mixed")
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "ff"])
def test_full_size_sampled_rows(K, prec):
    """The 100000-point, d = 16 ill-conditioned workload with 4 right-hand
    sides: GPU product on all rows, oracle on 48 sampled rows."""
    w = make_c2_mixed()
    rng = np.random.default_rng(2)
    V = rng.standard_normal((w.m, w.N))
    rows = np.sort(rng.choice(w.N, 48, replace=False))
    got = K.krr_kmatvec(to_dev(w.X), w.kernel, w.sigma, w.lam, to_dev(V), prec=prec)
    got = got.cpu().numpy()[:, rows]
    ref = O.kmatvec(w.X, w.kernel, w.sigma, w.lam, V, rows)
    if prec == "fp64":
        np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    elif prec == "ff":
        bound = f32_product_bound(w.X, w.kernel, w.sigma, w.lam, V, rows)
        assert np.all(np.abs(got - ref) <= 2e-12 * bound)
    else:
        bound = f32_product_bound(w.X, w.kernel, w.sigma, w.lam, V, rows)
        assert np.all(np.abs(got - ref) <= 2e-5 * bound)


@pytest.mark.parametrize("kern", KERNS)
@pytest.mark.parametrize("N,Nt,d,m", [(1, 1, 1, 1), (700, 65, 8, 4), (3000, 1025, 16, 2),
                                      (513, 2000, 20, 16)])
def test_prediction(K, kern, N, Nt, d, m):
    rng = np.random.default_rng(N + Nt + d + kern)
    X = rng.standard_normal((N, d))
    T = rng.standard_normal((Nt, d)) * 1.3
    alpha = rng.standard_normal((m, N))
    ref = O.predict(X, kern, 1.1, alpha, T)
    bound = O.predict(X, kern, 1.1, np.abs(alpha), T)
    got64 = K.krr_predict(X, kern, 1.1, alpha, T, prec="fp64")
    np.testing.assert_allclose(got64, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    got32 = K.krr_predict(to_dev(X), kern, 1.1, to_dev(alpha), to_dev(T), prec="mixed")
    assert np.all(np.abs(got32.cpu().numpy() - ref) <= 2e-5 * bound + 1e-30)


@pytest.mark.parametrize("N,d,ms", [(1, 2, 1), (777, 8, 2), (3001, 5, 2), (1500, 16, 1)])
def test_batched_settings_product(K, N, d, ms):
    """Eight (kernel, sigma) settings sharing the tile generation, each with
    its own shifts; every block equals the single-setting oracle product."""
    rng = np.random.default_rng(N + d)
    means = 3.0 * rng.standard_normal((4, d))
    X = means[rng.integers(0, 4, N)] + 0.5 * rng.standard_normal((N, d))
    kerns = [O.MATERN52] * 4 + [O.LAPLACE_L1] * 3 + [O.GAUSSIAN]
    sigmas = [0.5, 1.0, 2.0, 4.0, 0.5, 1.0, 2.0, 1.5]
    S = len(kerns)
    lams = rng.uniform(1e-3, 1.0, S * ms)
    V = rng.standard_normal((S * ms, N))
    got = K.krr_kmatvec_batched(X, kerns, sigmas, lams, V)
    for q in range(S):
        for c in range(ms):
            col = q * ms + c
            ref = O.kmatvec(X, kerns[q], sigmas[q], lams[col], V[col])
            bound = O.kmatvec(X, kerns[q], sigmas[q], lams[col], np.abs(V[col]))
            assert np.all(np.abs(got[col] - ref[0]) <= 2e-5 * bound[0]), (q, c)


def test_autotuned_product(K):
    """With autotuning on, the first product of a shape on the FMA path times
    the candidate column tiles and keeps one; the product still meets the
    float32 bound, repeats bit for bit, and the choice is reported.  (The
    tcgen05 path's variant tuning is tested in test_gpu_tc5.py.)"""
    rng = np.random.default_rng(21)
    X = rng.standard_normal((20011, 8))
    V = rng.standard_normal((3, 20011))
    ref = O.kmatvec(X, O.GAUSSIAN, 1.1, 0.5, V, np.arange(0, 20011, 97))
    bound = f32_product_bound(X, O.GAUSSIAN, 1.1, 0.5, V, np.arange(0, 20011, 97))
    K.krr_set_product_path("fma")
    assert K.krr_autotune_choice(O.GAUSSIAN, 8, 3, 20011) == 0
    K.krr_set_autotune(True)
    try:
        a = K.krr_kmatvec(X, O.GAUSSIAN, 1.1, 0.5, V, prec="mixed")
        b = K.krr_kmatvec(X, O.GAUSSIAN, 1.1, 0.5, V, prec="mixed")
        splits = K.krr_autotune_choice(O.GAUSSIAN, 8, 3, 20011)
    finally:
        K.krr_set_autotune(False)
        K.krr_set_product_path("tensor")
    assert 1 <= splits <= (20011 + 63) // 64
    np.testing.assert_array_equal(a, b)
    assert np.all(np.abs(a[:, ::97] - ref) <= 2e-5 * bound)
