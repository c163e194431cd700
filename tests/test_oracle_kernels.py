"""Pins for the oracle's kernel functions and matrix-free product.

The three kernels are checked against independent library routines (the
normal density, the modified Bessel form of the Matern family), against
special values that a wrong factor would break, and against positive
semi-definiteness, which a wrong sign would break.
"""
import math

import numpy as np
import pytest
import scipy.special as sps
import scipy.stats as st

import oracle as O
from inputs import make_c1_plain_fp64


def matern_bessel(r, ell, nu):
    """General Matern correlation 2^{1-nu}/Gamma(nu) z^nu K_nu(z),
    z = sqrt(2 nu) r / ell (Rasmussen & Williams 2006, eq. 4.14)."""
    z = math.sqrt(2 * nu) * r / ell
    if z == 0:
        return 1.0
    return 2 ** (1 - nu) / sps.gamma(nu) * z ** nu * sps.kv(nu, z)


@pytest.mark.parametrize("kern", [O.GAUSSIAN, O.LAPLACE_L1, O.MATERN52])
def test_unit_diagonal(kern):
    x = np.array([0.3, -1.2, 2.0, 0.1])
    assert O.kappa(x, x, kern, 0.7) == 1.0


def test_gaussian_matches_normal_density():
    rng = np.random.default_rng(0)
    for _ in range(50):
        d = int(rng.integers(1, 9))
        sigma = float(rng.uniform(0.3, 3))
        x, y = rng.standard_normal(d), rng.standard_normal(d)
        # a product over coordinates of scaled 1-d normal densities
        ref = np.prod(st.norm.pdf(x - y, scale=sigma) * sigma * math.sqrt(2 * math.pi))
        assert O.kappa(x, y, O.GAUSSIAN, sigma) == pytest.approx(ref, rel=1e-13)


def test_laplace_is_l1_product_of_matern_half():
    rng = np.random.default_rng(1)
    for _ in range(50):
        d = int(rng.integers(1, 9))
        sigma = float(rng.uniform(0.3, 3))
        x, y = rng.standard_normal(d), rng.standard_normal(d)
        ref = np.prod([matern_bessel(abs(a - b), sigma, 0.5) for a, b in zip(x, y)])
        assert O.kappa(x, y, O.LAPLACE_L1, sigma) == pytest.approx(ref, rel=1e-12)
    # l1, not l2: the two distances differ for a diagonal step
    x, y = np.zeros(2), np.ones(2)
    assert O.kappa(x, y, O.LAPLACE_L1, 1.0) == pytest.approx(math.exp(-2.0), rel=1e-15)


def test_matern52_matches_bessel_form():
    rng = np.random.default_rng(2)
    for _ in range(50):
        d = int(rng.integers(1, 9))
        sigma = float(rng.uniform(0.3, 3))
        x, y = rng.standard_normal(d), rng.standard_normal(d)
        r = float(np.linalg.norm(x - y))
        ref = matern_bessel(r, sigma, 2.5)
        assert O.kappa(x, y, O.MATERN52, sigma) == pytest.approx(ref, rel=1e-11)


def test_special_values():
    sigma = 1.7
    x = np.zeros(3)
    e = np.array([1.0, 0.0, 0.0])
    # Gaussian at distance sigma: exp(-1/2)
    assert O.kappa(x, sigma * e, O.GAUSSIAN, sigma) == pytest.approx(math.exp(-0.5), rel=1e-15)
    # Laplace at l1 distance sigma: exp(-1)
    assert O.kappa(x, sigma * e, O.LAPLACE_L1, sigma) == pytest.approx(math.exp(-1), rel=1e-15)
    # Matern-5/2 at r = sigma / sqrt(5): (1 + 1 + 1/3) exp(-1)
    assert O.kappa(x, sigma / math.sqrt(5) * e, O.MATERN52, sigma) == \
        pytest.approx(7.0 / 3.0 * math.exp(-1), rel=1e-14)


@pytest.mark.parametrize("kern", [O.GAUSSIAN, O.LAPLACE_L1, O.MATERN52])
def test_kernel_matrix_psd_symmetric(kern):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((120, 5))
    A = O.kernel_block(X, kern, 1.3)
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > -1e-12


def test_kernel_block_subsets():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((50, 3))
    A = O.kernel_block(X, O.GAUSSIAN, 0.9)
    rows = np.array([3, 7, 49, 0])
    cols = np.array([10, 2])
    assert np.array_equal(O.kernel_block(X, O.GAUSSIAN, 0.9, rows, cols), A[np.ix_(rows, cols)])


@pytest.mark.parametrize("kern", [O.GAUSSIAN, O.LAPLACE_L1, O.MATERN52])
def test_kmatvec_equals_dense_product(kern):
    w = make_c1_plain_fp64(n=300)
    rng = np.random.default_rng(5)
    V = rng.standard_normal((3, w.N))
    lam = 0.37
    A = O.kernel_block(w.X, kern, w.sigma)
    ref = (A @ V.T + lam * V.T).T
    got = O.kmatvec(w.X, kern, w.sigma, lam, V)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    rows = np.array([299, 0, 17])
    np.testing.assert_array_equal(O.kmatvec(w.X, kern, w.sigma, lam, V, rows), got[:, rows])


def test_kcols_krows_products():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((200, 4))
    S = np.array([5, 9, 100, 150, 199])
    A = O.kernel_block(X, O.GAUSSIAN, 1.1)
    beta = rng.standard_normal((2, 5))
    u = rng.standard_normal((2, 200))
    np.testing.assert_allclose(O.kcols_matvec(X, O.GAUSSIAN, 1.1, S, beta),
                               (A[:, S] @ beta.T).T, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(O.krows_matvec(X, O.GAUSSIAN, 1.1, S, u),
                               (A[S, :] @ u.T).T, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("kern", [O.GAUSSIAN, O.LAPLACE_L1, O.MATERN52])
def test_predict_equals_block_of_stacked_matrix(kern):
    """Prediction = the (test, train) block of the kernel matrix of the
    stacked point set, applied to alpha."""
    rng = np.random.default_rng(7)
    X = rng.standard_normal((90, 4))
    T = rng.standard_normal((25, 4))
    alpha = rng.standard_normal((2, 90))
    Z = np.vstack([X, T])
    Akt = O.kernel_block(Z, kern, 1.2, np.arange(90, 115), np.arange(90))
    np.testing.assert_allclose(O.predict(X, kern, 1.2, alpha, T), (Akt @ alpha.T).T,
                               rtol=1e-12, atol=1e-13)
