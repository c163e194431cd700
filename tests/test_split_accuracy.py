"""Accuracy of the two-half fp16 split behind the tensor-core float32 product
(its inner products x_i . x_j of the Gaussian and Matern kernels, Sec. 2.1).

Restated here with numpy's float16 (no code shared with the CUDA path):
h = fp16(x), l = fp16(x - h) represents x to 2^-22 |x|, and the three-term
inner product h_i.h_j + h_i.l_j + l_i.h_j, summed in float32 from
c_i + c_j, gives kernel values whose error stays far inside the float32
product bound the GPU parity tests apply (2e-5 of sum_j |a_ij v_j| per row).
"""
import numpy as np
import pytest

import oracle as O
from inputs import make_c2_mixed

LOG2E = 1.4426950408889634


def split16(v):
    h = v.astype(np.float32).astype(np.float16)
    l = (v - h.astype(np.float64)).astype(np.float32).astype(np.float16)
    return h, l


def test_split_represents_to_2_pow_minus_22():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.standard_normal(20000) * s for s in (1e-3, 0.3, 1.0, 40.0, 9000.0)])
    h, l = split16(v)
    err = np.abs(v - h.astype(np.float64) - l.astype(np.float64))
    # relative 2^-22 for normal halves; subnormal lo parts add at most 2^-25 absolute
    assert np.all(err <= 2.0 ** -22 * np.abs(v) + 2.0 ** -25)


def split_gaussian_matrix(X, sigma):
    """Kernel values by the tensor path's arithmetic: centred, scaled, split
    coordinates; float32 accumulation starting at c_i + c_j, small terms
    first; 2^acc."""
    x = (X - X.mean(axis=0)) * (np.sqrt(LOG2E) / sigma)
    h, l = split16(x)
    hd, ld = h.astype(np.float64), l.astype(np.float64)
    e = hd + ld
    c = (-0.5 * (e * e).sum(axis=1)).astype(np.float32)
    f32 = np.float32
    acc = (c[:, None] + c[None, :]).astype(f32)
    for a, b in ((ld, hd), (hd, ld), (hd, hd)):
        acc = (acc + (a @ b.T).astype(f32)).astype(f32)
    return np.exp2(acc.astype(np.float64))


@pytest.mark.parametrize("sigma", [0.5, 1.5, 4.0])
def test_split_kernel_values_within_float32_bound(sigma):
    w = make_c2_mixed(n=1500)
    X = w.X
    A = O.kernel_block(X, O.GAUSSIAN, sigma)
    As = split_gaussian_matrix(X, sigma)
    # entrywise: far below the float32 product's per-entry budget (measured
    # 1.3e-6 at sigma = 0.5; dropping the two correction terms gives 3.4e-3)
    assert np.abs(As - A).max() <= 3e-6
    # the product bound of the parity tests, with room to spare
    V = np.random.default_rng(1).standard_normal((3, X.shape[0]))
    got = V @ As.T
    ref = V @ A.T
    bound = np.abs(V) @ A.T
    assert np.all(np.abs(got - ref) <= 3e-6 * bound)


def test_near_duplicates_keep_kernel_value_near_one():
    """Near-duplicate rows (1e-6 jitter) have A_ij within 1e-5 of 1; the split
    arithmetic keeps their argument's cancellation error small."""
    w = make_c2_mixed(n=800)
    As = split_gaussian_matrix(w.X, 0.5)
    A = O.kernel_block(w.X, O.GAUSSIAN, 0.5)
    close = A > 1 - 1e-5
    assert close.sum() > w.X.shape[0]          # the diagonal and the duplicates
    assert np.abs(As[close] - A[close]).max() <= 3e-6
