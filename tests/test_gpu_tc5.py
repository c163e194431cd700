"""GPU parity of the tcgen05 fused product (the default float32 product of
the Gaussian and Matern kernels) against the oracle.

The product forms D = x_i . x_j + c_i + c_j with fp16 two-half splits on the
tensor cores (Sec. 2.1: both kernels are functions of |x_i - x_j|^2 =
-2 (x_i . x_j + c_i + c_j) after centring and scaling), kernel values and the
sums over V in float32, so every entry meets the float32 product bound of the
other float32 paths, |Y - Y_oracle| <= 2e-5 (A|V| + lambda|V|).  The cases
cover each split layout (c-part in a spare position of the last coordinate
block for d mod 16 = 1..10, in a block of its own otherwise; one or two
coordinate blocks), ragged sizes around the 128-column and 256-row tiles,
grids whose CTAs span several row blocks, every epilogue variant, and
right-hand-side counts that take one or two launches.
"""
import numpy as np
import pytest

import oracle as O
from gpu_common import f32_product_bound, require_gpu, to_dev

pytestmark = pytest.mark.gpu

TC_KERNS = [O.GAUSSIAN, O.MATERN52]


@pytest.fixture(scope="module")
def K():
    k = require_gpu()
    k.krr_set_product_path("tensor")
    yield k
    k.krr_set_product_variant(0)


def _case(N, d, m, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, d)) * scale, rng.standard_normal((m, N))


@pytest.mark.parametrize("kern", TC_KERNS)
@pytest.mark.parametrize("N,d,m", [(1, 1, 1), (127, 5, 2), (129, 10, 3), (255, 11, 4),
                                   (257, 16, 4), (383, 17, 8), (1000, 26, 5), (1031, 27, 1),
                                   (2049, 32, 11), (3000, 16, 16), (4099, 3, 7)])
def test_tcgen05_product_layouts(K, kern, N, d, m):
    X, V = _case(N, d, m, N * 3 + d + m + kern)
    ref = O.kmatvec(X, kern, 1.1, 0.5, V)
    bound = f32_product_bound(X, kern, 1.1, 0.5, V)
    got = K.krr_kmatvec(X, kern, 1.1, 0.5, V, prec="mixed")
    assert np.all(np.abs(got - ref) <= 2e-5 * bound)


@pytest.mark.parametrize("variant", list(range(1, 12)))
@pytest.mark.parametrize("kern", TC_KERNS)
def test_tcgen05_product_variants(K, kern, variant):
    """Every epilogue variant meets the bound; variants differ from each
    other only at the rounding level (the order of the column-group sums, or
    for 8..11 the tensor-core sums of split kernel values and right-hand
    sides)."""
    X, V = _case(2500, 16, 4, 11 + kern)
    ref = O.kmatvec(X, kern, 0.8, 0.3, V)
    bound = f32_product_bound(X, kern, 0.8, 0.3, V)
    try:
        K.krr_set_product_variant(variant)
        got = K.krr_kmatvec(X, kern, 0.8, 0.3, V, prec="mixed")
    finally:
        K.krr_set_product_variant(0)
    assert np.all(np.abs(got - ref) <= 2e-5 * bound)
    base = K.krr_kmatvec(X, kern, 0.8, 0.3, V, prec="mixed")
    assert np.all(np.abs(got - base) <= 1e-5 * bound)


@pytest.mark.parametrize("variant", [8, 9, 10])
@pytest.mark.parametrize("kern", TC_KERNS)
@pytest.mark.parametrize("N,d,m", [(1, 1, 1), (127, 5, 2), (257, 16, 4), (383, 17, 8),
                                   (1031, 27, 1), (2049, 32, 11), (4099, 3, 7)])
def test_tcgen05_tensor_sums_layouts(K, kern, variant, N, d, m):
    """The tensor-core sums over V (variants 8..11) on every split layout,
    one or two launches, right-hand-side counts that fill one B fragment
    (m <= 4: v_hi and v_lo slots side by side) or two (m = 5..8), and ragged
    tile edges (zero right-hand sides beyond N)."""
    X, V = _case(N, d, m, N * 5 + d + m + kern + variant)
    ref = O.kmatvec(X, kern, 1.1, 0.5, V)
    bound = f32_product_bound(X, kern, 1.1, 0.5, V)
    try:
        K.krr_set_product_variant(variant)
        got = K.krr_kmatvec(X, kern, 1.1, 0.5, V, prec="mixed")
    finally:
        K.krr_set_product_variant(0)
    assert np.all(np.abs(got - ref) <= 2e-5 * bound)


@pytest.mark.parametrize("variant", [3, 8])
def test_tcgen05_product_column_scales(K, variant):
    """Right-hand sides of very different magnitudes, one of them zero: the
    tensor-core sums scale each column by its own power of two (the FMA sums
    need none); both meet the componentwise bound."""
    X, V = _case(3001, 16, 5, 77)
    V[0] *= 1e-30
    V[1] *= 1e30
    V[2] = 0.0
    V[4] *= 3e-3
    ref = O.kmatvec(X, O.GAUSSIAN, 0.9, 0.2, V)
    bound = f32_product_bound(X, O.GAUSSIAN, 0.9, 0.2, V)
    try:
        K.krr_set_product_variant(variant)
        got = K.krr_kmatvec(X, O.GAUSSIAN, 0.9, 0.2, V, prec="mixed")
    finally:
        K.krr_set_product_variant(0)
    assert np.all(np.abs(got - ref) <= 2e-5 * bound)
    assert np.all(got[2] == 0.0)


def test_tcgen05_product_is_deterministic(K):
    """Partial sums are reduced in a fixed order: the same call twice gives
    the same bits."""
    X, V = _case(5000, 16, 4, 5)
    a = K.krr_kmatvec(X, O.GAUSSIAN, 0.7, 0.1, V, prec="mixed")
    b = K.krr_kmatvec(X, O.GAUSSIAN, 0.7, 0.1, V, prec="mixed")
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("N", [20000, 39041])
def test_tcgen05_product_multi_segment(K, N):
    """Grids where each CTA's range of (row block, column tile) pairs crosses
    row-block boundaries, so row blocks are summed from several CTAs' segment
    partials; sampled rows against the oracle, including the first and last
    rows of row blocks."""
    X, V = _case(N, 16, 4, N, scale=0.5)
    got = K.krr_kmatvec(to_dev(X), O.GAUSSIAN, 0.6, 0.2, to_dev(V), prec="mixed").cpu().numpy()
    rng = np.random.default_rng(N)
    edges = np.array([0, 255, 256, 511, 512, N // 2, N - 257, N - 256, N - 1])
    rows = np.unique(np.concatenate([edges, rng.choice(N, 40, replace=False)]))
    ref = O.kmatvec(X, O.GAUSSIAN, 0.6, 0.2, V, rows)
    bound = f32_product_bound(X, O.GAUSSIAN, 0.6, 0.2, V, rows)
    assert np.all(np.abs(got[:, rows] - ref) <= 2e-5 * bound)


def test_tcgen05_near_duplicates(K):
    """The ill-conditioned regime (twins at 1e-6 after scaling): the c_i + c_j
    pieces and the split keep D accurate where |x_i - x_j| is tiny."""
    rng = np.random.default_rng(9)
    X = rng.random((3000, 16))
    X[1500:] = X[:1500] + 1e-6 * rng.standard_normal((1500, 16))
    V = rng.standard_normal((4, 3000))
    for kern in TC_KERNS:
        ref = O.kmatvec(X, kern, 0.5, 1e-3, V)
        bound = f32_product_bound(X, kern, 0.5, 1e-3, V)
        got = K.krr_kmatvec(X, kern, 0.5, 1e-3, V, prec="mixed")
        assert np.all(np.abs(got - ref) <= 2e-5 * bound), kern


def test_tcgen05_autotuner_report(K):
    """With autotuning on, the first product of a shape times every valid
    variant; the report gives the choice and positive times for the timed
    ones (variants 2, 4-7, 10 and 11 serve m <= 4 only)."""
    X, V = _case(6001, 12, 8, 21)
    try:
        K.krr_set_autotune(True)
        got = K.krr_kmatvec(X, O.GAUSSIAN, 0.9, 0.2, V, prec="mixed")
    finally:
        K.krr_set_autotune(False)
    v, ms = K.krr_autotune_variant(O.GAUSSIAN, 12, 8, 6001)
    timed = {1, 3, 8, 9}
    assert v in timed
    assert all((ms[v - 1] > 0) == (v in timed) for v in range(1, 12))
    ref = O.kmatvec(X, O.GAUSSIAN, 0.9, 0.2, V)
    assert np.all(np.abs(got - ref) <= 2e-5 * f32_product_bound(X, O.GAUSSIAN, 0.9, 0.2, V))


def test_bounded_wait_gives_up_and_reports(K):
    """The product's bounded mbarrier wait, on a barrier that nothing
    completes, gives up after its budget (about half a millisecond here),
    raises the device fault flag, and the host reads KRR_ETIMEOUT; the flag is
    cleared and the context stays usable: the next product is correct."""
    assert K.krr_check_bounded_wait(1_000_000) == "KRR_ETIMEOUT"
    assert K.krr_check_bounded_wait(0) == "KRR_ETIMEOUT"
    X, V = _case(700, 16, 4, 77)
    ref = O.kmatvec(X, O.GAUSSIAN, 1.1, 0.5, V)
    bound = f32_product_bound(X, O.GAUSSIAN, 1.1, 0.5, V)
    got = K.krr_kmatvec(X, O.GAUSSIAN, 1.1, 0.5, V, prec="mixed")
    assert np.all(np.abs(got - ref) <= 2e-5 * bound)
