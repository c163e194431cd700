"""Pins for the counter-based generator and the pivot sampler of Alg. 3.

Philox4x64-10 is checked against numpy's independent implementation (numpy
increments its counter before each block, so numpy's counter c yields the
block of counter c + 1).  The sampler is checked against an independent
restatement of the fixed-point reading (Python integers, numpy's Philox,
np.searchsorted) and against exact enumerated probabilities.
"""
import numpy as np
import pytest
import scipy.stats as st

import oracle as O

TAG_PIVOTS = 0x5250434850495653


def numpy_philox_block(ctr, key):
    c = list(ctr)
    # numpy adds one to the counter (with carry) before producing a block
    for i in range(4):
        if c[i] == 0:
            c[i] = (1 << 64) - 1
        else:
            c[i] -= 1
            break
    bg = np.random.Philox(counter=np.array(c, dtype=np.uint64),
                          key=np.array(list(key), dtype=np.uint64))
    return bg.random_raw(4).astype(np.uint64)


@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (0, 0)),
    ((0, 0, 0, 0), (0, 0)),
    ((12345, 678, 9, 10), (2**64 - 1, 42)),
    ((2**64 - 1, 2**64 - 1, 2**64 - 1, 2**64 - 1), (2**64 - 1, 2**64 - 1)),
    ((3, 7, 0, 0), (1, TAG_PIVOTS)),
])
def test_philox_matches_numpy(ctr, key):
    np.testing.assert_array_equal(O.philox4x64(ctr, key), numpy_philox_block(ctr, key))


def test_philox_random_counters():
    rng = np.random.default_rng(7)
    for _ in range(200):
        ctr = [int(v) for v in rng.integers(0, 2**63, size=4, dtype=np.int64)]
        key = [int(v) for v in rng.integers(0, 2**63, size=2, dtype=np.int64)]
        np.testing.assert_array_equal(O.philox4x64(ctr, key), numpy_philox_block(ctr, key))


def independent_sample(dres, seed, t, ndraw, dfloor=0.0):
    N = len(dres)
    fbits = 62 - int(np.ceil(np.log2(N))) if N > 1 else 62
    w = [int(np.floor(min(v, 1.0) * 2.0 ** fbits)) if (v > 0 and v > dfloor) else 0
         for v in dres]
    W = np.cumsum(np.array(w, dtype=object))
    tot = int(W[-1])
    if tot == 0:
        return np.zeros(0, dtype=np.int64)
    Wu = np.array([int(v) for v in W], dtype=np.uint64)
    out = []
    for j in range(ndraw):
        u = int(numpy_philox_block((t, j, 0, 0), (seed, TAG_PIVOTS))[0])
        target = (u * tot) >> 64
        out.append(int(np.searchsorted(Wu, np.uint64(target), side="right")))
    return np.array(out, dtype=np.int64)


def test_fixed_point_bits():
    assert O.fixed_point_bits(1) == 62
    assert O.fixed_point_bits(2) == 61
    assert O.fixed_point_bits(4096) == 50
    assert O.fixed_point_bits(4097) == 49
    assert O.fixed_point_bits(100_000) == 62 - 17


@pytest.mark.parametrize("N", [1, 2, 5, 64, 1000, 4097])
def test_sampler_matches_independent_restatement(N):
    rng = np.random.default_rng(N)
    dres = rng.random(N)
    dres[rng.random(N) < 0.3] = 0.0
    dres[0] = -1e-17          # a slightly negative residual counts as zero
    if N > 3:
        dres[3] = 1.0
    for t in range(4):
        got = O.rpc_sample(dres, 99, t, 50)
        ref = independent_sample(dres, 99, t, 50)
        np.testing.assert_array_equal(got, ref)
    floor = float(np.median(dres))
    np.testing.assert_array_equal(O.rpc_sample(dres, 5, 1, 50, floor),
                                  independent_sample(dres, 5, 1, 50, floor))


def test_sampler_all_zero_returns_nothing():
    assert O.rpc_sample(np.zeros(10), 1, 0, 5).size == 0
    assert O.rpc_sample(-np.ones(10), 1, 0, 5).size == 0


def test_sampler_never_draws_zero_weight():
    dres = np.zeros(1000)
    dres[[17, 500, 999]] = [0.2, 1e-9, 0.7]
    draws = np.concatenate([O.rpc_sample(dres, 3, t, 100) for t in range(50)])
    assert set(np.unique(draws)) <= {17, 500, 999}
    # residuals at or below the floor carry no weight
    dres[[3, 4]] = [1e-13, O.drop_threshold(1000)]
    draws = np.concatenate([O.rpc_sample(dres, 3, t, 100, O.drop_threshold(1000))
                            for t in range(50)])
    assert set(np.unique(draws)) <= {17, 500, 999}


@pytest.mark.parametrize("dres", [
    [0.5, 0.25, 0.125, 0.125],
    [1.0, 1.0, 1.0, 1e-3, 0.0, 0.3],
    [0.9, 0.1],
])
def test_sampler_enumerated_probabilities(dres):
    dres = np.array(dres)
    fb = O.fixed_point_bits(len(dres))
    w = np.array([O.fixed_point_weight(v, fb) for v in dres], dtype=np.float64)
    p = w / w.sum()
    draws = np.concatenate([O.rpc_sample(dres, 11, t, 1000) for t in range(400)])
    counts = np.bincount(draws, minlength=len(dres)).astype(float)
    pos = p > 0
    assert counts[~pos].sum() == 0
    chi2 = ((counts[pos] - p[pos] * len(draws)) ** 2 / (p[pos] * len(draws))).sum()
    assert st.chi2.sf(chi2, pos.sum() - 1) > 1e-6
