"""The allocation-free float64 product, called through the C ABI.

Callers that cannot allocate device memory on their call path (a serving
loop that reserved its memory up front, a plug-in that only receives
framework-owned buffers) use krr_kmatvec_f64_noalloc, whose scratch is a
static device array.  Its output must match the allocating krr_kmatvec
(float64) within the float64 product tolerance, on two calls in a row that
share the array, and the oracle's product within the same tolerance.
Collected last so a stop-at-first-failure run has already run every other
test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_product_matches_allocating_product():
    import torch
    import paper_2304_12465_gb300 as K
    from inputs import make_c1_plain_fp64

    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    lib = K.load()
    w = make_c1_plain_fp64(n=3000)
    rng = np.random.default_rng(42)
    X = torch.from_numpy(w.X).cuda()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (m, kern) in enumerate([(4, 0), (3, 2)]):
        V = torch.from_numpy(rng.standard_normal((m, w.N))).cuda()
        Y = torch.full((m, w.N), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.krr_kmatvec_f64_noalloc(_ptr(X), w.N, w.d, kern, w.sigma, w.lam, _ptr(V), m,
                                         _ptr(Y), stream)
        assert st == 0, lib.krr_last_error().decode()
        ref = K.krr_kmatvec(X, kern, w.sigma, w.lam, V, prec="fp64")
        got, want = Y.cpu().numpy(), ref.cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max(),
                                   err_msg=f"call {call}")
        ora = O.kmatvec(w.X, kern, w.sigma, w.lam, V.cpu().numpy())
        np.testing.assert_allclose(got, ora, rtol=1e-12, atol=1e-12 * np.abs(ora).max(),
                                   err_msg=f"call {call} vs oracle")


def test_noalloc_product_near_the_scratch_limit():
    """m = 16 at N = 20000: the scratch holds 2^21 / (16 N) = 6 column splits,
    fewer than the allocating product would choose, so the split count is
    clamped to what fits; sampled rows against the oracle and all rows
    against the allocating product."""
    import torch
    import paper_2304_12465_gb300 as K

    lib = K.load()
    rng = np.random.default_rng(7)
    N, d, m = 20000, 8, 16
    Xn = rng.standard_normal((N, d))
    Vn = rng.standard_normal((m, N))
    X, V = torch.from_numpy(Xn).cuda(), torch.from_numpy(Vn).cuda()
    Y = torch.full((m, N), float("nan"), dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.krr_kmatvec_f64_noalloc(_ptr(X), N, d, 0, 1.2, 0.3, _ptr(V), m, _ptr(Y), stream)
    assert st == 0, lib.krr_last_error().decode()
    got = Y.cpu().numpy()
    want = K.krr_kmatvec(X, 0, 1.2, 0.3, V, prec="fp64").cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    rows = np.sort(rng.choice(N, 64, replace=False))
    ora = O.kmatvec(Xn, 0, 1.2, 0.3, Vn, rows)
    np.testing.assert_allclose(got[:, rows], ora, rtol=1e-12, atol=1e-12 * np.abs(ora).max())


def test_noalloc_rejects_oversize_and_host_memory():
    import torch
    import paper_2304_12465_gb300 as K

    lib = K.load()
    n = (1 << 21) // 4 + 1            # N x padded(4) just above the scratch
    X = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    V = torch.zeros((4, n), dtype=torch.float64, device="cuda")
    Y = torch.zeros((4, n), dtype=torch.float64, device="cuda")
    st = lib.krr_kmatvec_f64_noalloc(_ptr(X), n, 2, 0, 1.0, 0.1, _ptr(V), 4, _ptr(Y), None)
    assert st == 1 and "scratch" in lib.krr_last_error().decode()
    Xh = np.zeros((8, 2))
    st = lib.krr_kmatvec_f64_noalloc(C.c_void_p(Xh.ctypes.data), 8, 2, 0, 1.0, 0.1, _ptr(V),
                                     1, _ptr(Y), None)
    assert st == 1 and "device pointers" in lib.krr_last_error().decode()
