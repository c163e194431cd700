"""CPU checks of the C ABI boundary: the library builds and loads, exports every
function include/krr.h declares, the Python binding covers them, and argument
validation answers KRR_EINVAL before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "krr.h")


def declared_functions():
    text = open(HEADER).read()
    return re.findall(r"KRR_API\s+(?:krr_status|void|const char \*|uint64_t|double)\s*(\w+)\s*\(", text)


@pytest.fixture(scope="module")
def lib():
    import paper_2304_12465_gb300 as K
    return K.load()


def test_header_declares_the_calls():
    names = declared_functions()
    for must in ("krr_rpcholesky", "krr_pcg_solve", "krill_build", "krill_solve",
                 "krr_kmatvec", "krr_rpc_sample", "krr_sparse_sign", "krr_precond_apply"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    import paper_2304_12465_gb300 as K
    assert set(declared_functions()) == set(K.SIGNATURES)


def test_only_abi_symbols_are_exported():
    import subprocess
    import paper_2304_12465_gb300 as K
    K.load()
    out = subprocess.run(["nm", "-D", "--defined-only", K.library_path()], capture_output=True,
                         text=True).stdout
    text_syms = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(declared_functions()) <= text_syms
    assert not [s for s in text_syms if s.startswith("_ZN3krr")]


def test_version(lib):
    assert b"sm_103a" in lib.krr_version()


def _einval(status, lib, fragment):
    assert status == 1
    assert fragment in lib.krr_last_error().decode()


def test_argument_validation_before_any_launch(lib):
    X = np.zeros((4, 2))
    V = np.zeros((1, 4))
    Y = np.zeros((1, 4))
    p = lambda a: C.c_void_p(a.ctypes.data)
    _einval(lib.krr_kmatvec(p(X), 0, 2, 0, 1.0, 0.1, p(V), 1, p(Y), 0, None), lib, "N must")
    _einval(lib.krr_kmatvec(p(X), 4, 0, 0, 1.0, 0.1, p(V), 1, p(Y), 0, None), lib, "d must")
    _einval(lib.krr_kmatvec(p(X), 4, 33, 0, 1.0, 0.1, p(V), 1, p(Y), 0, None), lib, "d must")
    _einval(lib.krr_kmatvec(p(X), 4, 2, 7, 1.0, 0.1, p(V), 1, p(Y), 0, None), lib, "kernel")
    _einval(lib.krr_kmatvec(p(X), 4, 2, 0, -1.0, 0.1, p(V), 1, p(Y), 0, None), lib, "sigma")
    _einval(lib.krr_kmatvec(p(X), 4, 2, 0, float("nan"), 0.1, p(V), 1, p(Y), 0, None), lib,
            "sigma")
    _einval(lib.krr_kmatvec(p(X), 4, 2, 0, 1.0, 0.1, p(V), 17, p(Y), 0, None), lib, "m must")
    _einval(lib.krr_kmatvec(p(X), 4, 2, 0, 1.0, 0.1, p(V), 1, p(Y), 9, None), lib, "precision")
    h = C.c_void_p()
    _einval(lib.krr_rpcholesky(p(X), 4, 2, 0, 1.0, 5, 0, 0, None, C.byref(h)), lib, "k must")
    _einval(lib.krr_rpcholesky(p(X), 4, 2, 0, 1.0, 2, 129, 0, None, C.byref(h)), lib, "block")
    _einval(lib.krr_pivoted_cholesky(p(X), 4, 2, 0, 1.0, 2, 0, 0, 3, None, C.byref(h)), lib,
            "pivot rule")
    assert not h.value
    info = None
    _einval(lib.krr_pcg_solve(p(X), 4, 2, 0, 1.0, p(Y), 1, 0.0, None, 1e-6, 0, 0, p(Y), None,
                              info), lib, "mu")
    _einval(lib.krr_pcg_solve(p(X), 4, 2, 0, 1.0, p(Y), 1, 1e-3, None, 1.5, 0, 0, p(Y), None,
                              info), lib, "tol")
    rows = np.zeros((4, 2), dtype=np.int32)
    _einval(lib.krr_sparse_sign(4, 3, 4, 0, p(rows), p(V), None), lib, "zeta")
    _einval(lib.krr_sparse_sign(4, 8, 65, 0, p(rows), p(V), None), lib, "zeta")
    _einval(lib.krr_rpc_sample(p(V), 4, 0.0, 0, 0, 0, p(rows), C.byref(C.c_int()), None), lib,
            "ndraw")


def test_product_path_selection(lib):
    """krr_set_product_path takes the three documented paths, and
    krr_set_product_variant the variants 0..11 (host state only); anything
    else is refused."""
    _einval(lib.krr_set_product_path(3), lib, "product path")
    _einval(lib.krr_set_product_path(-1), lib, "product path")
    assert lib.krr_set_product_path(2) == 0
    assert lib.krr_set_product_path(1) == 0
    assert lib.krr_set_product_path(0) == 0
    _einval(lib.krr_set_product_variant(12), lib, "variant")
    _einval(lib.krr_set_product_variant(-1), lib, "variant")
    for v in range(12):
        assert lib.krr_set_product_variant(v) == 0
    assert lib.krr_set_product_variant(0) == 0


def test_autotune_variant_report_untuned(lib):
    """Before any product has run, no shape is tuned: variant 0, zero times."""
    v = C.c_int(-1)
    ms = (C.c_float * 11)(*([1.0] * 11))
    assert lib.krr_autotune_variant(0, 16, 4, 100000, C.byref(v), ms) == 0
    assert v.value == 0 and list(ms) == [0.0] * 11
    _einval(lib.krr_autotune_variant(0, 33, 4, 100, C.byref(v), ms), lib, "shape")


def test_server_footprint_is_host_only_and_monotone(lib):
    """The admission estimate needs no device and grows with every size."""
    def fp(N, d, m, k):
        b = C.c_double()
        assert lib.krr_server_footprint(N, d, m, k, C.byref(b)) == 0
        return b.value
    base = fp(20000, 8, 4, 1000)
    assert base > 20000 * 1000 * 12          # at least the float64 + float32 factor
    assert fp(40000, 8, 4, 1000) > base
    assert fp(20000, 16, 4, 1000) > base   # same float-float tile height as d = 8
    assert fp(20000, 8, 16, 1000) > base
    assert fp(20000, 8, 4, 2000) > base
    assert fp(20000, 8, 4, 0) < base
    b = C.c_double()
    _einval(lib.krr_server_footprint(0, 8, 4, 10, C.byref(b)), lib, "shape")
    _einval(lib.krr_server_footprint(100, 8, 17, 10, C.byref(b)), lib, "shape")
    _einval(lib.krr_server_footprint(100, 8, 4, 101, C.byref(b)), lib, "shape")


def test_server_config_validation(lib):
    import paper_2304_12465_gb300._native as N_
    h = C.c_void_p()
    for cfg, frag in [(N_.ServerConfig(0, 4, 1, 0, 0.0), "max_slots"),
                      (N_.ServerConfig(65, 4, 1, 0, 0.0), "max_slots"),
                      (N_.ServerConfig(4, 0, 1, 0, 0.0), "iters_per_step"),
                      (N_.ServerConfig(4, 65, 1, 0, 0.0), "iters_per_step"),
                      (N_.ServerConfig(4, 4, 1, 0, -1.0), "hbm_budget"),
                      (N_.ServerConfig(4, 4, 1, 9, 0.0), "build_threads"),
                      (N_.ServerConfig(4, 4, 1, -1, 0.0), "build_threads")]:
        _einval(lib.krr_server_create(C.byref(cfg), C.byref(h)), lib, frag)
        assert not h.value
    X = np.zeros((4, 2))
    rid = C.c_int64()
    p = C.c_void_p(X.ctypes.data)
    _einval(lib.krr_server_submit(None, p, 4, 2, 0, 1.0, p, 1, 1e-3, 1, 0, 1e-6, 10, p,
                                  C.byref(rid)), lib, "NULL")
    n = C.c_int()
    _einval(lib.krr_server_poll(None, None, 0, C.byref(n)), lib, "NULL")
    _einval(lib.krr_server_step(None, None), lib, "server")


def test_server_checkpoint_validation(lib):
    import paper_2304_12465_gb300._native as N_
    _einval(lib.krr_server_evict(None, 0), lib, "server")
    _einval(lib.krr_server_resume(None, 0), lib, "server")
    n = C.c_size_t()
    _einval(lib.krr_server_export(None, 0, None, C.byref(n)), lib, "NULL")
    rid = C.c_int64()
    _einval(lib.krr_server_import(None, None, 0, None, None, None, C.byref(rid)), lib, "NULL")
    pr = N_.RequestProgress()
    _einval(lib.krr_server_progress(None, 0, C.byref(pr)), lib, "NULL")


def test_bounded_wait_budget_validated_before_any_launch(lib):
    """krr_check_bounded_wait refuses a budget outside 0 .. 2^31 cycles with
    KRR_EINVAL before it touches the device (no GPU needed)."""
    _einval(lib.krr_check_bounded_wait(-1, None), lib, "wait budget")
    _einval(lib.krr_check_bounded_wait((1 << 31) + 1, None), lib, "wait budget")


def test_pcg_graph_switch_is_host_state(lib):
    """krr_set_pcg_graphs only sets host state (callable without a GPU)."""
    lib.krr_set_pcg_graphs(0)
    lib.krr_set_pcg_graphs(1)
