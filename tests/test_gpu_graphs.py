"""CUDA-graph replay of the PCG iterations (krr_set_pcg_graphs).

After its first iteration every PCG run replays captured chunks of 16, 4 or 1
whole iterations and reads the convergence flags back once per replay.
Converged columns freeze on the device, so a replay that runs past
convergence changes nothing: the iterates, iteration counts and statuses are
bit for bit those of launch-at-a-time stepping, in every precision path, the
batched solve and KRILL.  The host read-backs fall from one per iteration to
one per replay.
"""
import numpy as np
import pytest

from inputs import make_c1_plain_fp64, make_c2_mixed, make_c3_batched, make_c4_krill
from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    K = require_gpu()
    yield K
    K.krr_set_pcg_graphs(True)


def both(K, fn):
    K.krr_set_pcg_graphs(False)
    eager = fn()
    K.krr_set_pcg_graphs(True)
    graphs = fn()
    return eager, graphs


def same_solve(eager, graphs):
    (a0, i0), (a1, i1) = eager, graphs
    np.testing.assert_array_equal(np.asarray(a1), np.asarray(a0))
    for key in ("status", "iters", "outer_refinements", "rel_residual", "escalated"):
        assert i1[key] == i0[key], key
    assert i0["graph_replays"] == 0
    return i0, i1


@pytest.mark.parametrize("prec", ["fp64", "ff", "mixed"])
def test_single_solve_identical(K, prec):
    w = make_c1_plain_fp64(n=3000)
    f = K.krr_rpcholesky(w.X, w.kernel, w.sigma, 150, 15, 0)
    tol = 1e-6 if prec == "mixed" else 1e-10
    i0, i1 = same_solve(*both(K, lambda: K.krr_pcg_solve(
        w.X, w.kernel, w.sigma, w.Y, w.mu, f, tol=tol, prec=prec)))
    f.free()
    assert i0["status"] == "KRR_OK"
    assert i1["graph_replays"] > 0
    assert i1["host_checks"] < i0["host_checks"]


def test_fixed_iteration_count_and_budget(K):
    """tol = 0 runs exactly maxit iterations in both modes (chunks never run
    past the budget); the counts and iterates agree."""
    w = make_c1_plain_fp64(n=2000)
    f = K.krr_rpcholesky(w.X, w.kernel, w.sigma, 100, 10, 0)
    for maxit in (1, 2, 17, 37):
        i0, i1 = same_solve(*both(K, lambda: K.krr_pcg_solve(
            w.X, w.kernel, w.sigma, w.Y, w.mu, f, tol=1e-300, maxit=maxit, prec="fp64")))
        assert i1["iters"] == maxit and i1["status"] == "KRR_ENOCONV"
    f.free()


def test_ill_conditioned_mixed_identical(K):
    """Near-duplicate workload (refinement, several inner solves, 4 columns
    converging at different iterations)."""
    w = make_c2_mixed(n=12_000, k=300)
    f = K.krr_rpcholesky(w.X, w.kernel, w.sigma, w.k, 30, 1)
    i0, i1 = same_solve(*both(K, lambda: K.krr_pcg_solve(
        w.X, w.kernel, w.sigma, w.Y, w.mu, f, tol=w.tol, prec="mixed")))
    f.free()
    assert i1["status"] == "KRR_OK" and i1["iters"] > 50
    # one read-back per replay plus the few of each run's eager start
    assert i1["host_checks"] * 4 < i0["host_checks"]


def test_batched_solve_identical(K):
    w = make_c3_batched(n=3000, k=120)
    settings = [(2, 1.0), (1, 2.0)]
    factors = [K.krr_rpcholesky(w.X, k, s, w.k, 20, seed=q) for q, (k, s) in enumerate(settings)]
    Y = np.repeat(w.Y, 4, axis=0)
    _, i1 = same_solve(*both(K, lambda: K.krr_pcg_solve_batched(
        w.X, [k for k, _ in settings], [s for _, s in settings], factors, [1e-4, 1e-6], Y,
        tol=1e-8)))
    for f in factors:
        f.free()
    assert i1["status"] == "KRR_OK" and i1["graph_replays"] > 0


def test_krill_identical(K):
    w = make_c4_krill(n=4000, k=150)
    P = K.krill_build(w.X, w.kernel, w.sigma, w.centers, w.mu, seed=11)
    _, i1 = same_solve(*both(K, lambda: K.krill_solve(P, w.Y, tol=1e-8)))
    assert i1["status"] == "KRR_OK" and i1["graph_replays"] > 0
