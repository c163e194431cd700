"""GPU tests of the serving engine (continuous batching of Alg. 1 solves).

Every result must (a) be the same whether the request is served alone or in
a mix with others -- bit for bit, since each request's work decomposition
and summation order are its own -- and (b) meet the tolerance on the
float64 relative residual measured by the oracle's product.
"""
import numpy as np
import pytest

import oracle as O
from inputs import make_serving_request
from gpu_common import require_gpu, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-6

# uneven N (ragged tiles), d off the 4/8/16/32 classes (5, 12), every kernel,
# 1..16 right-hand sides, mu from 1e-8 to 1e-4, k = N / 10
REQS = [
    dict(N=1500, d=4, kernel=O.GAUSSIAN, sigma=0.8, mu=1e-5, m=1, seed=11),
    dict(N=2600, d=5, kernel=O.LAPLACE_L1, sigma=1.5, mu=1e-6, m=3, seed=12),
    dict(N=4100, d=16, kernel=O.MATERN52, sigma=0.6, mu=1e-7, m=8, seed=13),
    dict(N=3333, d=32, kernel=O.GAUSSIAN, sigma=2.0, mu=1e-8, m=16, seed=14),
    dict(N=1029, d=12, kernel=O.MATERN52, sigma=0.4, mu=1e-4, m=2, seed=15),
    dict(N=5000, d=8, kernel=O.LAPLACE_L1, sigma=0.3, mu=1e-5, m=5, seed=16),
]
for r in REQS:
    r["k"] = r["N"] // 10


@pytest.fixture(scope="module")
def K():
    return require_gpu()


@pytest.fixture(scope="module")
def data():
    return [make_serving_request(r) for r in REQS]


def submit(srv, r, X, Y, **kw):
    return srv.submit(X, r["kernel"], r["sigma"], Y, r["mu"], r["k"], tol=TOL, maxit=3000,
                      seed=r["seed"], **kw)


@pytest.fixture(scope="module")
def alone(K, data):
    """Each request served with nothing else on the server."""
    out = []
    with K.KrrServer(max_slots=8, iters_per_step=4) as srv:
        for r, (X, Y) in zip(REQS, data):
            rid = submit(srv, r, X, Y)
            done = srv.drain()
            assert len(done) == 1 and done[0]["id"] == rid
            out.append(done[0])
    return out


def test_alone_results_meet_tolerance(K, data, alone):
    for r, (X, Y), res in zip(REQS, data, alone):
        assert res["status_name"] == "KRR_OK", (r, res)
        lam = r["mu"] * r["N"]
        R = Y - O.kmatvec(X, r["kernel"], r["sigma"], lam, res["alpha"])
        rel = np.linalg.norm(R, axis=1) / np.linalg.norm(Y, axis=1)
        assert rel.max() <= TOL * 1.001, (r, rel.max())
        # the engine's float-float residual agrees with the oracle's float64 one
        assert abs(res["rel_residual"] - rel.max()) <= 1e-9, (res["rel_residual"], rel.max())
        assert res["rank"] > 0 and res["iters"] > 0


def test_mix_equals_alone(K, data, alone):
    """Staggered arrivals: three requests start, the rest arrive while they
    iterate; every result equals the alone run bit for bit."""
    with K.KrrServer(max_slots=8, iters_per_step=4) as srv:
        ids = {}
        for i in (3, 0, 5):
            ids[submit(srv, REQS[i], *data[i])] = i
        done = []
        for _ in range(6):
            srv.step()
            done += srv.poll()
        for i in (1, 4, 2):
            ids[submit(srv, REQS[i], *data[i])] = i
        done += srv.drain()
        st = srv.stats()
    assert len(done) == len(REQS)
    assert st["max_concurrent"] >= 2
    for res in done:
        i = ids[res["id"]]
        assert res["status_name"] == "KRR_OK"
        np.testing.assert_array_equal(res["alpha"], alone[i]["alpha"])
        assert res["iters"] == alone[i]["iters"]
        assert res["outer_refinements"] == alone[i]["outer_refinements"]


@pytest.mark.parametrize("use_graph,U", [(False, 1), (True, 7)])
def test_step_shape_does_not_change_results(K, data, alone, use_graph, U):
    with K.KrrServer(max_slots=8, iters_per_step=U, use_graph=use_graph) as srv:
        ids = {submit(srv, r, X, Y): i for i, (r, (X, Y)) in enumerate(zip(REQS, data))}
        done = srv.drain()
    for res in done:
        np.testing.assert_array_equal(res["alpha"], alone[ids[res["id"]]]["alpha"])


def test_admission_by_budget(K, data, alone):
    """A budget that fits about one request at a time: requests wait in the
    queue, the admitted footprint never exceeds the budget, results unchanged."""
    fps = [K.krr_server_footprint(r["N"], r["d"], r["m"], r["k"]) for r in REQS]
    budget = 1.05 * max(fps)
    with K.KrrServer(max_slots=8, iters_per_step=4, hbm_budget_bytes=budget) as srv:
        ids = {submit(srv, r, X, Y): i for i, (r, (X, Y)) in enumerate(zip(REQS, data))}
        queued_seen = 0
        done = []
        while True:
            left = srv.step()
            st = srv.stats()
            assert st["reserved_bytes"] <= budget
            queued_seen = max(queued_seen, st["queued"])
            done += srv.poll()
            if left == 0:
                break
        st = srv.stats()
    assert queued_seen > 0
    assert st["peak_reserved_bytes"] <= budget
    for res in done:
        np.testing.assert_array_equal(res["alpha"], alone[ids[res["id"]]]["alpha"])
    # arrival order is kept: admission times are non-decreasing in request id
    t = [r["t_admit"] for r in sorted(done, key=lambda r: r["id"])]
    assert t == sorted(t)


def test_request_larger_than_budget_is_refused(K, data):
    r = REQS[2]
    with K.KrrServer(max_slots=2, hbm_budget_bytes=1e6) as srv:
        with pytest.raises(K.KrrError) as e:
            submit(srv, r, *data[2])
        assert e.value.status == 2   # KRR_ENOMEM


def test_iteration_budget_exhausted(K, data):
    r = REQS[3]
    with K.KrrServer(max_slots=2) as srv:
        srv.submit(data[3][0], r["kernel"], r["sigma"], data[3][1], r["mu"], r["k"], tol=TOL,
                   maxit=3, seed=r["seed"])
        (res,) = srv.drain()
    assert res["status_name"] == "KRR_ENOCONV"
    assert res["iters"] <= 3
    assert np.all(np.isfinite(res["alpha"])) and res["rel_residual"] > TOL


def test_device_arrays(K, data, alone):
    r, (X, Y) = REQS[1], data[1]
    with K.KrrServer(max_slots=2) as srv:
        submit(srv, r, to_dev(X), to_dev(Y))
        (res,) = srv.drain()
    assert res["alpha"].is_cuda
    np.testing.assert_array_equal(res["alpha"].cpu().numpy(), alone[1]["alpha"])


def test_full_size_request_sampled_rows(K):
    """The largest serving request shape (N = 200000, d = 32, 16 right-hand
    sides, k = 1000): the reported residual meets the tolerance and sampled
    rows of the oracle's residual are consistent with it."""
    r = dict(N=200_000, d=32, kernel=O.MATERN52, sigma=1.0, mu=1e-6, m=16, seed=21, k=1000)
    X, Y = make_serving_request(r)
    with K.KrrServer(max_slots=2) as srv:
        submit(srv, r, to_dev(X), to_dev(Y))
        (res,) = srv.drain()
    assert res["status_name"] == "KRR_OK"
    assert res["rel_residual"] <= TOL
    alpha = res["alpha"].cpu().numpy()
    rows = np.sort(np.random.default_rng(0).choice(r["N"], 48, replace=False))
    lam = r["mu"] * r["N"]
    Rs = Y[:, rows] - O.kmatvec(X, r["kernel"], r["sigma"], lam, alpha, rows)
    ynorm = np.linalg.norm(Y, axis=1)
    assert np.all(np.abs(Rs) <= TOL * ynorm[:, None])


def test_evict_resume_and_checkpoint(K, data, alone):
    """A request evicted during its first inner solve resumes on the same
    server, and a checkpoint exported from one server finishes on another;
    both results are bit-identical to the uninterrupted solve."""
    i = 3                         # 16 right-hand sides, several refinements
    r, (X, Y) = REQS[i], data[i]
    assert alone[i]["outer_refinements"] >= 2

    def run_into_first_inner_solve(srv, rid):
        for _ in range(100000):
            srv.step()
            if srv.progress(rid)["state_name"] == "iterating":
                break
        for _ in range(3):          # the first inner solve is under way
            srv.step()
        assert srv.progress(rid)["state_name"] == "iterating"

    with K.KrrServer(max_slots=4, iters_per_step=4) as srv:
        rid = submit(srv, r, X, Y)
        run_into_first_inner_solve(srv, rid)
        srv.evict(rid)
        for _ in range(100000):
            srv.step()
            if srv.progress(rid)["state_name"] == "parked":
                break
        pr = srv.progress(rid)
        assert pr["state_name"] == "parked" and pr["outer_refinements"] >= 1
        assert srv.stats()["reserved_bytes"] == 0
        srv.resume(rid)
        (res,) = srv.drain()
    np.testing.assert_array_equal(res["alpha"], alone[i]["alpha"])
    assert res["iters"] == alone[i]["iters"]

    with K.KrrServer(max_slots=4, iters_per_step=4) as a:
        rid = submit(a, r, X, Y)
        run_into_first_inner_solve(a, rid)
        a.evict(rid)
        while a.progress(rid)["state_name"] != "parked":
            a.step()
        blob = a.export(rid)
        with pytest.raises(K.KrrError):
            a.progress(rid)
    assert len(blob) > 2 * 8 * r["N"] * r["m"]
    with K.KrrServer(max_slots=4, iters_per_step=1, use_graph=False) as b:
        with pytest.raises(K.KrrError):
            b.import_(b"not a checkpoint" * 10, X, Y)
        b.import_(blob, X, Y)
        (res,) = b.drain()
    np.testing.assert_array_equal(res["alpha"], alone[i]["alpha"])
    assert res["iters"] == alone[i]["iters"]
    assert res["outer_refinements"] == alone[i]["outer_refinements"]


def test_escalated_request(K):
    """A request whose float32 inner iterations stall (wide Gaussian, mu =
    1e-8) is continued in higher precision by the server and meets the
    tolerance against the oracle; its result is the same alone and in a mix."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3000, 4))
    Y = np.stack([np.sin(X @ rng.standard_normal(4)) for _ in range(2)])
    hard = dict(N=3000, d=4, kernel=O.GAUSSIAN, sigma=3.0, mu=1e-8, m=2, seed=1, k=300)
    with K.KrrServer(max_slots=4) as srv:
        submit(srv, hard, X, Y)
        (res,) = srv.drain()
    assert res["status_name"] == "KRR_OK" and res["escalated"] == 1
    R = Y - O.kmatvec(X, O.GAUSSIAN, 3.0, 1e-8 * 3000, res["alpha"])
    rel = np.linalg.norm(R, axis=1) / np.linalg.norm(Y, axis=1)
    assert rel.max() <= TOL * 1.001
    easy = dict(N=2000, d=8, kernel=O.LAPLACE_L1, sigma=1.0, mu=1e-5, m=3, seed=2, k=200)
    Xe, Ye = make_serving_request(easy)
    with K.KrrServer(max_slots=4) as srv:
        ids = {submit(srv, hard, X, Y): "hard", submit(srv, easy, Xe, Ye): "easy"}
        done = {ids[d["id"]]: d for d in srv.drain()}
    np.testing.assert_array_equal(done["hard"]["alpha"], res["alpha"])
    assert done["easy"]["status_name"] == "KRR_OK"


def test_large_requests_on_tcgen05_product(K, data):
    """Requests of N >= 32768 with the Gaussian or Matern kernel take the
    single-problem tcgen05 product as launches of their own (m = 10 as groups
    of 8 and 2 right-hand sides): each result is the same bit for bit alone
    and among other requests, and sampled rows of the oracle's float64
    residual meet the tolerance."""
    big = [dict(N=40_000, d=16, kernel=O.GAUSSIAN, sigma=0.7, mu=1e-6, m=4, seed=31, k=400),
           dict(N=36_000, d=8, kernel=O.MATERN52, sigma=1.0, mu=1e-5, m=10, seed=32, k=360)]
    bdata = [make_serving_request(r) for r in big]
    alone_big = []
    with K.KrrServer(max_slots=4, iters_per_step=4) as srv:
        for r, (X, Y) in zip(big, bdata):
            submit(srv, r, X, Y)
            (res,) = srv.drain()
            assert res["status_name"] == "KRR_OK", res
            alone_big.append(res)
    with K.KrrServer(max_slots=6, iters_per_step=4) as srv:
        ids = {submit(srv, r, X, Y): i for i, (r, (X, Y)) in enumerate(zip(big, bdata))}
        small = {submit(srv, REQS[i], *data[i]): None for i in (0, 2)}
        done = srv.drain()
    assert len(done) == len(ids) + len(small)
    for res in done:
        if res["id"] not in ids:
            assert res["status_name"] == "KRR_OK"
            continue
        i = ids[res["id"]]
        np.testing.assert_array_equal(res["alpha"], alone_big[i]["alpha"])
        assert res["iters"] == alone_big[i]["iters"]
    for r, (X, Y), res in zip(big, bdata, alone_big):
        rows = np.sort(np.random.default_rng(1).choice(r["N"], 48, replace=False))
        lam = r["mu"] * r["N"]
        Rs = Y[:, rows] - O.kmatvec(X, r["kernel"], r["sigma"], lam, res["alpha"], rows)
        ynorm = np.linalg.norm(Y, axis=1)
        assert np.all(np.abs(Rs) <= TOL * ynorm[:, None]), r
        assert res["rel_residual"] <= TOL
