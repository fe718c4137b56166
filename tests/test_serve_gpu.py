"""Continuous-batching server (pmlsh_serve_*): every request's result equals
pmlsh_knn on that request alone, whether it ran alone or batched with others
of uneven size and k; timeouts, cancellation and memory admission behave."""
import math
import threading

import numpy as np
import pytest

import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_05537_gb300 as pm  # noqa: E402


@pytest.fixture(scope="module")
def served():
    X, Q, _, _ = datagen.mixture(20_000, 64, 40, (0.5, 2.0), seed=11, nq=6000)
    ix = pm.Index(torch.from_numpy(X).cuda(), leaf_size=128)
    yield ix, Q
    ix.close()


def _requests(Q, count, seed):
    rng = np.random.default_rng(seed)
    reqs, at = [], 0
    for _ in range(count):
        size = int(np.exp(rng.uniform(0, math.log(300))))
        k = int(rng.choice([1, 10, 50]))
        rows = Q[at % len(Q): at % len(Q) + size]
        if len(rows) == 0:
            rows = Q[:size]
        at += size
        reqs.append((np.ascontiguousarray(rows), k))
    return reqs


def test_results_same_alone_and_in_the_mix(served):
    ix, Q = served
    reqs = _requests(Q, 48, seed=1)
    srv = pm.Server(ix, slots=3, max_batch_queries=2048)
    tickets = [None] * len(reqs)

    def client(part):
        for i in range(part, len(reqs), 4):
            tickets[i] = srv.submit(reqs[i][0], k=reqs[i][1])
    threads = [threading.Thread(target=client, args=(p,)) for p in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    outs = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["queries"] == sum(len(r) for r, _ in reqs)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for (rows, k), (ids, dd) in zip(reqs, outs):
        alone = ix.knn(rows, k=k, with_stats=False)
        assert np.array_equal(ids, alone["ids"])
        assert np.array_equal(dd, alone["dists"])


def test_tiny_memory_budget_runs_batches_one_at_a_time(served):
    ix, Q = served
    reqs = _requests(Q, 12, seed=2)
    srv = pm.Server(ix, slots=3, mem_budget_bytes=1)
    tickets = [srv.submit(r, k=k) for r, k in reqs]
    outs = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs)
    for (rows, k), (ids, _) in zip(reqs, outs):
        assert np.array_equal(ids, ix.knn(rows, k=k, with_stats=False)["ids"])


def test_timeout_cancel_and_stop(served):
    ix, Q = served
    srv = pm.Server(ix, slots=1, max_batch_queries=64)
    big = srv.submit(Q[:3000], k=50)
    smalls = [srv.submit(Q[3000 + 10 * i: 3010 + 10 * i], k=10) for i in range(20)]
    # an immediate wait either finds the result or times out, leaving the ticket valid
    try:
        srv.wait(smalls[-1], timeout_ms=0)
        waited = True
    except pm.PmlshError as e:
        assert e.code == 3   # ETIMEOUT
        waited = False
    srv.stop()
    outcomes = []
    for t in [big] + smalls[:-1] + ([] if waited else [smalls[-1]]):
        try:
            srv.wait(t, timeout_ms=60_000)
            outcomes.append("ok")
        except pm.PmlshError as e:
            assert e.code == 5   # ECANCELED
            outcomes.append("cancelled")
    assert "ok" in outcomes   # the running batch finished
    st = srv.stats()
    assert st["canceled"] == outcomes.count("cancelled")
    with pytest.raises(pm.PmlshError) as e:
        srv.submit(Q[:4], k=1)
    assert e.value.code == 5
    srv.close()


def test_invalid_requests_rejected(served):
    ix, Q = served
    srv = pm.Server(ix, slots=1)
    with pytest.raises(pm.PmlshError):
        srv.submit(Q[:4], k=0)
    with pytest.raises(pm.PmlshError):
        srv.submit(Q[:4], k=10, c=0.9)
    with pytest.raises(pm.PmlshError):
        srv.wait(123456)
    srv.close()


@pytest.mark.slow
def test_c5_serving_full_size():
    # serving workload: n = 2*10^6, d = 256 resident; an open-loop stream of
    # requests of log-uniform size in [1, 4096] with k in {1, 10, 100} from
    # four client threads; every result equals pmlsh_knn on that request
    # alone, and a query sample equals the oracle's
    import time
    import oracle
    w = datagen.workload("c5")
    X, Q = w["X"], w["Q"]
    ix = pm.Index(torch.from_numpy(X).cuda(), leaf_size=256)
    rng = np.random.default_rng(7)
    reqs = []
    for _ in range(40):
        size = int(np.exp(rng.uniform(0.0, math.log(4096.0))))
        q0 = int(rng.integers(0, len(Q) - size + 1))
        reqs.append((np.ascontiguousarray(Q[q0:q0 + size]), int(rng.choice([1, 10, 100]))))
    srv = pm.Server(ix, slots=3)
    tickets = [None] * len(reqs)

    def client(part):
        for i in range(part, len(reqs), 4):
            time.sleep(0.002)
            tickets[i] = srv.submit(reqs[i][0], k=reqs[i][1], precision=pm.PMLSH_BF16_TENSOR)
    threads = [threading.Thread(target=client, args=(p,)) for p in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    outs = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    for (rows, k), (ids, dd) in zip(reqs, outs):
        alone = ix.knn(rows, k=k, with_stats=False)
        assert np.array_equal(ids, alone["ids"]) and np.array_equal(dd, alone["dists"])
    # a sample of the requests' queries against the oracle
    A = ix.projection()
    rows, k = reqs[0]
    sel = rows[:4]
    t, _, _ = oracle.params(15, 1.5, 1 / math.e)
    ref = oracle.knn(X, A, sel, k, 1.5, t, oracle.budget(len(X), 0.2809, k),
                     oracle.rmin_auto(X, 0.2809, k, 1.5, 3), 0)
    assert np.array_equal(outs[0][0][:4], ref["ids"])
    assert np.array_equal(outs[0][1][:4], ref["dists"].astype(np.float32))
    ix.close()


def test_non_finite_options_rejected_and_server_keeps_serving(served):
    # options that pmlsh_knn rejects are rejected at submit; a request whose
    # options equal no other (NaN compares unequal) could otherwise never be
    # batched, so the server must keep serving after such attempts
    ix, Q = served
    srv = pm.Server(ix, slots=2, max_batch_queries=512)
    for bad in (dict(r_min=float("nan")), dict(t=float("nan")), dict(c=float("inf")),
                dict(r_min=float("inf"))):
        with pytest.raises(pm.PmlshError):
            srv.submit(Q[:4], k=5, **bad)
    rows = np.ascontiguousarray(Q[:37])
    ids, dd = srv.wait(srv.submit(rows, k=5), timeout_ms=60_000)
    srv.close()
    alone = ix.knn(rows, k=5, with_stats=False)
    np.testing.assert_array_equal(ids, alone["ids"])
    np.testing.assert_array_equal(dd, alone["dists"])


def test_memory_admission_bounds_resident_scratch(served):
    # admission counts every slot's resident scratch plus the growth charged
    # to running batches: with no batch needing more than the budget by
    # itself, the total never passes the budget.  beta = 1 keeps the budget
    # rule (whose selection buffers grow with the data) out of play.
    ix, Q = served
    cap = 600
    budget = int(1.6 * max(ix.workspace_bytes(cap, k) for k in (1, 10, 50)))
    reqs = _requests(Q, 40, seed=3)
    srv = pm.Server(ix, slots=3, max_batch_queries=cap, mem_budget_bytes=budget)
    tickets = [None] * len(reqs)

    def client(part):
        for i in range(part, len(reqs), 4):
            tickets[i] = srv.submit(reqs[i][0], k=reqs[i][1], beta=1.0)
    threads = [threading.Thread(target=client, args=(p,)) for p in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    outs = [srv.wait(t, with_err=True) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs)
    assert 0 < st["peak_bytes"] <= budget and st["resident_bytes"] <= budget
    for (rows, k), (ids, dd, ee) in zip(reqs, outs):
        alone = ix.knn(rows, k=k, beta=1.0, with_stats=False)
        assert np.array_equal(ids, alone["ids"]) and np.array_equal(dd, alone["dists"])
        # the per-result error bound of pmlsh_knn is passed through
        assert np.array_equal(ee, alone["err"])
