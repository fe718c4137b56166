"""Parity of the CUDA closest-pair path (Algorithm 4, through the C ABI) with
the FP64 oracle on the same leaf hierarchy (exported by the library and fed
to the oracle as data).  Pairs, distances and Algorithm 4's trace (count, ub
after the self-joins, FindLCA nodes, nodes examined) must be identical."""
import math

import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_05537_gb300 as pm  # noqa: E402


def _both(X, A, k, gamma, T, leaf=16, t=None, m=None):
    m = A.shape[0] if m is None else m
    ix = pm.Index(torch.from_numpy(X).cuda(), m=m, leaf_size=leaf, proj=A)
    tt, _, _ = oracle.params(m, 1.5, 1 / math.e)
    if t is not None:
        tt = t
    got = ix.closest_pairs(k=k, gamma=gamma, T=T, t=tt)
    lay = ix.layout()
    ix.close()
    ref = oracle.cp_radius_filter(X, A, lay, k, tt, gamma, T)
    return got, ref


def _assert_same(got, ref):
    assert got["pairs"].tolist() == ref["pairs"].tolist()
    assert np.array_equal(got["dists"], ref["dists"].astype(np.float32))
    st = got["stats"]
    assert st["count"] == ref["count"]
    assert st["ub_self"] == ref["ub_self"] or (math.isinf(st["ub_self"]) and math.isinf(ref["ub_self"]))
    assert st["lca_nodes"] == ref["nodes"]
    assert st["nodes_done"] == ref["nodes_done"]


@pytest.mark.parametrize("n,d,clusters,k,gamma", [
    (600, 16, 6, 5, 3.0),
    (1500, 32, 12, 20, 1.5),
    (1000 + 13, 40, 8, 10, math.inf),
])
def test_cp_parity_random(n, d, clusters, k, gamma):
    X, _, _, _ = datagen.mixture(n, d, clusters, 1.0, seed=n)
    A = oracle.gen_projection(5, 15, d).astype(np.float32)
    T = int(math.ceil(0.0024 * n * (n - 1))) + k
    got, ref = _both(X, A, k, gamma, T)
    _assert_same(got, ref)


def test_cp_budget_cut_inside_a_node():
    # a small T makes count cross T inside a node: the cut keeps the
    # T + 1 - count smallest (projected distance, i, j)
    X, _, _, _ = datagen.mixture(800, 24, 5, 1.0, seed=9)
    A = oracle.gen_projection(6, 15, 24).astype(np.float32)
    ix = pm.Index(X, leaf_size=16, proj=A)
    self_pairs = ix.closest_pairs(k=5, gamma=1e9, T=10 ** 12)["stats"]["self_pairs"]
    ix.close()
    for extra in (1, 57, 400):
        got, ref = _both(X, A, 5, 1e9, self_pairs + extra)
        _assert_same(got, ref)
        assert ref["count"] == self_pairs + extra + 1


def test_cp_all_pairs_equals_exact_kcp():
    X = datagen.gaussian(400, 12, seed=4)
    A = oracle.gen_projection(7, 8, 12).astype(np.float32)
    # t large enough that every pair passes the projected-distance filter
    got, ref = _both(X, A, 15, math.inf, 400 * 399 // 2, m=8, t=1e6)
    _assert_same(got, ref)
    ep, ed = oracle.exact_kcp(X, 15)
    assert got["pairs"].tolist() == ep.tolist()
    assert np.array_equal(got["dists"], ed.astype(np.float32))


def test_cp_duplicates_tie_by_ids():
    base = datagen.gaussian(60, 10, seed=2)
    X = np.repeat(base, 3, axis=0)   # every point three times: many zero distances
    A = oracle.gen_projection(3, 15, 10).astype(np.float32)
    got, ref = _both(X, A, 30, 2.0, 10 ** 9)
    _assert_same(got, ref)
    assert np.all(got["dists"] == 0.0)


def test_cp_planted_pairs_c4_shape():
    # the closest-pair workload's structure at reduced n: 20 planted pairs at
    # distance 0.01 among a 500-cluster mixture in d = 512
    w = datagen.workload("c4", n=20_000)
    X, planted = w["X"], w["planted"]
    A = oracle.gen_projection(2, 15, 512).astype(np.float32)
    n = len(X)
    T = int(math.ceil(0.0024 * n * (n - 1))) + 10
    got, ref = _both(X, A, 10, 3.0, T)
    _assert_same(got, ref)
    planted_set = {tuple(p) for p in planted.tolist()}
    assert {tuple(p) for p in got["pairs"].tolist()} <= planted_set


@pytest.mark.slow
def test_cp_c4_full_size():
    # the closest-pair workload at full size (n = 100,000, d = 512)
    w = datagen.workload("c4")
    X, planted = w["X"], w["planted"]
    A = oracle.gen_projection(2, 15, 512).astype(np.float32)
    n = len(X)
    T = int(math.ceil(0.0024 * n * (n - 1))) + 10
    got, ref = _both(X, A, 10, 3.0, T)
    _assert_same(got, ref)
    planted_set = {tuple(p) for p in planted.tolist()}
    assert {tuple(p) for p in got["pairs"].tolist()} <= planted_set
