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


# ------------------------------------------------ Algorithm 3 (branch and bound)
def _bnb_both(X, A, k, T, leaf):
    ix = pm.Index(torch.from_numpy(X).cuda(), leaf_size=leaf, proj=A)
    got = ix.closest_pairs_bnb(k=k, T=T)
    ix.close()
    rp, rd = oracle.cp_bnb(X, A, T, k)
    return got, rp, rd


@pytest.mark.parametrize("n,d,clusters,k,T,leaf", [
    (800, 16, 6, 5, 40, 32),          # self-joins alone give T pairs: pruned search
    (1200, 32, 10, 10, 20000, 64),    # T beyond the self-join pairs: no bound at first
    (300, 8, 3, 7, 10 ** 9, 16),      # every pair: the exact kCP
    (1000 + 9, 40, 8, 12, 3000, 128), # ragged n, larger leaves
])
def test_cp_bnb_parity(n, d, clusters, k, T, leaf):
    X, _, _, _ = datagen.mixture(n, d, clusters, 1.0, seed=n + 1)
    A = oracle.gen_projection(8, 15, d).astype(np.float32)
    got, rp, rd = _bnb_both(X, A, k, T, leaf)
    assert got["pairs"].tolist() == rp.tolist()
    assert np.array_equal(got["dists"], rd.astype(np.float32))
    assert got["stats"]["count"] == min(T, n * (n - 1) // 2)


def test_cp_bnb_many_listed_leaf_pairs():
    # 20,000 points in four clusters, leaves of <= 16 points (L >= 1,250):
    # the first Mindist band lists the leaf pairs of overlapping balls in each
    # cluster, more than the 8,192 keys one block of the device sort of the
    # listing takes (the oracle keeps its T = 2,000 pairs by insertion, so T
    # stays small)
    n, k, T = 20000, 9, 2000
    X, _, _, _ = datagen.mixture(n, 8, 4, 1.0, seed=31)
    A = oracle.gen_projection(10, 15, 8).astype(np.float32)
    got, rp, rd = _bnb_both(X, A, k, T, 16)
    assert got["stats"]["lca_nodes"] > 8192
    assert got["pairs"].tolist() == rp.tolist()
    assert np.array_equal(got["dists"], rd.astype(np.float32))
    assert got["stats"]["count"] == T


def test_cp_bnb_duplicates_and_exact_kcp():
    # repeated points: many pairs at projected distance 0, ties by (i, j)
    base, _, _, _ = datagen.mixture(40, 12, 4, 1.0, seed=2)
    X = np.repeat(base, 6, axis=0)
    A = oracle.gen_projection(9, 15, 12).astype(np.float32)
    got, rp, rd = _bnb_both(X, A, 15, 500, 16)
    assert got["pairs"].tolist() == rp.tolist()
    assert np.array_equal(got["dists"], rd.astype(np.float32))
    got, rp, rd = _bnb_both(X, A, 15, 10 ** 9, 16)
    ep, ed = oracle.exact_kcp(X, 15)
    assert got["pairs"].tolist() == ep.tolist()
    assert np.array_equal(got["dists"], ed.astype(np.float32))


@pytest.mark.slow
def test_cp_bnb_c4_full_size():
    # Algorithm 3 on the closest-pair workload (n = 100,000, d = 512) with
    # T = ceil(0.0024 n (n-1)) + k ~ 2.4e7: the returned pairs are planted
    # pairs, their distances equal the FP64 distances, and the result equals
    # Algorithm 4's on the same index (both find the planted pairs first)
    w = datagen.workload("c4")
    X, planted = w["X"], w["planted"]
    A = oracle.gen_projection(2, 15, 512).astype(np.float32)
    n = len(X)
    T = int(math.ceil(0.0024 * n * (n - 1))) + 10
    ix = pm.Index(torch.from_numpy(X).cuda(), leaf_size=256, proj=A)
    got = ix.closest_pairs_bnb(k=10, T=T)
    rf = ix.closest_pairs(k=10, gamma=3.0, T=T, t=oracle.params(15, 1.5, 1 / math.e)[0])
    ix.close()
    assert got["stats"]["count"] == T
    planted_set = {tuple(p) for p in planted.tolist()}
    assert {tuple(p) for p in got["pairs"].tolist()} <= planted_set
    ex = np.sqrt(((X[got["pairs"][:, 0]].astype(np.float64) - X[got["pairs"][:, 1]].astype(np.float64)) ** 2).sum(1))
    assert np.allclose(got["dists"], ex, rtol=1e-6, atol=0)
    assert got["pairs"].tolist() == rf["pairs"].tolist()


@pytest.mark.parametrize("n,k,leaf", [
    (2, 1, 16),          # a single pair
    (3, 3, 16),          # k = n (n - 1) / 2
    (120, 1024, 16),     # the largest k (7,140 pairs)
])
def test_cp_extremes_both_algorithms(n, k, leaf):
    X, _, _, _ = datagen.mixture(n, 10, min(3, n), 1.0, seed=n + 5)
    A = oracle.gen_projection(12, 15, 10).astype(np.float32)
    T = 10 ** 9
    got, ref = _both(X, A, k, 3.0, T, leaf=leaf)
    _assert_same(got, ref)
    got, rp, rd = _bnb_both(X, A, k, T, leaf)
    assert got["pairs"].tolist() == rp.tolist()
    assert np.array_equal(got["dists"], rd.astype(np.float32))
    ep, ed = oracle.exact_kcp(X, k)
    assert got["pairs"].tolist() == ep.tolist()


# ------------------------------------------- setting of gamma (Sec. 6.3)

@pytest.mark.parametrize("n,d,leaf", [(600, 16, 16), (1100 + 7, 24, 64)])
def test_gamma_calibration_whole_index(n, d, leaf):
    # nsample >= n: the ratios of every pair of the index's own layout
    X, _, _, _ = datagen.mixture(n, d, 6, 1.0, seed=n)
    A = oracle.gen_projection(3, 15, d).astype(np.float32)
    ix = pm.Index(torch.from_numpy(X).cuda(), leaf_size=leaf, proj=A)
    lay = ix.layout()
    O = oracle.project(X, A)
    for pr in (0.85, 0.5, 1.0, 1.0 / (n * (n - 1) // 2)):
        assert ix.gamma_calibrate(pr, nsample=n) == oracle.gamma_calibrate(O, lay, pr)
    ix.close()


def test_gamma_calibration_sample_and_cp_default():
    # nsample < n: the library indexes the sampled rows with the index's own
    # projection and leaf capacity; the oracle draws the same ids and takes
    # the sample's layout (built through the public API) as data
    n, d, ns = 3000, 20, 700
    X, _, _, _ = datagen.mixture(n, d, 10, 1.0, seed=4)
    A = oracle.gen_projection(8, 15, d).astype(np.float32)
    ix = pm.Index(X, leaf_size=32, proj=A, seed=5)
    g = ix.gamma_calibrate(0.85, nsample=ns, seed=99)
    ids = oracle.gamma_sample(n, ns, 99)
    sub = pm.Index(X[ids], leaf_size=32, proj=A, seed=5)
    ref = oracle.gamma_calibrate(oracle.project(X[ids], A), sub.layout(), 0.85)
    sub.close()
    assert g == ref and g >= 0.5
    # gamma <= 0 in closest_pairs: calibrated on 10,000 points (here all)
    # of stream seed + 7, reported in the statistics
    k, T = 5, int(math.ceil(0.0024 * n * (n - 1))) + 5
    got = ix.closest_pairs(k=k, T=T, gamma=0.0)
    g0 = got["stats"]["gamma"]
    assert g0 == ix.gamma_calibrate(0.85, nsample=10000, seed=5 + 7)
    assert g0 == oracle.gamma_calibrate(oracle.project(X, A), ix.layout(), 0.85)
    tt, _, _ = oracle.params(15, 1.5, 1 / math.e)
    ref = oracle.cp_radius_filter(X, A, ix.layout(), k, tt, g0, T)
    _assert_same(got, ref)
    ix.close()


def test_gamma_calibration_rejects_bad_arguments():
    X, _, _, _ = datagen.mixture(100, 8, 3, 1.0, seed=1)
    ix = pm.Index(X, leaf_size=16)
    for pr, ns in ((0.0, 50), (1.5, 50), (0.85, 1), (0.85, 40000)):
        with pytest.raises(pm.PmlshError):
            ix.gamma_calibrate(pr, nsample=ns)
    ix.close()
