"""Algorithm 1, the (r,c)-BC query (pmlsh_rcbc), against the FP64 oracle,
and the guarantees of Sec. 5.3 measured over many random projections."""
import math

import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_05537_gb300 as pm  # noqa: E402

E = math.e


@pytest.fixture(scope="module")
def c1():
    w = datagen.workload("c1")
    A = oracle.gen_projection(2, 15, w["d"]).astype(np.float32)
    return w["X"], w["Q"], A


@pytest.mark.parametrize("precision", [pm.PMLSH_FP32_PLAIN, pm.PMLSH_BF16_TENSOR])
def test_rcbc_parity(c1, precision):
    # radii from "nothing" through "within c r" to "|C| >= beta n + 1"
    X, Q, A = c1
    ix = pm.Index(torch.from_numpy(X).cuda(), proj=A, leaf_size=64)
    O = oracle.project(X, A)
    t, _, _ = oracle.params(15, 1.5, 1 / E)
    seen = set()
    for beta in (0.01, 0.2809):
        Bbc = oracle.budget(len(X), beta, 1)
        for r in (2.0, 8.0, 12.0, 16.0, 40.0, 200.0):
            for c in (1.2, 2.0):
                ref_ids, ref_d, ref_nc = oracle.rcbc(X, A, Q, r, c, t, Bbc, Oproj=O)
                got = ix.rcbc(Q, r, c=c, beta=beta, precision=precision)
                fast = ix.rcbc(torch.from_numpy(Q).cuda(), r, c=c, beta=beta, precision=precision,
                               with_stats=False)
                assert np.array_equal(got["ids"], ref_ids)
                assert np.array_equal(got["dists"], ref_d.astype(np.float32))
                assert np.array_equal(fast["ids"], ref_ids) and np.array_equal(fast["dists"], got["dists"])
                assert np.array_equal(got["stats"]["ncand"], ref_nc)
                rule = got["stats"]["rule"]
                assert np.array_equal(rule == 2, ref_nc >= Bbc)
                assert np.all((rule == 0) == (ref_ids == -1))
                seen |= set(rule.tolist())
    ix.close()
    assert seen == {0, 1, 2}


def test_rcbc_edges(c1):
    X, Q, A = c1
    ix = pm.Index(X, proj=A, leaf_size=64)
    assert ix.rcbc(Q[:0], 5.0)["ids"].shape == (0,)
    with pytest.raises(pm.PmlshError):
        ix.rcbc(Q[:4], 0.0)
    with pytest.raises(pm.PmlshError):
        ix.rcbc(Q[:4], 5.0, c=1.0)
    # a query equal to a data point at a tiny radius returns that point
    got = ix.rcbc(X[:8], 1e-3, c=1.5)
    assert np.array_equal(got["ids"], np.arange(8)) and np.all(got["dists"] == 0)
    ix.close()


def test_rcbc_guarantee_over_projections():
    # Sec. 5.3: with beta = 2 alpha2 (Eq. 9, Lemma 5), whenever B(q, r)
    # holds a point, Algorithm 1 returns a point of B(q, c r) with
    # probability at least 1/2 - 1/e; measured over 12 projections x 48
    # queries at r = the exact nearest-neighbour distance
    X, Q, _, _ = datagen.mixture(4000, 32, 20, 1.0, seed=5, nq=48)
    _, ed = oracle.exact_knn(X, Q, 1)
    c = 1.5
    t, a2, _ = oracle.params(15, c, 1 / E)
    ok = []
    for seed in range(12):
        ix = pm.Index(torch.from_numpy(X).cuda(), leaf_size=64, seed=100 + seed)
        for qi in range(len(Q)):
            r = float(ed[qi, 0]) * (1 + 1e-9) + 1e-12
            got = ix.rcbc(Q[qi:qi + 1], r, c=c, beta=2 * a2, with_stats=False)
            ok.append(got["ids"][0] >= 0 and got["dists"][0] <= c * r)
        ix.close()
    assert np.mean(ok) >= 0.5 - 1 / E


def test_knn_c2_ann_rate_over_projections():
    # Theorem 1: Algorithm 2 returns a c^2-approximate nearest neighbour with
    # probability at least 1/2 - 1/e (beta = 2 alpha2); measured on the GPU
    # over 12 projections x 64 queries
    X, Q, _, _ = datagen.mixture(4000, 32, 20, 1.0, seed=6, nq=64)
    _, ed = oracle.exact_knn(X, Q, 1)
    c = 1.5
    _, a2, _ = oracle.params(15, c, 1 / E)
    ok = []
    for seed in range(12):
        ix = pm.Index(torch.from_numpy(X).cuda(), leaf_size=64, seed=200 + seed)
        got = ix.knn(Q, k=1, c=c, beta=2 * a2, with_stats=False)
        ok.extend((got["dists"][:, 0] <= c * c * ed[:, 0]).tolist())
        ix.close()
    assert np.mean(ok) >= 0.5 - 1 / E
