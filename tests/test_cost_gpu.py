"""Cost model of the PM-tree (Sec. 4.2) on the GPU index: the distance
distribution sample and CC / sum Pr[e] against the FP64 oracle, the pivot
monotonicity of Pr[e], and the leaf-size choice the model drives."""
import ctypes
import math

import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_05537_gb300 as pm  # noqa: E402


@pytest.fixture(scope="module")
def c1():
    w = datagen.workload("c1")
    return w["X"], w["Q"]


def _entries_for_oracle(ix):
    e = ix.leaf_entries()
    count = np.diff(ix.layout()["leaf_off"])
    return (count, e["radius"].astype(np.float64), e["ring_min"].astype(np.float64),
            e["ring_max"].astype(np.float64))


@pytest.mark.parametrize("leaf_size,npairs,seed", [(64, 5000, 7), (256, 65536, 1), (1024, 3, 9)])
def test_distance_sample_bit_identical_to_oracle(c1, leaf_size, npairs, seed):
    X, _ = c1
    ix = pm.Index(torch.from_numpy(X).cuda(), leaf_size=leaf_size)
    got = ix.distance_sample(npairs, seed)
    ref = oracle.distance_sample(ix.projected(), npairs, seed)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("s", [0, 1, 5, 8])
def test_cost_model_matches_oracle(c1, s):
    X, _ = c1
    ix = pm.Index(torch.from_numpy(X).cuda(), leaf_size=128, s=s)
    F = ix.distance_sample(20000, 3)
    count, rad, lo, hi = _entries_for_oracle(ix)
    assert lo.shape == (ix.leaves, s)
    rq = np.array([0.0, F[0], F[100] / 4, F[2000] / 2, F[10000], F[19999], 1e9])
    cc, en = ix.cost_model(F, rq)
    for r, a, b in zip(rq, cc, en):
        rc, re_ = oracle.cost_model(F, count, rad, lo, hi, r)
        assert a == pytest.approx(rc, rel=1e-12, abs=1e-12)
        assert b == pytest.approx(re_, rel=1e-12, abs=1e-12)
    # an unbounded radius reaches every point of every leaf
    assert cc[-1] == len(X) and en[-1] == ix.leaves


def test_cost_model_device_buffers_and_validation(c1):
    X, _ = c1
    ix = pm.Index(torch.from_numpy(X).cuda(), leaf_size=128)
    F = ix.distance_sample(4096, 5)
    Fd = torch.from_numpy(F).cuda()
    rq = torch.tensor([F[50], F[3000]], dtype=torch.float64, device="cuda")
    cc = torch.empty(2, dtype=torch.float64, device="cuda")
    L = pm.lib()
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    assert L.pmlsh_cost_model(ix._h, vp(Fd), 4096, vp(rq), 2, vp(cc), None,
                              pm._stream()) == 0
    ref, _ = ix.cost_model(F, rq.cpu().numpy())
    assert np.array_equal(cc.cpu().numpy(), ref)
    out = torch.empty(4096, dtype=torch.float64, device="cuda")
    assert L.pmlsh_distance_sample(ix._h, 4096, 5, vp(out), pm._stream()) == 0
    assert np.array_equal(out.cpu().numpy(), F)
    with pytest.raises(pm.PmlshError):
        ix.cost_model(F[::-1].copy(), [1.0])          # not ascending
    with pytest.raises(pm.PmlshError):
        ix.cost_model(F, [-1.0])                      # negative radius
    with pytest.raises(pm.PmlshError):
        ix.distance_sample(0, 1)


def test_pr_nonincreasing_in_pivot_count(c1):
    # Same seed and leaf size: the leaves do not depend on s and the pivots of
    # a smaller s are a prefix of a larger s (farthest-first), so every extra
    # pivot multiplies Pr[e] by a factor in [0, 1].
    X, _ = c1
    Xd = torch.from_numpy(X).cuda()
    idx = {s: pm.Index(Xd, leaf_size=128, s=s, seed=4) for s in (0, 2, 5, 8)}
    offs = [idx[s].layout()["leaf_off"] for s in idx]
    assert all(np.array_equal(offs[0], o) for o in offs)
    piv8 = idx[8].leaf_entries()["pivots"]
    for s in (2, 5):
        assert np.array_equal(idx[s].leaf_entries()["pivots"], piv8[:s])
    F = idx[0].distance_sample(20000, 2)
    rq = F[[10, 500, 2000, 8000, 15000]]
    prev = None
    for s in (0, 2, 5, 8):
        cc, en = idx[s].cost_model(F, rq)
        if prev is not None:
            assert np.all(cc <= prev[0]) and np.all(en <= prev[1])
        prev = (cc, en)


def test_model_tuned_leaf_size_minimises_modelled_cost(c1):
    # leaf_size = -1 keeps the candidate with the fewest modelled distance
    # computations L + CC(range(q, t r_min)); recompute them per candidate.
    X, Q = c1
    Xd = torch.from_numpy(X).cuda()
    chosen = pm.Index(Xd, leaf_size=-1, seed=3)
    t, _, _ = pm.params(15, 1.5, 1 / math.e)
    W = {}
    for M in (128, 256, 512):
        ix = pm.Index(Xd, leaf_size=M, seed=3)
        st = ix.knn(Q, k=10)["stats"]
        one = st["rounds"] == 1
        assert one.any()
        rmin = float(st["r"][one][0])
        F = ix.distance_sample(65536, 3 + 6)
        cc, _ = ix.cost_model(F, [t * rmin])
        W[M] = ix.leaves + cc[0]
    best = min(W, key=W.get)
    assert chosen.leaf_size == best, (chosen.leaf_size, W)
