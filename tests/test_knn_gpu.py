"""Parity of the CUDA (c,k)-ANN path (through the C ABI) with the FP64 oracle.

Every decision of Algorithm 2 (range membership, budget cut, k-th neighbour,
stop rules) is taken in FP64 where FP32 cannot decide, so ids, the per-query
trace (rounds, stop rule, |C|) and the FP32-rounded FP64 distances must be
identical to the oracle's.  The stated tolerance for distances is 1e-6
relative; the comparison below also checks they are the rounded FP64 values.
"""
import math

import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2107_05537_gb300 as pm  # noqa: E402

E = math.e


def _run_both(X, Q, A, k, c=1.5, beta=0.2809, r_min=None, stop_rule=0, leaf=64, s=5, m=None,
              t=None, device_inputs=True, precision=0, with_stats=True):
    m = A.shape[0] if m is None else m
    ix = pm.Index(torch.from_numpy(X).cuda() if device_inputs else X, m=m, s=s, leaf_size=leaf,
                  proj=A)
    tt, _, _ = oracle.params(m, c, 1 / E)
    if t is not None:
        tt = t
    rmin = r_min if r_min is not None else oracle.rmin_auto(X, beta, k, c, 3)
    B = oracle.budget(len(X), beta, k)
    ref = oracle.knn(X, A, Q, k, c, tt, B, rmin, stop_rule)
    Qin = torch.from_numpy(Q).cuda() if device_inputs else Q
    got = ix.knn(Qin, k=k, c=c, beta=beta, r_min=r_min if r_min is not None else 0.0,
                 stop_rule=stop_rule, t=tt, precision=precision, with_stats=with_stats)
    torch.cuda.synchronize()
    ix.close()
    return got, ref


def _to_np(a):
    return a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)


def _assert_parity(got, ref, trace=True):
    ids = _to_np(got["ids"])
    dd = _to_np(got["dists"])
    assert np.array_equal(ids, ref["ids"]), np.argwhere(ids != ref["ids"])[:5]
    # distances: the FP64 value rounded to FP32 (well within 1e-6 relative)
    assert np.array_equal(dd, ref["dists"].astype(np.float32))
    finite = np.isfinite(ref["dists"])
    rel = np.abs(dd[finite].astype(np.float64) - ref["dists"][finite]) / np.maximum(ref["dists"][finite], 1e-300)
    assert rel.max(initial=0) <= 1e-6
    err = _to_np(got["err"])
    assert np.allclose(err[finite], np.abs(dd[finite].astype(np.float64) - ref["dists"][finite]),
                       rtol=1e-6, atol=1e-30)
    if trace:
        st = got["stats"]
        assert np.array_equal(st["rounds"], ref["rounds"])
        assert np.array_equal(st["rule"], ref["rule"])
        assert np.array_equal(st["ncand"], ref["ncand"])
        assert np.array_equal(st["r"], ref["r"])


@pytest.fixture(scope="module")
def c1():
    w = datagen.workload("c1")
    A = oracle.gen_projection(2, 15, w["d"]).astype(np.float32)
    return w["X"], w["Q"], A


def test_projection_bit_identical_to_oracle(c1):
    X, Q, A = c1
    ix = pm.Index(torch.from_numpy(X).cuda(), proj=A, leaf_size=64)
    O = ix.projected()
    assert np.array_equal(O, oracle.project(X, A))
    assert np.array_equal(ix.projection(), A)
    ix.close()
    # the library's own projection: stream seed+2 of the counter generator
    ix = pm.Index(X, seed=7, leaf_size=128)
    assert np.array_equal(ix.projection(), oracle.gen_projection(9, 15, X.shape[1]).astype(np.float32))
    ix.close()


@pytest.mark.parametrize("stop_rule", [0, 1])
def test_c1_parity(c1, stop_rule):
    X, Q, A = c1
    got, ref = _run_both(X, Q, A, k=10, stop_rule=stop_rule)
    _assert_parity(got, ref)
    assert set(ref["rule"].tolist()) >= {1}


def test_c1_host_buffers_and_auto_t(c1):
    # host input/output buffers, t from alpha1 inside the library
    X, Q, A = c1
    ix = pm.Index(X, proj=A, leaf_size=128)
    got = ix.knn(Q, k=10)
    ix.close()
    t, _, _ = oracle.params(15, 1.5, 1 / E)
    ref = oracle.knn(X, A, Q, 10, 1.5, t, oracle.budget(len(X), 0.2809, 10),
                     oracle.rmin_auto(X, 0.2809, 10, 1.5, 3), 0)
    assert isinstance(got["ids"], np.ndarray)
    _assert_parity(got, ref)


def test_budget_rule2_path(c1):
    # a first radius that already holds more than B points: every query stops
    # by rule 2 with the B nearest in projected space
    X, Q, A = c1
    got, ref = _run_both(X, Q[:40], A, k=10, r_min=200.0)
    assert np.all(ref["rule"] == 2)
    _assert_parity(got, ref)


def test_small_beta_budget_and_multiround(c1):
    X, Q, A = c1
    got, ref = _run_both(X, Q[:50], A, k=5, beta=0.01, r_min=2.0)
    assert ref["rounds"].max() >= 2
    _assert_parity(got, ref)
    got, ref = _run_both(X, Q[:50], A, k=5, beta=0.01, r_min=2.0, stop_rule=1)
    _assert_parity(got, ref)


@pytest.mark.parametrize("n,d,m,leaf,s,k", [
    (1000 + 17, 37, 15, 64, 5, 7),     # ragged n, d not a multiple of 32
    (300, 8, 3, 16, 0, 1),             # m = 3, no pivots, k = 1
    (50, 20, 16, 64, 5, 50),           # n < leaf size, k = n
    (2500, 64, 15, 1024, 8, 20),       # largest leaf, most pivots
])
def test_shapes_and_edges(n, d, m, leaf, s, k):
    X, Q, _, _ = datagen.mixture(n, d, 7, 1.0, seed=n, nq=33)
    A = oracle.gen_projection(11, m, d).astype(np.float32)
    for rmin in (None, 0.5):
        got, ref = _run_both(X, Q, A, k=k, leaf=leaf, s=s, r_min=rmin, beta=0.1)
        _assert_parity(got, ref)


@pytest.mark.parametrize("precision", [pm.PMLSH_FP32_PLAIN, pm.PMLSH_BF16_TENSOR])
@pytest.mark.parametrize("n,d,m,leaf,s,k,nq", [
    (1, 4, 15, 16, 5, 1, 5),           # a single point
    (700, 1, 1, 16, 3, 9, 40),         # d = 1, m = 1
    (600, 24, 15, 64, 5, 256, 20),     # the largest k
])
def test_extreme_shapes(n, d, m, leaf, s, k, nq, precision):
    X, Q, _, _ = datagen.mixture(n, d, min(7, n), 1.0, seed=n + d, nq=nq)
    A = oracle.gen_projection(11, m, d).astype(np.float32)
    got, ref = _run_both(X, Q, A, k=k, leaf=leaf, s=s, beta=0.1, precision=precision)
    _assert_parity(got, ref)


def test_duplicate_points_tie_by_id():
    # 40 copies of each of 25 points: every distance ties 40 ways
    base, Q, _, _ = datagen.mixture(25, 16, 5, 1.0, seed=3, nq=20)
    X = np.repeat(base, 40, axis=0)
    A = oracle.gen_projection(5, 15, 16).astype(np.float32)
    for beta in (0.2809, 0.02):
        got, ref = _run_both(X, Q, A, k=30, beta=beta, leaf=32)
        _assert_parity(got, ref)


def test_queries_equal_to_data_points(c1):
    X, _, A = c1
    Q = X[::250].copy()
    got, ref = _run_both(X, Q, A, k=10)
    _assert_parity(got, ref)
    assert np.all(_to_np(got["dists"])[:, 0] == 0.0)


def test_empty_batch(c1):
    X, Q, A = c1
    ix = pm.Index(X, proj=A)
    r = ix.knn(Q[:0], k=3)
    assert r["ids"].shape == (0, 3)
    ix.close()


def test_invalid_arguments_rejected(c1):
    X, Q, A = c1
    ix = pm.Index(X, proj=A)
    with pytest.raises(pm.PmlshError):
        ix.knn(Q, k=0)
    with pytest.raises(pm.PmlshError):
        ix.knn(Q, k=10, c=1.0)
    with pytest.raises(pm.PmlshError):
        ix.knn(Q, k=10, beta=1.5)
    with pytest.raises(pm.PmlshError):
        ix.knn(Q, k=len(X) + 1)
    ix.close()


@pytest.mark.slow
def test_c2_full_size_sampled_parity():
    # the throughput workload at full size, in the launch configuration the
    # benchmark times (all 10,000 queries in one call); 48 sampled queries are
    # checked against the oracle one by one
    w = datagen.workload("c2")
    X, Q = w["X"], w["Q"]
    A = oracle.gen_projection(2, 15, 128).astype(np.float32)
    ix = pm.Index(torch.from_numpy(X).cuda(), proj=A, leaf_size=256)
    got = ix.knn(torch.from_numpy(Q).cuda(), k=50, c=1.5, beta=0.2809)
    torch.cuda.synchronize()
    ix.close()
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(len(Q), size=48, replace=False))
    t, _, _ = oracle.params(15, 1.5, 1 / E)
    ref = oracle.knn(X, A, Q[sample], 50, 1.5, t, oracle.budget(len(X), 0.2809, 50),
                     oracle.rmin_auto(X, 0.2809, 50, 1.5, 3), 0)
    sub = dict(ids=got["ids"][sample], dists=got["dists"][sample], err=got["err"][sample],
               stats={k2: v[sample] for k2, v in got["stats"].items()})
    # t from the library's own Eq. 9 solver may differ from the oracle's in
    # the last bit; the trace check still holds unless a point sits exactly
    # at the radius
    _assert_parity(sub, ref)


def test_query_projection_entry_point(c1):
    X, Q, A = c1
    ix = pm.Index(X, proj=A)
    ref = oracle.project(Q, A)
    o64, o32 = ix.project(torch.from_numpy(Q).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(o64.cpu().numpy(), ref)
    assert np.array_equal(o32.cpu().numpy(), ref.astype(np.float32))
    h64, h32 = ix.project(Q[:7])
    assert np.array_equal(h64, ref[:7])
    ix.close()


# ------------------------------------------- tensor-core range counts

TENSOR = pm.PMLSH_BF16_TENSOR


@pytest.mark.parametrize("stop_rule", [0, 1])
def test_c1_parity_tensor(c1, stop_rule):
    X, Q, A = c1
    got, ref = _run_both(X, Q, A, k=10, stop_rule=stop_rule, precision=TENSOR)
    _assert_parity(got, ref)


@pytest.mark.parametrize("n,d,m,leaf,s,k,nq", [
    (1000 + 17, 37, 15, 64, 5, 7, 33),     # ragged n and d
    (300, 8, 3, 16, 0, 1, 129),            # m = 3, one query past a 128-query tile
    (50, 20, 16, 64, 5, 50, 1),            # n < leaf size, k = n, one query
    (2500, 64, 15, 1024, 8, 20, 257),      # leaves of 1024 points: four 256-row tiles
])
def test_shapes_and_edges_tensor(n, d, m, leaf, s, k, nq):
    X, Q, _, _ = datagen.mixture(n, d, 7, 1.0, seed=n, nq=nq)
    A = oracle.gen_projection(11, m, d).astype(np.float32)
    for rmin in (None, 0.5):
        got, ref = _run_both(X, Q, A, k=k, leaf=leaf, s=s, r_min=rmin, beta=0.1, precision=TENSOR)
        _assert_parity(got, ref)


def test_tensor_rule2_multiround_and_duplicates(c1):
    X, Q, A = c1
    got, ref = _run_both(X, Q[:40], A, k=10, r_min=200.0, precision=TENSOR)
    _assert_parity(got, ref)
    got, ref = _run_both(X, Q[:50], A, k=5, beta=0.01, r_min=2.0, precision=TENSOR)
    _assert_parity(got, ref)
    base, Qd, _, _ = datagen.mixture(25, 16, 5, 1.0, seed=3, nq=20)
    Xd = np.repeat(base, 40, axis=0)
    Ad = oracle.gen_projection(5, 15, 16).astype(np.float32)
    got, ref = _run_both(Xd, Qd, Ad, k=30, beta=0.02, leaf=32, precision=TENSOR)
    _assert_parity(got, ref)


def test_tensor_far_from_origin():
    # a common offset of 1000 makes ||o'||^2 + ||q'||^2 - 2 q'.o' cancel
    # heavily: far more pairs fall back to the exact test, results unchanged
    X, Q, _, _ = datagen.mixture(3000, 32, 10, 1.0, seed=21, nq=200)
    X = X + np.float32(1000.0)
    Q = Q + np.float32(1000.0)
    A = oracle.gen_projection(4, 15, 32).astype(np.float32)
    got, ref = _run_both(X, Q, A, k=10, precision=TENSOR)
    _assert_parity(got, ref)


def test_tensor_trace_equals_fp32_path(c1):
    # identical counts and band lists: every statistic of the two modes agrees
    X, Q, A = c1
    ix = pm.Index(torch.from_numpy(X).cuda(), proj=A, leaf_size=128)
    a = ix.knn(Q, k=10, precision=pm.PMLSH_FP32_PLAIN)
    b = ix.knn(Q, k=10, precision=TENSOR)
    ix.close()
    assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["dists"], b["dists"])
    for key in ("rounds", "rule", "ncand", "r", "fp64"):
        assert np.array_equal(a["stats"][key], b["stats"][key]), key


def test_tensor_needs_the_split_operand(c1):
    X, Q, A = c1
    ix = pm.Index(X, proj=A, bf16_shadow=False)
    with pytest.raises(pm.PmlshError):
        ix.knn(Q[:4], k=3, precision=TENSOR)
    assert ix.knn(Q[:4], k=3)["ids"].shape == (4, 3)
    ix.close()


@pytest.mark.slow
def test_c2_full_size_sampled_parity_tensor():
    w = datagen.workload("c2")
    X, Q = w["X"], w["Q"]
    A = oracle.gen_projection(2, 15, 128).astype(np.float32)
    ix = pm.Index(torch.from_numpy(X).cuda(), proj=A, leaf_size=256)
    Qd = torch.from_numpy(Q).cuda()
    got = ix.knn(Qd, k=50, c=1.5, beta=0.2809, precision=TENSOR)
    plain = ix.knn(Qd, k=50, c=1.5, beta=0.2809)
    fast = ix.knn(Qd, k=50, c=1.5, beta=0.2809, precision=TENSOR, with_stats=False)
    torch.cuda.synchronize()
    ix.close()
    assert torch.equal(got["ids"], plain["ids"]) and torch.equal(got["dists"], plain["dists"])
    assert torch.equal(got["ids"], fast["ids"]) and torch.equal(got["dists"], fast["dists"])
    assert torch.equal(got["err"], fast["err"])
    for key in ("rounds", "rule", "ncand", "r", "fp64"):
        assert np.array_equal(got["stats"][key], plain["stats"][key]), key
    rng = np.random.default_rng(1)
    sample = np.sort(rng.choice(len(Q), size=32, replace=False))
    t, _, _ = oracle.params(15, 1.5, 1 / E)
    ref = oracle.knn(X, A, Q[sample], 50, 1.5, t, oracle.budget(len(X), 0.2809, 50),
                     oracle.rmin_auto(X, 0.2809, 50, 1.5, 3), 0)
    sub = dict(ids=got["ids"][sample], dists=got["dists"][sample], err=got["err"][sample],
               stats={k2: v[sample] for k2, v in got["stats"].items()})
    _assert_parity(sub, ref)


# Without statistics the exact range count runs only where the bounds of
# |S_i| from whole leaves straddle min(B, n); band points of the visited
# leaves are then decided in FP64 by the verification.  Results are the
# oracle's in every regime: rule 1 (bounds far below B), a radius whose
# lower bound already reaches B (rule 2 without a count), bounds that
# straddle B (the exact count runs), several rounds, rule 3 (B > n).
@pytest.mark.parametrize("precision", [pm.PMLSH_FP32_PLAIN, pm.PMLSH_BF16_TENSOR])
@pytest.mark.parametrize("kw", [
    dict(k=10),
    dict(k=10, r_min=200.0),
    dict(k=5, beta=0.01, r_min=2.0),
    dict(k=5, beta=0.01, r_min=2.0, stop_rule=1),
    dict(k=10, beta=0.05, r_min=8.0),
    dict(k=10, beta=1.0, r_min=400.0),
])
def test_no_stats_path_parity(c1, precision, kw):
    X, Q, A = c1
    got, ref = _run_both(X, Q[:64], A, precision=precision, with_stats=False, **kw)
    assert got.get("stats") is None
    _assert_parity(got, ref, trace=False)


@pytest.mark.parametrize("n,d,m,leaf,s,k", [
    (1000 + 17, 37, 15, 64, 5, 7),
    (300, 8, 3, 16, 0, 1),
    (50, 20, 16, 64, 5, 50),
])
def test_no_stats_path_shapes(n, d, m, leaf, s, k):
    X, Q, _, _ = datagen.mixture(n, d, 7, 1.0, seed=n, nq=33)
    A = oracle.gen_projection(11, m, d).astype(np.float32)
    for rmin in (None, 0.5):
        got, ref = _run_both(X, Q, A, k=k, leaf=leaf, s=s, r_min=rmin, beta=0.1, with_stats=False)
        _assert_parity(got, ref, trace=False)


def test_no_stats_path_sub_batch_of_straddling_queries(c1):
    # radii for which some queries' bounds straddle B and others do not: the
    # exact count runs on a gathered sub-batch (k_gather_sub), results equal
    # the oracle's, and the sweep also covers rounds without any count
    X, Q, A = c1
    seen_sub, seen_none = [], []
    # projected clusters of this workload lie ~600 apart with radius ~45, so
    # the counts of different queries cross B = 510 at r of about 80-120
    for beta, rmin in ((0.05, 3.0), (0.05, 60.0), (0.05, 80.0), (0.05, 100.0), (0.05, 120.0),
                       (0.2809, 3.0)):
        pm.profile(True)
        pm.profile_read()
        got, ref = _run_both(X, Q[:64], A, k=10, beta=beta, r_min=rmin, with_stats=False)
        prof = pm.profile_read()
        pm.profile(False)
        _assert_parity(got, ref, trace=False)
        if "k_gather_sub" in prof:
            seen_sub.append((beta, rmin))
        if "k_count" not in prof and "k_count_tc" not in prof:
            seen_none.append((beta, rmin))
    assert seen_sub and seen_none, (seen_sub, seen_none)


def test_no_stats_straddle_decided_by_band_points():
    # A = I (m = d = 2), a query at the origin, a clump well inside the first
    # radius R = t r_min, 200 points on the circle of radius R (their FP32
    # distances lie inside the FP32 error band of R, so no FP32 test decides
    # them) and far points; B lies between the clump and clump + circle, so
    # the query's bounds straddle B and its exact count (k_gather_sub, FP64
    # at the band) decides rule 2; results equal the oracle's with and
    # without statistics
    c, k, rmin = 1.5, 5, 10.0
    t, _, _ = oracle.params(2, c, 1 / E)
    R = t * rmin
    rng = np.random.default_rng(7)
    inner = rng.uniform(-0.1, 0.1, size=(40, 2)) * R
    ang = rng.uniform(0.0, 2.0 * np.pi, size=200)
    ring = np.stack([R * np.cos(ang), R * np.sin(ang)], 1)
    far = rng.normal(size=(260, 2)) * R + 20.0 * R
    X = np.concatenate([inner, ring, far]).astype(np.float32)
    Q = np.array([[0.0, 0.0], [20.0 * R, 20.0 * R], [0.0, 0.5]], dtype=np.float32)
    A = np.eye(2, dtype=np.float32)
    beta = 0.2   # B = 105: 40 sure points, 240 possible
    assert 40 < oracle.budget(len(X), beta, k) <= 240
    pm.profile(True)
    pm.profile_read()
    got, ref = _run_both(X, Q, A, k=k, c=c, beta=beta, r_min=rmin, leaf=16, s=0, with_stats=False)
    prof = pm.profile_read()
    pm.profile(False)
    _assert_parity(got, ref, trace=False)
    assert "k_gather_sub" in prof and "k_band64" in prof, sorted(prof)
    full, _ = _run_both(X, Q, A, k=k, c=c, beta=beta, r_min=rmin, leaf=16, s=0)
    _assert_parity(full, ref)


@pytest.mark.slow
def test_c3_full_size_sampled_parity():
    # high-dimensional workload: n = 10^6, d = 960, anisotropic clusters;
    # all 1,000 queries on the GPU for three (c, k) settings, a query sample
    # against the oracle, and the statistics-free path against the full one
    w = datagen.workload("c3")
    X, Q = w["X"], w["Q"]
    A = oracle.gen_projection(2, 15, X.shape[1]).astype(np.float32)
    ix = pm.Index(torch.from_numpy(X).cuda(), proj=A, leaf_size=256)
    torch.cuda.synchronize()
    Qd = torch.from_numpy(Q).cuda()
    O = oracle.project(X, A)
    rng = np.random.default_rng(3)
    sample = np.sort(rng.choice(len(Q), size=12, replace=False))
    for c, k in ((1.2, 1), (1.5, 10), (2.0, 100)):
        got = ix.knn(Qd, k=k, c=c, beta=0.2809, precision=TENSOR)
        fast = ix.knn(Qd, k=k, c=c, beta=0.2809, with_stats=False)
        torch.cuda.synchronize()
        assert torch.equal(got["ids"], fast["ids"]) and torch.equal(got["dists"], fast["dists"])
        t, _, _ = oracle.params(15, c, 1 / E)
        ref = oracle.knn(X, A, Q[sample], k, c, t, oracle.budget(len(X), 0.2809, k),
                         oracle.rmin_auto(X, 0.2809, k, c, 3), 0, Oproj=O)
        sub = dict(ids=got["ids"][sample], dists=got["dists"][sample], err=got["err"][sample],
                   stats={k2: v[sample] for k2, v in got["stats"].items()})
        _assert_parity(sub, ref)
    ix.close()


def test_autotuned_leaf_size(c1):
    # leaf_size = 0: the build times each candidate capacity and keeps one;
    # results do not depend on the layout
    X, Q, A = c1
    ix = pm.Index(torch.from_numpy(X).cuda(), proj=A, leaf_size=0)
    assert ix.leaf_size in (128, 256, 512)
    t, _, _ = oracle.params(15, 1.5, 1 / E)
    ref = oracle.knn(X, A, Q, 10, 1.5, t, oracle.budget(len(X), 0.2809, 10),
                     oracle.rmin_auto(X, 0.2809, 10, 1.5, 3), 0)
    got = ix.knn(torch.from_numpy(Q).cuda(), k=10, t=t)
    _assert_parity(got, ref)
    ix.close()


# BF16 first-pass verification (PMLSH_BF16_VERIFY, and with the tensor-core
# count PMLSH_BF16_RERANK): BF16 residual rows bound each candidate's
# distance, the candidates that can reach the k-th upper bound are reranked
# from the FP32 rows, FP64 where FP32 cannot decide; ids, distances, error
# bounds and the trace equal the oracle's.
VERIFY = pm.PMLSH_BF16_VERIFY
RERANK = pm.PMLSH_BF16_RERANK


@pytest.mark.parametrize("precision", [VERIFY, RERANK])
@pytest.mark.parametrize("stop_rule", [0, 1])
def test_c1_parity_bf16_verify(c1, stop_rule, precision):
    X, Q, A = c1
    got, ref = _run_both(X, Q, A, k=10, stop_rule=stop_rule, precision=precision)
    _assert_parity(got, ref)


@pytest.mark.parametrize("n,d,m,leaf,s,k", [
    (1000 + 17, 37, 15, 64, 5, 7),
    (300, 8, 3, 16, 0, 1),
    (50, 20, 16, 64, 5, 50),
    (2500, 64, 15, 1024, 8, 20),
])
def test_shapes_and_edges_bf16_verify(n, d, m, leaf, s, k):
    X, Q, _, _ = datagen.mixture(n, d, 7, 1.0, seed=n, nq=33)
    A = oracle.gen_projection(11, m, d).astype(np.float32)
    for rmin in (None, 0.5):
        got, ref = _run_both(X, Q, A, k=k, leaf=leaf, s=s, r_min=rmin, beta=0.1, precision=VERIFY)
        _assert_parity(got, ref)


@pytest.mark.parametrize("n,d,m,leaf,s,k,nq", [
    (1, 4, 15, 16, 5, 1, 5),
    (700, 1, 1, 16, 3, 9, 40),
    (600, 24, 15, 64, 5, 256, 20),
])
def test_extreme_shapes_bf16_verify(n, d, m, leaf, s, k, nq):
    X, Q, _, _ = datagen.mixture(n, d, min(7, n), 1.0, seed=n + d, nq=nq)
    A = oracle.gen_projection(11, m, d).astype(np.float32)
    got, ref = _run_both(X, Q, A, k=k, leaf=leaf, s=s, beta=0.1, precision=RERANK)
    _assert_parity(got, ref)


def test_bf16_verify_duplicates_and_far_from_origin():
    # 40 copies of each of 25 points (ties 40 ways at every distance), and a
    # data set far from the origin (large residual rounding relative to the
    # distances): the first pass must hand such queries to the rerank, or
    # to the FP32 verification, without changing a result
    base, Q, _, _ = datagen.mixture(25, 16, 5, 1.0, seed=3, nq=20)
    X = np.repeat(base, 40, axis=0)
    A = oracle.gen_projection(5, 15, 16).astype(np.float32)
    for beta in (0.2809, 0.02):
        got, ref = _run_both(X, Q, A, k=30, beta=beta, leaf=32, precision=VERIFY)
        _assert_parity(got, ref)
    X, Q, _, _ = datagen.mixture(3000, 48, 6, 1.0, seed=8, nq=40)
    X = X + 1000.0
    Q = Q + 1000.0
    A = oracle.gen_projection(6, 15, 48).astype(np.float32)
    got, ref = _run_both(X, Q, A, k=10, precision=RERANK)
    _assert_parity(got, ref)


@pytest.mark.parametrize("kw", [
    dict(k=10),
    dict(k=10, r_min=200.0),
    dict(k=5, beta=0.01, r_min=2.0),
    dict(k=10, beta=1.0, r_min=400.0),
])
def test_no_stats_path_parity_bf16_verify(c1, kw):
    X, Q, A = c1
    got, ref = _run_both(X, Q[:64], A, precision=RERANK, with_stats=False, **kw)
    assert got.get("stats") is None
    _assert_parity(got, ref, trace=False)


@pytest.mark.slow
def test_c2_full_size_sampled_parity_bf16_verify():
    w = datagen.workload("c2")
    X, Q = w["X"], w["Q"]
    A = oracle.gen_projection(2, 15, 128).astype(np.float32)
    ix = pm.Index(torch.from_numpy(X).cuda(), proj=A, leaf_size=256)
    Qd = torch.from_numpy(Q).cuda()
    got = ix.knn(Qd, k=50, c=1.5, beta=0.2809, precision=RERANK)
    plain = ix.knn(Qd, k=50, c=1.5, beta=0.2809)
    fast = ix.knn(Qd, k=50, c=1.5, beta=0.2809, precision=RERANK, with_stats=False)
    torch.cuda.synchronize()
    ix.close()
    assert torch.equal(got["ids"], plain["ids"]) and torch.equal(got["dists"], plain["dists"])
    assert torch.equal(got["ids"], fast["ids"]) and torch.equal(got["dists"], fast["dists"])
    assert torch.equal(got["err"], fast["err"])
    for key in ("rounds", "rule", "ncand", "r"):
        assert np.array_equal(got["stats"][key], plain["stats"][key]), key
    rng = np.random.default_rng(2)
    sample = np.sort(rng.choice(len(Q), size=32, replace=False))
    t, _, _ = oracle.params(15, 1.5, 1 / E)
    ref = oracle.knn(X, A, Q[sample], 50, 1.5, t, oracle.budget(len(X), 0.2809, 50),
                     oracle.rmin_auto(X, 0.2809, 50, 1.5, 3), 0)
    sub = dict(ids=got["ids"][sample], dists=got["dists"][sample], err=got["err"][sample],
               stats={k2: v[sample] for k2, v in got["stats"].items()})
    _assert_parity(sub, ref)


@pytest.mark.slow
def test_c3_full_size_sampled_parity_bf16_verify():
    w = datagen.workload("c3")
    X, Q = w["X"], w["Q"]
    A = oracle.gen_projection(2, 15, X.shape[1]).astype(np.float32)
    ix = pm.Index(torch.from_numpy(X).cuda(), proj=A, leaf_size=256)
    Qd = torch.from_numpy(Q).cuda()
    O = oracle.project(X, A)
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(len(Q), size=10, replace=False))
    for c, k in ((1.2, 1), (1.5, 10), (2.0, 100)):
        got = ix.knn(Qd, k=k, c=c, beta=0.2809, precision=RERANK)
        plain = ix.knn(Qd, k=k, c=c, beta=0.2809, with_stats=False)
        torch.cuda.synchronize()
        assert torch.equal(got["ids"], plain["ids"]) and torch.equal(got["dists"], plain["dists"])
        t, _, _ = oracle.params(15, c, 1 / E)
        ref = oracle.knn(X, A, Q[sample], k, c, t, oracle.budget(len(X), 0.2809, k),
                         oracle.rmin_auto(X, 0.2809, k, c, 3), 0, Oproj=O)
        sub = dict(ids=got["ids"][sample], dists=got["dists"][sample], err=got["err"][sample],
                   stats={k2: v[sample] for k2, v in got["stats"].items()})
        _assert_parity(sub, ref)
    ix.close()


def test_bf16_verify_needs_the_residual_rows(c1):
    X, Q, A = c1
    ix = pm.Index(X, proj=A, bf16_shadow=False)
    with pytest.raises(pm.PmlshError):
        ix.knn(Q[:4], k=3, precision=VERIFY)
    ix.close()
