"""Pins for the FP64 oracle: each test ties an oracle function to something
other than itself -- a closed form, a value printed in the paper, a textbook
special case, an invariant of the method or brute force on tiny inputs."""
import math

import numpy as np
import pytest

import datagen
import oracle
from conftest import golden

E = math.e


# --------------------------------------------------------------- chi^2 / Eq. 9
def test_chi2_closed_form_m2():
    # chi^2(2) is exponential with mean 2: Pr[X > x] = exp(-x/2), so the
    # upper quantile is -2 ln(alpha) (Lemma 3 with m = 2).
    for x in (0.1, 1.0, 3.7, 12.0, 40.0):
        assert oracle.chi2_sf(x, 2) == pytest.approx(math.exp(-x / 2), rel=1e-13)
    for a in (0.9, 1 / E, 0.1, 1e-4):
        assert oracle.chi2_isf(a, 2) == pytest.approx(-2 * math.log(a), rel=1e-12)


def test_chi2_closed_form_m1_and_m4():
    # chi^2(1): Pr[X > x] = erfc(sqrt(x/2)); chi^2(4): exp(-x/2)(1 + x/2).
    for x in (0.01, 0.5, 2.0, 9.0, 30.0):
        assert oracle.chi2_sf(x, 1) == pytest.approx(math.erfc(math.sqrt(x / 2)), rel=1e-11)
        assert oracle.chi2_sf(x, 4) == pytest.approx(math.exp(-x / 2) * (1 + x / 2), rel=1e-12)


def test_chi2_against_scipy():
    st = pytest.importorskip("scipy.stats")
    for m in (3, 8, 15, 16, 40):
        for a in (0.9, 0.5, 1 / E, 0.05, 1e-3):
            assert oracle.chi2_isf(a, m) == pytest.approx(st.chi2.isf(a, m), rel=1e-10)


def test_eq9_printed_cp_alpha2():
    g = golden("params.json")
    t, a2, beta = oracle.params(g["m"], g["cp_c"], g["alpha1"])
    # the paper prints alpha2 = 0.0024 to four decimals
    assert round(a2, g["cp_alpha2_decimals"]) == g["cp_alpha2_printed"]
    assert beta == pytest.approx(2 * a2)
    # t^2 = chi^2_{1/e}(15); E1 of Lemma 4: Pr[r' > t r] = alpha1 exactly
    assert oracle.chi2_sf(t * t, 15) == pytest.approx(1 / E, rel=1e-12)
    # second line of Eq. 9: Pr[chi^2 > t^2/c^2] = 1 - alpha2
    assert oracle.chi2_sf(t * t / 4.0, 15) == pytest.approx(1 - a2, rel=1e-12)


def test_eq9_nn_printed_values_not_reproducible():
    # Recorded discrepancy: the printed alpha2 = 0.1405 at c = 1.5 does not
    # follow from Eq. 9 with m = 15, alpha1 = 1/e.
    g = golden("params.json")
    _, a2, _ = oracle.params(15, g["nn_printed"]["c"], g["alpha1"])
    assert abs(a2 - g["nn_printed"]["alpha2"]) > 0.05
    assert a2 == pytest.approx(0.04835, abs=5e-5)


def test_budget_integer_rounding():
    assert oracle.budget(10_000, 0.2809, 10) == 2819
    assert oracle.budget(1_000_000, 0.2809, 50) == 280_950
    assert oracle.budget(10, 0.4, 1) == 5          # Example 3: beta n = 4 -> 5
    assert oracle.budget(10, 0.45, 1) == 6         # ceil(4.5) + 1
    assert oracle.budget(3, 1.0, 2) == 5


# ------------------------------------------------ projection, Lemmas 1 - 3
def test_projection_entries_standard_normal():
    A = oracle.gen_projection(7, 16, 4096).ravel()
    assert abs(A.mean()) < 4 / math.sqrt(A.size)
    assert A.var() == pytest.approx(1.0, abs=0.03)
    # fourth moment of N(0,1) is 3 (uniform or Rademacher entries would fail)
    assert np.mean(A ** 4) == pytest.approx(3.0, abs=0.15)
    # deterministic in the seed, different across seeds
    assert np.array_equal(A, oracle.gen_projection(7, 16, 4096).ravel())
    assert not np.array_equal(A, oracle.gen_projection(8, 16, 4096).ravel())


def test_projection_identity_and_columns():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((50, 6)).astype(np.float32)
    O = oracle.project(X, np.eye(6, dtype=np.float32))
    assert np.array_equal(O, X.astype(np.float64))
    A = rng.standard_normal((4, 6)).astype(np.float32)
    O = oracle.project(np.eye(6, dtype=np.float32), A)
    assert np.array_equal(O, A.T.astype(np.float64))


def _ks_stat(samples, cdf):
    s = np.sort(samples)
    n = len(s)
    F = np.array([cdf(v) for v in s])
    return max(np.max(np.arange(1, n + 1) / n - F), np.max(F - np.arange(n) / n))


def test_lemma1_ratio_is_chi2():
    # Lemma 1: r'^2 / r^2 ~ chi^2(m) over random projections (m = 15).
    m, d, reps = 15, 32, 1500
    rng = np.random.default_rng(3)
    o1 = rng.standard_normal(d).astype(np.float32)
    o2 = rng.standard_normal(d).astype(np.float32)
    r2 = float(np.sum((o1.astype(np.float64) - o2) ** 2))
    ratios = []
    for s in range(reps):
        A = oracle.gen_projection(1000 + s, m, d).astype(np.float32)
        O = oracle.project(np.stack([o1, o2]), A)
        ratios.append(float(np.sum((O[0] - O[1]) ** 2)) / r2)
    ks = _ks_stat(np.array(ratios), lambda x: 1 - oracle.chi2_sf(x, m))
    assert ks < 1.63 / math.sqrt(reps)      # KS test at the 1% level
    # Lemma 2: r'^2/m is unbiased for r^2
    assert np.mean(ratios) / m == pytest.approx(1.0, abs=4 * math.sqrt(2 / m / reps))


def test_lemma3_tail_probabilities():
    # P2 of Lemma 3: Pr[r' > r sqrt(chi^2_alpha(m))] = alpha, checked with a
    # binomial 4-sigma band over many random point pairs and projections.
    m, d, reps, alpha = 15, 24, 4000, 1 / E
    rng = np.random.default_rng(5)
    A = oracle.gen_projection(11, m * reps, d).astype(np.float32).reshape(reps, m, d)
    P = rng.standard_normal((reps, 2, d)).astype(np.float32)
    hits = 0
    thr = math.sqrt(oracle.chi2_isf(alpha, m))
    lo_thr = math.sqrt(oracle.chi2_isf(1 - alpha / 3, m))
    lo_hits = 0
    for s in range(reps):
        O = oracle.project(P[s], A[s])
        rp = math.sqrt(float(np.sum((O[0] - O[1]) ** 2)))
        r = oracle.dist(P[s, 0], P[s, 1])
        hits += rp > r * thr
        lo_hits += rp < r * lo_thr          # P1 with alpha/3
    sd = math.sqrt(alpha * (1 - alpha) / reps)
    assert abs(hits / reps - alpha) < 4 * sd
    sd1 = math.sqrt(alpha / 3 * (1 - alpha / 3) / reps)
    assert abs(lo_hits / reps - alpha / 3) < 4 * sd1


# ----------------------------------------------------------- Algorithm 2
def test_example3_trace():
    g = golden("example3_knn.json")
    X = np.array(g["points"], dtype=np.float32)
    Q = np.array([g["q"]], dtype=np.float32)
    A = np.eye(2, dtype=np.float32)
    B = oracle.budget(len(X), g["beta"], g["k"])
    e = g["expect"]
    assert B == e["budget"]
    # the two range queries of the example
    O = oracle.project(X, A)
    pd = np.sqrt(np.sum(O ** 2, axis=1))
    for i, cnt in enumerate(e["range_counts"]):
        R = g["t"] * g["r_min"] * g["c"] ** i
        assert int(np.sum(pd <= R)) == cnt
    for stop_rule in (0, 1):
        r = oracle.knn(X, A, Q, g["k"], g["c"], g["t"], B, g["r_min"], stop_rule)
        assert r["rounds"][0] == e["rounds"]
        assert r["rule"][0] == e["rule"]
        assert r["ncand"][0] == e["ncand"]
        assert r["ids"][0].tolist() == e["ids"]
        assert r["dists"][0, 0] == pytest.approx(e["dist"], rel=1e-15)


def _c1_small(n=3000, nq=30, d=32, seed=0):
    X, Q, _, _ = datagen.mixture(n, d, 20, 1.0, seed=seed, nq=nq)
    return X, Q


def test_identity_projection_gives_exact_knn():
    # With A = I (m = d) projected and original distances coincide, so every
    # range set is an exact ball and every stop rule returns the exact top-k.
    X, Q = _c1_small(n=2000, nq=25, d=12)
    A = np.eye(12, dtype=np.float32)
    ei, ed = oracle.exact_knn(X, Q, 7)
    for beta, rmin in ((0.05, 0.5), (0.3, 3.0), (1.0, 0.2)):
        B = oracle.budget(len(X), beta, 7)
        for sr in (0, 1):
            r = oracle.knn(X, A, Q, 7, 1.5, 1.2, B, rmin, sr)
            assert np.array_equal(r["ids"], ei)
            assert np.array_equal(r["dists"], ed)


def test_whole_dataset_round_gives_exact_knn():
    # B > n and a first radius that covers every point: C = D (rule 3).
    X, Q = _c1_small()
    A = oracle.gen_projection(2, 15, X.shape[1]).astype(np.float32)
    t, _, _ = oracle.params(15, 1.5, 1 / E)
    ei, ed = oracle.exact_knn(X, Q, 10)
    r = oracle.knn(X, A, Q, 10, 1.5, t, oracle.budget(len(X), 1.0, 10), 1e6, 0)
    assert np.all(r["rule"] == 3) and np.all(r["ncand"] == len(X))
    assert np.array_equal(r["ids"], ei)


def test_knn_invariants():
    X, Q = _c1_small(n=4000, nq=40)
    A = oracle.gen_projection(2, 15, X.shape[1]).astype(np.float32)
    t, _, _ = oracle.params(15, 1.5, 1 / E)
    k, c = 10, 1.5
    B = oracle.budget(len(X), 0.2809, k)
    O = oracle.project(X, A)
    qp = oracle.project(Q, A)
    for rmin in (0.5, 2.0, oracle.rmin_auto(X, 0.2809, k, c, 3)):
        for sr in (0, 1):
            r = oracle.knn(X, A, Q, k, c, t, B, rmin, sr, Oproj=O)
            for qi in range(len(Q)):
                ids, dd = r["ids"][qi], r["dists"][qi]
                assert len(set(ids.tolist())) == k
                assert np.all(np.diff(dd) >= 0)
                # distances are the true distances of the returned ids
                for i, v in zip(ids[:3], dd[:3]):
                    assert v == oracle.dist(X[i], Q[qi])
                pd = np.sqrt(np.sum((O - qp[qi]) ** 2, axis=1))
                last_r = r["r"][qi] if not (sr == 0 and r["rule"][qi] == 1) else r["r"][qi] / c
                R = t * last_r
                S = np.flatnonzero(pd <= R)
                if r["rule"][qi] == 2:
                    assert r["ncand"][qi] == B and len(S) >= B
                else:
                    assert r["ncand"][qi] == len(S)
                    # rule 1: at least k verified points within c r
                    if r["rule"][qi] == 1:
                        assert np.sum(np.sqrt(np.sum((X[S].astype(np.float64) - Q[qi]) ** 2, axis=1)) <= c * r["r"][qi]) >= k
                # every returned id lies in the final range set
                assert set(ids.tolist()) <= set(S.tolist())
                # radius schedule r = r_min c^i
                assert r["r"][qi] == pytest.approx(rmin * c ** (r["rounds"][qi] - (sr == 1 or r["rule"][qi] != 1)), rel=1e-12)


def test_candidate_nesting_and_budget_selection():
    # Rule 2 keeps the B nearest in projected space (ties by id): they must
    # contain every point of the previous (smaller) range set.
    X, Q = _c1_small(n=3000, nq=10)
    A = oracle.gen_projection(9, 15, X.shape[1]).astype(np.float32)
    t = 4.0
    O = oracle.project(X, A)
    qp = oracle.project(Q, A)
    B = 400
    r = oracle.knn(X, A, Q, 5, 1.5, t, B, 0.3, 0, Oproj=O)
    for qi in range(len(Q)):
        if r["rule"][qi] != 2:
            continue
        pd = np.sqrt(np.sum((O - qp[qi]) ** 2, axis=1))
        order = np.lexsort((np.arange(len(X)), pd))[:B]
        prev = np.flatnonzero(pd <= t * r["r"][qi] / 1.5)
        assert set(prev.tolist()) <= set(order.tolist())
        ex = np.sqrt(np.sum((X[order].astype(np.float64) - Q[qi]) ** 2, axis=1))
        best = order[np.lexsort((order, ex))[:5]]
        assert r["ids"][qi].tolist() == best.tolist()


def test_duplicates_tie_break_by_id():
    X = np.zeros((50, 4), dtype=np.float32)
    X[:, 0] = np.repeat(np.arange(5), 10).astype(np.float32)
    Q = np.array([[2.0, 0, 0, 0]], dtype=np.float32)
    A = oracle.gen_projection(1, 4, 4).astype(np.float32)
    r = oracle.knn(X, A, Q, 15, 2.0, 3.0, oracle.budget(50, 0.5, 15), 0.5, 0)
    assert r["ids"][0].tolist() == list(range(20, 30)) + list(range(10, 15))


def test_theorem1_success_rate():
    # Theorem 1: a c^2-ANN answer with probability >= 1/2 - 1/e.
    X, Q = _c1_small(n=3000, nq=60)
    A = oracle.gen_projection(2, 15, X.shape[1]).astype(np.float32)
    t, a2, _ = oracle.params(15, 1.5, 1 / E)
    B = oracle.budget(len(X), 2 * a2, 1)
    r = oracle.knn(X, A, Q, 1, 1.5, t, B, oracle.rmin_auto(X, 2 * a2, 1, 1.5, 3), 0)
    _, ed = oracle.exact_knn(X, Q, 1)
    ok = np.mean(r["dists"][:, 0] <= 1.5 ** 2 * ed[:, 0])
    assert ok >= 0.5 - 1 / E


def test_rmin_rule_quantile():
    # two points: every sampled pair is that pair, so r* is their distance
    X = np.array([[0, 0, 0], [3, 4, 0]], dtype=np.float32)
    assert oracle.rmin_auto(X, 0.3, 1, 1.5, 9, 100) == pytest.approx(5.0 / 1.5)
    # identical points: fallback 1.0
    assert oracle.rmin_auto(np.ones((5, 3), np.float32), 0.3, 1, 1.5, 9, 100) == 1.0
    # 1-D points 0..99: quantile of sampled |i - j| at p = (beta n + k)/n
    X = np.arange(100, dtype=np.float32)[:, None]
    v = oracle.rmin_auto(X, 0.5, 0, 2.0, 4, 20000)
    # |i-j| for i,j uniform on 0..99 has median close to 29
    assert 27 / 2 <= v <= 31 / 2


# ----------------------------------------------------------- Algorithm 1
def test_rcbc_with_identity_projection():
    X, Q = _c1_small(n=1500, nq=20, d=8)
    A = np.eye(8, dtype=np.float32)
    ei, ed = oracle.exact_knn(X, Q, 1)
    for r in (0.5, 2.0, 5.0):
        ids, dd, nc = oracle.rcbc(X, A, Q, r, 2.0, 1.0, 10 ** 9)
        for qi in range(len(Q)):
            if ed[qi, 0] <= r:           # B(q, r) covers a point: returned
                assert ids[qi] == ei[qi, 0]
            if ed[qi, 0] > 2.0 * r:      # B(q, c r) empty: nothing
                assert ids[qi] == -1


# ----------------------------------------------------- brute force / CP
def test_exact_knn_brute_force():
    X, Q = _c1_small(n=500, nq=10, d=5)
    ids, dd = oracle.exact_knn(X, Q, 6)
    for qi in range(len(Q)):
        dv = np.sqrt(((X.astype(np.float64) - Q[qi].astype(np.float64)) ** 2).sum(1))
        order = np.lexsort((np.arange(len(X)), dv))[:6]
        assert ids[qi].tolist() == order.tolist()
        assert np.allclose(dd[qi], dv[order], rtol=1e-14)


def test_exact_kcp_brute_force():
    X = datagen.gaussian(120, 4, seed=3)
    pairs, dd = oracle.exact_kcp(X, 9)
    Xd = X.astype(np.float64)
    allp = [(np.sqrt(((Xd[i] - Xd[j]) ** 2).sum()), i, j)
            for i in range(len(X)) for j in range(i + 1, len(X))]
    allp.sort()
    assert [[i, j] for _, i, j in allp[:9]] == pairs.tolist()
    assert np.allclose(dd, [v for v, _, _ in allp[:9]], rtol=1e-14)


def test_cp_example_of_algorithm4():
    g = golden("cp_example.json")
    X = np.array(g["points"], dtype=np.float32)
    A = np.eye(2, dtype=np.float32)
    e = g["expect"]
    r = oracle.cp_radius_filter(X, A, g["layout"], g["k"], g["t"], g["gamma"], g["T"])
    assert r["pairs"].tolist() == e["pairs"]
    assert r["dists"].tolist() == e["dists"]
    assert r["ub_self"] == e["ub_self"]
    assert g["gamma"] * g["t"] * r["ub_self"] == e["R"]
    assert r["nodes"] == e["lca_nodes"]
    assert r["count"] == e["count"]
    i, j = e["skipped_pair"]
    assert oracle.dist(X[i], X[j]) == pytest.approx(e["skipped_pair_pd"])


def _bisect_layout(X, leaf):
    """A hierarchy for tests: recursive median split on coordinate 0 / 1."""
    n = len(X)
    perm = np.argsort(X[:, 0], kind="stable")
    leaf_off = list(range(0, n, leaf)) + [n]
    L = len(leaf_off) - 1
    nodes = []

    def mk(lo, hi):
        idx = len(nodes)
        nodes.append([lo, hi, -1, -1])
        if hi - lo > 1:
            mid = (lo + hi) // 2
            nodes[idx][2] = mk(lo, mid)
            nodes[idx][3] = mk(mid, hi)
        return idx
    mk(0, L)
    nd = np.array(nodes)
    return dict(perm=perm, leaf_off=np.array(leaf_off), node_lo=nd[:, 0],
                node_hi=nd[:, 1], node_left=nd[:, 2], node_right=nd[:, 3])


def test_cp_all_pairs_budget_is_exact_kcp():
    # T >= n(n-1)/2, gamma = inf and a t so large that every pair passes the
    # projected filter: every cross-leaf pair is examined, so the answer is
    # the exact k closest pairs (the NLJ result).
    X = datagen.gaussian(150, 6, seed=5)
    A = oracle.gen_projection(3, 4, 6).astype(np.float32)
    lay = _bisect_layout(X, 8)
    r = oracle.cp_radius_filter(X, A, lay, 12, 1e6, math.inf, 150 * 149 // 2)
    ep, ed = oracle.exact_kcp(X, 12)
    assert r["pairs"].tolist() == ep.tolist()
    assert np.array_equal(r["dists"], ed)


def test_cp_node_ball_covers():
    X = datagen.gaussian(300, 5, seed=6)
    A = oracle.gen_projection(3, 5, 5).astype(np.float32)
    O = oracle.project(X, A)
    perm = np.random.default_rng(0).permutation(300).astype(np.int32)
    ro, rad = oracle.node_ball(O, perm, 10, 90)
    dd = np.sqrt(((O[perm[10:90]] - ro) ** 2).sum(1))
    assert np.max(dd) == rad
    assert np.allclose(ro, 0.5 * (O[perm[10:90]].min(0) + O[perm[10:90]].max(0)))


def test_metrics_eq11_eq12():
    assert oracle.overall_ratio([[1.0, 2.0]], [[1.0, 1.0]]) == 1.5
    assert oracle.recall([[1, 2, 3]], [[3, 4, 1]]) == pytest.approx(2 / 3)


def test_stop_rule_placement_readings():
    # Identity projection, t = 2, c = 1.5, r_min = 1, k = 1: the only point of
    # the first range set lies at 1.8, inside c^2 r but outside c r.  As
    # printed, rule 1 is tested at the loop top after r <- c r and fires
    # before a second range query; the Algorithm-1 form tests c r of the same
    # round, fails, and runs a second range query first.
    X = np.array([[1.8, 0], [0, 2.5], [-4, 0], [0, -6]], dtype=np.float32)
    Q = np.zeros((1, 2), dtype=np.float32)
    A = np.eye(2, dtype=np.float32)
    lit = oracle.knn(X, A, Q, 1, 1.5, 2.0, 100, 1.0, 0)
    bc = oracle.knn(X, A, Q, 1, 1.5, 2.0, 100, 1.0, 1)
    assert (lit["rounds"][0], lit["rule"][0], lit["ncand"][0]) == (1, 1, 1)
    assert (bc["rounds"][0], bc["rule"][0], bc["ncand"][0]) == (2, 1, 2)
    assert lit["ids"][0, 0] == bc["ids"][0, 0] == 0


# ------------------------------------------------- Algorithm 3 (B&B CP)
def test_cp_bnb_all_pairs_is_exact_kcp():
    # T >= n(n-1)/2 keeps every pair: the verified top-k is the exact kCP
    X, _ = _c1_small(n=300, nq=1, d=16)
    A = oracle.gen_projection(2, 15, 16).astype(np.float32)
    pb, db = oracle.cp_bnb(X, A, 10 ** 9, 7)
    pe, de = oracle.exact_kcp(X, 7)
    assert np.array_equal(pb, pe) and np.array_equal(db, de)


def test_cp_bnb_identity_projection_is_exact_kcp():
    # A = I (m = d): projected and original distances coincide, so the T
    # nearest projected pairs hold the exact k nearest for any T >= k
    X, _ = _c1_small(n=400, nq=1, d=8)
    A = np.eye(8, dtype=np.float32)
    pe, de = oracle.exact_kcp(X, 5)
    for T in (5, 6, 50):
        pb, db = oracle.cp_bnb(X, A, T, 5)
        assert np.array_equal(pb, pe) and np.array_equal(db, de)


def test_cp_bnb_against_numpy_brute_force():
    # an independent brute force: all pair distances in the projected space
    # (numpy, FP64), the T smallest by (distance, i, j), then the k smallest
    # original distances among them
    X, _ = _c1_small(n=250, nq=1, d=24)
    A = oracle.gen_projection(7, 15, 24).astype(np.float32)
    O = A.astype(np.float64) @ X.astype(np.float64).T
    i, j = np.triu_indices(len(X), 1)
    pd = np.sqrt(((O[:, i] - O[:, j]) ** 2).sum(0))
    T, k = 40, 6
    sel = np.lexsort((j, i, pd))[:T]
    od = np.sqrt(((X[i[sel]].astype(np.float64) - X[j[sel]].astype(np.float64)) ** 2).sum(1))
    top = np.lexsort((j[sel], i[sel], od))[:k]
    pb, db = oracle.cp_bnb(X, A, T, k)
    assert np.array_equal(pb, np.stack([i[sel][top], j[sel][top]], 1))
    assert np.allclose(db, od[top], rtol=1e-12, atol=0)


# ------------------------------------------------- cost model (Sec. 4.2)
def test_cost_model_hand_example():
    # Two nodes, two pivots, F the empirical CDF of {1..8}: values worked by
    # hand from Pr[e] and CC (tests/golden/cost_model_example.json), exact
    # binary fractions; the second radius puts arguments on sample values.
    g = golden("cost_model_example.json")
    for c in g["cases"]:
        cc, en = oracle.cost_model(g["F_sample"], g["count"], g["radius"], g["hr_min"], g["hr_max"], c["rq"])
        assert cc == c["cc"] and en == c["expected_nodes"]


def test_cost_model_unbounded_radius_accesses_every_node():
    # r_q beyond every distance: each factor of Pr[e] is 1 - 0 or 1, so every
    # node is accessed and CC = sum N(e) = n.
    rng = np.random.default_rng(3)
    F = np.sort(rng.uniform(0, 10, 500))
    cnt = rng.integers(1, 300, 40)
    rad = rng.uniform(0, 3, 40)
    lo = rng.uniform(0, 5, (40, 4))
    hi = lo + rng.uniform(0, 5, (40, 4))
    cc, en = oracle.cost_model(F, cnt, rad, lo, hi, 1e6)
    assert cc == float(cnt.sum()) and en == 40.0


def test_cost_model_point_nodes_without_pivots():
    # s = 0 and nodes of radius 0: Pr[e] = F(r_q), CC = n F(r_q); F from
    # numpy's sorted search (the empirical CDF counts samples <= x).
    rng = np.random.default_rng(4)
    F = np.sort(rng.exponential(2.0, 1000))
    cnt = rng.integers(1, 50, 30)
    n = int(cnt.sum())
    for rq in (0.0, 0.3, F[17], 1.9, F[999], 50.0):
        cc, en = oracle.cost_model(F, cnt, np.zeros(30), np.zeros((30, 0)), np.zeros((30, 0)), rq)
        Fq = np.searchsorted(F, rq, side="right") / len(F)
        assert cc == pytest.approx(n * Fq, rel=1e-14) and en == pytest.approx(30 * Fq, rel=1e-14)


def test_cost_model_single_point_nodes_equal_brute_force_range_count():
    # With one point per node, no pivots and F taken over all ordered pairs
    # (i != j), CC = n F(r_q) = n/(n-1) times the mean number of other points
    # within r_q of a query drawn from D: brute force over all pairs.
    rng = np.random.default_rng(5)
    O = rng.normal(size=(60, 5))
    D = np.sqrt(((O[:, None, :] - O[None, :, :]) ** 2).sum(-1))
    off = D[~np.eye(60, dtype=bool)]
    F = np.sort(off)
    for rq in (0.5, 1.5, 2.5, 4.0):
        cc, _ = oracle.cost_model(F, np.ones(60, dtype=np.int64), np.zeros(60), np.zeros((60, 0)),
                                  np.zeros((60, 0)), rq)
        mean_count = ((D <= rq).sum(1) - 1).mean()
        assert cc == pytest.approx(60 / 59 * mean_count, rel=1e-12)


def test_distance_sample_two_points_and_brute_force():
    # two points at distance 5: every sampled pair is (0, 1) or (1, 0)
    O = np.array([[0.0, 0.0], [3.0, 4.0]])
    v = oracle.distance_sample(O, 200, 11)
    assert np.all(v == 5.0)
    # the sampled pairs recomputed with numpy norms, sorted
    rng = np.random.default_rng(6)
    O = rng.normal(size=(97, 15)) * 10
    npairs, seed = 3000, 21
    v = oracle.distance_sample(O, npairs, seed)
    ref = []
    for s in range(npairs):
        i = oracle.splitmix64(seed, 2 * s) % 97
        j = oracle.splitmix64(seed, 2 * s + 1) % 97
        if j == i:
            j = (j + 1) % 97
        ref.append(np.linalg.norm(O[i] - O[j]))
    assert np.all(np.diff(v) >= 0)
    np.testing.assert_allclose(v, np.sort(ref), rtol=1e-13)


def test_splitmix64_published_outputs():
    # the first three outputs of SplitMix64 (Steele, Lea, Flood, OOPSLA 2014)
    # from state 0, as published with its reference implementation
    assert [oracle.splitmix64(0, i) for i in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_cp_budget_cut_inside_a_node_hand_counted():
    # Algorithm 4's budget T reached inside a node (reading: the node's
    # candidates are cut to the T + 1 - count smallest by (projected
    # distance, i, j)); the projection onto the first coordinate makes the
    # kept and the dropped pairs change the answer
    g = golden("cp_tcut_example.json")
    X = np.array(g["points"], dtype=np.float32)
    A = np.array(g["proj"], dtype=np.float32)
    for case in g["cases"]:
        r = oracle.cp_radius_filter(X, A, g["layout"], g["k"], g["t"], g["gamma"], case["T"])
        assert r["pairs"].tolist() == case["pairs"]
        assert r["dists"].tolist() == [math.sqrt(v) for v in case["dists_sq"]]
        assert r["count"] == case["count"]
        assert r["ub_self"] == math.sqrt(g["ub_self_sq"])
        assert r["nodes"] == 1 and r["nodes_done"] == 1


def test_gamma_hand_worked_example():
    # Sec. 6.3: gamma with Pr(gamma) = p for the ratio of the LCA radius to
    # the projected distance, on a hand-worked three-leaf hierarchy
    g = golden("gamma_example.json")
    O = np.array(g["coords"], dtype=np.float64)[:, None]
    lay = g["layout"]
    for e, r in enumerate(g["radii"]):
        lo, hi = lay["leaf_off"][lay["node_lo"][e]], lay["leaf_off"][lay["node_hi"][e]]
        assert oracle.node_ball(O, lay["perm"], lo, hi)[1] == r
    for p, want in g["expect"]:
        assert oracle.gamma_calibrate(O, lay, p) == want


def _numpy_gamma(O, lay, p):
    # independent restatement: node balls from numpy, the lowest common node
    # as the node with the fewest leaves whose range holds both leaves
    perm = np.asarray(lay["perm"])
    loff = np.asarray(lay["leaf_off"])
    nlo, nhi = np.asarray(lay["node_lo"]), np.asarray(lay["node_hi"])
    rad = []
    for e in range(len(nlo)):
        P = O[perm[loff[nlo[e]]:loff[nhi[e]]]]
        c = 0.5 * (P.min(0) + P.max(0))
        rad.append(np.sqrt(((P - c) ** 2).sum(1)).max())
    leaf_of = np.searchsorted(loff, np.arange(len(perm)), side="right") - 1
    ratios = []
    for a in range(len(perm)):
        for b in range(a + 1, len(perm)):
            la, lb = leaf_of[a], leaf_of[b]
            holds = [e for e in range(len(nlo)) if nlo[e] <= min(la, lb) and max(la, lb) < nhi[e]]
            e = min(holds, key=lambda x: (nhi[x] - nlo[x], x))
            dv = np.sqrt(((O[perm[a]] - O[perm[b]]) ** 2).sum())
            ratios.append(rad[e] / dv if dv > 0 else (np.inf if rad[e] > 0 else 0.0))
    return float(np.quantile(np.array(ratios), p, method="inverted_cdf")), np.array(ratios)


@pytest.mark.parametrize("seed,n,leaf", [(1, 40, 4), (2, 57, 6), (3, 33, 33)])
def test_gamma_against_numpy_brute_force(seed, n, leaf):
    X = datagen.gaussian(n, 7, seed=seed)
    A = oracle.gen_projection(seed, 3, 7).astype(np.float32)
    O = oracle.project(X, A)
    lay = _bisect_layout(X, leaf)
    for p in (0.85, 0.5, 0.97, 1.0):
        want, ratios = _numpy_gamma(O, lay, p)
        got = oracle.gamma_calibrate(O, lay, p)
        assert got == pytest.approx(want, rel=1e-12)
        # a node's ball holds both points, so their distance is at most 2R
        assert ratios.min() >= 0.5 * (1 - 1e-12) and got >= 0.5 * (1 - 1e-12)


def test_gamma_coincident_projections():
    # R / 0: +inf for a node of positive radius, 0 for a zero-radius node
    O = np.array([[1.0], [1.0], [4.0], [4.0]])
    lay = dict(perm=[0, 1, 2, 3], leaf_off=[0, 2, 4], node_lo=[0, 0, 1], node_hi=[2, 1, 2],
               node_left=[1, -1, -1], node_right=[2, -1, -1])
    # pairs: two zero-radius leaves (ratio 0 each), four cross pairs at
    # distance 3 under the root of radius 1.5 (ratio 0.5 each)
    assert oracle.gamma_calibrate(O, lay, 2 / 6) == 0.0
    assert oracle.gamma_calibrate(O, lay, 1.0) == 0.5
    lay1 = dict(perm=[0, 1, 2, 3], leaf_off=[0, 4], node_lo=[0], node_hi=[1],
                node_left=[-1], node_right=[-1])
    assert oracle.gamma_calibrate(O, lay1, 1.0) == math.inf


def test_gamma_sample_ids():
    for n, np_ in ((100, 10), (37, 37), (20, 50), (1000, 999)):
        ids = oracle.gamma_sample(n, np_, 11)
        assert len(ids) == min(n, np_)
        assert np.all(np.diff(ids) > 0) and ids[0] >= 0 and ids[-1] < n
    assert oracle.gamma_sample(37, 100, 5).tolist() == list(range(37))
    # the first draw of the shuffle: entry 0 swaps with v_0 mod n
    v0 = oracle.splitmix64(11, 0) % 100
    assert v0 in oracle.gamma_sample(100, 1, 11).tolist()
