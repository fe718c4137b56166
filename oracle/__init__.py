"""FP64 CPU oracle for PM-LSH (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does: the
oracle and the CUDA path share no code.

This module is a ctypes wrapper over ``pmlsh_oracle.c`` (plain C, FP64); see
that file for the arithmetic and the paper passage each function follows.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmlsh_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle with gcc (FP contraction off, OpenMP when present)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", _SRC, "-o", _OUT + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_OUT + ".tmp", _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_OUT)
        d, i64, i32, u64, p = (ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                               ctypes.c_uint64, ctypes.c_void_p)
        L.orc_splitmix64.restype = u64
        L.orc_splitmix64.argtypes = [u64, u64]
        L.orc_gen_projection.argtypes = [u64, i32, i32, p]
        L.orc_chi2_sf.restype = d
        L.orc_chi2_sf.argtypes = [d, i32]
        L.orc_chi2_isf.restype = d
        L.orc_chi2_isf.argtypes = [d, i32]
        L.orc_params.argtypes = [i32, d, d, p, p, p]
        L.orc_budget.restype = i64
        L.orc_budget.argtypes = [i64, d, i64]
        L.orc_project.argtypes = [p, i64, i32, p, i32, p]
        L.orc_dist.restype = d
        L.orc_dist.argtypes = [p, p, i32]
        L.orc_pdist.restype = d
        L.orc_pdist.argtypes = [p, p, i32]
        L.orc_rmin_auto.restype = d
        L.orc_rmin_auto.argtypes = [p, i64, i32, d, i64, d, u64, i64]
        L.orc_knn.restype = i32
        L.orc_knn.argtypes = [p, p, i64, i32, p, i32, p, i64, i64, d, d, i64,
                              p, i32, p, p, p, p, p, p]
        L.orc_rcbc.restype = i32
        L.orc_rcbc.argtypes = [p, p, i64, i32, p, i32, p, i64, d, d, d, i64,
                               p, p, p]
        L.orc_exact_knn.restype = i32
        L.orc_exact_knn.argtypes = [p, i64, i32, p, i64, i64, p, p]
        L.orc_cp_bnb.restype = i32
        L.orc_cp_bnb.argtypes = [p, p, i64, i32, i32, i64, i64, p, p]
        L.orc_exact_kcp.restype = i32
        L.orc_exact_kcp.argtypes = [p, i64, i32, i64, p, p]
        L.orc_node_ball.argtypes = [p, i32, p, i64, i64, p, p]
        L.orc_distance_sample.argtypes = [p, i64, i32, u64, i64, p]
        L.orc_cost_model.argtypes = [p, i64, i64, p, p, i32, p, p, d, p]
        L.orc_cost_model.restype = d
        L.orc_cp_radius_filter.restype = i32
        L.orc_cp_radius_filter.argtypes = [p, p, i64, i32, i32, p, p, i64,
                                           p, p, p, p, i64, i64, d, d, i64,
                                           p, p, p, p, p, p]
        L.orc_gamma_sample.restype = i64
        L.orc_gamma_sample.argtypes = [i64, i64, u64, p]
        L.orc_gamma_calibrate.restype = i32
        L.orc_gamma_calibrate.argtypes = [p, i64, i32, p, p, i64, p, p, p, p, i64, d, p]
        L.orc_num_threads.restype = i32
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def num_threads():
    return lib().orc_num_threads()


def splitmix64(seed, i):
    return lib().orc_splitmix64(seed, i)


def gen_projection(seed, m, d):
    """Sec. 3.2 / Eq. 3: FP64 Gaussian projection [m, d] from the seed."""
    A = np.empty((m, d), dtype=np.float64)
    lib().orc_gen_projection(seed, m, d, _ptr(A))
    return A


def chi2_sf(x, m):
    return lib().orc_chi2_sf(float(x), int(m))


def chi2_isf(alpha, m):
    """Lemma 3: upper quantile chi^2_alpha(m)."""
    return lib().orc_chi2_isf(float(alpha), int(m))


def params(m, c, alpha1):
    """Eq. 9: returns (t, alpha2, beta = 2 alpha2)."""
    t, a2, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_params(m, c, alpha1, ctypes.byref(t), ctypes.byref(a2),
                     ctypes.byref(b))
    return t.value, a2.value, b.value


def budget(n, beta, k):
    return lib().orc_budget(n, beta, k)


def project(X, A32):
    """Eq. 3: FP64 projected coordinates [n, m] with the FP32 matrix A32."""
    X, A32 = _f32(X), _f32(A32)
    n, d = X.shape
    m = A32.shape[0]
    out = np.empty((n, m), dtype=np.float64)
    lib().orc_project(_ptr(X), n, d, _ptr(A32), m, _ptr(out))
    return out


def dist(x, y):
    x, y = _f32(x), _f32(y)
    return lib().orc_dist(_ptr(x), _ptr(y), x.shape[0])


def rmin_auto(X, beta, k, c, seed, npairs=10000):
    """Sec. 5.2 r_min rule (reading: r* = lower F-hat quantile, r_min = r*/c)."""
    X = _f32(X)
    n, d = X.shape
    return lib().orc_rmin_auto(_ptr(X), n, d, beta, k, c, seed, npairs)


def knn(X, A32, Q, k, c, t, B, rmin, stop_rule=0, Oproj=None):
    """Algorithm 2.  Returns dict of ids, dists (FP64), rounds, rule, ncand, r."""
    X, A32, Q = _f32(X), _f32(A32), _f32(Q)
    n, d = X.shape
    m = A32.shape[0]
    nq = Q.shape[0]
    if Oproj is None:
        Oproj = project(X, A32)
    Oproj = np.ascontiguousarray(Oproj, dtype=np.float64)
    rm = np.broadcast_to(np.asarray(rmin, dtype=np.float64), (nq,)).copy()
    ids = np.empty((nq, k), dtype=np.int64)
    dists = np.empty((nq, k), dtype=np.float64)
    rounds = np.empty(nq, dtype=np.int32)
    rule = np.empty(nq, dtype=np.int32)
    ncand = np.empty(nq, dtype=np.int64)
    rfin = np.empty(nq, dtype=np.float64)
    rc = lib().orc_knn(_ptr(X), _ptr(Oproj), n, d, _ptr(A32), m, _ptr(Q), nq,
                       k, c, t, B, _ptr(rm), stop_rule, _ptr(ids), _ptr(dists),
                       _ptr(rounds), _ptr(rule), _ptr(ncand), _ptr(rfin))
    if rc != 0:
        raise ValueError("orc_knn rejected its arguments (%d)" % rc)
    return dict(ids=ids, dists=dists, rounds=rounds, rule=rule, ncand=ncand,
                r=rfin)


def rcbc(X, A32, Q, r, c, t, Bbc, Oproj=None):
    """Algorithm 1 for one radius r: returns (id or -1, dist, |C|) per query."""
    X, A32, Q = _f32(X), _f32(A32), _f32(Q)
    n, d = X.shape
    m = A32.shape[0]
    nq = Q.shape[0]
    if Oproj is None:
        Oproj = project(X, A32)
    Oproj = np.ascontiguousarray(Oproj, dtype=np.float64)
    ids = np.empty(nq, dtype=np.int64)
    dd = np.empty(nq, dtype=np.float64)
    nc = np.empty(nq, dtype=np.int64)
    lib().orc_rcbc(_ptr(X), _ptr(Oproj), n, d, _ptr(A32), m, _ptr(Q), nq,
                   r, c, t, Bbc, _ptr(ids), _ptr(dd), _ptr(nc))
    return ids, dd, nc


def cp_bnb(X, A32, T, k, Oproj=None):
    """Algorithm 3: the T pairs nearest in the projected space, verified;
    returns (pairs [k,2] int64 with i < j, FP64 distances [k])."""
    X, A32 = _f32(X), _f32(A32)
    n, d = X.shape
    m = A32.shape[0]
    if Oproj is None:
        Oproj = project(X, A32)
    Oproj = np.ascontiguousarray(Oproj, dtype=np.float64)
    pairs = np.empty((k, 2), dtype=np.int64)
    dd = np.empty(k, dtype=np.float64)
    if lib().orc_cp_bnb(_ptr(X), _ptr(Oproj), n, d, m, int(T), int(k), _ptr(pairs), _ptr(dd)):
        raise ValueError("bad arguments")
    return pairs, dd


def exact_knn(X, Q, k):
    X, Q = _f32(X), _f32(Q)
    n, d = X.shape
    nq = Q.shape[0]
    ids = np.empty((nq, k), dtype=np.int64)
    dists = np.empty((nq, k), dtype=np.float64)
    if lib().orc_exact_knn(_ptr(X), n, d, _ptr(Q), nq, k, _ptr(ids), _ptr(dists)):
        raise ValueError("bad k")
    return ids, dists


def exact_kcp(X, k):
    X = _f32(X)
    n, d = X.shape
    pairs = np.empty((k, 2), dtype=np.int64)
    dists = np.empty(k, dtype=np.float64)
    if lib().orc_exact_kcp(_ptr(X), n, d, k, _ptr(pairs), _ptr(dists)):
        raise ValueError("bad k")
    return pairs, dists


def node_ball(Oproj, perm, lo, hi):
    Oproj = np.ascontiguousarray(Oproj, dtype=np.float64)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    m = Oproj.shape[1]
    ro = np.empty(m, dtype=np.float64)
    rad = ctypes.c_double()
    lib().orc_node_ball(_ptr(Oproj), m, _ptr(perm), lo, hi, _ptr(ro),
                        ctypes.byref(rad))
    return ro, rad.value


def cp_radius_filter(X, A32, layout, k, t, gamma, T, Oproj=None):
    """Algorithm 4 on the hierarchy `layout` (dict with perm, leaf_off,
    node_lo, node_hi, node_left, node_right).  Returns dict."""
    X, A32 = _f32(X), _f32(A32)
    n, d = X.shape
    m = A32.shape[0]
    if Oproj is None:
        Oproj = project(X, A32)
    Oproj = np.ascontiguousarray(Oproj, dtype=np.float64)
    perm = np.ascontiguousarray(layout["perm"], dtype=np.int32)
    loff = np.ascontiguousarray(layout["leaf_off"], dtype=np.int64)
    nlo = np.ascontiguousarray(layout["node_lo"], dtype=np.int64)
    nhi = np.ascontiguousarray(layout["node_hi"], dtype=np.int64)
    nl = np.ascontiguousarray(layout["node_left"], dtype=np.int32)
    nr = np.ascontiguousarray(layout["node_right"], dtype=np.int32)
    L = loff.shape[0] - 1
    nn = nlo.shape[0]
    pairs = np.empty((k, 2), dtype=np.int64)
    dists = np.empty(k, dtype=np.float64)
    cnt, ubs, nodes, done = (ctypes.c_int64(), ctypes.c_double(),
                             ctypes.c_int64(), ctypes.c_int64())
    rc = lib().orc_cp_radius_filter(
        _ptr(X), _ptr(Oproj), n, d, m, _ptr(perm), _ptr(loff), L, _ptr(nlo),
        _ptr(nhi), _ptr(nl), _ptr(nr), nn, k, t, gamma, T, _ptr(pairs),
        _ptr(dists), ctypes.byref(cnt), ctypes.byref(ubs), ctypes.byref(nodes),
        ctypes.byref(done))
    if rc != 0:
        raise ValueError("orc_cp_radius_filter rejected its arguments")
    return dict(pairs=pairs, dists=dists, count=cnt.value, ub_self=ubs.value,
                nodes=nodes.value, nodes_done=done.value)


def gamma_sample(n, nprime, seed):
    """Sec. 6.3 sample: the sorted ids of min(nprime, n) distinct points
    (partial Fisher-Yates shuffle driven by the SplitMix64 stream `seed`)."""
    ids = np.empty(max(1, min(int(nprime), int(n))), dtype=np.int64)
    k = lib().orc_gamma_sample(int(n), int(nprime), seed, _ptr(ids))
    return ids[:k]


def gamma_calibrate(Oproj, layout, pr=0.85):
    """Sec. 6.3: gamma = lower empirical pr-quantile of R_LCA / ||o1', o2'||
    over all pairs of the points of `layout` (Oproj indexed by point id)."""
    Oproj = np.ascontiguousarray(Oproj, dtype=np.float64)
    n, m = Oproj.shape
    perm = np.ascontiguousarray(layout["perm"], dtype=np.int32)
    loff = np.ascontiguousarray(layout["leaf_off"], dtype=np.int64)
    nlo = np.ascontiguousarray(layout["node_lo"], dtype=np.int64)
    nhi = np.ascontiguousarray(layout["node_hi"], dtype=np.int64)
    nl = np.ascontiguousarray(layout["node_left"], dtype=np.int32)
    nr = np.ascontiguousarray(layout["node_right"], dtype=np.int32)
    g = ctypes.c_double()
    rc = lib().orc_gamma_calibrate(_ptr(Oproj), n, m, _ptr(perm), _ptr(loff), loff.shape[0] - 1,
                                   _ptr(nlo), _ptr(nhi), _ptr(nl), _ptr(nr), nlo.shape[0],
                                   float(pr), ctypes.byref(g))
    if rc != 0:
        raise ValueError("orc_gamma_calibrate rejected its arguments")
    return g.value


def distance_sample(Oproj, npairs, seed):
    """Sec. 4.2: sorted FP64 projected distances of `npairs` sampled pairs
    (the sample whose empirical CDF estimates F(x) = Pr[||o_i, o_j|| <= x])."""
    Oproj = np.ascontiguousarray(Oproj, dtype=np.float64)
    n, m = Oproj.shape
    out = np.empty(int(npairs), dtype=np.float64)
    lib().orc_distance_sample(_ptr(Oproj), n, m, seed, int(npairs), _ptr(out))
    return out


def cost_model(F, count, radius, hr_min, hr_max, rq):
    """Sec. 4.2: (CC, sum of Pr[e]) of range(q, rq) over the nodes given by
    their entry counts [nn], radii [nn] and pivot rings [nn][s]."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    count = np.ascontiguousarray(count, dtype=np.int64)
    radius = np.ascontiguousarray(radius, dtype=np.float64)
    hr_min = np.ascontiguousarray(hr_min, dtype=np.float64).reshape(len(count), -1)
    hr_max = np.ascontiguousarray(hr_max, dtype=np.float64).reshape(len(count), -1)
    s = hr_min.shape[1]
    en = ctypes.c_double()
    cc = lib().orc_cost_model(_ptr(F), len(F), len(count), _ptr(count), _ptr(radius), s,
                              _ptr(hr_min), _ptr(hr_max), float(rq), ctypes.byref(en))
    return cc, en.value


def overall_ratio(dists, exact_dists):
    """Eq. 11 / Eq. 13, averaged over the rows given."""
    d = np.asarray(dists, dtype=np.float64)
    e = np.asarray(exact_dists, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(e > 0, d / np.where(e > 0, e, 1), 1.0)
    return float(np.mean(r))


def recall(ids, exact_ids):
    """Eq. 12, averaged over the rows given."""
    ids = np.atleast_2d(ids)
    ex = np.atleast_2d(exact_ids)
    hits = [len(set(a.tolist()) & set(b.tolist())) / len(b) for a, b in zip(ids, ex)]
    return float(np.mean(hits))
