"""GB300 PM-LSH: Python binding of libpmlsh.so (argument marshalling only).

Every step of the query and build path runs in the library's CUDA kernels;
this module only converts arrays to pointers, allocates output tensors with
PyTorch and passes the current CUDA stream.  If the compiled library is
missing, every call raises: there is no CPU fallback.
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpmlsh.so")

PMLSH_FP32_PLAIN = 0
PMLSH_BF16_TENSOR = 1
PMLSH_BF16_VERIFY = 2
PMLSH_BF16_RERANK = 3
STOP_LITERAL = 0
STOP_BC_CONSISTENT = 1

_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ETIMEOUT", 4: "ECUDA",
           5: "ECANCELED", 6: "EINTERNAL"}


class PmlshError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("pmlsh %s: %s" % (_STATUS.get(code, code), msg))
        self.code = code


class BuildOpts(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("s", ctypes.c_int), ("leaf_size", ctypes.c_int),
                ("cp_leaf_size", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("proj", ctypes.c_void_p), ("rmin_pairs", ctypes.c_int64),
                ("bf16_shadow", ctypes.c_int)]


class KnnOpts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("c", ctypes.c_double), ("alpha1", ctypes.c_double),
                ("beta", ctypes.c_double), ("r_min", ctypes.c_double),
                ("precision", ctypes.c_int), ("t", ctypes.c_double),
                ("stop_rule", ctypes.c_int)]


class CpOpts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("c", ctypes.c_double), ("alpha1", ctypes.c_double),
                ("alpha2", ctypes.c_double), ("T", ctypes.c_int64), ("gamma", ctypes.c_double),
                ("t", ctypes.c_double)]


class CpStats(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("ub_self", ctypes.c_double),
                ("lca_nodes", ctypes.c_int64), ("nodes_done", ctypes.c_int64),
                ("self_pairs", ctypes.c_int64), ("fp64_checks", ctypes.c_int64),
                ("t", ctypes.c_double), ("T", ctypes.c_int64), ("gamma", ctypes.c_double)]


class ServeOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("max_batch_queries", ctypes.c_int64),
                ("mem_budget_bytes", ctypes.c_int64)]


class ServeStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "completed", "queries", "batches",
                                               "deferred", "canceled", "queue_depth")] + \
               [(f, ctypes.c_double) for f in ("p50_ms", "p99_ms", "mean_ms", "qps")] + \
               [(f, ctypes.c_int64) for f in ("resident_bytes", "peak_bytes")]


class QueryStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("stop_rule", ctypes.c_int32),
                ("n_cand", ctypes.c_int64), ("r_final", ctypes.c_double),
                ("fp64_checks", ctypes.c_int32), ("leaves_visited", ctypes.c_int32),
                ("n_verified", ctypes.c_int64), ("first_pass_fallbacks", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


# numpy view of pmlsh_query_stats (same field offsets as the ctypes struct)
_QSTATS_DT = np.dtype({"names": [f for f, _ in QueryStats._fields_],
                       "formats": [np.dtype(t._type_) for _, t in QueryStats._fields_],
                       "offsets": [getattr(QueryStats, f).offset for f, _ in QueryStats._fields_],
                       "itemsize": ctypes.sizeof(QueryStats)})

# name -> (restype, argtypes); the exported C ABI of include/pmlsh.h
_P = ctypes.c_void_p
_SIGS = {
    "pmlsh_params": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, _P, _P, _P]),
    "pmlsh_budget": (ctypes.c_int64, [ctypes.c_int64, ctypes.c_double, ctypes.c_int64]),
    "pmlsh_build_opts_default": (None, [_P]),
    "pmlsh_build": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, _P, _P, _P]),
    "pmlsh_free": (None, [_P]),
    "pmlsh_index_info": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "pmlsh_get_projection": (ctypes.c_int, [_P, _P]),
    "pmlsh_get_projected": (ctypes.c_int, [_P, _P]),
    "pmlsh_export_layout": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "pmlsh_export_leaf_entries": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "pmlsh_distance_sample": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_uint64, _P, _P]),
    "pmlsh_cost_model": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P, _P, _P]),
    "pmlsh_project": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P]),
    "pmlsh_project_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P]),
    "pmlsh_knn_opts_default": (None, [_P]),
    "pmlsh_knn": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P, _P, _P, _P]),
    "pmlsh_rcbc": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_double, _P, _P, _P, _P, _P]),
    "pmlsh_cp_opts_default": (None, [_P]),
    "pmlsh_closest_pair": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "pmlsh_closest_pair_bnb": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "pmlsh_gamma_calibrate": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, _P, _P]),
    "pmlsh_serve_opts_default": (None, [_P]),
    "pmlsh_serve_create": (ctypes.c_int, [_P, _P, _P]),
    "pmlsh_serve_submit": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "pmlsh_serve_wait": (ctypes.c_int, [_P, ctypes.c_uint64, _P, _P, _P, ctypes.c_int]),
    "pmlsh_rmin": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, ctypes.c_double, _P]),
    "pmlsh_knn_workspace_bytes": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _P]),
    "pmlsh_serve_stop": (ctypes.c_int, [_P]),
    "pmlsh_serve_stats": (ctypes.c_int, [_P, _P]),
    "pmlsh_serve_destroy": (ctypes.c_int, [_P]),
    "pmlsh_profile": (ctypes.c_int, [ctypes.c_int]),
    "pmlsh_profile_read": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int64]),
    "pmlsh_launch_count": (ctypes.c_longlong, []),
    "pmlsh_last_error": (ctypes.c_char_p, []),
    "pmlsh_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Loads the in-tree library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise PmlshError(4, "libpmlsh.so not built (%s); run "
                             "`python -m paper_2107_05537_gb300.build`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code):
    if code != 0:
        raise PmlshError(code, lib().pmlsh_last_error().decode())


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    if torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def _as_f32(a):
    """Returns (object keeping memory alive, pointer) for a 2-D float32 array
    (numpy or torch, host or device)."""
    torch = _torch()
    if isinstance(a, torch.Tensor):
        t = a.detach()
        if t.dtype != torch.float32:
            t = t.float()
        t = t.contiguous()
        return t, ctypes.c_void_p(t.data_ptr())
    arr = np.ascontiguousarray(a, dtype=np.float32)
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


def params(m=15, c=1.5, alpha1=1 / math.e):
    """Eq. 9: returns (t, alpha2, beta = 2 alpha2)."""
    t, a2, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().pmlsh_params(m, c, alpha1, ctypes.byref(t), ctypes.byref(a2), ctypes.byref(b)))
    return t.value, a2.value, b.value


def budget(n, beta, k):
    return lib().pmlsh_budget(n, beta, k)


def version():
    return lib().pmlsh_version().decode()


def profile(enable=True):
    """Per-kernel CUDA-event timing of every library launch (on/off)."""
    _check(lib().pmlsh_profile(1 if enable else 0))


def profile_read():
    """{kernel: (launches, total_ms)} since the last read (waits for events)."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().pmlsh_profile_read(buf, len(buf)))
    return {k: (v[0], v[1]) for k, v in json.loads(buf.value.decode()).items()}


def launch_count():
    return lib().pmlsh_launch_count()


class Index:
    """A PM-LSH index resident on the current CUDA device."""

    def __init__(self, X, m=15, s=5, leaf_size=256, seed=0, proj=None, rmin_pairs=10000,
                 bf16_shadow=True):
        L = lib()
        o = BuildOpts()
        L.pmlsh_build_opts_default(ctypes.byref(o))
        o.m, o.s, o.leaf_size, o.seed, o.rmin_pairs = m, s, leaf_size, seed, rmin_pairs
        o.bf16_shadow = 1 if bf16_shadow else 0
        keep = []
        if proj is not None:
            pa, pp = _as_f32(proj)
            keep.append(pa)
            o.proj = pp
        xa, xp = _as_f32(X)
        n, d = int(xa.shape[0]), int(xa.shape[1])
        h = ctypes.c_void_p()
        _check(L.pmlsh_build(xp, n, d, ctypes.byref(o), _stream(), ctypes.byref(h)))
        self._h = h
        self.n, self.d, self.m, self.seed = n, d, m, seed
        nl, ns = ctypes.c_int64(), ctypes.c_int64()
        lsz = ctypes.c_int()
        _check(L.pmlsh_index_info(h, None, None, None, ctypes.byref(nl), ctypes.byref(lsz),
                                  ctypes.byref(ns)))
        self.leaves, self.leaf_size, self.nodes = nl.value, lsz.value, ns.value

    def close(self):
        if getattr(self, "_h", None):
            lib().pmlsh_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def projection(self):
        A = np.empty((self.m, self.d), dtype=np.float32)
        _check(lib().pmlsh_get_projection(self._h, A.ctypes.data_as(ctypes.c_void_p)))
        return A

    def projected(self):
        O = np.empty((self.n, self.m), dtype=np.float64)
        _check(lib().pmlsh_get_projected(self._h, O.ctypes.data_as(ctypes.c_void_p)))
        return O

    def layout(self):
        perm = np.empty(self.n, dtype=np.int32)
        loff = np.empty(self.leaves + 1, dtype=np.int64)
        nlo = np.empty(self.nodes, dtype=np.int64)
        nhi = np.empty(self.nodes, dtype=np.int64)
        nl = np.empty(self.nodes, dtype=np.int32)
        nr = np.empty(self.nodes, dtype=np.int32)
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().pmlsh_export_layout(self._h, ptr(perm), ptr(loff), ptr(nlo), ptr(nhi),
                                         ptr(nl), ptr(nr)))
        return dict(perm=perm, leaf_off=loff, node_lo=nlo, node_hi=nhi, node_left=nl,
                    node_right=nr)

    def leaf_entries(self):
        """PM-tree entries of the leaves (Sec. 4.1) as the Eq. 5 test uses
        them: dict of centre [L, m], radius [L], ring_min / ring_max [L, s],
        pivots [s, m] (FP32) and s."""
        ns = ctypes.c_int()
        _check(lib().pmlsh_export_leaf_entries(self._h, ctypes.byref(ns), None, None, None, None, None))
        s = ns.value
        centre = np.empty((self.leaves, self.m), dtype=np.float32)
        radius = np.empty(self.leaves, dtype=np.float32)
        rmin = np.empty((self.leaves, s), dtype=np.float32)
        rmax = np.empty((self.leaves, s), dtype=np.float32)
        piv = np.empty((s, self.m), dtype=np.float32)
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().pmlsh_export_leaf_entries(self._h, None, ptr(centre), ptr(radius), ptr(rmin), ptr(rmax),
                                               ptr(piv)))
        return dict(s=s, centre=centre, radius=radius, ring_min=rmin, ring_max=rmax, pivots=piv)

    def distance_sample(self, npairs=65536, seed=0):
        """Sec. 4.2: sorted FP64 projected distances of `npairs` sampled
        pairs (the sample whose empirical CDF estimates F)."""
        out = np.empty(int(npairs), dtype=np.float64)
        _check(lib().pmlsh_distance_sample(self._h, int(npairs), int(seed), out.ctypes.data_as(ctypes.c_void_p),
                                           _stream()))
        return out

    def cost_model(self, F_sorted, rq):
        """Sec. 4.2: (CC [nr], sum of Pr[e] [nr]) of range(q, rq) over the
        leaves, F the empirical CDF of F_sorted."""
        F = np.ascontiguousarray(F_sorted, dtype=np.float64)
        r = np.ascontiguousarray(np.atleast_1d(rq), dtype=np.float64)
        cc = np.empty(len(r), dtype=np.float64)
        en = np.empty(len(r), dtype=np.float64)
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().pmlsh_cost_model(self._h, ptr(F), len(F), ptr(r), len(r), ptr(cc), ptr(en), _stream()))
        return cc, en

    def project(self, Q):
        """Eq. 3 for query rows: returns (FP64 [nq, m], FP32 [nq, m]) on the
        device of Q (numpy for host input)."""
        torch = _torch()
        qa, qp = _as_f32(Q)
        nq = int(qa.shape[0])
        if isinstance(qa, torch.Tensor) and qa.is_cuda:
            o64 = torch.empty((nq, self.m), dtype=torch.float64, device=qa.device)
            o32 = torch.empty((nq, self.m), dtype=torch.float32, device=qa.device)
            p64, p32 = ctypes.c_void_p(o64.data_ptr()), ctypes.c_void_p(o32.data_ptr())
        else:
            o64 = np.empty((nq, self.m), dtype=np.float64)
            o32 = np.empty((nq, self.m), dtype=np.float32)
            p64, p32 = o64.ctypes.data_as(ctypes.c_void_p), o32.ctypes.data_as(ctypes.c_void_p)
        _check(lib().pmlsh_project(self._h, qp, nq, p64, p32, _stream()))
        return o64, o32

    def rmin_rule(self, beta=0.2809, k=10, c=1.5):
        """The Sec. 5.2 first radius knn() uses when r_min <= 0."""
        r = ctypes.c_double()
        _check(lib().pmlsh_rmin(self._h, float(beta), int(k), float(c), ctypes.byref(r)))
        return r.value

    def workspace_bytes(self, nq, k=10, precision=PMLSH_FP32_PLAIN):
        """Device scratch knn() reserves for a batch of nq queries."""
        b = ctypes.c_int64()
        _check(lib().pmlsh_knn_workspace_bytes(self._h, int(nq), int(k), int(precision), ctypes.byref(b)))
        return b.value

    def gamma_calibrate(self, pr=0.85, nsample=10000, seed=None):
        """Sec. 6.3 setting of gamma (seed defaults to the index seed + 7,
        the stream closest_pairs uses when it calibrates)."""
        g = ctypes.c_double()
        sd = self.seed + 7 if seed is None else seed
        _check(lib().pmlsh_gamma_calibrate(self._h, float(pr), int(nsample), sd, ctypes.byref(g), _stream()))
        return g.value

    def closest_pairs(self, k=10, c=1.5, alpha1=1 / math.e, alpha2=0.0024, T=0, gamma=0.0, t=0.0):
        """Algorithm 4 (gamma <= 0: calibrated, Sec. 6.3).  Returns
        dict(pairs [k,2] int64, dists [k] f32, stats)."""
        o = CpOpts()
        lib().pmlsh_cp_opts_default(ctypes.byref(o))
        o.k, o.c, o.alpha1, o.alpha2, o.T, o.gamma, o.t = k, c, alpha1, alpha2, T, gamma, t
        pairs = np.empty((k, 2), dtype=np.int64)
        dists = np.empty(k, dtype=np.float32)
        st = CpStats()
        _check(lib().pmlsh_closest_pair(self._h, ctypes.byref(o), pairs.ctypes.data_as(ctypes.c_void_p),
                                        dists.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st),
                                        _stream()))
        return dict(pairs=pairs, dists=dists,
                    stats={f: getattr(st, f) for f, _ in CpStats._fields_})

    def rcbc(self, Q, r, c=1.5, alpha1=1 / math.e, beta=0.2809, precision=PMLSH_FP32_PLAIN, t=0.0,
             with_stats=True):
        """Algorithm 1 ((r,c)-BC) at radius r.  Returns dict(ids [nq] int64,
        dists [nq] f32, stats) in numpy (host) form; -1 / inf for "nothing"."""
        qa, qp = _as_f32(Q)
        nq = int(qa.shape[0])
        o = KnnOpts()
        lib().pmlsh_knn_opts_default(ctypes.byref(o))
        o.c, o.alpha1, o.beta, o.precision, o.t = c, alpha1, beta, precision, t
        ids = np.empty(nq, dtype=np.int64)
        dists = np.empty(nq, dtype=np.float32)
        stats = (QueryStats * max(1, nq))() if with_stats else None
        _check(lib().pmlsh_rcbc(self._h, qp, nq, float(r), ctypes.byref(o),
                                ids.ctypes.data_as(ctypes.c_void_p), dists.ctypes.data_as(ctypes.c_void_p),
                                ctypes.cast(stats, ctypes.c_void_p) if stats is not None else None,
                                _stream()))
        res = dict(ids=ids, dists=dists)
        if with_stats:
            sv = np.frombuffer(stats, dtype=_QSTATS_DT, count=nq) if nq else np.zeros(0, _QSTATS_DT)
            res["stats"] = dict(rule=sv["stop_rule"].copy(), ncand=sv["n_cand"].copy(),
                                rounds=sv["rounds"].copy())
        return res

    def closest_pairs_bnb(self, k=10, T=0, alpha2=0.0024):
        """Algorithm 3 (branch and bound).  Returns dict(pairs, dists, stats)."""
        o = CpOpts()
        lib().pmlsh_cp_opts_default(ctypes.byref(o))
        o.k, o.T, o.alpha2 = k, T, alpha2
        pairs = np.empty((k, 2), dtype=np.int64)
        dists = np.empty(k, dtype=np.float32)
        st = CpStats()
        _check(lib().pmlsh_closest_pair_bnb(self._h, ctypes.byref(o), pairs.ctypes.data_as(ctypes.c_void_p),
                                            dists.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st), _stream()))
        return dict(pairs=pairs, dists=dists,
                    stats={f: getattr(st, f) for f, _ in CpStats._fields_})

    def knn(self, Q, k=10, c=1.5, alpha1=1 / math.e, beta=0.2809, r_min=0.0,
            precision=PMLSH_FP32_PLAIN, stop_rule=STOP_LITERAL, t=0.0, out=None,
            with_err=True, with_stats=True):
        """Algorithm 2 for the rows of Q.  Outputs live on the GPU when Q is a
        CUDA tensor (or when `out` tensors are given), else in numpy arrays.
        Returns dict(ids, dists, err, stats)."""
        torch = _torch()
        qa, qp = _as_f32(Q)
        nq = int(qa.shape[0])
        o = KnnOpts()
        lib().pmlsh_knn_opts_default(ctypes.byref(o))
        o.k, o.c, o.alpha1, o.beta, o.r_min = k, c, alpha1, beta, r_min
        o.precision, o.stop_rule, o.t = precision, stop_rule, t
        on_gpu = isinstance(qa, torch.Tensor) and qa.is_cuda
        if out is not None:
            ids, dists, err = out
        elif on_gpu:
            ids = torch.empty((nq, k), dtype=torch.int64, device=qa.device)
            dists = torch.empty((nq, k), dtype=torch.float32, device=qa.device)
            err = torch.empty((nq, k), dtype=torch.float32, device=qa.device) if with_err else None
        else:
            ids = np.empty((nq, k), dtype=np.int64)
            dists = np.empty((nq, k), dtype=np.float32)
            err = np.empty((nq, k), dtype=np.float32) if with_err else None

        def ptr(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                return ctypes.c_void_p(a.data_ptr())
            return a.ctypes.data_as(ctypes.c_void_p)
        stats = (QueryStats * max(1, nq))() if with_stats else None
        _check(lib().pmlsh_knn(self._h, qp, nq, ctypes.byref(o), ptr(ids), ptr(dists), ptr(err),
                               ctypes.cast(stats, ctypes.c_void_p) if stats is not None else None,
                               _stream()))
        res = dict(ids=ids, dists=dists, err=err)
        if with_stats:
            sv = np.frombuffer(stats, dtype=_QSTATS_DT, count=nq) if nq else np.zeros(0, _QSTATS_DT)
            res["stats"] = dict(
                rounds=sv["rounds"].copy(), rule=sv["stop_rule"].copy(),
                ncand=sv["n_cand"].copy(), r=sv["r_final"].copy(), fp64=sv["fp64_checks"].copy(),
                nver=sv["n_verified"].copy(), leaves=sv["leaves_visited"].copy(),
                fallbacks=sv["first_pass_fallbacks"].copy())
        return res


class Server:
    """Continuous-batching server over an Index (see pmlsh_serve_* in pmlsh.h)."""

    def __init__(self, index, slots=3, max_batch_queries=16384, mem_budget_bytes=8 << 30):
        L = lib()
        o = ServeOpts()
        L.pmlsh_serve_opts_default(ctypes.byref(o))
        o.slots, o.max_batch_queries, o.mem_budget_bytes = slots, max_batch_queries, mem_budget_bytes
        h = ctypes.c_void_p()
        _check(L.pmlsh_serve_create(index._h, ctypes.byref(o), ctypes.byref(h)))
        self._h, self.index, self._k = h, index, {}

    def submit(self, Q, k=10, c=1.5, alpha1=1 / math.e, beta=0.2809, r_min=0.0,
               stop_rule=STOP_LITERAL, t=0.0, precision=PMLSH_FP32_PLAIN):
        Q = np.ascontiguousarray(Q, dtype=np.float32)
        o = KnnOpts()
        lib().pmlsh_knn_opts_default(ctypes.byref(o))
        o.k, o.c, o.alpha1, o.beta, o.r_min, o.stop_rule, o.t = k, c, alpha1, beta, r_min, stop_rule, t
        o.precision = precision
        tk = ctypes.c_uint64()
        _check(lib().pmlsh_serve_submit(self._h, Q.ctypes.data_as(ctypes.c_void_p), Q.shape[0],
                                        ctypes.byref(o), ctypes.byref(tk)))
        self._k[tk.value] = (Q.shape[0], k)
        return tk.value

    def wait(self, ticket, timeout_ms=-1, with_err=False):
        """(ids, dists), or (ids, dists, err) with `with_err` (|returned -
        FP64 distance| per result)."""
        nq, k = self._k.get(ticket, (1, 1))
        ids = np.empty((nq, k), dtype=np.int64)
        dd = np.empty((nq, k), dtype=np.float32)
        ee = np.empty((nq, k), dtype=np.float32) if with_err else None
        rc = lib().pmlsh_serve_wait(self._h, ticket, ids.ctypes.data_as(ctypes.c_void_p),
                                    dd.ctypes.data_as(ctypes.c_void_p),
                                    ee.ctypes.data_as(ctypes.c_void_p) if with_err else None,
                                    int(timeout_ms))
        if rc != 3:
            self._k.pop(ticket, None)
        _check(rc)
        return (ids, dd, ee) if with_err else (ids, dd)

    def stats(self):
        s = ServeStats()
        _check(lib().pmlsh_serve_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServeStats._fields_}

    def stop(self):
        _check(lib().pmlsh_serve_stop(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().pmlsh_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
