#!/usr/bin/env python
"""Throughput benchmark of the PM-LSH (c,k)-ANN query path on GB300.

One step = one batch of the throughput workload (n = 1,000,000 points,
d = 128, a 1,000-cluster Gaussian mixture, 10,000 queries, m = 15, c = 1.5,
k = 50, beta = 0.2809, alpha1 = 1/e) through pmlsh_knn: query projection,
the range rounds of Algorithm 2, the budget cut, verification, top-k and the
stop rules.  The index is built once before the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank serves its own copy
of the batch against its own replica of the index (no collective on the data
path), so `value` is the aggregate queries/s of all ranks ("scaling": weak).
`--impl reference` times the FP64 CPU oracle on the host cores on bounded
samples of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "c-ANN queries/s at fixed ratio, 1M×128 k=50; serve p50/p99 ms vs plain FP32"
K, C, BETA, M_PROJ = 50, 1.5, 0.2809, 15
# precision modes of pmlsh_knn (bits: 1 tensor-core count, 2 BF16 first-pass verification)
PRECISIONS = {"fp32": 0, "bf16": 1, "verify": 2, "rerank": 3}
ALPHA1 = 1 / math.e


def workload_desc(nq):
    return ("c-ANN, n=1,000,000 d=128 FP32, Gaussian mixture of 1,000 clusters "
            "(centres N(0,100 I), sigma U[0.5,2]), %d queries from the same mixture, "
            "m=15, c=1.5, k=50, beta=0.2809, alpha1=1/e, r_min by the Sec. 5.2 rule, "
            "leaf size autotuned, seed 0" % nq)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region: start()
    returns once the first sample has arrived (or after wait_s), begin()/end()
    mark the region, and stop() summarises the samples taken inside it and the
    first one after it.  Samples are placed by nvidia-smi's own timestamp (its
    output may reach the pipe in bursts); lines without a readable timestamp
    are placed by arrival, and if no sample falls in the region all are used."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, interval_ms=100, exe="nvidia-smi"):
        self.gpu = gpu_index
        self.interval_ms = interval_ms
        self.exe = exe
        self.p = None
        self.lines = []
        self.t0 = self.t1 = None
        self.reader = None

    def _read(self):
        try:
            for line in self.p.stdout:
                self.lines.append((time.time(), line))
        except Exception:
            pass

    def start(self, wait_s=2.0):
        import threading
        try:
            self.p = subprocess.Popen([self.exe, "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
            t = time.time()
            while not self.lines and time.time() - t < wait_s and self.p.poll() is None:
                time.sleep(0.005)
        except Exception:
            self.p = None

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(text):
        import datetime
        try:
            return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except Exception:
            return None

    def stop(self):
        if self.p is None:
            return None
        try:
            # wait for one more sample after the region closes
            t = time.time()
            while (self.t1 is not None and not any(ts > self.t1 for ts, _ in self.lines)
                   and time.time() - t < 5 * self.interval_ms / 1000.0 + 1.0 and self.p.poll() is None):
                time.sleep(0.005)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            if self.reader is not None:
                self.reader.join(timeout=5)
        except Exception:
            return None
        rows = []
        for arrived, line in list(self.lines):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                rows.append((self._stamp(f[0]) or arrived, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        if not rows:
            return None
        t0 = self.t0 if self.t0 is not None else float("-inf")
        t1 = self.t1 if self.t1 is not None else float("inf")
        after = [r[0] for r in rows if r[0] > t1]
        last = min(after) if after else t1
        pick = [r for r in rows if t0 <= r[0] <= last] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = {nm for r in pick for nm, v in zip(names, r[3]) if v.lower().startswith("active")}
        return {"sm_mhz": statistics.median(r[1] for r in pick), "sm_max_mhz": max(r[2] for r in pick),
                "reasons": sorted(reasons), "samples": len(pick), "interval_ms": self.interval_ms}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def traffic_record():
    """DRAM bytes per query of each profiled kernel (ncu), with the hash of
    the source file they were taken from: a changed source voids them."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def cpu_baseline(X, Q, A, budget_s=15.0):
    """The FP64 oracle, as it stands, on a bounded sample of the queries."""
    import oracle
    t, _, _ = oracle.params(M_PROJ, C, ALPHA1)
    B = oracle.budget(len(X), BETA, K)
    O = oracle.project(X, A)
    rmin = oracle.rmin_auto(X, BETA, K, C, 3)
    t0 = time.perf_counter()
    probe = 32
    oracle.knn(X, A, Q[:probe], K, C, t, B, rmin, 0, Oproj=O)
    per_q = (time.perf_counter() - t0) / probe
    ns = int(max(probe, min(len(Q), budget_s / max(per_q, 1e-6))))
    t0 = time.perf_counter()
    oracle.knn(X, A, Q[:ns], K, C, t, B, rmin, 0, Oproj=O)
    el = time.perf_counter() - t0
    # one query per call: the oracle parallelises over queries, so this is
    # the single-thread time per query
    single = 8
    t0 = time.perf_counter()
    for i in range(single):
        oracle.knn(X, A, Q[i:i + 1], K, C, t, B, rmin, 0, Oproj=O)
    st_ms = (time.perf_counter() - t0) * 1000 / single
    return {"value": ns / el, "unit": "queries/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "first %d of the %d queries (FP64 Algorithm 2, OpenMP over queries), "
                      "%.1f s" % (ns, len(Q), el),
            "single_thread_ms_per_query": st_ms, "cpu": cpu_model()}


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (model name, else implementer
    and part), with the machine type."""
    import platform
    name = ""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read().splitlines()
        for key in ("model name", "CPU part"):
            vals = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith(key)]
            if vals:
                name = vals[0] if key == "model name" else "CPU part " + vals[0]
                break
    except OSError:
        pass
    return ("%s (%s)" % (name, platform.machine())).strip() if name else platform.machine()


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import datagen
    import oracle
    w = datagen.workload("c2")
    X, Q = w["X"], w["Q"]
    A = oracle.gen_projection(2, M_PROJ, X.shape[1]).astype(np.float32)
    t, _, _ = oracle.params(M_PROJ, C, ALPHA1)
    B = oracle.budget(len(X), BETA, K)
    O = oracle.project(X, A)
    rmin = oracle.rmin_auto(X, BETA, K, C, 3)
    per_step = args.ref_queries
    for s in range(args.warmup):
        oracle.knn(X, A, Q[s * per_step % len(Q):][:per_step], K, C, t, B, rmin, 0, Oproj=O)
    total = 0.0
    for s in range(args.steps):
        q0 = (args.warmup + s) * per_step % len(Q)
        t0 = time.perf_counter()
        oracle.knn(X, A, Q[q0:q0 + per_step], K, C, t, B, rmin, 0, Oproj=O)
        total += time.perf_counter() - t0
    v = per_step * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total * 1000 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(per_step) + " (sample of %d queries per step)" % per_step},
            "cpu_baseline": {"value": v, "unit": "queries/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "cpu": cpu_model(),
                             "sample": "%d queries per step, %d steps" % (per_step, args.steps)},
            "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def source_sha(rel):
    """sha256 of one source file, or of several concatenated in order."""
    import hashlib
    h = hashlib.sha256()
    for r in ([rel] if isinstance(rel, str) else rel):
        with open(os.path.join(ROOT, r), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def timed_steps(step, steps, flush, stream, tag, profile=False):
    """K steps, L2 flushed before each, CUDA events on the launch stream.
    The steps run inside the NVTX range `tag` (a profiler can select them).
    With `profile`, the library brackets every launch with events and the
    per-kernel totals are returned (the step time then includes those event
    records, so headline numbers come from an unprofiled pass)."""
    import torch
    import paper_2107_05537_gb300 as pm
    pm.profile(bool(profile))
    pm.profile_read()
    launches0 = pm.launch_count()
    total_ms, res = 0.0, None
    try:
        torch.cuda.nvtx.range_push(tag)
        nvtx = True
    except Exception:
        nvtx = False
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = step()
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
    if nvtx:
        torch.cuda.nvtx.range_pop()
    launches = pm.launch_count() - launches0
    prof = pm.profile_read()
    pm.profile(False)
    return total_ms, res, prof, launches


def serve_leg(pm, ix, Q, prec, rate_qps, seconds, seed):
    """Open-loop Poisson request stream through the continuous-batching
    server: request sizes log-uniform in [1, 4096], k uniform in {1, 10, 100},
    c = 1.5; returns the server's latency and throughput figures."""
    import threading
    rng = np.random.default_rng(seed)
    mean_size = (4096 - 1) / math.log(4096)
    reqs, t = [], 0.0
    while t < seconds:
        t += rng.exponential(mean_size / rate_qps)
        size = int(np.exp(rng.uniform(0.0, math.log(4096.0))))
        q0 = int(rng.integers(0, len(Q) - size + 1))
        reqs.append((t, q0, size, int(rng.choice([1, 10, 100]))))
    srv = pm.Server(ix, slots=3, max_batch_queries=16384)
    tickets = []

    def producer():
        t0 = time.perf_counter()
        for at, q0, size, k in reqs:
            dt = at - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(Q[q0:q0 + size], k=k, c=C, beta=BETA, precision=prec))
    th = threading.Thread(target=producer)
    th.start()
    th.join()
    for tk in tickets:
        srv.wait(tk)
    st = srv.stats()
    srv.close()
    return {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "qps": st["qps"], "requests": st["completed"], "queries": st["queries"],
            "batches": st["batches"]}


def knn_leg(pm, ix, Q, k, c, beta, prec, steps, warmup, flush, stream, tag, r_min=0.0):
    """One (c,k)-ANN setting timed like the main step (statistics-free call,
    L2 flushed between steps), then once with statistics for the trace and
    the verified rows behind the k_verify roofline."""
    import torch
    nq, d = Q.shape
    ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    er = torch.empty((nq, k), dtype=torch.float32, device="cuda")

    def step():
        return ix.knn(Q, k=k, c=c, alpha1=ALPHA1, beta=beta, r_min=r_min, precision=prec,
                      out=(ids, dd, er), with_stats=False)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ms, _, _, launches = timed_steps(step, steps, flush, stream, tag)
    _, _, prof, _ = timed_steps(step, steps, flush, stream, "profiled_" + tag, profile=True)
    st = ix.knn(Q, k=k, c=c, alpha1=ALPHA1, beta=beta, r_min=r_min, precision=prec)["stats"]
    nver = int(st["nver"].sum())
    out = {"k": k, "c": c, "beta": beta, "queries": int(nq), "value": nq * steps / (ms / 1000.0),
           "unit": "queries/s", "ms_per_step": ms / steps, "gpu_launches": launches,
           "trace": {"mean_rounds": float(st["rounds"].mean()), "mean_candidates": float(st["ncand"].mean()),
                     "mean_verified": float(st["nver"].mean()),
                     "first_pass_fallback_queries": int((st["fallbacks"] > 0).sum()),
                     "rule_counts": np.bincount(st["rule"], minlength=4).tolist()},
           "kernels": {k2: {"launches": v[0], "ms": round(v[1], 4)} for k2, v in prof.items()}}
    if "k_verify" in prof:
        lv, mv = prof["k_verify"]
        # verified rows' bytes and the query rows and results, per launch,
        # as for the main step (rows of every round of the call)
        alg = (nver * d * 4.0 + nq * (d * 4.0 + k * 16.0)) * steps / lv
        pk, kind = peaks()
        ach = alg / (mv / lv / 1000.0) / 1e9
        out["k_verify_roofline"] = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                    "frac": ach / pk["hbm_gbs"], "algorithmic_bytes_per_launch": alg,
                                    "avg_launch_ms": mv / lv, "peak_kind": kind}
    return out


def leg_c2_budget(pm, ix, Q, prec, steps, warmup, flush, stream):
    """The throughput workload in the other regimes of Algorithm 2: with
    beta = 0.01 (B = 10,050) and the first radius of the Sec. 5.2 rule, about
    half of the queries' range sets pass the budget in round 1 (|S_i| from
    ~1k to ~100k) and rule 2 keeps the B nearest in projected space; with
    beta = 0.2809 and a first radius three growth steps below the rule, the
    radius grows over several rounds before rule 1 stops a query."""
    out = {}
    for nm, beta, scale in (("rule2", 0.01, 1.0), ("multiround", BETA, 1.0 / (C * C * C))):
        rmin = ix.rmin_rule(beta, K, C) * scale
        r = knn_leg(pm, ix, Q, K, C, beta, prec, steps, warmup, flush, stream, "timed_" + nm, r_min=rmin)
        r["r_min"] = rmin
        out[nm] = r
    out["workload"] = "1M x 128 throughput workload; rule2: beta = 0.01, r_min = Sec. 5.2 rule; " \
                      "multiround: beta = 0.2809, r_min = rule / c^3"
    return out


def leg_c3(pm, prec, steps, warmup, flush, stream):
    """High-dimensional workload: n = 10^6, d = 960, 1,000 clusters with
    covariance eigenvalues i^-1 (seeded rotation), 1,000 queries; (c, k) in
    {(1.2, 1), (1.5, 10), (2.0, 100)}; leaf size 256."""
    import torch
    import datagen
    w = datagen.workload("c3")
    t0 = time.perf_counter()
    ix = pm.Index(torch.from_numpy(w["X"]).cuda(), m=M_PROJ, leaf_size=256, seed=0)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    Qd = torch.from_numpy(w["Q"]).cuda()
    out = {"workload": "n=1,000,000 d=960 FP32, 1,000 clusters, eigenvalues i^-1, 1,000 queries, m=15, "
                       "beta=0.2809, leaf size 256", "build_s": build_s, "settings": []}
    for c, k in ((1.5, 10), (1.2, 1), (2.0, 100)):
        out["settings"].append(knn_leg(pm, ix, Qd, k, c, BETA, prec, steps, warmup, flush, stream,
                                       "timed_c3"))
    # BF16 first-pass verification against FP32 verification, same count
    # mode, at (c, k) = (1.5, 10): results compared element by element
    base = prec & ~2
    cmp = {}
    for nm, p2 in (("fp32_verify", base), ("bf16_verify", base | 2)):
        r = knn_leg(pm, ix, Qd, 10, 1.5, BETA, p2, steps, warmup, flush, stream, "timed_c3_verify")
        got = ix.knn(Qd, k=10, c=1.5, alpha1=ALPHA1, beta=BETA, precision=p2, with_stats=False)
        r["ids"] = got["ids"]
        r["dists"] = got["dists"]
        cmp[nm] = r
    same = bool(torch.equal(cmp["fp32_verify"].pop("ids"), cmp["bf16_verify"].pop("ids")) and
                torch.equal(cmp["fp32_verify"].pop("dists"), cmp["bf16_verify"].pop("dists")))
    out["verify_precision"] = {"k": 10, "c": 1.5, "results_identical": same, **cmp}
    ix.close()
    return out


def leg_c4(pm):
    """Closest pairs: n = 10^5, d = 512, 500 clusters plus 20 planted pairs at
    distance 0.01; k = 10, m = 15, alpha2 = 0.0024 (T = alpha2 n (n - 1) + k);
    gamma calibrated (Pr = 0.85 on 10^4 sampled points); Algorithm 4 with
    FindLCA and Algorithm 3 (branch and bound), each timed once after one
    untimed run, leaf size 16."""
    import torch
    import datagen
    w = datagen.workload("c4")
    X, planted = w["X"], w["planted"]
    ix = pm.Index(torch.from_numpy(X).cuda(), m=M_PROJ, leaf_size=16, seed=0)
    planted_set = {tuple(p) for p in planted.tolist()}
    out = {"workload": "n=100,000 d=512 FP32, 500 clusters + 20 planted pairs at 0.01, k=10, m=15, "
                       "alpha2=0.0024, leaf size 16"}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        pm.profile(True)
        pm.profile_read()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        prof = pm.profile_read()
        pm.profile(False)
        return r, el, prof

    g, el, _ = timed(lambda: ix.gamma_calibrate(0.85, nsample=10000))
    out["gamma"] = {"value": g, "pr": 0.85, "sample": 10000, "seconds": el}
    for nm, fn in (("radius_filter", lambda: ix.closest_pairs(k=10, gamma=g)),
                   ("branch_and_bound", lambda: ix.closest_pairs_bnb(k=10))):
        r, el, prof = timed(fn)
        dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
        out[nm] = {"seconds": el, "count": int(r["stats"]["count"]),
                   "top10_planted": sum(tuple(p) in planted_set for p in r["pairs"].tolist()),
                   "dominant_kernel": dom,
                   "kernels": {k2: {"launches": v[0], "ms": round(v[1], 4)} for k2, v in prof.items()}}
    ix.close()
    return out


def leg_c5(pm, seconds, main_name):
    """Serving workload: n = 2*10^6, d = 256 resident (2,000 clusters); an
    open-loop Poisson stream at 5k, 20k and 50k queries/s (request sizes
    log-uniform in [1, 4096], k in {1, 10, 100}, c = 1.5) through the
    continuous-batching server, the benchmark's precision mode vs FP32."""
    import torch
    import datagen
    w = datagen.workload("c5", nq=16384)
    ix = pm.Index(torch.from_numpy(w["X"]).cuda(), m=M_PROJ, leaf_size=256, seed=0)
    Q = w["Q"]
    out = {"workload": "n=2,000,000 d=256 FP32 resident, 2,000 clusters; Poisson arrivals, request sizes "
                       "log-uniform [1,4096], k in {1,10,100}, c=1.5, 3 slots", "seconds": seconds, "rates": {}}
    for rate in (5_000.0, 20_000.0, 50_000.0):
        out["rates"][str(int(rate))] = {
            nm: serve_leg(pm, ix, Q, p, rate, seconds, seed=7)
            for nm, p in ((main_name, PRECISIONS[main_name]), ("fp32", PRECISIONS["fp32"]))}
    ix.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=list(PRECISIONS),
                    help="fp32: CUDA-core count, FP32 verification; bf16: tensor-core count; "
                         "verify: BF16 first-pass verification; rerank: both")
    ap.add_argument("--nq", type=int, default=10_000)
    ap.add_argument("--leaf-size", type=int, default=0, help="leaf capacity M; 0 = autotuned by pmlsh_build")
    ap.add_argument("--ref-queries", type=int, default=96)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--serve-rate", type=float, default=50_000.0)
    ap.add_argument("--legs", default="budget,c3,c4,c5",
                    help="other workloads on the same line: budget,c3,c4,c5 (or none)")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch

    import datagen
    import paper_2107_05537_gb300 as pm
    torch.cuda.set_device(local)
    w = datagen.workload("c2", nq=args.nq)
    X, Q = w["X"], w["Q"]
    nq, d = Q.shape
    Xd = torch.from_numpy(X).cuda()
    t0 = time.perf_counter()
    ix = pm.Index(Xd, m=M_PROJ, leaf_size=args.leaf_size, seed=0)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    del Xd
    prec = PRECISIONS[args.precision]
    Qd = torch.from_numpy(Q).cuda()
    ids = torch.empty((nq, K), dtype=torch.int64, device="cuda")
    dd = torch.empty((nq, K), dtype=torch.float32, device="cuda")
    er = torch.empty((nq, K), dtype=torch.float32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    stream = torch.cuda.current_stream()

    # the timed call is the one a caller makes for results: ids, distances
    # and error bounds, no per-query statistics (with statistics the exact
    # |C| of every round is also counted; that form is timed beside it)
    def make_step(p, with_stats=False):
        return lambda: ix.knn(Qd, k=K, c=C, alpha1=ALPHA1, beta=BETA, precision=p, out=(ids, dd, er),
                              with_stats=with_stats)

    step = make_step(prec)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    if sampler:
        sampler.begin()
    total_ms, res, _, launches = timed_steps(step, args.steps, flush, stream, "timed_main")
    barrier(ws)
    torch.cuda.synchronize()
    if sampler:
        sampler.end()
    clocks = sampler.stop() if sampler else None
    # per-kernel CUDA-event times of the same steps, in a second pass
    prof_ms, _, prof, _ = timed_steps(step, args.steps, flush, stream, "profiled_main", profile=True)
    total_s = max_over_ranks(total_ms / 1000.0, ws)
    value = nq * args.steps * ws / total_s
    ids_main = ids.clone()
    dd_main = dd.clone()

    # the same batch with per-query statistics (exact |C| per round): the
    # trace, the verified rows behind the roofline, and its own speed
    sstep = make_step(prec, with_stats=True)
    sstep()
    sms, sres, _, _ = timed_steps(sstep, args.steps, flush, stream, "timed_stats")
    stats = sres["stats"]
    nver = int(stats["nver"].sum()) * args.steps
    with_stats = {"value": nq * args.steps * ws / max_over_ranks(sms / 1000.0, ws),
                  "ms_per_step": sms / args.steps,
                  "ids_identical": bool(torch.equal(ids, ids_main) and torch.equal(dd, dd_main))}

    # the other precision modes on the same batch: same results, own speed
    other = None
    if not args.no_fp32_compare:
        other = {}
        for nm, op in PRECISIONS.items():
            if op == prec:
                continue
            ostep = make_step(op)
            for _ in range(args.warmup):
                ostep()
            torch.cuda.synchronize()
            barrier(ws)
            oms, _, _, _ = timed_steps(ostep, args.steps, flush, stream, "timed_other")
            _, _, oprof, _ = timed_steps(ostep, args.steps, flush, stream, "profiled_other", profile=True)
            barrier(ws)
            os_ = max_over_ranks(oms / 1000.0, ws)
            other[nm] = {"value": nq * args.steps * ws / os_, "ms_per_step": os_ * 1000 / args.steps,
                         "ids_identical": bool(torch.equal(ids, ids_main)),
                         "dists_identical": bool(torch.equal(dd, dd_main)),
                         "kernels": {k2: {"launches": v[0], "ms": round(v[1], 4)} for k2, v in oprof.items()}}
            ids.copy_(ids_main)
            dd.copy_(dd_main)

    # quality at the operating point: Eq. 11 / Eq. 12 on a query sample
    # against exact neighbours (plain PyTorch FP64 on the GPU)
    with torch.no_grad():
        sq = torch.arange(0, nq, max(1, nq // 64), device="cuda")[:64]
        Xe = torch.from_numpy(X).cuda().double()
        Qe = Qd[sq].double()
        dist = torch.cdist(Qe, Xe)
        ex_d, ex_i = torch.topk(dist, K, largest=False)
        got_d = dd[sq].double()
        ratio = float((got_d / ex_d.clamp_min(1e-300)).mean())
        rec = float(np.mean([len(set(ids[q].tolist()) & set(ex_i[j].tolist())) / K
                             for j, q in enumerate(sq.tolist())]))
        del Xe, dist

    # end to end through the public API with host buffers (pinned), the
    # host->device copy of Q and the device->host copy of the results inside
    e2e = None
    if not args.no_e2e:
        Qh = torch.from_numpy(Q).pin_memory()
        idh = torch.empty((nq, K), dtype=torch.int64).pin_memory()
        ddh = torch.empty((nq, K), dtype=torch.float32).pin_memory()
        erh = torch.empty((nq, K), dtype=torch.float32).pin_memory()
        ix.knn(Qh.numpy(), k=K, c=C, beta=BETA, precision=prec, out=(idh.numpy(), ddh.numpy(), erh.numpy()),
               with_stats=False)
        el = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ix.knn(Qh.numpy(), k=K, c=C, beta=BETA, precision=prec,
                   out=(idh.numpy(), ddh.numpy(), erh.numpy()), with_stats=False)
            el += time.perf_counter() - t0
        el = max_over_ranks(el, ws)
        e2e = {"value": nq * args.steps * ws / el, "unit": "queries/s",
               "h2d_bytes_per_step": nq * d * 4, "d2h_bytes_per_step": nq * K * (8 + 4 + 4)}

    # roofline of the dominant kernel
    pk, pk_kind = peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    roof = None
    if dom:
        launches_dom, ms_dom = prof[dom]
        tr = traffic_record().get(dom)
        traffic = None
        if tr and tr.get("sha256") == source_sha(tr["source"]):
            traffic = tr["dram_bytes_per_query"] * nq * args.steps / launches_dom
        roof = {"bound": "hbm", "achieved": None, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": None, "kernel": dom, "traffic": traffic}
        if dom == "k_verify":
            # algorithmic bytes: the original-space row of every verified
            # candidate, the query rows, the k results (id, distance, error)
            alg = nver * d * 4.0 + args.steps * nq * (d * 4.0 + K * 16.0)
            achieved = alg / (ms_dom / 1000.0) / 1e9
            roof.update({"achieved": achieved, "frac": achieved / pk["hbm_gbs"],
                         "algorithmic_bytes_per_launch": alg / launches_dom,
                         "avg_launch_ms": ms_dom / launches_dom})
        roof["kernels"] = {k2: {"launches": v[0], "ms": round(v[1], 4)} for k2, v in prof.items()}
        # DRAM GB/s of each kernel with captured traffic (ncu bytes per query
        # scaled to the timed queries; the capture's source must be unchanged)
        for k2, tr2 in traffic_record().items():
            if k2 in prof and isinstance(tr2, dict) and tr2.get("sha256") == source_sha(tr2["source"]):
                b2 = tr2["dram_bytes_per_query"] * nq * args.steps
                roof["kernels"][k2].update({"dram_bytes_per_launch": b2 / prof[k2][0],
                                            "dram_gbs": b2 / (prof[k2][1] / 1000.0) / 1e9,
                                            "dram_frac": b2 / (prof[k2][1] / 1000.0) / 1e9 / pk["hbm_gbs"]})
        roof["peak_kind"] = pk_kind
        # the per-kernel times come from a second pass with every launch
        # bracketed by events; its step time, for comparison with ms_per_step
        roof["profiled_pass_ms_per_step"] = prof_ms / args.steps

    # serving: open-loop Poisson stream on the resident index, both precisions
    serve = None
    if rank == 0 and args.serve_seconds > 0:
        serve = {"rate_qps": args.serve_rate, "seconds": args.serve_seconds,
                 "note": "resident 1M x 128 index; request sizes log-uniform [1,4096], k in {1,10,100}"}
        for nm in dict.fromkeys((args.precision, "fp32")):
            serve[nm] = serve_leg(pm, ix, Q, PRECISIONS[nm], args.serve_rate, args.serve_seconds, seed=5)

    legs = {}
    want = set(x for x in args.legs.split(",") if x and x != "none")
    if rank == 0:
        lsteps, lwarm = max(3, min(args.steps, 10)), max(3, min(args.warmup, 3))
        if "budget" in want:
            legs["c2_budget"] = leg_c2_budget(pm, ix, Qd, prec, lsteps, lwarm, flush, stream)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        A = ix.projection()
        cpu = cpu_baseline(X, Q, A)

    # the other workloads (each with its own index; the throughput index is
    # freed first)
    ix_leaf = ix.leaf_size
    ix.close()
    del Qd, ids, dd, er
    torch.cuda.empty_cache()
    if rank == 0:
        if "c3" in want:
            legs["c3"] = leg_c3(pm, prec, lsteps, lwarm, flush, stream)
            torch.cuda.empty_cache()
        if "c4" in want:
            legs["c4"] = leg_c4(pm)
            torch.cuda.empty_cache()
        if "c5" in want and args.serve_seconds > 0:
            legs["c5_serve"] = leg_c5(pm, min(args.serve_seconds, 2.0), args.precision)
            torch.cuda.empty_cache()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_s * 1000 / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_desc(nq), "precision": args.precision,
                           "leaf_size": ix_leaf,
                           "leaf_size_choice": "autotuned over 128/256/512" if args.leaf_size == 0 else "fixed",
                           "l2": "flushed between steps (512 MB write)",
                           "parallelism": "replicas" if ws > 1 else "single"},
                "gpu_launches": launches,
                "quality": {"overall_ratio": ratio, "recall": rec, "sample_queries": int(len(sq))},
                "trace": {"mean_rounds": float(stats["rounds"].mean()),
                          "mean_candidates": float(stats["ncand"].mean()),
                          "mean_verified": float(stats["nver"].mean()),
                          "mean_leaves_visited": float(stats["leaves"].mean()),
                          "first_pass_fallback_queries": int((stats["fallbacks"] > 0).sum()),
                          "rule_counts": np.bincount(stats["rule"], minlength=4).tolist()},
                "build_s": build_s, "with_stats": with_stats, "other_precision": other, "serve": serve,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "legs": legs}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
