"""Sweep of the projection count m and the pivot count s with the PM-tree
cost model of Sec. 4.2 next to the measured query work.

For each (m, s) the index is built on a seeded Gaussian mixture, F is sampled
(pmlsh_distance_sample), and the model's CC and expected accessed leaves of
range(q, t r_min) (pmlsh_cost_model, t from Eq. 9 for m, r_min by the Sec. 5.2
rule) are printed beside the measured mean |C|, rounds and time per query of
pmlsh_knn (k = 10, c = 1.5, no statistics in the timed call).

Usage: python -m paper_2107_05537_gb300.cost_sweep [--n 100000] [--nq 2000]
Prints one JSON line per (m, s).
"""
import argparse
import json
import math
import os
import sys

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=100_000)
    ap.add_argument("--d", type=int, default=128)
    ap.add_argument("--clusters", type=int, default=100)
    ap.add_argument("--nq", type=int, default=2000)
    ap.add_argument("--m", default="8,12,15,16")
    ap.add_argument("--s", default="0,3,5,8")
    ap.add_argument("--leaf-size", type=int, default=256)
    args = ap.parse_args()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import datagen
    import paper_2107_05537_gb300 as pm

    X, Q, _, _ = datagen.mixture(args.n, args.d, args.clusters, (0.5, 2.0), seed=0, nq=args.nq)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    for m in [int(v) for v in args.m.split(",")]:
        t, _, _ = pm.params(m, 1.5, 1 / math.e)
        for s in [int(v) for v in args.s.split(",")]:
            ix = pm.Index(Xd, m=m, s=s, leaf_size=args.leaf_size)
            st = ix.knn(Qd[:256], k=10)["stats"]
            one = st["rounds"] == 1
            rmin = float(st["r"][one][0]) if one.any() else float("nan")
            F = ix.distance_sample(65536, 6)
            cc, nodes = ix.cost_model(F, [t * rmin]) if one.any() else ([float("nan")], [float("nan")])
            stats = ix.knn(Qd, k=10)["stats"]
            for _ in range(2):
                ix.knn(Qd, k=10, with_stats=False)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ix.knn(Qd, k=10, with_stats=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            print(json.dumps({"m": m, "s": s, "leaves": ix.leaves, "t": t, "r_min": rmin,
                              "model_cc": float(cc[0]), "model_leaves": float(nodes[0]),
                              "model_work": ix.leaves + float(cc[0]),
                              "mean_candidates": float(np.mean(stats["ncand"])),
                              "mean_rounds": float(np.mean(stats["rounds"])),
                              "us_per_query": 1e3 * ms / len(Q)}), flush=True)
            ix.close()


if __name__ == "__main__":
    main()
