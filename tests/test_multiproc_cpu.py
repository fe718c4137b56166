"""Multi-rank host logic of bench.py on the CPU: two processes joined by the
gloo backend (the path `bench.py --gpus N` takes under torchrun, minus the
GPU work) agree on the barrier, take the maximum time over ranks and scale
the aggregate throughput by the world size; the reference arm runs on rank 0
only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (ws, rank, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    # rank r "took" (r + 1) * 1.5 s: the job's time is the slowest rank's
    t = bench.max_over_ranks((rank + 1) * 1.5, w)
    value = 1000 * 3 * w / t   # 1000 queries x 3 steps per rank
    # the reference arm does nothing on ranks other than 0
    class A:
        steps, warmup, ref_queries = 1, 0, 1
    if rank != 0:
        bench.run_reference(A, w, rank)
    bench.barrier(w)
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write("%r %r\n" % (t, value))
    dist.destroy_process_group()


def test_two_rank_gloo_barrier_and_max(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       start_method="spawn", join=True)
    vals = [open(tmp_path / ("rank%d.txt" % r)).read().split() for r in range(ws)]
    for t, value in vals:
        assert float(t) == 3.0
        assert abs(float(value) - 2000.0) < 1e-9
