"""Host-side multi-rank logic of bench.py on CPU with gloo (world size 2): the slowest rank's
time is used on every rank, the whole-job rate counts every rank's units (weak scaling), and
the CPU reference arm runs on rank 0 only."""
import os
import socket
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    mx = bench.reduce_max_over_ranks(10.0 + 5.0 * rank)
    rate = bench.whole_job_rate(1000.0, mx, ws)
    env = bench.dist_env()

    class A:
        workload, warmup, steps, eps_pt2 = "tiny_n10", 0, 1, 0.0
    ref = bench.run_reference(A, ws, rank)
    dist.barrier()
    q.put((rank, mx, rate, env, ref is None))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, rate, env, ref_none in res:
        assert mx == 15.0                     # the slowest rank's time everywhere
        assert abs(rate - 2 * 1000.0 / 0.015) < 1e-6
        assert env == (2, rank, rank)
        assert ref_none == (rank != 0)        # reference arm: rank 0 only
