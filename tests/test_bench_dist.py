"""The multi-rank (torchrun) path of bench.py on CPU: two gloo ranks.

bench.py runs one process per GPU. Each rank solves its own seeded problem
(independent units, no data-path collective), and the ranks meet only at a
barrier and a max-reduction of their timings. Here the same helpers run on
the gloo backend: the max over ranks, the whole-job value from the slowest
rank's time, per-rank seeds that give different problems, and the reference
arm's rule that only rank 0 works.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.barrier(ws)
        t = bench.allmax(ws, 10.0 + 5.0 * rank)            # per-rank "ms"
        tb, A = bench.workload(64, seed=rank)
        v = bench.whole_job_tflops(ws, 1e12, t)
        # the reference arm: ranks other than 0 return at once without output
        class Args:
            n, steps, warmup, gpus = 64, 1, 0, ws
        if rank != 0:
            bench.run_reference(Args, ws, rank)
        out.put((rank, t, v, float(np.abs(tb.H).sum()), float(np.abs(A).sum())))
        bench.barrier(ws)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, h0, a0), (r1, t1, v1, h1, a1) = res
    assert t0 == t1 == 15.0                      # both ranks see the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 1e12 / 15e-3 / 1e12)   # all ranks' work / that time
    assert h0 != h1 and a0 != a1                 # each rank solves its own seeded problem
