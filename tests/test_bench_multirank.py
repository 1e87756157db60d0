"""The multi-GPU bench path on CPU ranks (gloo, world size 2): each rank
integrates its own batch, the job's time is the slowest rank's and its
orbit-steps the sum over ranks; ranks draw different seeded batches."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as td
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = 1.5 + rank            # rank 1 is the slow one
        steps = 1000 * (rank + 1)
        t, n = bench.aggregate_ranks(elapsed, steps)
        cells = bench.workload(rank)
        out.put((rank, t, n, float(cells[:, 3].sum())))
        td.barrier()
    finally:
        td.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_summed_steps():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, n, _ in res:
        assert t == 2.5 and n == 3000.0
    assert res[0][3] != res[1][3]          # each rank scans its own seeded batch


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate_ranks(2.0, 7) == (2.0, 7.0)
