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


def _rank_summary(rank, world, port, out):
    import torch.distributed as td
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        summ = {"n_chaotic": 3 + rank, "newton_iters": 100 * (rank + 1), "n_skip": rank, "orbit_steps": 1000,
                "n_final_fallback": 0, "max_dE": 1e-15 * (rank + 1), "max_dJ": 2e-16 * (2 - rank),
                "max_dJ_all": 3e-16, "max_dS": 1e-16, "status_count": [0, 10 + rank, 5, 0, 0, 0],
                "fli_mean": 2.0 + rank}
        out.put((rank, bench.aggregate_summary(summ)))
        td.barrier()
    finally:
        td.destroy_process_group()


def test_two_gloo_ranks_aggregate_the_scan_counters():
    """The job's scan object: counts and the status histogram summed over
    ranks, drifts maximised, the FLI mean weighted by finished orbits."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_summary, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, s in res:
        assert s["n_chaotic"] == 7 and s["newton_iters"] == 300 and s["n_skip"] == 1
        assert s["orbit_steps"] == 2000 and s["status_count"] == [0, 21, 10, 0, 0, 0]
        assert s["max_dE"] == 2e-15 and s["max_dJ"] == 4e-16 and s["max_dJ_all"] == 3e-16
        assert abs(s["fli_mean"] - (2.0 * 10 + 3.0 * 11) / 21) < 1e-12


def test_launch_check_spawns_or_insists_on_a_matching_world():
    import bench
    assert bench.launch_check(1, {}) is None
    assert bench.launch_check(4, {}) == 4
    assert bench.launch_check(2, {"WORLD_SIZE": "2"}) is None
    with pytest.raises(SystemExit):
        bench.launch_check(8, {"WORLD_SIZE": "1"})
    argv = bench.torchrun_argv(4, ["--gpus", "4", "--steps", "2"], 29511)
    assert argv[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in argv and "--master-addr=127.0.0.1" in argv
    assert argv[-4:] == ["--gpus", "4", "--steps", "2"]


@pytest.mark.slow
def test_bench_gpus_2_runs_two_ranks():
    """`bench.py --gpus 2` without a launcher starts two ranks through
    torch.distributed.run; with the reference arm (the CPU oracle) rank 0
    alone prints its line and both exit 0."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                       cwd=root, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
