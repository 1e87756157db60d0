"""Host logic of the benchmark's roofline: the algorithmic flop count and the
rule that recorded DRAM traffic is reported only for the kernel sources it
was captured with."""
import hashlib
import os

import pytest

import bench


def test_algorithmic_flops_per_orbit_step():
    per = 2 * bench.FLOPS_PER_TRAJ_STEP + bench.FLOPS_PER_ORBIT_STEP_EXTRA
    # two trajectories, one Newton iteration each: no further iterations
    assert bench.algorithmic_flops(1, 2) == pytest.approx(per)
    assert bench.algorithmic_flops(1000, 2000) == pytest.approx(1000 * per)
    # every iteration beyond each correction's first adds its cost
    assert bench.algorithmic_flops(1000, 2240) == pytest.approx(1000 * per + 240 * bench.FLOPS_PER_NEWTON_ITER)
    # fewer iterations than corrections (skipped solves) never subtract
    assert bench.algorithmic_flops(1000, 1500) == pytest.approx(1000 * per)
    assert bench.FLOPS_PER_TRAJ_STEP == 4 * 217 + 171 + 138 + 43


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    live = {}
    for path in bench.TRAFFIC_SOURCES:
        with open(os.path.join(bench.ROOT, path), "rb") as f:
            live[path] = hashlib.sha256(f.read()).hexdigest()
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES", live)
    for sched, nbytes in bench.TRAFFIC_BYTES_PER_RUN.items():
        assert bench.traffic_per_run(sched) == nbytes
    assert bench.traffic_per_run(99) is None
    stale = dict(live)
    stale[next(iter(stale))] = "0" * 64
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES", stale)
    assert all(bench.traffic_per_run(s) is None for s in bench.TRAFFIC_BYTES_PER_RUN)


def test_traffic_stays_below_the_algorithmic_bytes():
    # one read and one write of the state per orbit bound what a run must move
    n = 314 * 314
    for nbytes in bench.TRAFFIC_BYTES_PER_RUN.values():
        assert 0 < nbytes <= n * bench.STATE_BYTES_PER_ORBIT
