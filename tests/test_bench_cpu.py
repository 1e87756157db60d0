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


def test_oracle_agreement_counts_statuses_and_classes():
    import numpy as np
    g_status = np.array([1, 1, 1, 2, 1, 3])
    o_status = np.array([1, 1, 1, 2, 2, 3])
    g_fli = np.array([7.0, 2.0, 6.5, 9.0, 1.0, 0.0])
    o_fli = np.array([7.2, 2.1, 5.9, 9.0, 1.0, 0.0])
    a = bench.oracle_agreement(g_status, g_fli, o_status, o_fli, thr=6.0)
    assert a["orbits"] == 6 and a["status_agree"] == 5 / 6
    # finished in both: orbits 0, 1, 2; orbit 2 sits on opposite sides of 6
    assert a["class_orbits"] == 3 and a["class_agree"] == 2 / 3
    empty = bench.oracle_agreement([], [], [], [])
    assert empty["orbits"] == 0 and empty["status_agree"] is None and empty["class_agree"] is None


def test_register_occupancy_arithmetic():
    regs = {"_ZN6pnscan17k_integrate_queueILb0ELi2ELb0ELi4ELb1ELb0EEEvX": 253,
            "_ZN6pnscan17k_integrate_queueILb1ELi2ELb0ELi4ELb1ELb0EEEvX": 250,
            "_ZN6pnscan18k_integrate_staticILb0ELi4ELb0EEEvX": 210,
            "_ZN6pnscan16k_integrate_pairILb0ELi4ELb0EEEvX": 164}
    q = bench.register_occupancy({"schedule": 3, "block_size": 128, "register_variant": 4}, regs)
    # 253 -> 8,192 registers per warp: two 128-thread blocks, 8 warps per SM
    assert q == {"kernel": "k_integrate_queue", "registers_per_thread": 253, "block_size": 128,
                 "blocks_per_sm": 2, "warps_per_sm": 8}
    st = bench.register_occupancy({"schedule": 1, "block_size": 32}, regs)
    assert st["registers_per_thread"] == 210 and st["blocks_per_sm"] == 9 and st["warps_per_sm"] == 9
    pr = bench.register_occupancy({"schedule": 4, "block_size": 32}, regs)
    assert pr["registers_per_thread"] == 164 and pr["blocks_per_sm"] == 12
    assert bench.register_occupancy({"schedule": 2, "block_size": 128, "register_variant": 3}, regs) is None
    assert bench.register_occupancy({"schedule": 3}, {}) is None


def test_build_records_the_timed_kernels_registers():
    from paper_1802_00147_gb300 import build
    build.build()
    if not build.kernel_registers():
        build.build(force=True)
    regs = build.kernel_registers()
    q = bench.register_occupancy({"schedule": 3, "block_size": 128, "register_variant": 4}, regs)
    assert q is not None and 128 <= q["registers_per_thread"] <= 255 and q["blocks_per_sm"] >= 1
