"""Benchmark of the batched manifold-corrected PN scan on GB300.

One step = one pass of the whole hot path over one batch: grid set-up and
reference integrals on the device, integration of every orbit to t_end
(RK4 + manifold correction + FLI for both trajectories, in the schedule the
library's autotuner picks, replayed from a CUDA graph), final integrals and
the scan-level reduction.  Workload: the 314 x 314 (x0, theta) scan, seeded
synthetic cells, h = 1, t_end = 2e4.

The same JSON line also carries: the end-to-end rate through the C ABI with
host buffers, the roofline of the integrator, the CPU oracle's rate on the
host cores, the uneven 1e5-orbit batch, the same scan with the 2.5PN
radiation reaction, and the surrogate-adaptive 1024 x 1024 map against
integrating every cell (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(the reference arm of this build: plain FP64 C, OpenMP over orbits) on a
bounded sample of the same workload.  ``--profile`` runs the device path
alone (fixed shape, for ncu).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 orbit-steps/s (RK+manifold corr.+FLI), 314² scan; adaptive-scan speedup"
UNIT = "orbit-steps/s"
T_END = 2.0e4
H_STEP = 1.0

# Algorithmic FP64 flops of the kernel's formulation (fma = 2, add/sub/mul = 1,
# sqrt/rsqrt/reciprocal/division/log10 = 1 each), per trajectory-step:
#   4 x 217 (RHS) + 171 (RK4 stages) + 138 (correction: spin lengths, Newton
#   monomial set-up, scaling) + 43 (first Newton iteration, at alpha = beta = 1)
#   = 1220, plus 73 per further Newton iteration; per orbit-step two
#   trajectories, 5 for the termination test and 1.75 for the FLI
#   renormalisation amortised over 100 steps.
FLOPS_PER_TRAJ_STEP = 4 * 217 + 171 + 138 + 43
FLOPS_PER_NEWTON_ITER = 73
FLOPS_PER_ORBIT_STEP_EXTRA = 5 + 1.75
# With the 2.5PN radiation reaction each RK stage adds (rhs_rr): r.p, p.p,
# (n.p)^2, the A and B polynomials, the two scale factors, a = sr r + sp p and
# its addition to dp/dt, (dr/dt).a, L, J, J.L, |J|^-1 and the product (74), and
# the two reference-value updates (4): 78 per stage.
FLOPS_PER_RR_STAGE = 78
# Algorithmic DRAM bytes per orbit and run: the SoA state read once (main and
# shadow 2 x 12, reference integrals 8, FLI accumulator, t, beta, kappa1,
# kappa2: 37 doubles; nstep, status, Newton and skip counters, last kind:
# 5 int32) and written once (2 x 12 + 4 + 2 doubles, 5 int32).
STATE_BYTES_PER_ORBIT = (37 * 8 + 5 * 4) + (30 * 8 + 5 * 4)
# Nominal FP64 peak from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz.
FP64_PEAK_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the integrator
# over one scan_run of this workload, from ncu captures of
# `bench.py --profile --schedule S`, keyed by schedule.  Valid only
# for the kernel sources they were taken with: reported as null once any of
# these files differs from the recorded SHA-256.
TRAFFIC_SOURCES = {
    "paper_1802_00147_gb300/csrc/pn_device.cuh": "842840ddc516186f903346f6170f158988a3850a8ae369f0bc67e598617b7c45",
    "paper_1802_00147_gb300/csrc/pn_kernels.cu": "584e55448a9c6ef82addc40966aad17efda5c263909c36628465737020fc2ced",
    "paper_1802_00147_gb300/csrc/pn_kernels.cuh": "b96896c16a4511134e2587dfacf70a1be233dedbea094e41872b6caf91cdbc00",
}
# ncu --cache-control none, as the bench runs: the set-up kernels leave the
# state in L2 right before the run.
TRAFFIC_BYTES_PER_RUN = {3: 7795200 + 41977344,      # compacting schedule, chunk 62 (7 epochs)
                         2: 4466688 + 42416640}      # work-queue schedule, chunk 125 (one launch)


def traffic_per_run(schedule):
    import hashlib
    for path, digest in TRAFFIC_SOURCES.items():
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    return TRAFFIC_BYTES_PER_RUN.get(schedule)


def algorithmic_flops(orbit_steps, newton_iters):
    further = max(0, newton_iters - 2 * orbit_steps)     # iterations beyond each correction's first
    return (orbit_steps * (2 * FLOPS_PER_TRAJ_STEP + FLOPS_PER_ORBIT_STEP_EXTRA)
            + further * FLOPS_PER_NEWTON_ITER)


def workload(rank=0, orbits=0):
    from paper_1802_00147_gb300 import workloads as W
    cells = W.full_scan(seed=2 + rank)
    if orbits and orbits < cells.shape[0]:
        cells = W.subset(cells, orbits, seed=40)[0]
    return cells


def workload_desc(n):
    return {
        "workload": "314x314 (x0, theta) phase-space scan: x0 in [10,50], theta in [0,pi] "
                    "(both spins), beta~U[0.5,1], chi~U[0.5,1], seeded azimuths, p_y = 0.9 circular; "
                    "RK4 h=1 to t_end=2e4, manifold correction every step (Newton tol 1e-10), "
                    "FLI from two trajectories d0=1e-9 renormalised every 100 steps, threshold 6",
        "orbits": int(n), "h": H_STEP, "t_end": T_END,
        "l2": "inputs smaller than L2; a 256 MiB buffer is written before every timed step",
    }


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle
def cpu_oracle_rate(cells, target_s=15.0, steps_cap=20000):
    """Time the CPU oracle (OpenMP over orbits, all host cores) on a bounded
    sample of the workload to the benchmark's t_end; returns (orbit-steps/s,
    sample description, cores, seconds, (sample indices, oracle outputs))."""
    import oracle
    from paper_1802_00147_gb300 import workloads as W
    cores = oracle.max_threads()
    # calibrate on a small sample
    cal, _ = W.subset(cells, max(cores * 4, 64), seed=31)
    t0 = time.perf_counter()
    o = oracle.scan(oracle.setup_cells(cal[:, :9]), cal[:, W.BETA], H_STEP, 500, oracle.config())
    dt = time.perf_counter() - t0
    rate0 = o["t_stop"].sum() / H_STEP / dt
    nsteps = steps_cap
    m = int(max(cores, min(cells.shape[0], rate0 * target_s / nsteps)))
    m = max(cores, (m // cores) * cores)
    sub, idx = W.subset(cells, m, seed=32)
    y0 = oracle.setup_cells(sub[:, :9])
    t0 = time.perf_counter()
    o = oracle.scan(y0, sub[:, W.BETA], H_STEP, nsteps, oracle.config())
    dt = time.perf_counter() - t0
    steps_done = float(o["t_stop"].sum() / H_STEP)
    return (steps_done / dt, "%d seeded orbits of the 314x314 scan to t_end=%g (%d orbit-steps, %.1f s)"
            % (m, nsteps * H_STEP, steps_done, dt), cores, dt, (idx, o))


# The integrator each tuned shape runs (conservative, RK4), as the kernel
# symbols ptxas reports: k_integrate_queue<QM, MINB, SMEM, RK, ROLLED, RR>
# per register_variant, k_integrate_static<QM, RK, RR>, k_integrate_pair<QM, RK, RR>.
_QUEUE_VARIANT = {4: "k_integrate_queueILb0ELi2ELb0ELi4ELb1ELb0E", 2: "k_integrate_queueILb0ELi2ELb0ELi4ELb0ELb0E",
                  3: "k_integrate_queueILb0ELi3ELb1ELi4ELb1ELb0E"}


def register_occupancy(shape, registers):
    """Registers per thread of the integrator a tuned shape runs (from the
    build's ptxas report) and the resident blocks and warps per SM they allow
    (65,536 registers per SM, allocated per warp in units of 256)."""
    sched, block = shape.get("schedule"), shape.get("block_size") or 128
    if sched in (2, 3):
        key = _QUEUE_VARIANT.get(shape.get("register_variant") or 4)
    else:
        key = {1: "k_integrate_staticILb0ELi4ELb0E", 4: "k_integrate_pairILb0ELi4ELb0E"}.get(sched)
    found = [v for k, v in registers.items() if key and key in k]
    if len(found) != 1:
        return None
    regs = found[0]
    per_warp = -(-regs * 32 // 256) * 256
    blocks = min(32, 65536 // (per_warp * (block // 32)))
    return {"kernel": key.split("I")[0], "registers_per_thread": regs, "block_size": block,
            "blocks_per_sm": blocks, "warps_per_sm": blocks * block // 32}


def oracle_agreement(g_status, g_fli, o_status, o_fli, thr=6.0):
    """The timed run against the oracle on the same orbits (the CPU-baseline
    sample, integrated to the same t_end): fraction of equal statuses, and
    among the orbits both finished, fraction of equal classes (FLI > thr)."""
    g_status, o_status = np.asarray(g_status), np.asarray(o_status)
    same = g_status == o_status
    done = same & (o_status == 1)                # DONE in both numberings
    cls = (np.asarray(g_fli)[done] > thr) == (np.asarray(o_fli)[done] > thr)
    return {"orbits": int(o_status.size), "status_agree": float(same.mean()) if same.size else None,
            "class_orbits": int(cls.size), "class_agree": float(cls.mean()) if cls.size else None,
            "threshold": thr}


def cpu_oracle_rate_single_core(cells, m=64, nsteps=20000):
    """The oracle on one host core: m seeded orbits of the workload to t_end
    (about 1 s of CPU work); returns orbit-steps/s."""
    import oracle
    from paper_1802_00147_gb300 import workloads as W
    sub, _ = W.subset(cells, m, seed=33)
    y0 = oracle.setup_cells(sub[:, :9])
    t0 = time.perf_counter()
    o = oracle.scan(y0, sub[:, W.BETA], H_STEP, nsteps, oracle.config(), nthreads=1)
    dt = time.perf_counter() - t0
    return float(o["t_stop"].sum() / H_STEP) / dt


# -------------------------------------------------------------- reference
def run_reference(args, rank, world):
    if rank != 0:
        return
    cells = workload()
    # calibrate once; every step is the same bounded sample
    rate, sample, cores, dt, _ = cpu_oracle_rate(cells, target_s=8.0)
    import oracle
    from paper_1802_00147_gb300 import workloads as W
    m = int(sample.split()[0])
    sub, _ = W.subset(cells, m, seed=32)
    y0 = oracle.setup_cells(sub[:, :9])
    for _ in range(args.warmup):
        oracle.scan(y0, sub[:, W.BETA], H_STEP, int(T_END / H_STEP), oracle.config())
    t0 = time.perf_counter()
    steps = 0.0
    for _ in range(args.steps):
        o = oracle.scan(y0, sub[:, W.BETA], H_STEP, int(T_END / H_STEP), oracle.config())
        steps += float(o["t_stop"].sum() / H_STEP)
    dt = time.perf_counter() - t0
    value = steps / dt
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_desc(cells.shape[0]), sample=sample),
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "each step: " + sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def aggregate_ranks(elapsed_s, orbit_steps, device=None):
    """Whole-job timing across ranks: the slowest rank's time and the sum of
    every rank's orbit-steps (each rank integrates its own batch).  Single
    process when torch.distributed is not initialised."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return float(elapsed_s), float(orbit_steps)
    t = torch.tensor([float(elapsed_s), float(orbit_steps)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    mx = t[:1].clone()
    td.all_reduce(mx, op=td.ReduceOp.MAX)
    sm = t[1:].clone()
    td.all_reduce(sm, op=td.ReduceOp.SUM)
    return float(mx.item()), float(sm.item())


SUMMARY_SUM_KEYS = ("n_chaotic", "newton_iters", "n_skip", "orbit_steps", "n_final_fallback")
SUMMARY_MAX_KEYS = ("max_dE", "max_dJ", "max_dJ_all", "max_dS")


def aggregate_summary(summ, device=None):
    """The scan counters of the whole job: counts summed over ranks (the
    status histogram too), maximal drifts maximised, the FLI mean weighted by
    each rank's finished orbits.  Each rank scans its own batch, so this is
    the one exchange of the multi-GPU path, after the timed region."""
    import torch
    import torch.distributed as td
    out = {k: summ[k] for k in SUMMARY_SUM_KEYS + SUMMARY_MAX_KEYS + ("status_count", "fli_mean")}
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return out
    dev = device if device is not None else "cpu"
    done = float(summ["status_count"][1])
    sums = torch.tensor([float(summ[k]) for k in SUMMARY_SUM_KEYS] + [float(c) for c in summ["status_count"]]
                        + [summ["fli_mean"] * done], dtype=torch.float64, device=dev)
    maxs = torch.tensor([float(summ[k]) for k in SUMMARY_MAX_KEYS], dtype=torch.float64, device=dev)
    td.all_reduce(sums, op=td.ReduceOp.SUM)
    td.all_reduce(maxs, op=td.ReduceOp.MAX)
    sums = sums.cpu().tolist()
    maxs = maxs.cpu().tolist()
    ns = len(SUMMARY_SUM_KEYS)
    for i, k in enumerate(SUMMARY_SUM_KEYS):
        out[k] = int(round(sums[i]))
    out["status_count"] = [int(round(v)) for v in sums[ns:ns + 6]]
    out["fli_mean"] = sums[ns + 6] / max(1, out["status_count"][1])
    for i, k in enumerate(SUMMARY_MAX_KEYS):
        out[k] = maxs[i]
    return out


def torchrun_argv(nproc, argv, port):
    """The command that runs this script once per GPU of this node (one rank
    per GPU, rendezvous on 127.0.0.1) with the same arguments."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=%d" % nproc,
            "--master-addr=127.0.0.1", "--master-port=%d" % port, os.path.abspath(__file__)] + list(argv)


def launch_check(gpus, env):
    """None to run in this process, or the number of ranks to spawn.  Under
    a launcher (WORLD_SIZE set) --gpus must match the world size."""
    world = env.get("WORLD_SIZE")
    if world is None:
        return gpus if gpus > 1 else None
    if int(world) != gpus:
        raise SystemExit("bench.py: --gpus %d but WORLD_SIZE=%s: give --gpus the launcher's process count"
                         % (gpus, world))
    return None


# --------------------------------------------------------- adaptive scan
ADAPTIVE_N = 1024
ADAPTIVE_T_END = 1.0e4
# Adam steps per ensemble member (one persistent training launch, ~0.5 s).
# Every cell of this grid that the surrogate marks is marked for ensemble
# disagreement (none is predicted within 1 of the threshold), so a
# better-converged ensemble marks fewer cells: 4,000 steps marked 4.1 % of
# the grid, 12,000 steps 0.7 %.
ADAPTIVE_TRAIN_STEPS = 12000


def run_adaptive(cells_full, cells_full_d, fli_full_d, thr=6.0, band=1.0, spread_max=0.5):
    """Surrogate-adaptive 1024 x 1024 scan of the small-scan parameters vs
    integrating every cell: time-to-map and misclassification."""
    import torch
    from paper_1802_00147_gb300 import adaptive as A
    from paper_1802_00147_gb300 import workloads as W
    import paper_1802_00147_gb300 as pn

    small = W.small_scan(seed=1)
    grid = W.adaptive_grid(ADAPTIVE_N, seed=4)
    grid_d = torch.as_tensor(np.ascontiguousarray(grid[:, :9]), device="cuda")
    # warm-up of every timed path on tiny inputs: the first use of a PyTorch
    # CUDA operation (comparisons, masked indexing) loads its kernels, which
    # took seconds and would be charged to whichever path came first
    A.training_set([small[:32]], [10.0])
    A.full_map(grid_d[:64], 10.0, thr=thr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xs, ys = A.training_set([small], [ADAPTIVE_T_END])
    Xf = pn.adaptive_features(cells_full_d)
    X = torch.cat([Xs, Xf])
    y = torch.cat([ys, fli_full_d.float()])
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0          # integrating the small scan (the full one is reused)
    t0 = time.perf_counter()
    sur, hist = A.train_surrogate(X, y, members=5, steps=ADAPTIVE_TRAIN_STEPS, lr=3e-3, seed=1)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0

    A.adaptive_map(sur, grid_d[:4096], ADAPTIVE_T_END, thr=thr, band=band, spread_max=spread_max)  # warm-up
    full = A.full_map(grid_d, ADAPTIVE_T_END, thr=thr)
    sub, sub_idx = W.subset(grid, 4096, seed=6)
    sub_idx_d = torch.as_tensor(sub_idx, device="cuda")
    out = {"grid": "%dx%d" % (ADAPTIVE_N, ADAPTIVE_N), "t_end": ADAPTIVE_T_END, "members": 5,
           "train_steps": ADAPTIVE_TRAIN_STEPS, "train_rows": int(X.shape[0]), "train_s": train_s,
           "training_data_s": data_s,
           "train_loss_first_last": [float(hist[:, :20].mean()), float(hist[:, -200:].mean())],
           "plain_s": full["seconds"]}
    for name, th, bd, sp in [("thr6", thr, band, spread_max)]:
        res = A.adaptive_map(sur, grid_d, ADAPTIVE_T_END, thr=th, band=bd, spread_max=sp)
        truth = A.classes(full["fli"], full["status"], th)
        mis_all = float((res["cls"] != truth).float().mean().item())
        mis_sub = float((res["cls"][sub_idx_d] != truth[sub_idx_d]).float().mean().item())
        out[name] = {"thr": th, "band": bd, "spread_max": sp, "marked": res["n_marked"],
                     "marked_frac": res["n_marked"] / grid.shape[0], "adaptive_s": res["seconds"],
                     "surrogate_s": res["seconds_surrogate"],
                     "speedup": full["seconds"] / res["seconds"],
                     "speedup_incl_training": full["seconds"] / (res["seconds"] + train_s),
                     "speedup_incl_training_and_data": full["seconds"] / (res["seconds"] + train_s + data_s),
                     "misclassification_subset4096": mis_sub, "misclassification_all": mis_all,
                     "chaotic_frac": float(truth.float().mean().item())}
    sur.close()
    return out


# ------------------------------------- adaptive scan on a boundary-rich plane
def run_adaptive_boundary():
    """The surrogate-adaptive map and the no-learning coarse-grid map against
    integrating every cell, on the (theta1, theta2) plane of Sec. 3C, Fig. 7
    (512 x 512, RK4 h = 1 to t_end = 1e4, no merger or escape cut as in the
    paper's scan, threshold 5.8): a plane with an order/chaos boundary."""
    from paper_1802_00147_gb300 import adaptive as A
    rep = A.boundary_study(n=512, t_end=1.0e4, thr=5.8, stride=8, r_merge=0.0, r_escape=0.0)
    # the surrogate trained on the neighbouring planes only (x0 = 9.9 ... 10.4 at the same fraction of
    # the circular momentum): no cell of the mapped plane is integrated before the map
    tr = A.boundary_study(n=512, t_end=1.0e4, thr=5.8, stride=8, r_merge=0.0, r_escape=0.0,
                          train_x0=(9.9, 10.0, 10.3, 10.4))
    rep["surrogate_trained_on_other_planes"] = tr["surrogate"]
    for r in (rep["surrogate"], rep["baseline"], rep["surrogate_trained_on_other_planes"]):
        r["n_points"] = len(r.pop("points"))   # the sweeps stay out of the bench line: the chosen points go in
    return rep


# ----------------------------------------------------------- uneven batch
def run_uneven(n=100_000, t_end=2.0e4):
    """The uneven batch (mass ratio 0.1-1, isotropic spins, p_y 50-100% of
    circular; merger / escape / FLI-saturation cut-offs), autotuned schedule,
    one timed run through the CUDA graph."""
    import torch
    import paper_1802_00147_gb300 as pn
    from paper_1802_00147_gb300 import workloads as W
    cells = W.uneven_batch(n, seed=3)
    cd = torch.as_tensor(np.ascontiguousarray(cells[:, :9]), device="cuda")
    with pn.Scan(None, device=True, n=n, fli_cap=12.0) as s:
        s.setup(cd)
        shape = s.autotune(2000)
        for _ in range(2):                      # warm-up (and graph capture), then timed
            s.setup(cd)
            s.run(t_end, H_STEP)
            summ = s.summary()
        ms, _ = s.last_run_timing()
    return {"workload": "uneven batch: 1e5 orbits, beta~U[0.1,1], chi~U[0,1], isotropic spins, "
                        "x0~U[10,50], p_y 50-100% of circular; stops at r<6, r>1e3, FLI>=12; t_end 2e4",
            "schedule": shape, "kernel_ms": ms, "orbit_steps": summ["orbit_steps"],
            "value": summ["orbit_steps"] / (ms * 1e-3), "unit": UNIT,
            "status_count": summ["status_count"],
            "newton_iters_per_orbit_step": summ["newton_iters"] / max(1, summ["orbit_steps"]),
            "tflops_algorithmic": algorithmic_flops(summ["orbit_steps"], summ["newton_iters"]) / (ms * 1e-3) / 1e12}


# ------------------------------------------------------ radiation reaction
def run_dissipative(t_end=5.0e3):
    """The 314 x 314 scan with the 2.5PN radiation reaction (Eq. 6; the
    reference E and |J| carried by their integral-invariant relations,
    Sec. 3B), autotuned schedule: one timed run after a warm-up.  Close
    binaries merge early, so the batch is uneven."""
    import torch
    import paper_1802_00147_gb300 as pn
    cells = workload(0)
    n = cells.shape[0]
    cd = torch.as_tensor(np.ascontiguousarray(cells[:, :9]), device="cuda")
    with pn.Scan(None, device=True, n=n, radiation_reaction=1) as s:
        s.setup(cd)
        shape = s.autotune(1000)
        for _ in range(2):                      # warm-up (and graph capture), then timed
            s.setup(cd)
            s.run(t_end, H_STEP)
            summ = s.summary()
        ms, _ = s.last_run_timing()
    flops = (summ["orbit_steps"] * (2 * (FLOPS_PER_TRAJ_STEP + 4 * FLOPS_PER_RR_STAGE) + FLOPS_PER_ORBIT_STEP_EXTRA)
             + max(0, summ["newton_iters"] - 2 * summ["orbit_steps"]) * FLOPS_PER_NEWTON_ITER)
    achieved = flops / (ms * 1e-3) / 1e12
    return {"workload": "314x314 scan (as the headline) with the 2.5PN radiation reaction, harmonic gauge, "
                        "RK4 h=1 to t_end=5e3, merger cut r<6",
            "schedule": shape, "kernel_ms": ms,
            "orbit_steps": summ["orbit_steps"], "value": summ["orbit_steps"] / (ms * 1e-3), "unit": UNIT,
            "status_count": summ["status_count"],
            "newton_iters_per_orbit_step": summ["newton_iters"] / max(1, summ["orbit_steps"]),
            "tflops_algorithmic": achieved, "frac": achieved / FP64_PEAK_NOMINAL_TFLOPS,
            "max_dE_vs_reference": summ["max_dE"]}


# -------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1802_00147_gb300 as pn
    from paper_1802_00147_gb300 import build as pnbuild
    from paper_1802_00147_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    pnbuild.build()
    dist = world > 1
    if dist:
        import torch.distributed as td
    if args.profile and args.uneven:
        # the uneven batch (or a seeded subset of it), for profiling only
        cells_h = W.uneven_batch(args.orbits or 100_000, seed=3)
    else:
        cells_h = workload(rank, args.orbits)
    n = cells_h.shape[0]
    t_end = args.t_end
    dev = torch.device("cuda", local_rank)
    cells_d = torch.as_tensor(np.ascontiguousarray(cells_h[:, :9]), device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    sched_code = {"auto": 0, "static": 1, "queue": 2, "compact": 3, "pair": 4}[args.schedule]
    prof_opts = dict(schedule=sched_code, chunk_steps=args.chunk, block_size=args.block) if args.profile else {}
    if args.profile and args.dissipative:
        prof_opts["radiation_reaction"] = 1
    if args.profile and args.uneven:
        prof_opts["fli_cap"] = 12.0
    scan = pn.Scan(cells_h[:, W.BETA], device=True, **prof_opts)
    scan.setup(cells_d)
    if args.profile:
        shape = {"schedule": sched_code, "block_size": args.block or 0, "chunk_steps": args.chunk or 500,
                 "blocks_per_sm": 0}
        fp64_measured = float("nan")
    else:
        shape = scan.autotune(2000)
        fp64_measured = scan.fp64_peak(400_000)

    def step():
        flush.fill_(1)
        scan.setup(cells_d)
        scan.run(t_end, H_STEP)
        return scan.summary()          # final integrals + reduction; synchronises

    for _ in range(args.warmup):
        summ = step()
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    kern_ms = []
    run_launches = []
    steps_total = 0
    iters_total = 0
    with ClockSampler(local_rank) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            summ = step()
            ms_run, nl = scan.last_run_timing()
            kern_ms.append(ms_run)
            run_launches.append(nl)
            steps_total += summ["orbit_steps"]
            iters_total += summ["newton_iters"]
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            td.barrier()
    elapsed, steps_all = aggregate_ranks(ev0.elapsed_time(ev1) / 1e3, steps_total, dev if dist else None)
    value = steps_all / elapsed
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile_run": True, "orbits": n, "t_end": t_end, "value": value,
                              "ms_per_step": elapsed / args.steps * 1e3,
                              "kernel_ms": float(np.mean(kern_ms))}), flush=True)
        scan.close()
        return

    # end-to-end through the C ABI with host buffers (H2D of the cells and
    # D2H of the per-orbit results inside the timed region), with the shape
    # the device timing was tuned to
    tuned = {k: shape[k] for k in ("schedule", "block_size", "chunk_steps", "blocks_per_sm", "register_variant")
             if shape.get(k)}
    host = pn.Scan(cells_h[:, W.BETA], device=False, **tuned)
    cells9 = np.ascontiguousarray(cells_h[:, :9])
    out = dict(states=np.empty((n, 12)), integrals=np.empty((n, 6)), fli=np.empty(n),
               status=np.empty(n, np.int32), t_stop=np.empty(n))
    host.setup(cells9)
    host.run(t_end, H_STEP)
    pn.scan_read(host.h, **out)
    torch.cuda.synchronize()
    if dist:
        td.barrier()
    t0 = time.perf_counter()
    e2e_steps = 0
    e2e_k = max(1, args.steps)
    for _ in range(e2e_k):
        flush.fill_(1)
        host.setup(cells9)
        host.run(t_end, H_STEP)
        pn.scan_read(host.h, **out)
        e2e_steps += int(np.round(out["t_stop"].sum() / H_STEP))
    e2e_dt = time.perf_counter() - t0
    host.close()
    # whole job: the slowest rank's time, every rank's orbit-steps and bytes
    e2e_dt, e2e_steps = aggregate_ranks(e2e_dt, e2e_steps, dev if dist else None)
    h2d = cells9.nbytes * world
    d2h = sum(a.nbytes for a in out.values()) * world

    job_summary = aggregate_summary(summ, dev if dist else None)
    uneven = run_uneven() if (rank == 0 and args.adaptive) else None
    dissipative = run_dissipative() if (rank == 0 and args.adaptive) else None
    adaptive = None
    if args.adaptive and rank == 0:
        fli_full = scan.read()["fli"]
        adaptive = run_adaptive(cells_h, cells_d, fli_full)
        adaptive["boundary_plane"] = run_adaptive_boundary()

    if rank != 0:
        return
    ms_kernel = float(np.mean(kern_ms))
    flops = algorithmic_flops(summ["orbit_steps"], summ["newton_iters"])
    achieved = flops / (ms_kernel * 1e-3) / 1e12
    traffic = traffic_per_run(shape["schedule"])
    cpu_rate, cpu_sample, cores, _, (cpu_idx, cpu_out) = cpu_oracle_rate(cells_h, target_s=15.0)
    occupancy = register_occupancy(shape, pnbuild.kernel_registers())
    try:
        final = scan.read()
        host = {k: (v.cpu().numpy() if hasattr(v, "cpu") else np.asarray(v)) for k, v in final.items()}
        agreement = oracle_agreement(host["status"][cpu_idx], host["fli"][cpu_idx],
                                     cpu_out["status"], cpu_out["fli"])
    except Exception as e:          # a diagnostic must not cost the benchmark line
        agreement = {"error": repr(e)}
    cpu_rate_1 = cpu_oracle_rate_single_core(cells_h)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_desc(n), schedule=shape, parallelism="dp%d (independent scans)" % world),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_NOMINAL_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_NOMINAL_TFLOPS, "traffic": traffic,
                     "kernel": "k_integrate_queue",
                     "per": "scan_run: one integrator launch (queue schedule) or one per epoch with a "
                            "compaction between epochs (compacting schedule); achieved, flops and "
                            "traffic are per run",
                     "launches_per_run": int(run_launches[-1]), "kernel_ms": ms_kernel,
                     "flops_per_run": flops,
                     "traffic_algorithmic_bytes": int(n * STATE_BYTES_PER_ORBIT),
                     "peak_measured_dfma": fp64_measured,
                     "frac_of_measured": achieved / fp64_measured,
                     "occupancy": occupancy},
        "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": cpu_sample, "agreement_with_this_run": agreement,
                         "single_core_value": cpu_rate_1,
                         "single_core_sample": "64 seeded orbits of the 314x314 scan to t_end=2e4 on one core"},
        "e2e": {"value": e2e_steps / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        # per step: k_setup_cells, k_init, the run's integrator (+ compaction) launches,
        # k_finalize, k_reduce
        "gpu_launches": int(sum(4 + nl for nl in run_launches)),
        "clocks": clk.summary(),
        "adaptive": adaptive,
        "uneven": uneven,
        "dissipative": dissipative,
        "scan": job_summary,
    }
    print(json.dumps(line), flush=True)
    scan.close()


def run_profile_surrogate(steps):
    """Surrogate training alone, for ncu runs: 5 members on 20,000 seeded
    synthetic rows (the scan's input ranges, a smooth target); one untimed
    launch of 200 Adam steps, then one timed launch of `steps`."""
    import torch
    import paper_1802_00147_gb300 as pn
    from paper_1802_00147_gb300 import build as pnbuild
    pnbuild.build()
    rng = np.random.default_rng(4)
    X = np.stack([rng.uniform(10, 50, 20000), rng.uniform(0, np.pi, 20000), rng.uniform(0.1, 1, 20000),
                  rng.uniform(0, 1, 20000)], axis=1).astype(np.float32)
    y = (np.sin(X[:, 0] / 10) + 2.0).astype(np.float32)
    Xd, yd = torch.as_tensor(X, device="cuda"), torch.as_tensor(y, device="cuda")
    with pn.Surrogate(members=5, seed=11) as sur:
        sur.train(Xd, yd, steps=200, lr=3e-3, seed=5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist = sur.train(Xd, yd, steps=steps, lr=3e-3, seed=6)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    print(json.dumps({"profile_surrogate": True, "members": 5, "steps": steps, "seconds": dt,
                      "us_per_step": dt / steps * 1e6, "loss_last": float(hist[:, -1].mean())}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--orbits", type=int, default=0,
                    help="seeded subset of the 314x314 scan (0: all 98,596); profiling only")
    ap.add_argument("--t-end", type=float, default=T_END, help="integration time (profiling only)")
    ap.add_argument("--no-adaptive", dest="adaptive", action="store_false",
                    help="skip the uneven-batch and surrogate-adaptive 1024x1024 measurements")
    ap.add_argument("--schedule", choices=["auto", "static", "queue", "compact", "pair"], default="auto",
                    help="schedule for --profile runs (default: the library's AUTO choice)")
    ap.add_argument("--block", type=int, default=0, help="threads per block for --profile runs (0: default)")
    ap.add_argument("--chunk", type=int, default=0, help="steps per task for --profile runs (0: 500)")
    ap.add_argument("--profile", action="store_true",
                    help="time the device path only (no autotune, e2e or CPU leg) for ncu runs")
    ap.add_argument("--dissipative", action="store_true",
                    help="--profile runs with the 2.5PN radiation reaction")
    ap.add_argument("--uneven", action="store_true",
                    help="--profile runs on the uneven batch (--orbits of it; FLI cap 12)")
    ap.add_argument("--profile-surrogate", type=int, default=0, metavar="STEPS",
                    help="time STEPS steps of surrogate training alone (5 members), for ncu runs")
    args = ap.parse_args()
    if args.profile_surrogate:
        run_profile_surrogate(args.profile_surrogate)
        return
    spawn = launch_check(args.gpus, os.environ)
    if spawn:
        # one process per GPU: re-run this script under torch.distributed.run
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        sys.exit(subprocess.call(torchrun_argv(spawn, sys.argv[1:], port)))
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
