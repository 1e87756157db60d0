"""Scan studies built on the library's C ABI.

Quadrupole-monopole drift study: the small-scan parameter grid (equal
masses, chi = 1) with the spin-induced quadrupole-monopole term on and
kappa_i ~ U[1, 10] (Eqs. 4-5 with kappa multipliers), RK4 at h = 0.5 to
t_end = 1e5; the drift of E, |J| and the spin lengths over the orbits that
reach t_end is reported with and without the manifold correction
(Eqs. 10-13).

    python -m paper_1802_00147_gb300.studies qm [--n 1024] [--subset 65536] [--t-end 1e5]

The paper's own scans (Sec. 3C, Figs. 6-7), with the fifth-order base
integrator and the paper's FLI threshold 5.8; the FLI maps are written as
.npy files (no graphics):

    python -m paper_1802_00147_gb300.studies paper [--t-end 1e5] [--out DIR]

Newton-tolerance ablation (Sec. 3A, Fig. 4) over a scan grid: the energy
drift at t_end for eps = 1e-6, 1e-8, 1e-10 under both Newton stopping rules
(apply a step and then test it; stop before applying a step within eps),
RK5 at h = 1:

    python -m paper_1802_00147_gb300.studies newton [--n 64] [--t-end 1e4]

Correction ablation over the same grid: drift of E, |J| and |S_i| at t_end
with no correction, the spin lengths alone (Eq. 10), the spin lengths and
velocity scaling p = a p* to E0 (Sec. 1), and the full dual scaling:

    python -m paper_1802_00147_gb300.studies ablation [--n 64] [--t-end 1e4]

Gravitational waveforms (Eq. 14, Sec. 4, Fig. 10, conservative case): h_plus
and h_cross of the mass quadrupole field along the regular orbit 4 and the
chaotic case II orbit 2, observer on the z axis, written as .npy:

    python -m paper_1802_00147_gb300.studies waveform [--t-end 1e4] [--out DIR]

FLI against time (Sec. 3B, Fig. 3): case II orbits 1 (regular: power-law
growth) and 2 (chaotic: exponential growth), corrected RK5 to t = 1e5:

    python -m paper_1802_00147_gb300.studies fli [--t-end 1e5] [--out DIR]

Non-conservative orbit 3 (Sec. 3B, Fig. 5) with the 2.5PN radiation
reaction: |r|, the energy and its integral-invariant reference, sampled until
the merger cut, corrected and uncorrected RK5:

    python -m paper_1802_00147_gb300.studies orbit3 [--t-end 3e5] [--out DIR]

Fig. 10's non-conservative waveforms (radiation reaction on, until the
merger cut) for orbit 4 and case II orbit 2:

    python -m paper_1802_00147_gb300.studies waveform --dissipative [--out DIR]
"""
import argparse
import json
import time

import numpy as np

from . import ORBIT_DONE, Scan
from . import workloads as W


def drift_stats(out, spin_ref):
    """Relative drift of E, |J| and |S_i| over the orbits that reached t_end."""
    st = out["status"].cpu().numpy()
    I = out["integrals"].cpu().numpy()
    done = st == ORBIT_DONE
    dE = np.abs((I[done, 1] - I[done, 0]) / I[done, 0])
    dJ = np.abs((I[done, 3] - I[done, 2]) / I[done, 2])
    sr = spin_ref[done]
    dS = np.maximum(np.abs(I[done, 4] - sr[:, 0]) / sr[:, 0], np.abs(I[done, 5] - sr[:, 1]) / sr[:, 1])

    def q(a):
        return {"max": float(a.max()) if a.size else None, "median": float(np.median(a)) if a.size else None}

    return {"done": int(done.sum()), "status_count": np.bincount(st, minlength=6).tolist(),
            "dE": q(dE), "dJ": q(dJ), "dS": q(dS)}


def qm_drift_study(n=1024, subset=0, t_end=1.0e5, h=0.5, seed=5):
    import torch
    cells = W.qm_grid(n, seed=seed)
    if subset and subset < cells.shape[0]:
        cells = W.subset(cells, subset, seed=seed + 100)[0]
    m1 = cells[:, W.BETA] / (1 + cells[:, W.BETA])
    m2 = 1 / (1 + cells[:, W.BETA])
    spin_ref = np.stack([cells[:, W.CHI1] * m1 ** 2, cells[:, W.CHI2] * m2 ** 2], axis=1)
    cd = torch.as_tensor(np.ascontiguousarray(cells[:, :9]), device="cuda")
    report = {"grid": "%dx%d" % (n, n), "orbits": int(cells.shape[0]), "h": h, "t_end": t_end,
              "kappa": "U[1,10]", "use_qm": 1}
    for correct in (1, 0):
        with Scan(None, kappa1=cells[:, W.KAP1], kappa2=cells[:, W.KAP2], device=True, n=cells.shape[0],
                  use_qm=1, correct=correct) as s:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.setup(cd)
            s.run(t_end, h)
            out = s.read()
            summ = s.summary()
            dt = time.perf_counter() - t0
        r = drift_stats(out, spin_ref)
        r.update(seconds=dt, orbit_steps=summ["orbit_steps"], rate=summ["orbit_steps"] / dt,
                 n_chaotic=summ["n_chaotic"], n_final_fallback=summ["n_final_fallback"])
        report["corrected" if correct else "uncorrected"] = r
    return report


def paper_scans(t_end=1.0e5, h=1.0, thr=5.8, out_dir=None, n=314):
    """Fig. 6 (theta2 scans at theta1 = pi/2 and 0) and Fig. 7 (theta1-theta2
    plane) with RK5; no merger / escape cut-off (the paper integrates every
    orbit to t_end and discards unbound ones afterwards)."""
    import os
    import torch
    runs = {"fig6a_theta1_pi2": W.paper_theta2_scan(np.pi / 2, n), "fig6b_theta1_0": W.paper_theta2_scan(0.0, n),
            "fig7_theta1_theta2": W.paper_theta12_scan(n)}
    report = {"t_end": t_end, "h": h, "rk_order": 5, "fli_threshold": thr}
    for name, cells in runs.items():
        cd = torch.as_tensor(np.ascontiguousarray(cells[:, :9]), device="cuda")
        with Scan(None, device=True, n=cells.shape[0], rk_order=5, r_merge=0.0, r_escape=0.0) as s:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.setup(cd)
            s.run(t_end, h)
            out = s.read()
            dt = time.perf_counter() - t0
        fli = out["fli"].cpu().numpy()
        r = np.linalg.norm(out["states"].cpu().numpy()[:, :3], axis=1)
        bound = r < 100.0
        if out_dir:
            os.makedirs(out_dir, exist_ok=True)
            np.save(os.path.join(out_dir, name + "_fli.npy"), fli.reshape(-1, n) if fli.size > n else fli)
            np.save(os.path.join(out_dir, name + "_r_end.npy"), r)
        report[name] = {"orbits": int(fli.size), "seconds": dt, "bound_frac": float(bound.mean()),
                        "chaotic_frac_bound": float((fli[bound] > thr).mean()) if bound.any() else None,
                        "fli_median_bound": float(np.median(fli[bound])) if bound.any() else None}
    return report


def newton_tolerance_study(n=64, t_end=1.0e4, h=1.0, eps_list=(1e-6, 1e-8, 1e-10), seed=1, cond_switch=0.0):
    """Energy, |J| and spin-length drift at t_end on an n x n grid of the
    small-scan family (x0 in [15, 40], theta in [0, pi], m1 = m2, chi = 1)
    for each Newton tolerance and stopping rule.  Fig. 4 is about the
    paper's own correction, so by default the dual scaling is used at every
    step where it is not singular (cond_switch 0)."""
    import torch
    cells = W.grid_cells(n, n, 15.0, 40.0, seed)
    m1 = cells[:, W.BETA] / (1 + cells[:, W.BETA])
    m2 = 1 / (1 + cells[:, W.BETA])
    spin_ref = np.stack([cells[:, W.CHI1] * m1 ** 2, cells[:, W.CHI2] * m2 ** 2], axis=1)
    cd = torch.as_tensor(np.ascontiguousarray(cells[:, :9]), device="cuda")
    report = {"grid": "%dx%d" % (n, n), "orbits": int(cells.shape[0]), "h": h, "t_end": t_end, "rk_order": 5,
              "cond_switch": cond_switch}
    for apply_small in (1, 0):
        rule = "apply_then_test" if apply_small else "stop_before_applying"
        report[rule] = {}
        for eps in eps_list:
            with Scan(None, device=True, n=cells.shape[0], rk_order=5, newton_tol=eps,
                      newton_apply_small=apply_small, newton_cond_switch=cond_switch) as s:
                s.setup(cd)
                s.run(t_end, h)
                out = s.read()
            report[rule]["%g" % eps] = drift_stats(out, spin_ref)
    return report


def correction_ablation_study(n=64, t_end=1.0e4, h=1.0, rk_order=4, seed=1):
    """Drift at t_end for each correction mode (0 none, 1 dual scaling,
    2 spin lengths only, 3 spin lengths + velocity scaling) on an n x n grid
    of the small-scan family."""
    import torch
    cells = W.grid_cells(n, n, 15.0, 40.0, seed)
    m1 = cells[:, W.BETA] / (1 + cells[:, W.BETA])
    m2 = 1 / (1 + cells[:, W.BETA])
    spin_ref = np.stack([cells[:, W.CHI1] * m1 ** 2, cells[:, W.CHI2] * m2 ** 2], axis=1)
    cd = torch.as_tensor(np.ascontiguousarray(cells[:, :9]), device="cuda")
    names = {0: "none", 1: "dual_scaling", 2: "spin_lengths_only", 3: "velocity_scaling"}
    report = {"grid": "%dx%d" % (n, n), "orbits": int(cells.shape[0]), "h": h, "t_end": t_end,
              "rk_order": rk_order}
    for mode in (0, 1, 2, 3):
        with Scan(None, device=True, n=cells.shape[0], rk_order=rk_order, correct=mode) as s:
            s.setup(cd)
            s.run(t_end, h)
            out = s.read()
        report[names[mode]] = drift_stats(out, spin_ref)
    return report


def waveform_series(cells, t_end, every=10.0, h=1.0, R=1.0, P=(1.0, 0.0, 0.0), Q=(0.0, 1.0, 0.0),
                    until_stopped=False, **opts):
    """Sample (h_plus, h_cross) of the orbits of `cells` (n x >= 9) every
    `every` time units from t = 0 to t_end (or, with until_stopped, until
    every orbit has stopped): returns t (m), hp (m x n), hc (m x n)."""
    cells = np.ascontiguousarray(np.atleast_2d(cells), dtype=np.float64)
    kap = cells.shape[1] > W.KAP2
    ts, hps, hcs = [], [], []
    with Scan(cells[:, W.BETA], kappa1=cells[:, W.KAP1] if kap else None,
              kappa2=cells[:, W.KAP2] if kap else None, **opts) as s:
        s.setup(cells[:, :9])
        t = 0.0
        while True:
            hp, hc = s.waveform(R, P, Q)
            ts.append(t)
            hps.append(np.array(hp))
            hcs.append(np.array(hc))
            if t >= t_end - 1e-9 * every:
                break
            if until_stopped and t > 0.0 and np.all(s.read()["status"] != ORBIT_DONE):
                break
            t = min(t + every, t_end)
            s.run(t, h)
    return np.array(ts), np.array(hps), np.array(hcs)


def paper_waveforms(t_end=1.0e4, every=2.0, out_dir=None, dissipative=False):
    """Fig. 10: orbit 4 (regular) and case II orbit 2 (chaotic), corrected
    RK5, h = 1, P = x, Q = y, N = z, R = 1.  Conservative (upper panels), or
    with the 2.5PN radiation reaction until the merger cut r < 6 (lower
    panels, sampled at least every 1 M since they last about one orbit; the
    series written and summarised end where each orbit stopped)."""
    import os
    names, cells = W.paper_orbit_cells()
    names, cells = names[:2], cells[:2]
    if dissipative:
        opts = dict(rk_order=5, radiation_reaction=1, r_escape=0.0, until_stopped=True)
        every = min(every, 1.0)
    else:
        opts = dict(rk_order=5, r_merge=0.0, r_escape=0.0)
    t, hp, hc = waveform_series(cells, t_end, every, **opts)
    report = {"t_end": t_end, "every": every, "R": 1.0, "dissipative": bool(dissipative)}
    tag = "_dissipative" if dissipative else ""
    for j, k in enumerate(names):
        # the stretch before the orbit stopped (constant samples after it)
        moving = np.flatnonzero(np.diff(hp[:, j]) != 0.0)
        last = int(moving[-1]) + 2 if moving.size else 1
        report[k] = {"h_plus_rms": float(np.sqrt(np.mean(hp[:last, j] ** 2))),
                     "h_plus_max": float(np.abs(hp[:last, j]).max()),
                     "h_cross_rms": float(np.sqrt(np.mean(hc[:last, j] ** 2))),
                     "duration": float(t[last - 1])}
        if out_dir:
            os.makedirs(out_dir, exist_ok=True)
            np.save(os.path.join(out_dir, k + tag + "_waveform.npy"),
                    np.stack([t[:last], hp[:last, j], hc[:last, j]], axis=1))
    return report


def dissipative_series(cells, t_end, every=1000.0, h=1.0, **opts):
    """Orbits of `cells` with the 2.5PN radiation reaction (Eq. 6; Sec. 3B),
    sampled every `every` time units by runs to t1, t2, ... until t_end or
    until every orbit has stopped.  Returns a dict of arrays (m x n): t, r
    (|r| of the main trajectory), E, E_ref, J, J_ref (the integrals and their
    integral-invariant references), status."""
    cells = np.ascontiguousarray(np.atleast_2d(cells), dtype=np.float64)
    kap = cells.shape[1] > W.KAP2
    rec = {k: [] for k in ("t", "r", "E", "E_ref", "J", "J_ref", "status")}
    with Scan(cells[:, W.BETA], kappa1=cells[:, W.KAP1] if kap else None,
              kappa2=cells[:, W.KAP2] if kap else None, radiation_reaction=1, **opts) as s:
        s.setup(cells[:, :9])
        t = 0.0
        while t < t_end - 1e-9 * every:
            t = min(t + every, t_end)
            s.run(t, h)
            out = s.read()
            rec["t"].append(np.array(out["t_stop"]))
            rec["r"].append(np.linalg.norm(out["states"][:, 0:3], axis=1))
            rec["E_ref"].append(np.array(out["integrals"][:, 0]))
            rec["E"].append(np.array(out["integrals"][:, 1]))
            rec["J_ref"].append(np.array(out["integrals"][:, 2]))
            rec["J"].append(np.array(out["integrals"][:, 3]))
            rec["status"].append(np.array(out["status"]))
            if np.all(out["status"] != ORBIT_DONE):
                break
    return {k: np.array(v) for k, v in rec.items()}


def paper_orbit3(t_end=3.0e5, every=1000.0, h=1.0, out_dir=None):
    """Fig. 5: orbit 3 with radiation reaction, corrected and uncorrected
    RK5 (h = 1): the relative energy error against the integral-invariant
    reference (a), |r| decaying to the merger cut (b)."""
    import os
    names, cells = W.paper_orbit_cells()
    cell = cells[[names.index("orbit_3")]]
    report = {"t_end": t_end, "every": every, "h": h}
    for label, corr in (("corrected", 1), ("uncorrected", 0)):
        d = dissipative_series(cell, t_end, every, h, rk_order=5, correct=corr, r_escape=0.0)
        err = np.abs(d["E"][:, 0] - d["E_ref"][:, 0]) / np.abs(d["E_ref"][:, 0])
        report[label] = {"t_stop": float(d["t"][-1, 0]), "status": int(d["status"][-1, 0]),
                         "r_first": float(d["r"][0, 0]), "r_last": float(d["r"][-1, 0]),
                         "dE_rel_max": float(err.max()),
                         "dE_rel_at": {"%g" % d["t"][i, 0]: float(err[i])
                                       for i in sorted({len(err) // 10, len(err) // 2, len(err) - 1})}}
        if out_dir:
            os.makedirs(out_dir, exist_ok=True)
            np.save(os.path.join(out_dir, "orbit_3_%s.npy" % label),
                    np.stack([d["t"][:, 0], d["r"][:, 0], d["E"][:, 0], d["E_ref"][:, 0]], axis=1))
    return report


def fli_curves(cells, t_end, every=1000.0, h=1.0, **opts):
    """FLI(t) of the orbits of `cells` (n x >= 9), sampled every `every` time
    units by runs to t1, t2, ...: returns t (m) and fli (m x n)."""
    cells = np.ascontiguousarray(np.atleast_2d(cells), dtype=np.float64)
    kap = cells.shape[1] > W.KAP2
    ts, flis = [], []
    with Scan(cells[:, W.BETA], kappa1=cells[:, W.KAP1] if kap else None,
              kappa2=cells[:, W.KAP2] if kap else None, **opts) as s:
        s.setup(cells[:, :9])
        t = 0.0
        while t < t_end - 1e-9 * every:
            t = min(t + every, t_end)
            s.run(t, h)
            ts.append(t)
            flis.append(np.array(s.read()["fli"]))
    return np.array(ts), np.array(flis)


def paper_fli_curves(t_end=8.0e5, every=2000.0, out_dir=None, thr=5.8):
    """Fig. 3: FLI(t) of case II orbits 1 and 2, corrected RK5, h = 1.
    Orbit 2's exponential growth sets in near t = 8e5 (an uncorrected RK5 run
    at h = 0.25 agrees), so that is the default length."""
    import os
    names, cells = W.paper_orbit_cells()
    pick = [names.index("case_II_orbit_1"), names.index("case_II_orbit_2")]
    t, fli = fli_curves(cells[pick], t_end, every, rk_order=5, r_merge=0.0, r_escape=0.0)
    report = {"t_end": t_end, "every": every, "threshold": thr}
    for j, k in enumerate(("case_II_orbit_1", "case_II_orbit_2")):
        report[k] = {"fli_end": float(fli[-1, j]), "chaotic": bool(fli[-1, j] > thr),
                     "fli_at": {"%g" % t[i]: float(fli[i, j]) for i in (len(t) // 10 - 1, len(t) // 2 - 1, len(t) - 1)}}
        if out_dir:
            os.makedirs(out_dir, exist_ok=True)
            np.save(os.path.join(out_dir, k + "_fli.npy"), np.stack([t, fli[:, j]], axis=1))
    return report


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["qm", "paper", "newton", "ablation", "waveform", "fli", "orbit3"])
    ap.add_argument("--dissipative", action="store_true")
    ap.add_argument("--out", default=None)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--subset", type=int, default=0)
    ap.add_argument("--t-end", type=float, default=1.0e5)
    ap.add_argument("--h", type=float, default=0.5)
    a = ap.parse_args()
    if a.study == "qm":
        print(json.dumps(qm_drift_study(a.n, a.subset, a.t_end, a.h)), flush=True)
    elif a.study == "newton":
        print(json.dumps(newton_tolerance_study(a.n, a.t_end)), flush=True)
    elif a.study == "ablation":
        print(json.dumps(correction_ablation_study(a.n, a.t_end)), flush=True)
    elif a.study == "waveform":
        print(json.dumps(paper_waveforms(a.t_end, out_dir=a.out, dissipative=a.dissipative)), flush=True)
    elif a.study == "orbit3":
        print(json.dumps(paper_orbit3(a.t_end, out_dir=a.out)), flush=True)
    elif a.study == "fli":
        print(json.dumps(paper_fli_curves(a.t_end, out_dir=a.out)), flush=True)
    else:
        print(json.dumps(paper_scans(a.t_end, 1.0, out_dir=a.out)), flush=True)


if __name__ == "__main__":
    main()
