"""Surrogate-adaptive phase-space scan: a driver over the library's C ABI.

The map of a scan grid (chaotic or not, FLI > thr) is produced in five steps,
each a call into libpnscan:

1. ``adaptive_features``: the surrogate's inputs (x0, theta1, beta, chi1).
2. ``Surrogate.predict``: ensemble mean and spread of the FLI.
3. ``adaptive_select``: cells with |mean - thr| <= band or spread > spread_max
   (ordered compaction, their scan parameters gathered).
4. ``Scan``: the full FP64 integrator on the selected cells only.
5. ``adaptive_merge``: integrator result on the selected cells, surrogate
   class elsewhere.

The surrogate is trained (``Surrogate.train``) on FLI values the integrator
itself produced for other scans.  Keyword options of ``training_set``,
``adaptive_map`` and ``full_map`` are ``Scan`` options (``rk_order``,
``use_qm``, ``radiation_reaction``, ...), passed to every integration.
PyTorch provides device memory and the stream only.
"""
import time

import numpy as np

from . import Scan, Surrogate, adaptive_features, adaptive_features_fields, adaptive_interp_grid, \
    adaptive_merge, adaptive_select, ORBIT_DONE, ORBIT_FLI_SATURATED, ORBIT_NONFINITE


def _torch():
    import torch
    return torch


def integrate_cells(cells_d, t_end, h=1.0, **opts):
    """Integrate every cell of cells_d (n x >= 9 float64, CUDA) to t_end with the
    scan integrator; returns the device outputs of scan_read."""
    torch = _torch()
    cells9 = cells_d[:, :9].contiguous()
    n = int(cells9.shape[0])
    if n == 0:
        e = torch.empty(0, device="cuda")
        return dict(fli=e.double(), status=e.int(), states=torch.empty((0, 12), device="cuda").double())
    with Scan(None, device=True, n=n, **opts) as s:
        s.setup(cells9)
        s.run(t_end, h)
        return s.read()


def classes(fli, status, thr):
    """1 where the orbit reached t_end (or saturated) with FLI > thr."""
    torch = _torch()
    ok = (status == ORBIT_DONE) | (status == ORBIT_FLI_SATURATED)
    return (ok & (fli > thr)).to(torch.int8)


def features(cells_d, fields=None):
    """Surrogate inputs of cells_d: (x0, theta1, beta, chi1) by default, else
    the four cell fields named by index."""
    return adaptive_features(cells_d) if fields is None else adaptive_features_fields(cells_d, fields)


def training_set(cell_sets, t_ends, h=1.0, fields=None, **opts):
    """Surrogate training data from integrator runs: X (m x 4 float32) and the
    FLI (m float32) of every cell that did not become non-finite."""
    torch = _torch()
    Xs, ys = [], []
    for cells, t_end in zip(cell_sets, t_ends):
        cd = torch.as_tensor(np.ascontiguousarray(cells[:, :9]), device="cuda")
        out = integrate_cells(cd, t_end, h, **opts)
        keep = out["status"] != ORBIT_NONFINITE
        Xs.append(features(cd, fields)[keep])
        ys.append(out["fli"][keep].float())
    return torch.cat(Xs), torch.cat(ys)


def train_surrogate(X, y, members=5, steps=4000, lr=3e-3, seed=1, center=None, scale=None):
    kw = {} if center is None else dict(center=tuple(center), scale=tuple(scale))
    sur = Surrogate(members=members, seed=seed, **kw)
    hist = sur.train(X, y, steps=steps, lr=lr, seed=seed + 100)
    return sur, hist


def adaptive_map(sur, cells_d, t_end, h=1.0, thr=6.0, band=1.0, spread_max=0.5, fields=None, **opts):
    """Class map of the grid cells_d (n x 9 float64, CUDA) and its cost."""
    torch = _torch()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X = features(cells_d, fields)
    mean, spread = sur.predict(X)
    idx, sel = adaptive_select(mean, spread, thr, band, spread_max, cells=cells_d)
    t1 = time.perf_counter()
    out = integrate_cells(sel, t_end, h, **opts)
    cls = adaptive_merge(mean, thr, idx, out["fli"], out["status"])
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return dict(cls=cls, mean=mean, spread=spread, idx=idx, fli_sel=out["fli"], status_sel=out["status"],
                n_marked=int(idx.shape[0]), seconds=t2 - t0, seconds_surrogate=t1 - t0)


def full_map(cells_d, t_end, h=1.0, thr=6.0, **opts):
    """Class map from integrating every cell, and its cost."""
    torch = _torch()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = integrate_cells(cells_d, t_end, h, **opts)
    cls = classes(out["fli"], out["status"], thr)
    torch.cuda.synchronize()
    return dict(cls=cls, fli=out["fli"], status=out["status"], seconds=time.perf_counter() - t0)


def coarse_nodes(cells_d, n1, n2, stride):
    """The cells of every stride-th row and column of a row-major n1 x n2 grid."""
    return cells_d[:, :9].reshape(n1, n2, 9)[::stride, ::stride].reshape(-1, 9).contiguous()


def baseline_map(cells_d, n1, n2, stride, t_end, h=1.0, thr=6.0, band=1.0, spread_max=0.5, **opts):
    """The no-learning adaptive map of a row-major n1 x n2 grid: integrate the
    coarse grid of every stride-th cell, interpolate its FLI bilinearly (the
    spread of the four surrounding nodes as uncertainty), integrate the cells
    the same selection rule marks, merge.  The coarse integration is part of
    the cost."""
    torch = _torch()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nodes = coarse_nodes(cells_d, n1, n2, stride)
    out_c = integrate_cells(nodes, t_end, h, **opts)
    mean, spread = adaptive_interp_grid(out_c["fli"], out_c["status"], n1, n2, stride)
    idx, sel = adaptive_select(mean, spread, thr, band, spread_max, cells=cells_d)
    out = integrate_cells(sel, t_end, h, **opts)
    cls = adaptive_merge(mean, thr, idx, out["fli"], out["status"])
    torch.cuda.synchronize()
    return dict(cls=cls, mean=mean, spread=spread, idx=idx, n_nodes=int(nodes.shape[0]),
                n_marked=int(idx.shape[0]), seconds=time.perf_counter() - t0)


def operating_points(mean, spread, truth, thr, bands, spread_maxes):
    """For each (band, spread_max): the fraction of cells the selection marks
    and the misclassification of the merged map.  Integrated cells take the
    integrator's class, which is the full map's own on those cells, so the
    truth map stands in for integrating them."""
    torch = _torch()
    pred = (mean > thr).to(torch.int8)
    wrong = pred != truth
    nan = torch.isnan(mean)
    pts = []
    for band in bands:
        for sm in spread_maxes:
            marked = ((mean - thr).abs() <= band) | (spread > sm) | nan
            pts.append({"band": float(band), "spread_max": float(sm),
                        "marked_frac": float(marked.float().mean().item()),
                        "misclassification": float((wrong & ~marked).float().mean().item())})
    return pts


def cheapest(points, mis_max):
    """The operating point with the fewest marked cells whose
    misclassification is at most mis_max (None if there is none)."""
    ok = [p for p in points if p["misclassification"] <= mis_max]
    return min(ok, key=lambda p: p["marked_frac"]) if ok else None


def boundary_study(n=512, t_end=1.0e4, thr=5.8, stride=8, train_m=None, members=5, train_steps=20000,
                   bands=(0.125, 0.25, 0.375, 0.5, 0.625, 0.75, 0.875, 1.0, 1.5, 2.0, 3.0),
                   spread_maxes=(0.125, 0.25, 0.375, 0.5, 0.75, 1.0, 2.0, float("inf")),
                   mis_max=0.005, seed=11, target_clip=1.0, train_x0=None, **opts):
    """Surrogate-adaptive map against the no-learning coarse-grid map on the
    (theta1, theta2) plane of Sec. 3C, Fig. 7 (workloads.theta12_plane),
    which has an order/chaos boundary.

    Both methods get the same integration budget for what they learn from:
    the surrogate is trained on train_m random cells of the plane (default
    (n/stride)^2), the baseline interpolates the (n/stride)^2 nodes of every
    stride-th row and column.  Each is swept over the selection thresholds
    (band, spread_max) against the full map; the cheapest point with
    misclassification <= mis_max is then run end to end and timed.  Returns
    the report (times in seconds; cells_integrated and seconds_total count
    each method's training data or coarse nodes too).

    The surrogate's training targets are clipped to thr +- target_clip: the
    class depends only on the side of thr, and the FLIs of chaotic cells
    scatter widely (6-15 at t = 1e4), so an unclipped fit spends its
    capacity there.  Measured on the 512^2 plane at t = 1e4 (15.6 %
    chaotic) over the coarser sweep band in (0.25, 0.5, 1, 1.5, 2, 3),
    spread_max in (0.25, 0.5, 1, 2, inf): unclipped, the cheapest point at
    <= 0.5 % marks 48.7 % of the cells; clipped to +-2, 27.3 %; to +-1 with
    30,000 steps, 23.7 %; the coarse grid of stride 8, 22.7 %.  Over the
    default sweep: the coarse grid 22.5 %; the surrogate after 8,000,
    12,000, 20,000 and 30,000 Adam steps 23.6, 23.2, 20.1 and 19.7 %, i.e.
    2.69, 2.68, 2.45 and 2.50 s to map with its training and training data
    against the coarse grid's 2.49 s (the default: 20,000)."""
    from . import workloads as W
    torch = _torch()
    fields = (W.TH1, W.TH2, W.X0, W.BETA)
    center, scale = (np.pi / 2, np.pi / 2, 10.14, 1.0), (np.pi / 2, np.pi / 2, 1.0, 1.0)
    grid = W.theta12_plane(n)
    grid_d = torch.as_tensor(np.ascontiguousarray(grid[:, :9]), device="cuda")
    m = train_m or ((n - 1) // stride + 1) ** 2
    if train_x0:
        # transfer: training cells from the neighbouring planes only, none of the target plane
        train = np.concatenate([W.theta12_random(m, seed + k, x0=x) for k, x in enumerate(train_x0)])
    else:
        train = W.theta12_random(m, seed)
    # warm-up of every path on tiny inputs (first use of a PyTorch comparison
    # or masked index loads its kernels)
    training_set([train[:32]], [10.0], fields=fields, **opts)
    _, y_w = training_set([train], [10.0], fields=fields, **opts)   # the training set's own batch size
    if target_clip is not None:
        y_w.clamp(thr - target_clip, thr + target_clip)             # (its first use loads the kernel: ~1.3 s)
    full_map(grid_d[:64], 10.0, thr=thr, **opts)
    baseline_map(grid_d[:64 * 64], 64, 64, 8, 10.0, thr=thr, **opts)

    full = full_map(grid_d, t_end, thr=thr, **opts)
    truth = full["cls"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, y = training_set([train], [t_end], fields=fields, **opts)
    if target_clip is not None:
        # the class depends only on the side of thr: FLIs far beyond it
        # (chaotic FLIs scatter widely) are clipped so that the fit spends
        # its capacity near the boundary
        y = y.clamp(thr - target_clip, thr + target_clip)
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    sur, hist = train_surrogate(X, y, members=members, steps=train_steps, lr=3e-3, seed=seed,
                                center=center, scale=scale)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    mean_s, spread_s = sur.predict(features(grid_d, fields))
    nodes = coarse_nodes(grid_d, n, n, stride)
    out_c = integrate_cells(nodes, t_end, **opts)
    mean_b, spread_b = adaptive_interp_grid(out_c["fli"], out_c["status"], n, n, stride)
    pts_s = operating_points(mean_s, spread_s, truth, thr, bands, spread_maxes)
    pts_b = operating_points(mean_b, spread_b, truth, thr, bands, spread_maxes)
    best_s, best_b = cheapest(pts_s, mis_max), cheapest(pts_b, mis_max)
    sub_idx = torch.as_tensor(W.subset(grid, 4096, seed=6)[1], device="cuda")
    report = {"grid": "%dx%d" % (n, n), "plane": "theta1 x theta2 in [0, pi]^2, (beta, r, p_y) = (1, 10.14, 0.365), "
                                              "chi = 1 (Sec. 3C, Fig. 7)",
              "t_end": t_end, "thr": thr, "chaotic_frac": float(truth.float().mean().item()),
              "plain_s": full["seconds"], "mis_max": mis_max, "budget_cells": m,
              "surrogate": {"train_cells": int(train.shape[0]), "train_x0": list(train_x0) if train_x0 else None,
                            "members": members, "train_steps": train_steps, "target_clip": target_clip,
                            "training_data_s": data_s, "train_s": train_s, "points": pts_s, "chosen": best_s},
              "baseline": {"stride": stride, "nodes": int(nodes.shape[0]), "points": pts_b, "chosen": best_b}}
    if best_s is not None:
        res = adaptive_map(sur, grid_d, t_end, thr=thr, band=best_s["band"], spread_max=best_s["spread_max"],
                           fields=fields, **opts)
        wrong = res["cls"] != truth
        report["surrogate"].update(
            adaptive_s=res["seconds"], marked=res["n_marked"], marked_frac=res["n_marked"] / grid.shape[0],
            misclassification_all=float(wrong.float().mean().item()),
            misclassification_subset4096=float(wrong[sub_idx].float().mean().item()),
            speedup=full["seconds"] / res["seconds"],
            cells_integrated=res["n_marked"] + (0 if train_x0 else m),
            training_cells_other_planes=int(train.shape[0]) if train_x0 else 0,
            seconds_total=res["seconds"] + train_s + data_s,
            speedup_incl_training_and_data=full["seconds"] / (res["seconds"] + train_s + data_s))
    if best_b is not None:
        res = baseline_map(grid_d, n, n, stride, t_end, thr=thr, band=best_b["band"],
                           spread_max=best_b["spread_max"], **opts)
        wrong = res["cls"] != truth
        report["baseline"].update(
            seconds=res["seconds"], marked=res["n_marked"], marked_frac=res["n_marked"] / grid.shape[0],
            misclassification_all=float(wrong.float().mean().item()),
            misclassification_subset4096=float(wrong[sub_idx].float().mean().item()),
            cells_integrated=res["n_marked"] + res["n_nodes"], seconds_total=res["seconds"],
            speedup=full["seconds"] / res["seconds"])
    sur.close()
    return report
