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
