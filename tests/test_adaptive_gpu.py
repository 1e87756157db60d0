"""End-to-end surrogate-adaptive scan on the GPU.

The surrogate is trained on FLI values the integrator produced for the small
scan and a sample of the full scan; the adaptive map of a 96 x 96 grid of
the small-scan parameters is then compared with integrating every cell:
  * cells the adaptive scan integrates carry exactly the full scan's values
    (the integrator's result for an orbit does not depend on its batch);
  * the class map disagrees on at most 0.5 % of the cells.
The FLI threshold here is the median FLI of the grid (so that both classes
occur and the selection is exercised); band and spread limits as in the
adaptive-scan configuration scaled to that FLI range."""
import numpy as np
import pytest

from paper_1802_00147_gb300 import workloads as W

pytestmark = pytest.mark.gpu

T_END = 2000.0


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00147_gb300 import build
    build.build()
    from paper_1802_00147_gb300 import adaptive as A
    train_cells = np.concatenate([W.small_scan(seed=1), W.subset(W.full_scan(seed=2), 8000, seed=3)[0]])
    X, y = A.training_set([train_cells], [T_END])
    sur, hist = A.train_surrogate(X, y, members=5, steps=3000, lr=3e-3, seed=4)
    grid = W.grid_cells(96, 96, 15.0, 40.0, seed=9)
    cells_d = torch.as_tensor(np.ascontiguousarray(grid[:, :9]), device="cuda")
    return A, sur, hist.cpu().numpy(), cells_d


def test_surrogate_learns_the_integrator_fli(env):
    A, sur, hist, cells_d = env
    assert np.all(hist[:, -200:].mean(1) < 0.25 * hist[:, :20].mean(1))


def test_adaptive_map_matches_full_integration(env):
    import torch
    A, sur, hist, cells_d = env
    full = A.full_map(cells_d, T_END, thr=0.0)
    done = full["status"] == 1
    thr = float(torch.median(full["fli"][done]).item())
    full_cls = A.classes(full["fli"], full["status"], thr)
    res = A.adaptive_map(sur, cells_d, T_END, thr=thr, band=0.25, spread_max=0.25)
    n = cells_d.shape[0]
    assert 0 < res["n_marked"] < n
    idx = res["idx"].long()
    # integrated cells: bit-identical to the full scan
    assert torch.equal(res["fli_sel"], full["fli"][idx])
    assert torch.equal(res["status_sel"], full["status"][idx])
    mis = (res["cls"] != full_cls).float().mean().item()
    assert mis <= 0.005, (mis, res["n_marked"])


def test_training_is_what_saves_the_work(env):
    """What the trained network gains over the method without it, under the
    adaptive scan's own criteria (threshold 6, band 1, spread 0.5): an
    untrained ensemble (random members disagree everywhere) marks nearly
    every cell, so the adaptive map integrates almost the whole grid; the
    trained ensemble marks less than half as many, with the same agreement
    with the full integration."""
    import torch
    import paper_1802_00147_gb300 as pn
    A, sur, hist, cells_d = env
    full = A.full_map(cells_d, T_END, thr=6.0)
    untrained = pn.Surrogate(members=5, seed=77)
    try:
        raw = A.adaptive_map(untrained, cells_d, T_END, thr=6.0, band=1.0, spread_max=0.5)
    finally:
        untrained.close()
    trained = A.adaptive_map(sur, cells_d, T_END, thr=6.0, band=1.0, spread_max=0.5)
    n = cells_d.shape[0]
    assert raw["n_marked"] >= 0.8 * n, raw["n_marked"]
    assert trained["n_marked"] < 0.5 * raw["n_marked"], (trained["n_marked"], raw["n_marked"])
    for res in (raw, trained):
        assert (res["cls"] != full["cls"]).float().mean().item() <= 0.005


def test_scan_options_reach_every_integration(env):
    """With radiation reaction and RK5 passed through, the cells the adaptive
    scan integrates carry exactly the values of integrating the whole grid
    with the same options, and of a direct Scan of those cells."""
    import torch
    import paper_1802_00147_gb300 as pn
    A, sur, hist, cells_d = env
    opts = dict(radiation_reaction=1, rk_order=5)
    t_end = 500.0
    full = A.full_map(cells_d, t_end, thr=2.0, **opts)
    plain = A.full_map(cells_d, t_end, thr=2.0)
    assert not torch.equal(full["fli"], plain["fli"])          # the options changed the run
    res = A.adaptive_map(sur, cells_d, t_end, thr=2.0, band=0.5, spread_max=0.25, **opts)
    idx = res["idx"].long()
    assert res["n_marked"] > 0
    assert torch.equal(res["fli_sel"], full["fli"][idx])
    assert torch.equal(res["status_sel"], full["status"][idx])
    sel = cells_d[idx].cpu().numpy()
    with pn.Scan(sel[:, 6], **opts) as s:
        s.setup(sel)
        s.run(t_end, 1.0)
        direct = s.read()
    np.testing.assert_array_equal(direct["fli"], res["fli_sel"].cpu().numpy())


# ----------------------------------------- boundary-rich plane and baseline
def test_features_from_chosen_fields_are_exact():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1802_00147_gb300 as pn
    cells = W.theta12_random(1000, seed=3)[:, :9]
    X = pn.adaptive_features_fields(torch.as_tensor(np.ascontiguousarray(cells), device="cuda"),
                                    (W.TH1, W.TH2, W.X0, W.BETA)).cpu().numpy()
    np.testing.assert_array_equal(X, cells[:, [W.TH1, W.TH2, W.X0, W.BETA]].astype(np.float32))
    with pytest.raises(pn.ScanError):
        pn.adaptive_features_fields(torch.zeros((4, 9), dtype=torch.float64, device="cuda"), (0, 1, 2, 9))


def interp_reference(fli, status, n1, n2, stride):
    """Bilinear interpolation of the node values (0 where a node did not
    finish or saturate) and the max - min of the four surrounding nodes."""
    nc1, nc2 = (n1 - 1) // stride + 1, (n2 - 1) // stride + 1
    v = np.where((status == 1) | (status == 4), fli, 0.0).reshape(nc1, nc2)
    mean = np.zeros((n1, n2))
    spread = np.zeros((n1, n2))
    for i in range(n1):
        for j in range(n2):
            a0, b0 = i // stride, j // stride
            a1, b1 = min(a0 + 1, nc1 - 1), min(b0 + 1, nc2 - 1)
            wa = (i - a0 * stride) / stride if a1 > a0 else 0.0
            wb = (j - b0 * stride) / stride if b1 > b0 else 0.0
            q = [v[a0, b0], v[a0, b1], v[a1, b0], v[a1, b1]]
            top = q[0] + wb * (q[1] - q[0])
            bot = q[2] + wb * (q[3] - q[2])
            node = i % stride == 0 and j % stride == 0
            mean[i, j] = q[0] if node else top + wa * (bot - top)
            spread[i, j] = 0.0 if node else max(q) - min(q)
    return mean.ravel(), spread.ravel()


@pytest.mark.parametrize("n1, n2, stride", [(37, 29, 4), (64, 64, 8), (9, 1, 3)])
def test_interpolation_baseline_matches_reference(n1, n2, stride):
    """Ragged grids (the last node row short of the edge), a one-column
    grid, nodes that did not finish (counted as FLI 0)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1802_00147_gb300 as pn
    rng = np.random.default_rng(n1 * 100 + n2)
    nc = ((n1 - 1) // stride + 1) * ((n2 - 1) // stride + 1)
    fli = rng.uniform(0, 12, nc)
    status = rng.choice([1, 1, 1, 2, 4], nc).astype(np.int32)
    mean, spread = pn.adaptive_interp_grid(torch.as_tensor(fli, device="cuda"), torch.as_tensor(status, device="cuda"),
                                           n1, n2, stride)
    m_ref, s_ref = interp_reference(fli, status, n1, n2, stride)
    np.testing.assert_allclose(mean.cpu().numpy(), m_ref, rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(spread.cpu().numpy(), s_ref, rtol=2e-6, atol=2e-6)


def test_boundary_plane_study_is_consistent():
    """The surrogate and the coarse-grid baseline on a small (theta1, theta2)
    plane of Fig. 7: the end-to-end maps at each method's chosen operating
    point have exactly the misclassification the sweep predicted (integrated
    cells carry the full map's own classes), within the 0.5 % bound."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00147_gb300 import adaptive as A
    rep = A.boundary_study(n=96, t_end=5000.0, thr=5.8, stride=8, train_steps=4000, r_merge=0.0, r_escape=0.0)
    assert 0.02 < rep["chaotic_frac"] < 0.5, rep["chaotic_frac"]
    for k in ("surrogate", "baseline"):
        r = rep[k]
        assert r["chosen"] is not None, k
        assert r["misclassification_all"] == pytest.approx(r["chosen"]["misclassification"], abs=1e-12), k
        assert r["misclassification_all"] <= 0.005 and r["marked_frac"] == pytest.approx(r["chosen"]["marked_frac"])
    assert rep["baseline"]["cells_integrated"] == rep["baseline"]["marked"] + 144
