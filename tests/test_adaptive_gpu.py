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
