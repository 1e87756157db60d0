"""The seeded input generators: the paper's single orbits come out as the
initial states the golden fixture cites, and the scan grids have the
stated ranges, distributions and seeded reproducibility."""
import json
import os

import numpy as np

import oracle
from paper_1802_00147_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_orbits.json")


def golden_state(name):
    with open(GOLDEN) as f:
        g = json.load(f)[name]
    beta = g["beta"]
    m1, m2 = beta / (1 + beta), 1 / (1 + beta)
    y = np.r_[g["r"], g["p"], g["chi1"] * m1 * m1 * np.array(g["S1_hat"]),
              g["chi2"] * m2 * m2 * np.array(g["S2_hat"])].astype(float)
    return beta, y


def test_paper_orbit_cells_reproduce_the_cited_initial_states():
    names, cells = W.paper_orbit_cells()
    y = oracle.setup_cells(cells[:, :9])
    for j, name in enumerate(names):
        beta, yg = golden_state(name)
        assert cells[j, W.BETA] == beta
        # printed unit vectors carry 6 digits: normalised here, so 1e-6
        np.testing.assert_allclose(y[j], yg, rtol=0, atol=1e-6 * np.abs(yg).max(), err_msg=name)


def test_grids_have_their_stated_ranges_and_are_seeded():
    s = W.small_scan(seed=1)
    assert s.shape == (256, W.NFIELDS)
    assert s[:, W.X0].min() == 15.0 and s[:, W.X0].max() == 40.0
    assert s[:, W.TH1].min() == 0.0 and np.isclose(s[:, W.TH1].max(), np.pi)
    assert np.all(s[:, W.TH1] == s[:, W.TH2]) and np.all(s[:, W.BETA] == 1.0)
    assert np.all(s[:, W.PFAC] == 0.9) and np.all(s[:, W.CHI1] == 1.0)
    f = W.full_scan(seed=2)
    assert f.shape == (98596, W.NFIELDS)
    assert f[:, W.X0].min() == 10.0 and f[:, W.X0].max() == 50.0
    assert 0.5 <= f[:, W.BETA].min() and f[:, W.BETA].max() <= 1.0
    assert 0.5 <= f[:, W.CHI1].min() and f[:, W.CHI2].max() <= 1.0
    assert np.array_equal(f, W.full_scan(seed=2))
    assert not np.array_equal(f, W.full_scan(seed=3))
    u = W.uneven_batch(n=20000, seed=3)
    assert 0.1 <= u[:, W.BETA].min() and 0.5 <= u[:, W.PFAC].min() and u[:, W.PFAC].max() <= 1.0
    # isotropic spin directions: cos(theta) uniform on [-1, 1]
    c = np.cos(u[:, W.TH1])
    assert abs(c.mean()) < 0.03 and abs(np.mean(c * c) - 1.0 / 3.0) < 0.01
    q = W.qm_grid(64, seed=5)
    assert 1.0 <= q[:, W.KAP1].min() and q[:, W.KAP2].max() <= 10.0


def test_random_states_are_what_they_say():
    y, beta, k1, k2 = W.random_states(4000, seed=31)
    r = np.linalg.norm(y[:, 0:3], axis=1)
    assert 12.0 <= r.min() and r.max() <= 40.0
    m1, m2 = beta / (1 + beta), 1 / (1 + beta)
    assert np.all(np.linalg.norm(y[:, 6:9], axis=1) <= m1 * m1 + 1e-15)
    assert np.all(np.linalg.norm(y[:, 9:12], axis=1) <= m2 * m2 + 1e-15)
    # |p| between 60 % and 100 % of circular, plus a radial part of at most 10 %
    pt = np.linalg.norm(np.cross(y[:, 0:3] / r[:, None], y[:, 3:6]), axis=1) * np.sqrt(r)
    assert 0.6 - 1e-12 <= pt.min() and pt.max() <= 1.0 + 1e-12
    assert 0.2 <= beta.min() and beta.max() <= 1.0 and 1.0 <= k1.min() and k2.max() <= 10.0


def test_paper_scans_match_sec_3c():
    t2 = W.paper_theta2_scan(np.pi / 2)
    assert t2.shape[0] == 314 and np.allclose(np.diff(t2[:, W.TH2]), 0.01)
    assert np.all(t2[:, W.BETA] == 1.0 / 3.0) and np.all(t2[:, W.X0] == 5.65)
    g = W.paper_theta12_scan()
    assert g.shape[0] == 314 * 314 and np.all(g[:, W.X0] == 10.14)
    assert np.allclose(g[:, W.PFAC] / np.sqrt(10.14), 0.365)
