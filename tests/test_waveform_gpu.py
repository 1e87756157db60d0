"""Gravitational-wave polarisations (Eq. 14, Sec. 4) through the C ABI
against the oracle along the paper's orbits, and the closed form of a
Newtonian circular orbit.  Tolerances: over the first 500 M the states
agree to ~1e-12 relative (one ulp per step, not yet amplified), so
h_plus / h_cross agree to <= 1e-9 of the waveform amplitude."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def studies():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00147_gb300 import build
    build.build()
    from paper_1802_00147_gb300 import studies as st
    return st


def test_waveform_matches_oracle_along_paper_orbits(studies):
    from paper_1802_00147_gb300 import workloads as W
    names, cells = W.paper_orbit_cells()
    every, nsteps = 10, 500
    t, hp, hc = studies.waveform_series(cells, float(nsteps), every=float(every), r_merge=0.0, r_escape=0.0)
    assert t.shape == (nsteps // every + 1,) and hp.shape == (t.size, len(names))
    y0 = oracle.setup_cells(cells[:, :9])
    cfg = oracle.config(r_merge=0, r_escape=0)
    for j in range(len(names)):
        s = oracle.system(cells[j, W.BETA], pn_order=2, use_so=1, use_ss=1)
        states = np.vstack([y0[j], oracle.trace(y0[j], cells[j, W.BETA], 1.0, nsteps, every, cfg)])
        want = np.array([oracle.waveform(s, y) for y in states])
        amp = np.abs(want).max()
        assert np.abs(hp[:, j] - want[:, 0]).max() <= 1e-9 * amp, names[j]
        assert np.abs(hc[:, j] - want[:, 1]).max() <= 1e-9 * amp, names[j]


def test_waveform_of_a_circular_newtonian_orbit(studies):
    """pn_order 0, no spins, p_y = 1/sqrt(a): h_plus = -(4 eta / (R a)) cos 2wt,
    h_cross = -(4 eta / (R a)) sin 2wt, w = a^-3/2 (RK4 phase error over one
    orbit at h = 1 is ~1e-8)."""
    from paper_1802_00147_gb300 import workloads as W
    a, R, beta = 20.0, 50.0, 0.5
    c = np.zeros((1, W.NFIELDS))
    c[0, W.X0], c[0, W.PFAC], c[0, W.BETA] = a, 1.0, beta
    c[0, W.KAP1] = c[0, W.KAP2] = 1.0
    w = a ** -1.5
    T = 2 * np.pi / w
    t, hp, hc = studies.waveform_series(c, float(np.floor(T)), every=16.0, R=R, pn_order=0, use_so=0, use_ss=0)
    eta = beta / (1 + beta) ** 2
    amp = 4 * eta / (R * a)
    np.testing.assert_allclose(hp[:, 0], -amp * np.cos(2 * w * t), rtol=0, atol=1e-6 * amp)
    np.testing.assert_allclose(hc[:, 0], -amp * np.sin(2 * w * t), rtol=0, atol=1e-6 * amp)


def test_waveform_frame_rotation_and_distance(studies):
    """Rotating (P, Q) by psi about N turns (h_plus, h_cross) by 2 psi; the
    amplitude falls as 1/R."""
    from paper_1802_00147_gb300 import workloads as W
    names, cells = W.paper_orbit_cells()
    _, hp0, hc0 = studies.waveform_series(cells, 50.0, every=50.0, r_merge=0.0)
    psi = 0.7
    P = (np.cos(psi), np.sin(psi), 0.0)
    Q = (-np.sin(psi), np.cos(psi), 0.0)
    _, hp1, hc1 = studies.waveform_series(cells, 50.0, every=50.0, R=4.0, P=P, Q=Q, r_merge=0.0)
    c2, s2 = np.cos(2 * psi), np.sin(2 * psi)
    scale = np.abs(hp0).max()
    np.testing.assert_allclose(4.0 * hp1, c2 * hp0 + s2 * hc0, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(4.0 * hc1, -s2 * hp0 + c2 * hc0, rtol=0, atol=1e-13 * scale)
