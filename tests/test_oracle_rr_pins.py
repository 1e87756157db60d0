"""Pins of the oracle's 2.5PN radiation reaction (Eq. 6's a_2.5PN; Sec. 3B,
orbit 3, Fig. 5) against results that do not come from the oracle itself.

The paper takes a_2.5PN from Levin et al. (2011) without printing it.  The
oracle uses the leading-order two-parameter gauge family of Iyer & Will
(1993), harmonic gauge by default.  The pins:
- every gauge gives the quadrupole-formula losses (Peters & Mathews 1963)
  averaged over a Kepler orbit, for energy and angular momentum, at any
  eccentricity; on a circular orbit they hold instant by instant;
- the force is odd under time reversal and rotation covariant;
- a quasi-circular Newtonian inspiral follows r^4 = r0^4 - (256/5) eta t and
  merges when that reaches the cut;
- the integral-invariant relations (dE/dt = (dH/dp).a, d|J|/dt = J.(r x a)/|J|)
  track H and |J| of the full spinning Hamiltonian along an uncorrected run;
- the extended RK4 and fifth-order steps converge at orders 4 and 5;
- with the correction, H and |J| equal the evolving reference values.
"""
import json
import os

import numpy as np
import pytest

import oracle as orc

GAUGES = ((4.0, 5.0), (0.0, 0.0), (5.0 / 3.0, 3.0), (-1.0, 2.5))


def newtonian(beta=1.0):
    return orc.system(beta, pn_order=0, use_so=0, use_ss=0)


def kepler_state(a, e, E):
    """Relative Newtonian orbit (M = 1) at eccentric anomaly E: state with
    p = v, and dt/dE."""
    b = a * np.sqrt(1.0 - e * e)
    nmean = a ** -1.5
    Edot = nmean / (1.0 - e * np.cos(E))
    y = np.zeros(12)
    y[0:3] = (a * (np.cos(E) - e), b * np.sin(E), 0.0)
    y[3:6] = (-a * np.sin(E) * Edot, b * np.cos(E) * Edot, 0.0)
    return y


def peters(a, e, eta):
    """Orbit-averaged losses per unit reduced mass, M = 1 (Peters & Mathews
    1963; Peters 1964): <dE/dt>, <dL/dt>."""
    dE = -(32.0 / 5.0) * eta * a ** -5 * (1 + 73.0 / 24.0 * e**2 + 37.0 / 96.0 * e**4) / (1 - e * e) ** 3.5
    dL = -(32.0 / 5.0) * eta * a ** -3.5 * (1 + 7.0 / 8.0 * e**2) / (1 - e * e) ** 2
    return dE, dL


@pytest.mark.parametrize("gauge", GAUGES)
def test_circular_orbit_loses_energy_at_the_quadrupole_rate(gauge):
    # on a circular orbit (n.v = 0, v^2 = u) every gauge gives
    # dE/dt = -(32/5) eta u^5 and dL/dt = dE/dt / omega, omega = u^(3/2)
    for beta in (1.0, 0.4):
        s = newtonian(beta)
        for r in (8.0, 20.0, 55.0):
            y = kepler_state(r, 0.0, 0.7)
            a = orc.rr_accel(s, y, gauge)
            u = 1.0 / r
            assert y[3:6] @ a == pytest.approx(-(32.0 / 5.0) * s.eta * u**5, rel=1e-13)
            assert np.cross(y[0:3], a)[2] == pytest.approx(-(32.0 / 5.0) * s.eta * u**3.5, rel=1e-13)
            # along -v only
            assert np.linalg.norm(np.cross(a, y[3:6])) <= 1e-13 * np.linalg.norm(a) * np.linalg.norm(y[3:6])


@pytest.mark.parametrize("gauge", GAUGES)
@pytest.mark.parametrize("e", (0.2, 0.5, 0.8))
def test_orbit_averaged_losses_are_those_of_peters_and_mathews(gauge, e):
    # time average over one period by the trapezoid rule in the eccentric
    # anomaly (spectrally accurate for a smooth periodic integrand):
    # <f> = (1/2 pi) int f(E) (1 - e cos E) dE
    s = newtonian(0.6)
    a_axis = 25.0
    N = 2048
    dE = dL = 0.0
    for E in 2.0 * np.pi * np.arange(N) / N:
        y = kepler_state(a_axis, e, E)
        acc = orc.rr_accel(s, y, gauge)
        w = 1.0 - e * np.cos(E)
        dE += (y[3:6] @ acc) * w
        dL += np.cross(y[0:3], acc)[2] * w
    pE, pL = peters(a_axis, e, s.eta)
    assert dE / N == pytest.approx(pE, rel=1e-10)
    assert dL / N == pytest.approx(pL, rel=1e-10)


def test_force_is_odd_under_time_reversal_and_rotation_covariant():
    s = orc.system(0.5, pn_order=2)
    rng = np.random.default_rng(7)
    y = np.zeros(12)
    y[0:3] = rng.normal(size=3) * 9.0
    y[3:6] = rng.normal(size=3) * 0.2
    a = orc.rr_accel(s, y)
    yr = y.copy()
    yr[3:6] = -y[3:6]
    np.testing.assert_allclose(orc.rr_accel(s, yr), -a, rtol=1e-14, atol=0)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    yq = y.copy()
    yq[0:3] = q @ y[0:3]
    yq[3:6] = q @ y[3:6]
    np.testing.assert_allclose(orc.rr_accel(s, yq), q @ a, rtol=1e-12, atol=1e-12 * np.abs(a).max())
    # proportional to eta at fixed state
    s2 = orc.system(1.0, pn_order=2)
    np.testing.assert_allclose(orc.rr_accel(s2, y) / s2.eta, a / s.eta, rtol=1e-14)


def test_quasicircular_inspiral_follows_the_closed_form():
    # Newtonian binary with radiation reaction: adiabatic circular inspiral
    # r^4 = r0^4 - (256/5) eta t; the start on an exactly circular orbit
    # leaves an eccentricity of order (64/5) eta r0^(-5/2) ~ 2e-3
    cfg = orc.config(pn_order=0, use_so=0, use_ss=0, correct=1, rr=1, fli_renorm=0, r_merge=6.0)
    r0 = 20.0
    y0 = np.zeros(12)
    y0[0] = r0
    y0[4] = r0 ** -0.5
    eta = 0.25
    T = 8000
    tr = orc.trace(y0, 1.0, 1.0, T, every=1, cfg=cfg)
    r = np.linalg.norm(tr[:, 0:3], axis=1)
    t = np.arange(1, T + 1, dtype=float)
    pred = (r0**4 - 256.0 / 5.0 * eta * t) ** 0.25
    assert np.max(np.abs(r / pred - 1.0)) < 3e-3
    assert r[-1] < 0.8 * r0
    out = orc.scan(y0[None], 1.0, 1.0, 20000, cfg=cfg)
    assert out["status"][0] == orc.MERGED
    t_merge = (r0**4 - 6.0**4) / (256.0 / 5.0 * eta)
    assert out["t_stop"][0] == pytest.approx(t_merge, rel=2e-3)


def _run14(s, y14, h, n, rk_order=4):
    for _ in range(n):
        y14 = orc.rk_step_rr(s, y14, h, rk_order)
    return y14


def test_integral_invariant_relations_track_the_full_hamiltonian():
    # uncorrected run of a spinning binary with every term (2PN, SO, SS, QM)
    # and radiation reaction: the reference values carried by the integral-
    # invariant relations stay on H(y(t)) and |J(y(t))| to the integration
    # error while both change by far more
    s = orc.system(0.5, kappa1=3.0, kappa2=6.0, pn_order=2, use_qm=1)
    y = orc.setup_cells(np.array([[20.0, 1.05, 0.8, 0.3, 2.0, 1.1, 0.5, 0.9, 0.7]]))[0]
    I0 = orc.integrals(s, y)
    y14 = np.concatenate([y, I0[:2]])
    y14 = _run14(s, y14, 0.5, 2000)
    I = orc.integrals(s, y14[:12])
    assert I[0] - I0[0] < -0.02 * abs(I0[0])        # energy radiated (about 6 %)
    assert I[1] - I0[1] < -0.01 * I0[1]             # angular momentum radiated (about 2 %)
    assert abs(y14[12] - I[0]) < 1e-9 * abs(I0[0])  # RK4 error at h = 0.5: about 3e-11
    assert abs(y14[13] - I[1]) < 1e-9 * I0[1]
    # spin lengths are untouched by the radiation reaction
    np.testing.assert_allclose(I[2:4], I0[2:4], rtol=1e-11)


@pytest.mark.parametrize("rk_order,slope", ((4, 4), (5, 5)))
def test_extended_steps_converge_at_their_order(rk_order, slope):
    s = orc.system(1.0, pn_order=2)
    y = orc.setup_cells(np.array([[9.0, 1.0, 1.0, 0.0, 1.3, 0.0, 1.0, 1.0, 1.0]]))[0]
    I0 = orc.integrals(s, y)
    y14 = np.concatenate([y, I0[:2]])
    T = 40.0
    ref = _run14(s, y14, T / 640, 640, rk_order)
    errs = []
    for n in (20, 40):
        errs.append(np.max(np.abs(_run14(s, y14, T / n, n, rk_order) - ref)))
    order = np.log2(errs[0] / errs[1])
    assert slope - 0.4 < order < slope + 0.6, (errs, order)


def golden_orbit(name):
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_orbits.json")) as f:
        g = json.load(f)[name]
    beta = g["beta"]
    m1, m2 = beta / (1 + beta), 1 / (1 + beta)
    y = np.r_[g["r"], g["p"], g["chi1"] * m1 * m1 * np.array(g["S1_hat"]),
              g["chi2"] * m2 * m2 * np.array(g["S2_hat"])].astype(float)
    return beta, y


@pytest.mark.parametrize("rk_order", (4, 5))
def test_correction_holds_the_evolving_reference_values(rk_order):
    # orbit 3 of Sec. 3B with radiation reaction
    beta, y0 = golden_orbit("orbit_3")
    s = orc.system(beta, pn_order=2)
    I0 = orc.integrals(s, y0)
    cfg = orc.config(rr=1, rk_order=rk_order, fli_renorm=100)
    out = orc.scan(y0[None], beta, 2.0, 3000, cfg=cfg)
    assert out["status"][0] == orc.DONE
    E0, E, J0, J = out["integrals"][0, :4]
    assert E0 < I0[0] and J0 < I0[1]               # the references moved (energy radiated)
    assert abs(E - E0) <= 1e-13 * abs(E0)
    assert abs(J - J0) <= 1e-13 * J0
    # without the correction the same run drifts off the references
    cfg0 = orc.config(rr=1, rk_order=rk_order, correct=0, fli_renorm=100)
    out0 = orc.scan(y0[None], beta, 2.0, 3000, cfg=cfg0)
    E0u, Eu = out0["integrals"][0, :2]
    assert abs(Eu - E0u) > 10 * abs(E - E0)


def test_orbit3_spirals_in_with_its_energy_on_the_reference():
    """Fig. 5 (soft): orbit 3 decays until the merger cut; with the correction
    the energy stays on the integral-invariant reference at every sample
    (no secular growth, Fig. 5a); uncorrected RK5 drifts off it."""
    beta, y0 = golden_orbit("orbit_3")
    errs, errs0, binding = [], [], []
    for T in (25_000, 50_000, 100_000):
        out = orc.scan(y0[None], beta, 2.0, T // 2, orc.config(rr=1, rk_order=5, r_escape=0))
        out0 = orc.scan(y0[None], beta, 2.0, T // 2, orc.config(rr=1, rk_order=5, r_escape=0, correct=0))
        E0, E = out["integrals"][0, :2]
        errs.append(abs(E - E0) / abs(E0))
        E0u, Eu = out0["integrals"][0, :2]
        errs0.append(abs(Eu - E0u) / abs(E0u))
        binding.append(abs(E0))
    assert max(errs) <= 1e-14
    assert errs0[-1] > 1e3 * max(errs)
    assert binding[0] < binding[1] < binding[2]    # |E| grows: the binary hardens
    out = orc.scan(y0[None], beta, 2.0, 200_000, orc.config(rr=1, rk_order=5, r_escape=0))
    assert out["status"][0] == orc.MERGED and 2.0e5 < out["t_stop"][0] < 3.5e5


def test_scalar_J_reference_matches_the_vector_form():
    # d|J|/dt = J.(r x a)/|J| integrated as a scalar (the oracle) against the
    # vector dJ/dt = r x a integrated beside it by a plain RK4 of this test,
    # on the same RK4 stages of the full spinning Hamiltonian: the norms agree
    # to the integration error
    s = orc.system(0.7, kappa1=2.0, kappa2=4.0, pn_order=2, use_qm=1)
    y = orc.setup_cells(np.array([[18.0, 1.0, 0.6, 0.2, 2.3, 1.7, 0.7, 0.8, 0.6]]))[0]
    I0 = orc.integrals(s, y)
    y14 = np.concatenate([y, I0[:2]])
    Jv = I0[4:7].copy()
    h = 0.5

    def f(z14, jv):
        d = orc.rhs_rr(s, z14)
        a = orc.rr_accel(s, z14[:12])
        return d, np.cross(z14[0:3], a)

    for _ in range(1200):
        k1, j1 = f(y14, Jv)
        k2, j2 = f(y14 + 0.5 * h * k1, Jv)
        k3, j3 = f(y14 + 0.5 * h * k2, Jv)
        k4, j4 = f(y14 + h * k3, Jv)
        y_next = orc.rk_step_rr(s, y14, h)
        Jv = Jv + h * (j1 + 2 * j2 + 2 * j3 + j4) / 6.0
        y14 = y_next
    assert abs(np.linalg.norm(Jv) - y14[13]) <= 1e-10 * y14[13]
    assert abs(y14[13] - I0[1]) > 1e-3 * I0[1]          # |J| did change
    # and the vector reference stays on J(y) of the state
    np.testing.assert_allclose(Jv, orc.integrals(s, y14[:12])[4:7], rtol=1e-9, atol=1e-9 * I0[1])


def test_ablation_modes_restore_what_they_claim_under_radiation_reaction():
    # orbit 3 with radiation reaction to t = 6000 (RK4, h = 2): velocity
    # scaling (mode 3) holds E on its moving reference but not |J|; spin
    # lengths alone (mode 2) hold neither; the dual scaling holds both
    beta, y0 = golden_orbit("orbit_3")
    s = orc.system(beta, pn_order=2)
    I0 = orc.integrals(s, y0)
    res = {}
    for mode in (0, 1, 2, 3):
        out = orc.scan(y0[None], beta, 2.0, 3000, orc.config(rr=1, correct=mode, fli_renorm=0))
        E0, E, J0, J, S1, S2 = out["integrals"][0]
        res[mode] = (abs(E - E0) / abs(E0), abs(J - J0) / J0, abs(S1 - I0[2]) / I0[2], abs(S2 - I0[3]) / I0[3])
    assert max(res[1]) <= 1e-14
    assert res[3][0] <= 1e-14 and res[3][1] > 100 * res[1][1] and max(res[3][2:]) <= 1e-14
    assert res[2][0] > 100 * res[1][0] and max(res[2][2:]) <= 1e-14
    assert res[0][0] > 100 * res[1][0] and res[0][1] > 100 * res[1][1]
