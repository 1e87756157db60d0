"""Pins of the CPU oracle against things other than itself (no GPU needed).

Every pin is chosen so that a plausible slip in the oracle -- a dropped term,
a wrong sign or coefficient, a transposed operand -- fails one of them:

* central finite differences of H       -> analytic gradient (all terms)
* Eqs. 8-9 of arXiv:1802.00147 as printed -> spin gradients Omega_i of H
* gauge-invariant 2PN circular-orbit energy E(x) (closed form) -> 1PN/2PN orbital terms
* Kepler closure after one period (closed form T = 2 pi a^{3/2}) -> H_N, RK4
* conservation of J = L + S1 + S2 and |S_i| by the flow        -> Eqs. 6-7 signs
* time reversal (r, p, S) -> (r, -p, -S)                         -> RK4 + correction
* RK4 global error order 4
* exact restoration of E, |J|, |S_i| by the correction (Eqs. 10-13)
* the Newton root of Eq. 13 vs an independent 2-D root finder, and its
  quadratic convergence (a wrong Jacobian entry would make it linear)
* FLI of an integrable orbit grows as a power law; the paper's case II
  orbits 1 / 2 are regular / chaotic (Sec. 3B, Fig. 3)
* the Newton tolerance matters only under the stop-before-applying rule,
  and then sets the energy error's size (Fig. 4)
"""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_orbits.json")


def paper_orbit(name):
    with open(GOLDEN) as f:
        g = json.load(f)[name]
    beta = g["beta"]
    m1, m2 = beta / (1 + beta), 1 / (1 + beta)
    y = np.r_[g["r"], g["p"], g["chi1"] * m1 * m1 * np.array(g["S1_hat"]),
              g["chi2"] * m2 * m2 * np.array(g["S2_hat"])].astype(float)
    return beta, y


def random_state(rng, r_lo=8.0, r_hi=30.0):
    r = rng.uniform(r_lo, r_hi)
    d = rng.normal(size=3)
    rv = r * d / np.linalg.norm(d)
    pv = rng.normal(size=3) * (0.6 / np.sqrt(r))
    S1 = rng.normal(size=3) * 0.1
    S2 = rng.normal(size=3) * 0.1
    return np.r_[rv, pv, S1, S2]


# ------------------------------------------------------------------ gradient
@pytest.mark.parametrize("beta", [1.0, 0.5, 0.2])
def test_gradient_matches_central_differences(orc, beta):
    rng = np.random.default_rng(11)
    s = orc.system(beta, kappa1=2.5, kappa2=7.0, pn_order=2, use_so=1, use_ss=1, use_qm=1)
    for _ in range(5):
        y = random_state(rng)
        g = orc.gradient(s, y)
        fd = np.zeros(12)
        for i in range(12):
            e = np.zeros(12)
            e[i] = 1e-5 * max(1.0, abs(y[i]))
            fd[i] = (orc.hamiltonian(s, y + e) - orc.hamiltonian(s, y - e)) / (2 * e[i])
        scale = np.abs(g).max()
        assert np.max(np.abs(g - fd)) < 1e-7 * scale, (g, fd)


@pytest.mark.parametrize("term", ["1PN", "2PN", "SO", "S1S2", "QM"])
def test_each_term_is_differentiated(orc, term):
    """Gradient of each Hamiltonian term alone (others off) against FD of that term."""
    rng = np.random.default_rng(5)
    flags = dict(pn_order=0, use_so=0, use_ss=0, use_qm=0)
    if term == "1PN":
        flags["pn_order"] = 1
    elif term == "2PN":
        flags["pn_order"] = 2
    else:
        flags[{"SO": "use_so", "S1S2": "use_ss", "QM": "use_qm"}[term]] = 1
    s = orc.system(0.4, kappa1=3.0, kappa2=2.0, **flags)
    y = random_state(rng)
    g = orc.gradient(s, y)
    fd = np.zeros(12)
    for i in range(12):
        e = np.zeros(12)
        e[i] = 1e-5 * max(1.0, abs(y[i]))
        fd[i] = (orc.hamiltonian(s, y + e) - orc.hamiltonian(s, y - e)) / (2 * e[i])
    # subtract the Newtonian part, which every configuration contains
    assert np.max(np.abs(g - fd)) < 1e-7 * np.abs(g).max()


# ------------------------------------------------- Eqs. 8-9 (spin precession)
def omega_paper(beta, y):
    """Omega_1, Omega_2 exactly as printed in Eqs. 8-9 (QM on, kappa = 1)."""
    r, p, S1, S2 = y[:3], y[3:6], y[6:9], y[9:12]
    eta = beta / (1 + beta) ** 2
    rr = np.linalg.norm(r)
    n = r / rr
    L = np.cross(r, p)
    O1 = ((2 + 3 / (2 * beta)) * L / rr ** 3 + (3 * n * (S2 @ n) - S2) / (eta * rr ** 3)
          + 3 / rr ** 3 * (1 + 1 / beta) ** 2 * n * (S1 @ n))
    O2 = ((2 + 3 * beta / 2) * L / rr ** 3 + (3 * n * (S1 @ n) - S1) / (eta * rr ** 3)
          + 3 / rr ** 3 * (1 + beta) ** 2 * n * (S2 @ n))
    return O1, O2


@pytest.mark.parametrize("beta", [1.0, 1 / 3, 0.15])
def test_spin_gradients_reproduce_eqs_8_9(orc, beta):
    rng = np.random.default_rng(7)
    s = orc.system(beta, pn_order=2, use_so=1, use_ss=1, use_qm=1)
    for _ in range(4):
        y = random_state(rng)
        fd = np.zeros(6)
        for i in range(6):
            e = np.zeros(12)
            e[6 + i] = 1e-6
            fd[i] = (orc.hamiltonian(s, y + e) - orc.hamiltonian(s, y - e)) / 2e-6
        O1, O2 = omega_paper(beta, y)
        rr = np.linalg.norm(y[:3])
        # Eqs. 8-9 drop the -S_i part of the QM gradient (it is parallel to S_i
        # and drops out of Omega_i x S_i); add it back for a component check.
        O1_full = O1 - (1 + 1 / beta) ** 2 * y[6:9] / rr ** 3
        O2_full = O2 - (1 + beta) ** 2 * y[9:12] / rr ** 3
        assert np.allclose(fd[:3], O1_full, rtol=1e-7, atol=1e-12 * np.abs(O1).max())
        assert np.allclose(fd[3:], O2_full, rtol=1e-7, atol=1e-12 * np.abs(O2).max())
        # and the precession the printed Omegas generate equals the oracle's EOM
        dy = orc.rhs(s, y)
        assert np.allclose(dy[6:9], np.cross(O1, y[6:9]), rtol=1e-12, atol=1e-18)
        assert np.allclose(dy[9:12], np.cross(O2, y[9:12]), rtol=1e-12, atol=1e-18)


# --------------------------------------------- 2PN circular-orbit energy E(x)
def circular_energy_numeric(orc, s, r):
    """Circular orbit of the oracle's H at separation r: returns (x, E)."""
    from scipy.optimize import brentq

    def radial_force(py):
        # dH/dr at fixed angular momentum L = r p_y:  dH/dx - (p_y / r) dH/dp_y
        y = np.r_[r, 0, 0, 0, py, 0, np.zeros(6)]
        g = orc.gradient(s, y)
        return g[0] - (py / r) * g[4]

    py = brentq(radial_force, 0.5 / np.sqrt(r), 1.5 / np.sqrt(r), xtol=1e-17, rtol=1e-15)
    y = np.r_[r, 0, 0, 0, py, 0, np.zeros(6)]
    omega = orc.gradient(s, y)[4] / r          # d(phi)/dt = (dH/dp_y) / r
    return omega ** (2.0 / 3.0), orc.hamiltonian(s, y)


def circular_energy_closed_form(x, eta):
    """Gauge-invariant 2PN binding energy per unit reduced mass of a circular
    orbit, x = (M omega)^{2/3} (standard PN result, e.g. Blanchet 2014)."""
    return -0.5 * x * (1 - (0.75 + eta / 12) * x - (27 / 8 - 19 * eta / 8 + eta ** 2 / 24) * x ** 2)


@pytest.mark.parametrize("beta", [1.0, 1 / 3])
def test_circular_orbit_energy_matches_2pn_closed_form(orc, beta):
    s = orc.system(beta, pn_order=2, use_so=0, use_ss=0, use_qm=0)
    eta = s.eta
    ratios = []
    for r in (100.0, 200.0, 400.0):
        x, E = circular_energy_numeric(orc, s, r)
        resid = E - circular_energy_closed_form(x, eta)
        ratios.append(resid / x ** 4)   # the first omitted (3PN) order
    ratios = np.array(ratios)
    # an error in any 1PN / 2PN coefficient leaves a residual ~x^2 or ~x^3,
    # whose ratio to x^4 would grow by 2x-4x per halving of x
    assert np.all(np.abs(ratios) < 20), ratios
    assert np.max(np.abs(np.diff(ratios))) < 0.1 * np.max(np.abs(ratios)) + 0.05, ratios


# ------------------------------------------------------------ Kepler limit
def kepler_system(orc):
    return orc.system(1.0, pn_order=0, use_so=0, use_ss=0, use_qm=0)


def test_kepler_orbit_closes_after_one_period(orc):
    s = kepler_system(orc)
    y0 = np.r_[10.0, 0, 0, 0, 0.28, 0, np.zeros(6)]
    E = orc.hamiltonian(s, y0)
    a = -1 / (2 * E)
    T = 2 * np.pi * a ** 1.5
    errs = []
    for N in (1000, 2000):
        y = y0.copy()
        h = T / N
        for _ in range(N):
            y = orc.rk4_step(s, y, h)
        errs.append(np.linalg.norm(y[:3] - y0[:3]) / 10.0)
    assert errs[1] < 1e-8
    assert 10 < errs[0] / errs[1] < 24      # RK4: global error ~ h^4
    # eccentricity from the closed form e = sqrt(1 + 2 E L^2)
    L = 10.0 * 0.28
    e = np.sqrt(1 + 2 * E * L * L)
    assert abs(e - (1 - 10.0 * 0.28 ** 2)) < 1e-12   # apocentre start: e = 1 - r v^2


@pytest.mark.parametrize("cond_switch", [0.0, None])
def test_kepler_period_and_correction(orc, cond_switch):
    """With the manifold correction on, E and |J| stay exact and the orbit
    still closes after one closed-form period -- with the dual scaling at
    every step (cond_switch 0: it is never singular on this e = 0.22
    ellipse), and with the split scaling taking the steps near r = a where
    the dual scaling is ill-conditioned (the default)."""
    s = kepler_system(orc)
    y0 = np.r_[10.0, 0, 0, 0, 0.28, 0, np.zeros(6)]
    ref = orc.integrals(s, y0)[:4]
    E = ref[0]
    T = 2 * np.pi * (-1 / (2 * E)) ** 1.5
    N = 2000
    y = y0.copy()
    codes = []
    for _ in range(N):
        y = orc.rk4_step(s, y, T / N)
        y, code, it, _ = orc.correct(s, y, ref, cond_switch=cond_switch)
        codes.append(code)
    assert set(codes) == ({0} if cond_switch == 0.0 else {0, 3}), set(codes)
    I = orc.integrals(s, y)
    assert abs(I[0] - E) < 1e-15
    assert abs(I[1] - ref[1]) < 1e-14
    assert np.linalg.norm(y[:3] - y0[:3]) / 10.0 < 1e-8


# ------------------------------------------------------ conservation of J
def test_flow_conserves_J_vector_and_spin_lengths(orc):
    rng = np.random.default_rng(3)
    s = orc.system(0.5, kappa1=4.0, kappa2=2.0, pn_order=2, use_so=1, use_ss=1, use_qm=1)
    y = random_state(rng, 12, 14)
    I0 = orc.integrals(s, y)
    drift = {}
    for h in (0.1, 0.05):
        yy = y.copy()
        for _ in range(int(round(50 / h))):
            yy = orc.rk4_step(s, yy, h)
        I = orc.integrals(s, yy)
        drift[h] = np.linalg.norm(I[4:7] - I0[4:7]) / np.linalg.norm(I0[4:7])
        assert abs(I[2] - I0[2]) < 1e-9 * I0[2]
        assert abs(I[3] - I0[3]) < 1e-9 * I0[3]
    assert drift[0.05] < 1e-9
    # the drift is RK4 truncation (shrinks ~16x per halving), not a wrong EOM
    assert drift[0.1] / max(drift[0.05], 1e-300) > 6


def test_wrong_spin_sign_would_break_J(orc):
    """Planted-mistake control: precessing the spins the other way (S x Omega)
    does not conserve J, so the test above can fail."""
    rng = np.random.default_rng(3)
    s = orc.system(0.5, pn_order=2, use_so=1, use_ss=1, use_qm=0)
    y = random_state(rng, 12, 14)

    def bad_rhs(y):
        dy = orc.rhs(s, y)
        dy[6:] = -dy[6:]
        return dy

    I0 = orc.integrals(s, y)
    h = 0.05
    for _ in range(1000):
        k1 = bad_rhs(y)
        k2 = bad_rhs(y + h / 2 * k1)
        k3 = bad_rhs(y + h / 2 * k2)
        k4 = bad_rhs(y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    I = orc.integrals(s, y)
    assert np.linalg.norm(I[4:7] - I0[4:7]) / np.linalg.norm(I0[4:7]) > 1e-6


# ------------------------------------------------------------ time reversal
def test_time_reversal_returns_to_start(orc):
    rng = np.random.default_rng(9)
    s = orc.system(0.5, kappa1=3.0, kappa2=1.5, pn_order=2, use_so=1, use_ss=1, use_qm=1)
    y0 = random_state(rng, 12, 16)
    ref = orc.integrals(s, y0)[:4]
    flip = np.r_[np.ones(3), -np.ones(9)]
    y = y0.copy()
    for _ in range(400):
        y = orc.rk4_step(s, y, 0.05)
        y, _, _, _ = orc.correct(s, y, ref)
    y = y * flip
    ref_b = orc.integrals(s, y)[:4]
    assert abs(ref_b[0] - ref[0]) < 1e-15 and abs(ref_b[1] - ref[1]) < 1e-13
    for _ in range(400):
        y = orc.rk4_step(s, y, 0.05)
        y, _, _, _ = orc.correct(s, y, ref_b)
    y = y * flip
    assert np.linalg.norm(y[:3] - y0[:3]) / np.linalg.norm(y0[:3]) < 1e-10
    assert np.linalg.norm(y[3:6] - y0[3:6]) / np.linalg.norm(y0[3:6]) < 1e-10
    assert np.linalg.norm(y[6:] - y0[6:]) / np.linalg.norm(y0[6:]) < 1e-10


# ---------------------------------------------------------------- RK4 order
def test_rk4_energy_error_is_fourth_order(orc):
    beta, y0 = paper_orbit("case_II_orbit_1")
    s = orc.system(beta)
    E0 = orc.hamiltonian(s, y0)
    err = []
    for h in (1.0, 0.5):
        y = y0.copy()
        for _ in range(int(round(200 / h))):
            y = orc.rk4_step(s, y, h)
        err.append(abs(orc.hamiltonian(s, y) - E0))
    assert 10 < err[0] / err[1] < 24


def test_rk5_energy_error_is_fifth_order(orc):
    """The fifth-order Dormand-Prince weights: halving h shrinks the global
    energy error ~32x (a wrong tableau entry drops the order)."""
    beta, y0 = paper_orbit("case_II_orbit_1")
    s = orc.system(beta)
    E0 = orc.hamiltonian(s, y0)
    err = []
    for h in (2.0, 1.0):
        y = y0.copy()
        for _ in range(int(round(400 / h))):
            y = orc.rk5_step(s, y, h)
        err.append(abs(orc.hamiltonian(s, y) - E0))
    assert 22 < err[0] / err[1] < 45, err


def test_rk5_kepler_closure(orc):
    s = kepler_system(orc)
    y0 = np.r_[10.0, 0, 0, 0, 0.28, 0, np.zeros(6)]
    T = 2 * np.pi * (-1 / (2 * orc.hamiltonian(s, y0))) ** 1.5
    errs = []
    for N in (500, 1000):
        y = y0.copy()
        for _ in range(N):
            y = orc.rk5_step(s, y, T / N)
        errs.append(np.linalg.norm(y[:3] - y0[:3]) / 10.0)
    assert errs[1] < 1e-9 and 22 < errs[0] / errs[1] < 45, errs


# ------------------------------------------------------ manifold correction
def test_correction_restores_all_six_integrals(orc):
    rng = np.random.default_rng(21)
    for beta in (1.0, 0.3):
        s = orc.system(beta, kappa1=2.0, kappa2=5.0, use_qm=1)
        for _ in range(5):
            y0 = random_state(rng, 10, 25)
            ref = orc.integrals(s, y0)
            y = orc.rk4_step(s, y0, 15.0)             # a crude step: visible errors
            Ibad = orc.integrals(s, y)
            assert abs(Ibad[0] - ref[0]) > 1e-12 * abs(ref[0])
            y, code, it, (a, b) = orc.correct(s, y, ref[:4])
            assert code in (0, 3) and it <= 6
            I = orc.integrals(s, y)
            assert abs(I[0] - ref[0]) <= 1e-14 * abs(ref[0])
            assert abs(I[1] - ref[1]) <= 1e-14 * ref[1]
            assert abs(I[2] - ref[2]) <= 1e-15 * ref[2]
            assert abs(I[3] - ref[3]) <= 1e-15 * ref[3]


def test_correction_is_identity_on_the_manifold(orc):
    rng = np.random.default_rng(4)
    s = orc.system(0.7)
    y0 = random_state(rng, 10, 25)
    ref = orc.integrals(s, y0)[:4]
    y, code, it, (a, b) = orc.correct(s, y0, ref)
    assert code == 0 and it == 1
    assert abs(a - 1) < 1e-15 and abs(b - 1) < 1e-15
    assert np.allclose(y, y0, rtol=1e-15, atol=0)


def test_newton_root_matches_independent_root_finder(orc):
    """The (alpha, beta) of Eq. 13 from the oracle's Newton equal the root that
    scipy's hybrid solver finds for the same two conditions."""
    from scipy.optimize import root
    rng = np.random.default_rng(8)
    s = orc.system(0.6)
    y0 = random_state(rng, 12, 20)
    ref = orc.integrals(s, y0)[:4]
    ystar = orc.rk4_step(s, y0, 5.0)
    # spins first (Eq. 10), exactly as the oracle does
    S = ystar.copy()
    for i, L in ((6, ref[2]), (9, ref[3])):
        S[i:i + 3] = S[i:i + 3] * (L / np.linalg.norm(S[i:i + 3]))

    def F(v):
        a, b = v
        yb = S.copy()
        yb[:3] = b * S[:3]
        yb[3:6] = a * S[3:6]
        I = orc.integrals(s, yb)
        return [(I[0] - ref[0]) / abs(ref[0]), (I[1] - ref[1]) / ref[1]]

    sol = root(F, [1.0, 1.0], method="hybr", options=dict(xtol=1e-15))
    _, code, _, (a, b) = orc.correct(s, ystar, ref)
    assert code == 0
    assert abs(a - sol.x[0]) < 1e-12 and abs(b - sol.x[1]) < 1e-12


def test_correction_restores_integrals_on_random_states(orc):
    """Over random states, mass ratios and kappas, a crude RK4 step followed by
    the correction (Eqs. 10-13) restores what its outcome code promises: the
    dual scaling (code 0) E, |J| and both spin lengths to rounding; the
    split scaling (code 3) E, |J| and the spin lengths, with r unchanged; the
    velocity scaling (code 2) E and the spin lengths, with r unchanged."""
    rng = np.random.default_rng(123)
    seen = set()
    for _ in range(60):
        beta = rng.uniform(0.1, 1.0)
        s = orc.system(beta, kappa1=rng.uniform(1, 10), kappa2=rng.uniform(1, 10),
                       pn_order=2, use_so=1, use_ss=1, use_qm=1)
        y0 = random_state(rng, 10.0, 40.0)
        I0 = orc.integrals(s, y0)
        ref = np.array(I0[:4])
        y1 = orc.rk4_step(s, y0, rng.uniform(2.0, 6.0))
        y2, code, it, _ = orc.correct(s, y1, ref)
        I2 = orc.integrals(s, y2)
        seen.add(code)
        assert code in (0, 2, 3), code
        assert abs(I2[0] - I0[0]) <= 1e-13 * abs(I0[0])
        assert abs(I2[2] - I0[2]) <= 1e-14 * I0[2] and abs(I2[3] - I0[3]) <= 1e-14 * I0[3]
        if code in (0, 3):
            assert abs(I2[1] - I0[1]) <= 1e-13 * I0[1]
            assert it >= 1
        if code in (2, 3):
            np.testing.assert_array_equal(y2[:3], y1[:3])
    assert 0 in seen


def test_newton_converges_quadratically(orc):
    """Newton's method with the exact Jacobian converges quadratically,
    e_{k+1} <= C e_k^2, while a wrong Jacobian entry (a sign, a transposed
    derivative) gives linear convergence at best.  From a crude RK step the
    dual-scaling iterates of Eq. 13 are followed for 6 steps: while the error
    is above rounding, each error is bounded by a fixed multiple of the
    square of the previous one (and the ratio e_{k+1} / e_k collapses)."""
    for name in ("case_II_orbit_1", "case_II_orbit_2"):
        beta, y0 = paper_orbit(name)
        s = orc.system(beta, pn_order=2, use_so=1, use_ss=1)
        I0 = orc.integrals(s, y0)
        ref = np.array([I0[0], I0[1], I0[2], I0[3]])
        y = orc.rk4_step(s, y0, 25.0)
        for k in (0, 1):                      # spins on their fixed lengths first (Eq. 10)
            S = y[6 + 3 * k:9 + 3 * k]
            y[6 + 3 * k:9 + 3 * k] = S * (ref[2 + k] / np.linalg.norm(S))
        a, b = orc.newton_trace(s, y, ref, kmax=6)
        assert a.size == 6
        err = np.maximum(np.abs(a - a[-1]), np.abs(b - b[-1]))[:-1]
        e = np.r_[max(abs(1 - a[-1]), abs(1 - b[-1])), err]     # e_0 at the start (1, 1)
        assert e[0] > 1e-6, (name, e)                           # a visible first correction
        for k in range(len(e) - 1):
            if e[k] < 1e-13:
                break
            assert e[k + 1] <= 50.0 * e[k] ** 2 + 1e-14, (name, k, e)   # + rounding of the limit
        assert e[2] <= 1e-3 * e[1], (name, e)


def test_singular_scaling_falls_back_to_velocity_scaling(orc):
    """Where alpha p.dH/dp = beta r.dH/dr the dual scaling has no unique
    solution; the oracle then restores E by scaling p alone (velocity
    scaling) and leaves r unchanged."""
    s = orc.system(1.0, pn_order=0, use_so=0, use_ss=0, use_qm=0)
    # Newtonian: p.dH/dp - r.dH/dr = p^2 - 1/r = 0 on the circle p = 1/sqrt(r)
    r = 20.0
    y = np.r_[r, 0, 0, 0, 1 / np.sqrt(r), 0, np.zeros(6)]
    ref = orc.integrals(s, y)[:4].copy()
    ref[0] -= 1e-9
    y2, code, it, (a, b) = orc.correct(s, y, ref)
    assert code == 2 and b == 1.0
    assert np.array_equal(y2[:3], y[:3])
    assert np.allclose(y2[3:6], a * y[3:6], rtol=0, atol=0)
    assert abs(orc.hamiltonian(s, y2) - ref[0]) <= 1e-16
    # closed form: p'^2/2 - 1/r = E0  ->  a = sqrt(2 (E0 + 1/r)) / p
    assert abs(a - np.sqrt(2 * (ref[0] + 1 / r)) / (1 / np.sqrt(r))) < 1e-15


def newtonian_point_at_semi_major_axis(e, a=25.0, tilt=0.3):
    """A Kepler ellipse (G = M = 1, reduced units) at r = a, where p^2 = 1/r
    and the dual scaling is singular; radial momentum fraction |p_r|/|p| = e.
    The orbital plane is tilted about x so that every component is used."""
    r = a
    p = 1.0 / np.sqrt(a)
    # at r = a: cos(nu) = -e, radial speed e / sqrt(a), tangential sqrt(1 - e^2) / sqrt(a)
    pr, pt = e * p, np.sqrt(1.0 - e * e) * p
    c, s_ = np.cos(tilt), np.sin(tilt)
    n = np.array([1.0, 0.0, 0.0])
    t = np.array([0.0, c, s_])
    return np.r_[r * n, pr * n + pt * t, np.zeros(6)], pr, pt


@pytest.mark.parametrize("e", [0.1, 0.3, 0.6])
def test_split_scaling_restores_both_integrals_where_the_dual_scaling_is_singular(orc, e):
    """Newtonian (no spins): at r = a the dual scaling's Jacobian vanishes
    (p.dH/dp = p^2 = 1/r = r.dH/dr).  The split scaling p = a p_t + g p_r
    (r kept) then restores both integrals, in closed form: |J| = a |L*| fixes
    a = J0 / |L*|, and (a^2 p_t^2 + g^2 p_r^2) / 2 - 1/r = E0 fixes g."""
    s = orc.system(1.0, pn_order=0, use_so=0, use_ss=0, use_qm=0)
    y, pr, pt = newtonian_point_at_semi_major_axis(e)
    ref = orc.integrals(s, y)[:4].copy()
    ref[0] *= 1 + 3e-9
    ref[1] *= 1 - 2e-9
    y2, code, it, (a, g) = orc.correct(s, y, ref)
    assert code == 3, code
    np.testing.assert_array_equal(y2[:3], y[:3])
    a_cf = ref[1] / (y[0] * pt)
    g_cf = np.sqrt(2 * (ref[0] + 1 / y[0]) - (a_cf * pt) ** 2) / pr
    assert abs(a - a_cf) <= 1e-15 and abs(g - g_cf) <= 1e-14 / e, (a - a_cf, g - g_cf)
    I2 = orc.integrals(s, y2)
    assert abs(I2[0] - ref[0]) <= 1e-15 * abs(ref[0]) and abs(I2[1] - ref[1]) <= 1e-15 * ref[1]
    # the momentum moved within the plane of r and p, only along p_t and p_r
    n = y[:3] / np.linalg.norm(y[:3])
    d = y2[3:6] - y[3:6]
    assert abs(np.dot(d, np.cross(n, y[3:6]))) <= 1e-18


def test_split_scaling_is_not_used_near_circular_orbits(orc):
    """Near a circular orbit E and |J| cannot be moved independently (their
    gradients are parallel on the circle), so the split scaling is as
    ill-conditioned as the dual one: below split_min the correction falls
    back to the velocity scaling of E alone (code 2)."""
    s = orc.system(1.0, pn_order=0, use_so=0, use_ss=0, use_qm=0)
    y, pr, pt = newtonian_point_at_semi_major_axis(0.01)      # (|p_r|/|p|)^2 = 1e-4 < 1e-3
    ref = orc.integrals(s, y)[:4].copy()
    ref[0] *= 1 + 3e-9
    y2, code, _, _ = orc.correct(s, y, ref)
    assert code == 2
    y3, code3, _, _ = orc.correct(s, y, ref, split_min=1e-5)
    assert code3 == 3


@pytest.mark.slow
def test_integrable_orbits_stay_regular():
    """Without spins the PN two-body problem is integrable, so every orbit's
    FLI grows as a power law: over 160 orbits of eccentricities ~0-0.4 and
    mass ratios 0.3-1 none exceeds 5 at t = 1e5 (a corrected run whose kicks
    differed between the two trajectories would climb past it)."""
    import oracle as orc
    rng = np.random.default_rng(5)
    n = 160
    x0 = rng.uniform(12, 40, n)
    pf = rng.uniform(0.75, 1.12, n)
    beta = rng.uniform(0.3, 1, n)
    y0 = np.zeros((n, 12))
    y0[:, 0] = x0
    y0[:, 4] = pf / np.sqrt(x0)
    o = orc.scan(y0, beta, 1.0, 100_000, orc.config(r_merge=0, r_escape=0))
    assert o["fli"].max() < 5.0, np.sort(o["fli"])[-5:]
    I = o["integrals"]
    assert np.max(np.abs(I[:, 3] - I[:, 2]) / I[:, 2]) <= 1e-14


# ------------------------------------------------------------------ FLI
def test_fli_of_integrable_orbit_grows_as_power_law(orc):
    beta, y0 = paper_orbit("case_I_orbit_1")
    cfg = orc.config(r_merge=0, r_escape=0)
    f4 = orc.scan(y0[None], beta, 1.0, 10_000, cfg)["fli"][0]
    f5 = orc.scan(y0[None], beta, 1.0, 100_000, cfg)["fli"][0]
    assert f5 < 5.0
    assert f5 - f4 < 1.6        # ~log10(10) per decade, not exponential


@pytest.mark.slow
def test_fli_classifies_paper_case_II_orbits(orc):
    """Sec. 3B / Fig. 3: case II orbit 1 regular (power-law FLI), orbit 2
    chaotic (exponential FLI), at the 5.8 threshold of Sec. 3C, with the
    paper's corrected RK5.  Orbit 2's exponential growth sets in late: an
    uncorrected RK5 run at h = 0.25 (energy error 2e-5) gives FLI 3.8, 5.2
    and 7.3 at t = 1e5, 4e5 and 8e5, and orbit 1 3.4, 4.5 and 4.6; so the
    classes are compared at t = 8e5."""
    with open(GOLDEN) as f:
        thr = json.load(f)["fli_threshold"]["value"]
    cfg = orc.config(r_merge=0, r_escape=0, rk_order=5)
    b1, y1 = paper_orbit("case_II_orbit_1")
    b2, y2 = paper_orbit("case_II_orbit_2")
    f1 = orc.scan(y1[None], b1, 1.0, 800_000, cfg)["fli"][0]
    f2 = orc.scan(y2[None], b2, 1.0, 800_000, cfg)["fli"][0]
    assert f1 < thr < f2, (f1, f2)


@pytest.mark.slow
def test_fli_does_not_depend_on_the_step_where_the_dual_scaling_is_ill_conditioned(orc):
    """Rounding in the correction's F reaches the state amplified by the
    inverse conditioning of the scaling; where the two FLI trajectories get
    different kicks, the separation grows from the kicks alone, and the
    kicks scale with the truncation error, i.e. with h.  With the split
    scaling taking the dual scaling's ill-conditioned band (cond_switch),
    case II orbit 2's FLI at t = 8e5 is the same at h = 1 and 0.5 within
    the indicator's spread, and near the uncorrected h = 0.25 run's 7.3;
    with the dual scaling down to its 1e-5 guard it is 35 at h = 1 and 18 at
    h = 0.5."""
    b2, y2 = paper_orbit("case_II_orbit_2")
    f = {}
    for sw in (None, 0.0):
        for h in (1.0, 0.5):
            kw = {} if sw is None else dict(cond_switch=sw)
            cfg = orc.config(r_merge=0, r_escape=0, fli_renorm=int(round(100 / h)), **kw)
            f[sw, h] = orc.scan(y2[None], b2, h, int(8e5 / h), cfg)["fli"][0]
    assert abs(f[None, 1.0] - f[None, 0.5]) < 1.0 and 5.8 < f[None, 1.0] < 9.0, f
    assert f[0.0, 1.0] > 20 and abs(f[0.0, 1.0] - f[0.0, 0.5]) > 10, f


def test_corrected_energy_error_at_table_2_level(orc):
    """Table 2: with correction the energy error at t = 1e4 is ~1e-15 (case I)
    and <= 1e-11 (case II)."""
    cfg = orc.config(r_merge=0, r_escape=0)
    for name in ("case_I_orbit_1", "case_I_orbit_2", "case_II_orbit_1", "case_II_orbit_2"):
        beta, y0 = paper_orbit(name)
        I = orc.scan(y0[None], beta, 1.0, 10_000, cfg)["integrals"][0]
        assert abs(I[1] - I[0]) <= 1e-14 * abs(I[0]), name
        assert abs(I[3] - I[2]) <= 1e-14 * I[2], name


def test_uncorrected_rk4_drifts(orc):
    """Without correction the energy error grows (Table 2 'linear growth')."""
    beta, y0 = paper_orbit("case_II_orbit_2")
    cfg = orc.config(correct=0, r_merge=0, r_escape=0)
    e = []
    for T in (2000, 8000):
        I = orc.scan(y0[None], beta, 1.0, T, cfg)["integrals"][0]
        e.append(abs(I[1] - I[0]) / abs(I[0]))
    assert e[0] > 1e-11 and e[1] > 2 * e[0]


def test_newton_tolerance_ablation_fig_4(orc):
    """Fig. 4 / Sec. 3A: the energy error depends on the Newton tolerance eps
    of the scale factors only under the rule that stops BEFORE applying a
    step already within eps.  Then the error follows the uncorrected drift
    until the pending step exceeds eps, so its size is set by eps (~7 eps
    here, a sawtooth whose first tooth is the linear growth of Fig. 4);
    under the default rule (apply the step, then test it) the error left is
    quadratic in eps (round-off from eps = 1e-8 down).  Orbit 4, corrected RK5, h = 1, 2e4 steps."""
    beta, y0 = paper_orbit("orbit_4")
    s = orc.system(beta, pn_order=2, use_so=1, use_ss=1)
    E0 = orc.hamiltonian(s, y0)
    worst = {}
    for apply_small in (1, 0):
        for eps in (1e-6, 1e-8, 1e-10):
            cfg = orc.config(newton_tol=eps, newton_apply_small=apply_small, rk_order=5,
                             r_merge=0, r_escape=0)
            tr = orc.trace(y0, beta, 1.0, 20_000, 1, cfg)
            worst[apply_small, eps] = max(abs(orc.hamiltonian(s, y) - E0) for y in tr) / abs(E0)
    for eps in (1e-6, 1e-8, 1e-10):
        # after an applied step Newton's remaining error is quadratic in it
        assert worst[1, eps] <= max(1e-13, 100 * eps * eps), (eps, worst[1, eps])
        assert worst[1, eps] <= 1e-4 * worst[0, eps]
        assert 0.1 * eps <= worst[0, eps] <= 100 * eps, (eps, worst[0, eps])
    assert worst[0, 1e-6] > 10 * worst[0, 1e-8] > 100 * worst[0, 1e-10]


def test_correction_modes_restore_what_they_claim(orc):
    """The correction ablations: mode 2 (Eq. 10 alone) restores the spin
    lengths and leaves r, p as the RK step left them; mode 3 (velocity
    scaling, Sec. 1) restores the spin lengths and E0 by scaling p alone, so
    r and the direction of p are untouched and |J| is not restored."""
    beta, y0 = paper_orbit("case_II_orbit_2")
    s = orc.system(beta, pn_order=2, use_so=1, use_ss=1)
    I0 = orc.integrals(s, y0)
    ref = np.array([I0[0], I0[1], I0[2], I0[3]])
    y = orc.rk4_step(s, y0, 15.0)                  # a crude step: every integral is off
    Iy = orc.integrals(s, y)
    assert abs(Iy[0] - I0[0]) > 1e-9 * abs(I0[0]) and abs(Iy[1] - I0[1]) > 1e-9 * I0[1]
    y2, code2, it2, _ = orc.correct(s, y, ref, mode=orc.MODE_SPINS)
    I2 = orc.integrals(s, y2)
    assert code2 == 1 and it2 == 0
    np.testing.assert_array_equal(y2[:6], y[:6])
    assert abs(I2[2] - I0[2]) <= 1e-15 * I0[2] and abs(I2[3] - I0[3]) <= 1e-15 * I0[3]
    y3, code3, it3, (a, b) = orc.correct(s, y, ref, mode=orc.MODE_VELOCITY)
    I3 = orc.integrals(s, y3)
    assert code3 == 2 and it3 >= 1 and b == 1.0
    np.testing.assert_array_equal(y3[:3], y[:3])
    np.testing.assert_array_equal(y3[6:], y2[6:])
    np.testing.assert_allclose(y3[3:6], a * y[3:6], rtol=1e-15)
    assert abs(I3[0] - I0[0]) <= 1e-14 * abs(I0[0])
    assert abs(I3[1] - I0[1]) > 1e-9 * I0[1]


def test_correction_ablation_drifts(orc):
    """Over 5000 steps of case II orbit 2: with no correction E, |J| and |S_i|
    drift; Eq. 10 alone fixes |S_i| only; velocity scaling adds E; the dual
    scaling holds all of them at round-off."""
    beta, y0 = paper_orbit("case_II_orbit_2")
    drift = {}
    for mode in (0, 1, 2, 3):
        cfg = orc.config(correct=mode, r_merge=0, r_escape=0)
        o = orc.scan(y0[None], beta, 1.0, 5000, cfg)
        I = o["integrals"][0]
        s0 = np.linalg.norm(y0[6:9]), np.linalg.norm(y0[9:12])
        drift[mode] = (abs(I[1] - I[0]) / abs(I[0]), abs(I[3] - I[2]) / I[2],
                       max(abs(I[4] - s0[0]) / s0[0], abs(I[5] - s0[1]) / s0[1]))
    dE, dJ, dS = zip(*(drift[m] for m in (0, 1, 2, 3)))
    assert dE[0] > 1e-10 and dJ[0] > 1e-11 and dS[0] > 1e-12
    assert dE[1] <= 1e-14 and dJ[1] <= 1e-14 and dS[1] <= 1e-15
    assert dS[2] <= 1e-15 and dE[2] > 1e-10 and dJ[2] > 1e-11
    assert dS[3] <= 1e-15 and dE[3] <= 1e-14 and dJ[3] > 1e-11


# ---------------------------------------------------- gravitational waves
def test_waveform_of_a_circular_orbit(orc):
    """Quadrupole field of a Newtonian circular orbit of radius a, face-on
    (N = z, P = x, Q = y): h_plus = -(4 eta / (R a)) cos 2 phi and
    h_cross = -(4 eta / (R a)) sin 2 phi at orbital phase phi; amplitude
    proportional to eta / R."""
    for beta in (1.0, 0.4):
        s = orc.system(beta, pn_order=0, use_so=0, use_ss=0)
        eta = beta / (1 + beta) ** 2
        a, R = 20.0, 1e3
        w = a ** -1.5
        for phi in np.linspace(0.0, 2 * np.pi, 13):
            y = np.zeros(12)
            y[:3] = a * np.cos(phi), a * np.sin(phi), 0.0
            y[3:6] = a * w * -np.sin(phi), a * w * np.cos(phi), 0.0
            hp, hc = orc.waveform(s, y, R)
            amp = 4 * eta / (R * a)
            assert abs(hp + amp * np.cos(2 * phi)) <= 1e-14 * amp
            assert abs(hc + amp * np.sin(2 * phi)) <= 1e-14 * amp


def test_waveform_is_spin_two_under_frame_rotation(orc):
    """Rotating the radiation frame (P, Q) by psi about N turns (h_plus,
    h_cross) by 2 psi, for any state (a spin-2 field)."""
    beta, y = paper_orbit("case_II_orbit_2")
    s = orc.system(beta, pn_order=2, use_so=1, use_ss=1)
    h0 = np.array(orc.waveform(s, y, 100.0))
    for psi in (0.3, 1.1, 2.5):
        P = (np.cos(psi), np.sin(psi), 0.0)
        Q = (-np.sin(psi), np.cos(psi), 0.0)
        h = np.array(orc.waveform(s, y, 100.0, P, Q))
        c, sn = np.cos(2 * psi), np.sin(2 * psi)
        want = np.array([c * h0[0] + sn * h0[1], -sn * h0[0] + c * h0[1]])
        np.testing.assert_allclose(h, want, rtol=0, atol=1e-14 * np.abs(h0).max())


# ---------------------------------------------------- set-up and statuses
def test_setup_cell_geometry(orc):
    cells = np.array([[20.0, 0.9, 0.7, 1.1, 2.0, 4.0, 0.5, 0.8, 0.6]])
    y = orc.setup_cells(cells)[0]
    m1, m2 = 0.5 / 1.5, 1 / 1.5
    assert np.allclose(y[:3], [20, 0, 0]) and np.allclose(y[3:6], [0, 0.9 / np.sqrt(20), 0])
    assert abs(np.linalg.norm(y[6:9]) - 0.8 * m1 ** 2) < 1e-16
    assert abs(np.linalg.norm(y[9:12]) - 0.6 * m2 ** 2) < 1e-16
    assert abs(np.arccos(y[8] / np.linalg.norm(y[6:9])) - 0.7) < 1e-13
    assert abs(np.arctan2(y[10], y[9]) - (4.0 - 2 * np.pi)) < 1e-13


def test_termination_statuses(orc):
    beta = 1.0
    cells = np.array([[20.0, 0.9, 1.0, 0.0, 1.0, 1.0, 1.0, 1.0, 1.0],     # runs to the end
                      [9.0, 0.45, 1.0, 0.0, 1.0, 1.0, 1.0, 1.0, 1.0],     # plunges: r < 6
                      [20.0, 2.0, 1.0, 0.0, 1.0, 1.0, 1.0, 1.0, 1.0]])    # unbound: r > 1e3
    y0 = orc.setup_cells(cells)
    out = orc.scan(y0, beta, 1.0, 8000, orc.config())
    assert list(out["status"]) == [orc.DONE, orc.MERGED, orc.ESCAPED]
    assert out["t_stop"][0] == 8000.0 and out["t_stop"][1] < 8000 and out["t_stop"][2] < 8000
    bad = y0[:1].copy()
    bad[0, 4] = np.nan
    out = orc.scan(bad, beta, 1.0, 10, orc.config())
    assert out["status"][0] == orc.NONFINITE and out["t_stop"][0] == 1.0
    b2, y2 = paper_orbit("case_II_orbit_2")
    out = orc.scan(y2[None], b2, 1.0, 100_000, orc.config(r_merge=0, r_escape=0, fli_cap=4.0))
    assert out["status"][0] == orc.FLI_SATURATED and out["t_stop"][0] % 100 == 0
