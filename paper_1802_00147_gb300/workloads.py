"""Seeded synthetic scan workloads (inputs only -- none of the method's arithmetic).

Both the CUDA path and the CPU oracle receive the arrays made here; the
initial-condition set-up itself (spin vectors, circular momentum, shadow
offset) is computed independently by each side.

A *cell* is one orbit's scan parameters, 11 FP64 fields:

    0 x0      initial separation, r = (x0, 0, 0)
    1 pfac    p_y as a fraction of the Newtonian circular momentum 1/sqrt(x0)
    2 theta1  polar angle of S1 from the z axis (the initial L direction)
    3 phi1    azimuth of S1
    4 theta2  polar angle of S2
    5 phi2    azimuth of S2
    6 beta    mass ratio m1/m2 <= 1 (Sec. 2 of arXiv:1802.00147)
    7 chi1    dimensionless spin magnitude of body 1
    8 chi2    dimensionless spin magnitude of body 2
    9 kappa1  quadrupole-monopole multiplier of body 1 (1 = black hole)
   10 kappa2  quadrupole-monopole multiplier of body 2

The scans stand in for the paper's phase-space scans (Sec. 3C, Figs. 6-7,
Table 3), which use no external dataset.  Random draws use numpy's PCG64
generator with the given seed.  ``random_states`` draws explicit states in
random orientations instead of cells; both sides receive the same states.
"""
import numpy as np

NFIELDS = 11
X0, PFAC, TH1, PH1, TH2, PH2, BETA, CHI1, CHI2, KAP1, KAP2 = range(NFIELDS)


def _grid(nx, nt, x_lo, x_hi):
    x0 = np.linspace(x_lo, x_hi, nx)
    th = np.linspace(0.0, np.pi, nt)
    X, T = np.meshgrid(x0, th, indexing="ij")
    return X.ravel(), T.ravel()


def grid_cells(nx, nt, x_lo, x_hi, seed, beta=None, chi=None, kappa=None, pfac=0.9):
    """(x0, theta) grid with both spins at polar angle theta and seeded azimuths.

    beta / chi / kappa: None for the fixed values 1, or a (lo, hi) range for a
    seeded uniform draw per cell (chi1, chi2 and kappa1, kappa2 drawn
    independently)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X, T = _grid(nx, nt, x_lo, x_hi)
    n = X.size
    c = np.zeros((n, NFIELDS))
    c[:, X0] = X
    c[:, PFAC] = pfac
    c[:, TH1] = T
    c[:, TH2] = T
    c[:, PH1] = rng.uniform(0.0, 2.0 * np.pi, n)
    c[:, PH2] = rng.uniform(0.0, 2.0 * np.pi, n)
    c[:, BETA] = 1.0 if beta is None else rng.uniform(beta[0], beta[1], n)
    if chi is None:
        c[:, CHI1] = c[:, CHI2] = 1.0
    else:
        c[:, CHI1] = rng.uniform(chi[0], chi[1], n)
        c[:, CHI2] = rng.uniform(chi[0], chi[1], n)
    if kappa is None:
        c[:, KAP1] = c[:, KAP2] = 1.0
    else:
        c[:, KAP1] = rng.uniform(kappa[0], kappa[1], n)
        c[:, KAP2] = rng.uniform(kappa[0], kappa[1], n)
    return c


def small_scan(seed=1):
    """16 x 16 = 256 orbits: x0 in [15, 40], theta in [0, pi], m1 = m2, chi = 1."""
    return grid_cells(16, 16, 15.0, 40.0, seed)


def full_scan(seed=2, nx=314, nt=314):
    """314 x 314 = 98,596 orbits: x0 in [10, 50], theta in [0, pi],
    beta ~ U[0.5, 1], chi_i ~ U[0.5, 1]."""
    return grid_cells(nx, nt, 10.0, 50.0, seed, beta=(0.5, 1.0), chi=(0.5, 1.0))


def uneven_batch(n=100_000, seed=3):
    """Uneven batch: beta ~ U[0.1, 1], chi_i ~ U[0, 1], isotropic spin
    directions, x0 ~ U[10, 50], p_y 50-100% of circular."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = np.zeros((n, NFIELDS))
    c[:, X0] = rng.uniform(10.0, 50.0, n)
    c[:, PFAC] = rng.uniform(0.5, 1.0, n)
    c[:, TH1] = np.arccos(rng.uniform(-1.0, 1.0, n))
    c[:, PH1] = rng.uniform(0.0, 2.0 * np.pi, n)
    c[:, TH2] = np.arccos(rng.uniform(-1.0, 1.0, n))
    c[:, PH2] = rng.uniform(0.0, 2.0 * np.pi, n)
    c[:, BETA] = rng.uniform(0.1, 1.0, n)
    c[:, CHI1] = rng.uniform(0.0, 1.0, n)
    c[:, CHI2] = rng.uniform(0.0, 1.0, n)
    c[:, KAP1] = c[:, KAP2] = 1.0
    return c


def adaptive_grid(n=1024, seed=4):
    """n x n grid of the small-scan parameters (x0 in [15, 40], theta in [0, pi])."""
    return grid_cells(n, n, 15.0, 40.0, seed)


def qm_grid(n=1024, seed=5):
    """n x n small-scan grid with kappa_i ~ U[1, 10] (quadrupole-monopole study)."""
    return grid_cells(n, n, 15.0, 40.0, seed, kappa=(1.0, 10.0))


def random_states(n, seed=31):
    """Seeded states in random orientations: |r| ~ U[12, 40] along an isotropic
    direction, p perpendicular to r in a random direction with |p| 60-100 %
    of the Newtonian circular value 1/sqrt(|r|), a small random radial part,
    and spin vectors of isotropic direction with |S_i| = chi_i m_i^2, chi_i ~
    U[0, 1].  Also beta ~ U[0.2, 1] and kappa_i ~ U[1, 10].  Returns
    (states n x 12, beta, kappa1, kappa2)."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def unit(m):
        v = rng.normal(size=(m, 3))
        return v / np.linalg.norm(v, axis=1, keepdims=True)

    r = rng.uniform(12.0, 40.0, n)
    nr = unit(n)
    t = unit(n)
    t = t - np.sum(t * nr, axis=1, keepdims=True) * nr
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    pmag = rng.uniform(0.6, 1.0, n) / np.sqrt(r)
    beta = rng.uniform(0.2, 1.0, n)
    m1, m2 = beta / (1 + beta), 1 / (1 + beta)
    y = np.zeros((n, 12))
    y[:, 0:3] = r[:, None] * nr
    y[:, 3:6] = pmag[:, None] * (t + rng.uniform(-0.1, 0.1, n)[:, None] * nr)
    y[:, 6:9] = (rng.uniform(0, 1, n) * m1 * m1)[:, None] * unit(n)
    y[:, 9:12] = (rng.uniform(0, 1, n) * m2 * m2)[:, None] * unit(n)
    return y, beta, rng.uniform(1, 10, n), rng.uniform(1, 10, n)


def subset(cells, m, seed=6):
    """A seeded subset of m cells (sorted indices) and the indices themselves."""
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = np.sort(rng.choice(cells.shape[0], size=min(m, cells.shape[0]), replace=False))
    return cells[idx], idx


def paper_cells(x0, p_y, beta, theta1, theta2, chi=1.0):
    """Cells of the paper's own scans: r = (x0, 0, 0), p = (0, p_y, 0), both
    spins in the x-z plane at polar angles theta1, theta2 (arrays), chi_i = chi."""
    theta1 = np.asarray(theta1, dtype=np.float64)
    theta2 = np.asarray(theta2, dtype=np.float64)
    theta1, theta2 = np.broadcast_arrays(theta1, theta2)
    n = theta1.size
    c = np.zeros((n, NFIELDS))
    c[:, X0] = x0
    c[:, PFAC] = p_y * np.sqrt(x0)
    c[:, TH1] = theta1.ravel()
    c[:, TH2] = theta2.ravel()
    c[:, BETA] = beta
    c[:, CHI1] = c[:, CHI2] = chi
    c[:, KAP1] = c[:, KAP2] = 1.0
    return c


def _polar(v):
    v = np.asarray(v, dtype=np.float64)
    v = v / np.linalg.norm(v)
    return float(np.arccos(np.clip(v[2], -1.0, 1.0))), float(np.arctan2(v[1], v[0]))


def paper_orbit_cells():
    """The paper's single orbits as cells, with polar / azimuthal spin angles
    from the printed unit vectors:
    - orbit 4 (Sec. 4): (beta, r, p_y) = (1, 10, 0.274), theta1 = 1.0 rad,
      theta2 = 1.325 rad in the x-z plane, chi = 1;
    - case II orbit 2 (Sec. 3B): (1, 10.14, 0.365), S1 = (0.13036, 0.262852,
      -0.955989), S2 = (0.118966, -0.13459, -0.983734), chi = 1;
    - case II orbit 1 (Sec. 3B): (1/3, 20, 0.2461), S1 = (sin 60, 0, cos 60),
      S2 = (sin 45, 0, cos 45), chi = 0.75;
    - orbit 3 (Sec. 3B, with radiation reaction): (1, 50, 0.140),
      S1 = (sin 45, 0, cos 45), S2 = (sin 30, 0, cos 30), chi = (1, 0.85).
    Returns (names, cells)."""
    names = ("orbit_4", "case_II_orbit_2", "case_II_orbit_1", "orbit_3")
    c = np.zeros((len(names), NFIELDS))
    rows = ((10.0, 0.274, 1.0, (np.sin(1.0), 0, np.cos(1.0)), (np.sin(1.325), 0, np.cos(1.325)), 1.0, 1.0),
            (10.14, 0.365, 1.0, (0.13036, 0.262852, -0.955989), (0.118966, -0.13459, -0.983734), 1.0, 1.0),
            (20.0, 0.2461, 1.0 / 3.0, (np.sin(np.pi / 3), 0, 0.5), (np.sqrt(0.5), 0, np.sqrt(0.5)), 0.75, 0.75),
            (50.0, 0.140, 1.0, (np.sqrt(0.5), 0, np.sqrt(0.5)), (0.5, 0, np.sqrt(0.75)), 1.0, 0.85))
    for k, (x0, py, beta, s1, s2, chi1, chi2) in enumerate(rows):
        c[k, X0] = x0
        c[k, PFAC] = py * np.sqrt(x0)
        c[k, TH1], c[k, PH1] = _polar(s1)
        c[k, TH2], c[k, PH2] = _polar(s2)
        c[k, BETA] = beta
        c[k, CHI1] = chi1
        c[k, CHI2] = chi2
        c[k, KAP1] = c[k, KAP2] = 1.0
    return names, c


def paper_theta2_scan(theta1, n=314):
    """Sec. 3C, Fig. 6: theta2 from 0 in steps of 0.01 (314 orbits), theta1
    fixed, (beta, r, p) = (1/3, 5.65, 0.765)."""
    return paper_cells(5.65, 0.765, 1.0 / 3.0, theta1, 0.01 * np.arange(n))


def theta12_plane(n):
    """The plane of Sec. 3C, Fig. 7 on an n x n grid: theta1, theta2 =
    linspace(0, pi, n) (row-major, theta1 slow), (beta, r, p) = (1, 10.14,
    0.365), chi = 1, spins in the x-z plane."""
    t = np.linspace(0.0, np.pi, n)
    T1, T2 = np.meshgrid(t, t, indexing="ij")
    return paper_cells(10.14, 0.365, 1.0, T1.ravel(), T2.ravel())


def theta12_random(m, seed, x0=10.14):
    """m cells of the same plane at seeded uniform (theta1, theta2) in [0, pi]^2;
    with another x0, the neighbouring plane at that separation and the same
    fraction of the circular momentum (p_y sqrt(x0) = 0.365 sqrt(10.14))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p_y = 0.365 * np.sqrt(10.14 / x0)
    return paper_cells(x0, p_y, 1.0, rng.uniform(0.0, np.pi, m), rng.uniform(0.0, np.pi, m))


def paper_theta12_scan(n=314):
    """Sec. 3C, Fig. 7: the (theta1, theta2) plane, both from 0 in steps of 0.01
    (314 x 314 orbits), (beta, r, p) = (1, 10.14, 0.365), chi = 1."""
    t = 0.01 * np.arange(n)
    T1, T2 = np.meshgrid(t, t, indexing="ij")
    return paper_cells(10.14, 0.365, 1.0, T1.ravel(), T2.ravel())
