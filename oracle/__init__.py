"""Plain FP64 CPU oracle for the manifold-corrected PN spinning-binary scan.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package.  It shares
no code with the CUDA library; see ``pn_oracle.c`` for the method and its
citations (arXiv:1802.00147, Sec. 2 Eqs. 1-13, Sec. 3).
"""
import ctypes as _ct
from contextlib import contextmanager as _contextmanager

import numpy as _np

from .build import build as _build

_lib = None

# conditioning guard of the split scaling (orc_config.split_min), and the
# dual scaling's conditioning below which the better-conditioned of the two
# is used (orc_config.cond_switch)
SPLIT_MIN = 1e-3
COND_SWITCH = 1e-2

# per-orbit status numbering of the oracle
RUNNING, DONE, MERGED, ESCAPED, FLI_SATURATED, NONFINITE = range(6)


class Config(_ct.Structure):
    _fields_ = [
        ("pn_order", _ct.c_int), ("use_so", _ct.c_int), ("use_ss", _ct.c_int), ("use_qm", _ct.c_int),
        ("correct", _ct.c_int),
        ("newton_tol", _ct.c_double), ("newton_max", _ct.c_int), ("det_min", _ct.c_double),
        ("fli_d0", _ct.c_double), ("fli_renorm", _ct.c_int), ("fli_cap", _ct.c_double),
        ("r_merge", _ct.c_double), ("r_escape", _ct.c_double), ("rk_order", _ct.c_int),
        ("newton_apply_small", _ct.c_int),
        ("rr", _ct.c_int), ("rr_gauge_a", _ct.c_double), ("rr_gauge_b", _ct.c_double),
        ("split_min", _ct.c_double), ("cond_switch", _ct.c_double),
    ]


class Sys(_ct.Structure):
    _fields_ = [
        ("beta", _ct.c_double), ("m1", _ct.c_double), ("m2", _ct.c_double), ("eta", _ct.c_double),
        ("kappa1", _ct.c_double), ("kappa2", _ct.c_double),
        ("pn_order", _ct.c_int), ("use_so", _ct.c_int), ("use_ss", _ct.c_int), ("use_qm", _ct.c_int),
    ]


def config(pn_order=2, use_so=1, use_ss=1, use_qm=0, correct=1, newton_tol=1e-10,
           newton_max=50, det_min=1e-5, fli_d0=1e-9, fli_renorm=100, fli_cap=0.0,
           r_merge=6.0, r_escape=1e3, rk_order=4, newton_apply_small=1, rr=0,
           rr_gauge_a=4.0, rr_gauge_b=5.0, split_min=SPLIT_MIN, cond_switch=COND_SWITCH):
    return Config(pn_order, use_so, use_ss, use_qm, correct, newton_tol, newton_max,
                  det_min, fli_d0, fli_renorm, fli_cap, r_merge, r_escape, rk_order, newton_apply_small,
                  rr, rr_gauge_a, rr_gauge_b, split_min, cond_switch)


def lib():
    global _lib
    if _lib is None:
        _lib = _declare(_ct.CDLL(_build()))
    return _lib


def load_variant(path):
    """Another build of pn_oracle.c (e.g. build.build_variant's) with the
    same signatures declared; use it through `using`."""
    return _declare(_ct.CDLL(path))


@_contextmanager
def using(L):
    """Run the functions of this module on the oracle library L."""
    global _lib
    old = _lib
    _lib = L
    try:
        yield L
    finally:
        _lib = old


def _declare(L):
    P = _ct.POINTER
    d, i, i64 = _ct.c_double, _ct.c_int, _ct.c_int64
    dp = P(d)
    L.orc_sys_init.argtypes = [P(Sys), d, d, d, i, i, i, i]
    for name in ("orc_H_newton", "orc_H_1pn", "orc_H_2pn", "orc_H_so", "orc_H_s1s2",
                 "orc_H_qm", "orc_hamiltonian"):
        f = getattr(L, name)
        f.argtypes = [P(Sys), dp]
        f.restype = d
    L.orc_gradient.argtypes = [P(Sys), dp, dp]
    L.orc_rhs.argtypes = [P(Sys), dp, dp]
    L.orc_rk4_step.argtypes = [P(Sys), dp, d]
    L.orc_rk5_step.argtypes = [P(Sys), dp, d]
    L.orc_integrals.argtypes = [P(Sys), dp, dp]
    L.orc_rr_accel.argtypes = [P(Sys), d, d, dp, dp]
    L.orc_rhs_rr.argtypes = [P(Sys), d, d, dp, dp]
    L.orc_rk_step_rr.argtypes = [P(Sys), d, d, i, dp, d]
    L.orc_correct.argtypes = [P(Sys), dp, dp, d, i, d, P(i), dp]
    L.orc_correct.restype = i
    L.orc_waveform.argtypes = [P(Sys), dp, d, dp, dp, dp]
    L.orc_newton_trace.argtypes = [P(Sys), dp, dp, i, dp, dp]
    L.orc_newton_trace.restype = i
    L.orc_correct_rule.argtypes = [P(Sys), dp, dp, d, i, d, d, d, i, i, P(i), dp]
    L.orc_correct_rule.restype = i
    L.orc_setup_cell.argtypes = [dp, dp]
    L.orc_scan.argtypes = [i64, dp, dp, dp, dp, P(Config), d, i64, dp, dp, dp, dp,
                           P(_ct.c_int32), dp, P(i64), P(_ct.c_int32), P(_ct.c_int32), i]
    L.orc_scan.restype = i
    L.orc_trace.argtypes = [dp, d, d, d, P(Config), d, i64, i64, dp]
    L.orc_trace.restype = i
    L.orc_max_threads.restype = i
    try:
        L.orc_ext_trace.argtypes = [dp, d, d, d, P(Config), d, i64, dp]
        L.orc_ext_trace.restype = i
    except AttributeError:      # an older build of the file, loaded for comparison
        pass
    return L


def _dp(a):
    return a.ctypes.data_as(_ct.POINTER(_ct.c_double))


def _vec(y):
    return _np.ascontiguousarray(y, dtype=_np.float64)


def system(beta, kappa1=1.0, kappa2=1.0, pn_order=2, use_so=1, use_ss=1, use_qm=0):
    s = Sys()
    lib().orc_sys_init(_ct.byref(s), float(beta), float(kappa1), float(kappa2),
                       pn_order, use_so, use_ss, use_qm)
    return s


def hamiltonian(s, y, term="total"):
    name = {"total": "orc_hamiltonian", "N": "orc_H_newton", "1PN": "orc_H_1pn",
            "2PN": "orc_H_2pn", "SO": "orc_H_so", "S1S2": "orc_H_s1s2", "QM": "orc_H_qm"}[term]
    y = _vec(y)
    return getattr(lib(), name)(_ct.byref(s), _dp(y))


def gradient(s, y):
    y = _vec(y)
    g = _np.zeros(12)
    lib().orc_gradient(_ct.byref(s), _dp(y), _dp(g))
    return g


def rhs(s, y):
    y = _vec(y)
    dy = _np.zeros(12)
    lib().orc_rhs(_ct.byref(s), _dp(y), _dp(dy))
    return dy


def rk4_step(s, y, h):
    y = _vec(y).copy()
    lib().orc_rk4_step(_ct.byref(s), _dp(y), float(h))
    return y


def rk5_step(s, y, h):
    y = _vec(y).copy()
    lib().orc_rk5_step(_ct.byref(s), _dp(y), float(h))
    return y


def rr_accel(s, y, gauge=(4.0, 5.0)):
    """2.5PN radiation-reaction acceleration a_2.5PN (Eq. 6) at the state y."""
    y = _vec(y)
    a = _np.zeros(3)
    lib().orc_rr_accel(_ct.byref(s), float(gauge[0]), float(gauge[1]), _dp(y), _dp(a))
    return a


def rhs_rr(s, y14, gauge=(4.0, 5.0)):
    """d/dt of (r, p, S1, S2, E, |J|) with radiation reaction."""
    y14 = _vec(y14)
    dy = _np.zeros(14)
    lib().orc_rhs_rr(_ct.byref(s), float(gauge[0]), float(gauge[1]), _dp(y14), _dp(dy))
    return dy


def rk_step_rr(s, y14, h, rk_order=4, gauge=(4.0, 5.0)):
    y14 = _vec(y14).copy()
    lib().orc_rk_step_rr(_ct.byref(s), float(gauge[0]), float(gauge[1]), int(rk_order), _dp(y14), float(h))
    return y14


def integrals(s, y):
    """(E, |J|, |S1|, |S2|, Jx, Jy, Jz)."""
    y = _vec(y)
    out = _np.zeros(7)
    lib().orc_integrals(_ct.byref(s), _dp(y), _dp(out))
    return out


def waveform(s, y, R=1.0, P=(1.0, 0.0, 0.0), Q=(0.0, 1.0, 0.0)):
    """(h_plus, h_cross) of the mass quadrupole field at distance R (Eq. 14)."""
    y = _vec(y)
    Pv, Qv = _vec(P), _vec(Q)
    out = _np.zeros(2)
    lib().orc_waveform(_ct.byref(s), _dp(y), float(R), _dp(Pv), _dp(Qv), _dp(out))
    return out[0], out[1]


def newton_trace(s, y, ref, kmax=8):
    """Dual-scaling Newton iterates (alpha_k, beta_k), k = 1..m <= kmax, of
    Eq. 13 at the state y = (r*, p*, S) from (1, 1), no stopping rule."""
    y, ref = _vec(y), _vec(ref)
    a, b = _np.zeros(kmax), _np.zeros(kmax)
    m = lib().orc_newton_trace(_ct.byref(s), _dp(y), _dp(ref), int(kmax), _dp(a), _dp(b))
    return a[:m], b[:m]


MODE_DUAL, MODE_SPINS, MODE_VELOCITY = 1, 2, 3


CORR_DUAL, CORR_NONE, CORR_VELOCITY, CORR_SPLIT = 0, 1, 2, 3


def correct(s, y, ref, newton_tol=1e-10, newton_max=50, det_min=1e-5, mode=MODE_DUAL, apply_small=1,
            split_min=None, cond_switch=None):
    """Returns (y_corrected, code, iters, (alpha, beta)); code 0 dual scaling,
    3 split scaling (singular dual scaling), 2 velocity scaling (both
    singular, or mode MODE_VELOCITY), 1 nothing applied beyond the spin
    lengths.  For code 3 (alpha, beta) are the factors (a, g) of the
    tangential and radial parts of p."""
    y = _vec(y).copy()
    ref = _vec(ref)
    it = _ct.c_int(0)
    ab = _np.zeros(2)
    split_min = SPLIT_MIN if split_min is None else split_min
    cond_switch = COND_SWITCH if cond_switch is None else cond_switch
    code = lib().orc_correct_rule(_ct.byref(s), _dp(y), _dp(ref), newton_tol, newton_max,
                                  det_min, float(split_min), float(cond_switch), int(apply_small), int(mode),
                                  _ct.byref(it), _dp(ab))
    return y, code, it.value, (ab[0], ab[1])


def setup_cells(cells):
    """cells: (n, 9) = (x0, pfac, theta1, phi1, theta2, phi2, beta, chi1, chi2)."""
    cells = _np.ascontiguousarray(cells, dtype=_np.float64).reshape(-1, 9)
    out = _np.zeros((cells.shape[0], 12))
    for i in range(cells.shape[0]):
        lib().orc_setup_cell(_dp(cells[i]), _dp(out[i]))
    return out


def scan(y0, beta, h, nsteps, cfg=None, kappa1=None, kappa2=None, nthreads=0):
    """Integrate n orbits with correction + FLI.  Returns a dict of arrays."""
    cfg = cfg or config()
    y0 = _np.ascontiguousarray(y0, dtype=_np.float64).reshape(-1, 12)
    n = y0.shape[0]
    beta = _np.ascontiguousarray(_np.broadcast_to(beta, (n,)), dtype=_np.float64)
    k1 = None if kappa1 is None else _np.ascontiguousarray(_np.broadcast_to(kappa1, (n,)), dtype=_np.float64)
    k2 = None if kappa2 is None else _np.ascontiguousarray(_np.broadcast_to(kappa2, (n,)), dtype=_np.float64)
    out = dict(y=_np.zeros((n, 12)), ys=_np.zeros((n, 12)), integrals=_np.zeros((n, 6)),
               fli=_np.zeros(n), status=_np.zeros(n, dtype=_np.int32), t_stop=_np.zeros(n),
               newton_iters=_np.zeros(n, dtype=_np.int64), n_skip=_np.zeros(n, dtype=_np.int32),
               last_kind=_np.zeros(n, dtype=_np.int32))
    P = _ct.POINTER
    rc = lib().orc_scan(n, _dp(y0), _dp(beta),
                        None if k1 is None else _dp(k1), None if k2 is None else _dp(k2),
                        _ct.byref(cfg), float(h), int(nsteps),
                        _dp(out["y"]), _dp(out["ys"]), _dp(out["integrals"]), _dp(out["fli"]),
                        out["status"].ctypes.data_as(P(_ct.c_int32)), _dp(out["t_stop"]),
                        out["newton_iters"].ctypes.data_as(P(_ct.c_int64)),
                        out["n_skip"].ctypes.data_as(P(_ct.c_int32)),
                        out["last_kind"].ctypes.data_as(P(_ct.c_int32)), int(nthreads))
    if rc != 0:
        raise ValueError("orc_scan rejected its arguments")
    return out


def trace(y0, beta, h, nsteps, every=1, cfg=None, kappa1=1.0, kappa2=1.0):
    cfg = cfg or config()
    y0 = _vec(y0)
    m = int(nsteps) // int(every)
    out = _np.zeros((m, 12))
    lib().orc_trace(_dp(y0), float(beta), float(kappa1), float(kappa2), _ct.byref(cfg),
                    float(h), int(nsteps), int(every), _dp(out))
    return out


def ext_trace(y0, beta, h, nsteps, cfg=None, kappa1=1.0, kappa2=1.0):
    """Final state of one corrected trajectory (no FLI shadow) after nsteps,
    computed in the library's arithmetic type (double, or long double in a
    build_variant with -DORC_LONG_DOUBLE); double in and out."""
    cfg = cfg or config()
    y0 = _vec(y0)
    out = _np.zeros(12)
    if lib().orc_ext_trace(_dp(y0), float(beta), float(kappa1), float(kappa2), _ct.byref(cfg), float(h),
                           int(nsteps), _dp(out)) != 0:
        raise ValueError("orc_ext_trace rejected its arguments")
    return out


def max_threads():
    return lib().orc_max_threads()
