"""The rounding floor the GPU parity tests assert against, checked on the CPU
with two builds of the same oracle: the reference build rounds every + and *
separately, the other contracts multiply-adds into FMAs, as the GPU kernels
do.  The two are the same algorithm, so everything between them is rounding.

Pinned here, on the small scan and on the uneven batch to t = 1000, with the
default correction and with the dual scaling kept down to its singular
guard (cond_switch 0):
  * statuses and stop times agree exactly;
  * every orbit's state lies within max(1e-10, 3x) its one-ulp spread;
  * every orbit's FLI lies within 3x its FLI spread over all 24 one-ulp
    moves (each component up and down) plus 1e-3 -- the per-orbit FLI floor
    of tests/test_gpu_parity.py -- while three moves alone are too few for
    the noisier cond_switch 0 correction;
  * with the default correction the two builds' FLIs differ by < 3e-3 (a
    median 1.6e-4), against up to 0.5 (median 6e-3) with cond_switch 0;
  * the class (FLI > 6) agrees on every orbit.
The FMA build needs FMA instructions: baseline on aarch64, -mfma on x86-64
(skipped where the CPU lacks them)."""
import os
import platform
import tempfile

import numpy as np
import pytest

import oracle
from oracle import build as ob
from paper_1802_00147_gb300 import workloads as W

from test_gpu_parity import block_relerr, ulp_spreads


def fma_flags():
    m = platform.machine().lower()
    if m in ("aarch64", "arm64"):
        return ["-ffp-contract=fast"]
    if m in ("x86_64", "amd64"):
        try:
            flags = open("/proc/cpuinfo").read()
        except OSError:
            return None
        return ["-mfma", "-ffp-contract=fast"] if " fma " in flags else None
    return None


@pytest.fixture(scope="module")
def fma_lib():
    flags = fma_flags()
    if flags is None:
        pytest.skip("no FMA instructions on this CPU")
    d = tempfile.mkdtemp()
    path = ob.build_variant(os.path.join(d, "libpnoracle_fma.so"), flags)
    return oracle.load_variant(path)


def run(cells, nsteps, y0=None, h=1.0, d0=1e-9, **kw):
    if y0 is None:
        y0 = oracle.setup_cells(cells[:, :9])
    return oracle.scan(y0, cells[:, W.BETA], h, nsteps, oracle.config(fli_d0=d0, **kw),
                       kappa1=cells[:, W.KAP1], kappa2=cells[:, W.KAP2])


@pytest.mark.slow
@pytest.mark.parametrize("cond_switch", [None, 0.0])
@pytest.mark.parametrize("which", ["small", "uneven"])
def test_fma_rounding_lies_within_the_per_orbit_floor(fma_lib, which, cond_switch):
    cells = W.small_scan(seed=1) if which == "small" else W.uneven_batch(n=1500, seed=3)
    nsteps = 1000
    kw = {} if cond_switch is None else dict(cond_switch=cond_switch)
    o = run(cells, nsteps, **kw)
    with oracle.using(fma_lib):
        f = run(cells, nsteps, **kw)
    y0 = oracle.setup_cells(cells[:, :9])
    s_state, s_fli3, _ = ulp_spreads(
        lambda y1, hh, idx, dd: run(cells if idx is None else cells[idx], nsteps, y0=y1, h=hh, d0=dd, **kw),
        y0, o, (0, 4, 6), 1.0)
    np.testing.assert_array_equal(f["status"], o["status"])
    np.testing.assert_array_equal(f["t_stop"], o["t_stop"])
    ok = o["status"] != oracle.NONFINITE
    err = block_relerr(f["y"][ok], o["y"][ok])
    assert np.all(err <= np.maximum(1e-10, 3 * s_state[ok]))
    done = o["status"] == oracle.DONE
    df = np.abs(f["fli"] - o["fli"])[done]
    assert np.all(df <= 3 * o["s_fli_all"][done] + 1e-3), np.max(df / (o["s_fli_all"][done] + 1e-300))
    if cond_switch == 0.0:
        # three moves underestimate the floor: some orbit exceeds 3x their spread
        assert np.any(df > 3 * s_fli3[done] + 1e-3)
        assert df.max() > 0.1
    else:
        assert df.max() < 3e-3 and np.median(df) < 1e-3, (df.max(), np.median(df))
    # the denser estimate contains the 24-move one
    idx = np.flatnonzero(done)[:2]
    assert np.all(o["refine_fli"](idx) >= o["s_fli_all"][idx])
    assert np.array_equal(f["fli"][done] > 6.0, o["fli"][done] > 6.0)


@pytest.mark.slow
def test_per_orbit_state_bound_catches_a_planted_mistake():
    """The GPU parity bound err_i <= max(1e-10, 3 s_i) has power: an oracle
    build whose spin-orbit coefficient (Eqs. 8-9's g1) is off by 1e-7
    relative lands beyond it on every orbit of the small scan at t = 1000
    (median error 1.2e-7), although it is the same program otherwise."""
    cells = W.small_scan(seed=1)
    nsteps = 1000
    o = run(cells, nsteps)
    y0 = oracle.setup_cells(cells[:, :9])
    s_state, _, _ = ulp_spreads(
        lambda y1, hh, idx, dd: run(cells if idx is None else cells[idx], nsteps, y0=y1, h=hh, d0=dd),
        y0, o, (0, 4, 6), 1.0)
    d = tempfile.mkdtemp()
    planted = oracle.load_variant(ob.build_variant(os.path.join(d, "libpnoracle_planted.so"),
                                                   ["-ffp-contract=off", "-DORC_PLANTED_SO_FACTOR=1.0000001"]))
    with oracle.using(planted):
        g = run(cells, nsteps)
    ok = o["status"] != oracle.NONFINITE
    err = block_relerr(g["y"][ok], o["y"][ok])
    assert np.all(err > np.maximum(1e-10, 3 * s_state[ok])), np.sort(err)[:3]
