"""The GPU's FP64 state against the extended-precision reference (the
oracle's plain C in long double, see tests/test_oracle_extended_precision.py)
over 1, 5 and 20 corrected RK4 and RK5 steps, through the C ABI: the parity
floor of tests/test_gpu_parity.py rests on the oracle's own one-ulp spread;
here both FP64 programs are measured against a third, wider one.  The FP64
oracle lies within 16 ulps of it (per block r, p, S1, S2); the kernels, which
fuse multiply-adds and evaluate H and its gradient in another formulation,
within BOUND_ULPS."""
import os
import tempfile

import numpy as np
import pytest

import oracle
from oracle import build as ob
from paper_1802_00147_gb300 import workloads as W

from test_oracle_extended_precision import ULP, block_relerr, cells, traces

pytestmark = pytest.mark.gpu

BOUND_ULPS = 32


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00147_gb300 import build
    build.build()
    import paper_1802_00147_gb300 as pn
    d = tempfile.mkdtemp()
    ld = oracle.load_variant(ob.build_variant(os.path.join(d, "libpnoracle_ld.so"),
                                              ["-ffp-contract=off", "-DORC_LONG_DOUBLE"]))
    return pn, ld


@pytest.mark.parametrize("rk", [4, 5])
def test_gpu_state_within_ulps_of_long_double(env, rk):
    pn, ld = env
    c = cells()
    cfg = oracle.config(r_merge=0, r_escape=0, rk_order=rk)
    for n in (1, 5, 20):
        s = pn.Scan(c[:, W.BETA], kappa1=c[:, W.KAP1], kappa2=c[:, W.KAP2], r_merge=0.0, r_escape=0.0, rk_order=rk)
        s.setup(c)
        s.run(float(n), 1.0)
        g = s.read()["states"]
        s.close()
        ref = traces(c, n, cfg, ld)
        e_gpu = block_relerr(g, ref) / ULP
        e_orc = block_relerr(traces(c, n, cfg), ref) / ULP
        assert e_gpu.max() <= BOUND_ULPS, (rk, n, e_gpu.max(), np.median(e_gpu), e_orc.max())
        # and statistically no farther than the FP64 oracle, within a factor 3
        assert np.median(e_gpu) <= 3 * np.median(e_orc) + 2, (rk, n, np.median(e_gpu), np.median(e_orc))
