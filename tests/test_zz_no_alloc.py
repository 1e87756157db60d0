"""scan_summary_noalloc: the scan reduction for callers that cannot allocate
device memory when they reduce (a framework whose caching allocator holds the
memory budget, a loop that must not allocate after start-up).  Checked through the C ABI against scan_summary, the
handle's reduction, on the same device arrays, on two calls in a row (the
second call reuses the library's fixed scratch that the first left behind).

Counts, maxima and sums of integers must agree exactly; the FLI mean agrees
to 1e-12 relative (the two reductions add in different orders); max_dS to
1e-15 absolute (the reference spin lengths are recomputed on the host here).
This file is named to be collected last."""
import numpy as np
import pytest

from paper_1802_00147_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_summary_matches_handle_summary_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00147_gb300 import build
    build.build()
    import paper_1802_00147_gb300 as pn

    cells = W.uneven_batch(n=5000, seed=17)
    s = pn.Scan(cells[:, W.BETA], device=True)
    s.setup(torch.as_tensor(cells[:, :9], device="cuda"))
    s.run(900.0, 1.0)
    out = s.read()
    diag = s.read_diag()
    ref = s.summary()
    s.close()

    beta = cells[:, W.BETA]
    m1, m2 = beta / (1 + beta), 1 / (1 + beta)
    spin_ref = torch.as_tensor(np.stack([cells[:, W.CHI1] * m1 ** 2, cells[:, W.CHI2] * m2 ** 2], axis=1),
                               device="cuda").contiguous()
    stream = torch.cuda.current_stream()
    for call in range(2):
        got = pn.scan_summary_noalloc(cells.shape[0], out["status"], out["fli"], out["integrals"],
                                      spin_ref, diag["newton_iters"], diag["n_skip"], diag["last_kind"],
                                      out["t_stop"], 1.0, 6.0, stream).as_dict()
        for k in ("n", "n_chaotic", "status_count", "newton_iters", "n_skip", "orbit_steps",
                  "n_final_fallback"):
            assert got[k] == ref[k], (call, k, got[k], ref[k])
        for k in ("max_dE", "max_dJ", "max_dJ_all", "fli_max"):
            assert got[k] == ref[k], (call, k, got[k], ref[k])
        assert got["fli_mean"] == pytest.approx(ref["fli_mean"], rel=1e-12)
        assert abs(got["max_dS"] - ref["max_dS"]) <= 1e-15
    assert ref["status_count"][pn.ORBIT_MERGED] > 0 and ref["status_count"][pn.ORBIT_DONE] > 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1802_00147_gb300 as pn
    with pytest.raises(pn.ScanError):
        pn.scan_summary_noalloc(2097153, None, None, None)
