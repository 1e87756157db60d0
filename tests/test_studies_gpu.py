"""Quadrupole-monopole drift study on a small seeded subset: with the
manifold correction the energy, |J| (dual-scaled final steps) and spin
lengths stay at rounding level; without it RK4 drifts by orders of
magnitude more (Table 2's 'linear growth')."""
import pytest

pytestmark = pytest.mark.gpu


def test_qm_drift_with_and_without_correction():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00147_gb300 import build
    build.build()
    from paper_1802_00147_gb300 import studies
    r = studies.qm_drift_study(n=64, subset=512, t_end=4000.0, h=0.5)
    c, u = r["corrected"], r["uncorrected"]
    assert c["done"] > 100 and u["done"] > 100
    assert c["dE"]["max"] <= 1e-12 and c["dS"]["max"] <= 1e-13
    assert c["dJ"]["median"] <= 1e-14
    assert u["dE"]["median"] > 1e3 * c["dE"]["median"]
    assert u["dJ"]["median"] > 1e2 * c["dJ"]["median"]
