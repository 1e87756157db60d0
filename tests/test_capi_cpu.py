"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every function include/*.h declares, and rejects bad calls without
touching a device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def pn():
    from paper_1802_00147_gb300 import build
    build.build()
    import paper_1802_00147_gb300 as pn
    pn.lib()
    return pn


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("scan_create", "scan_run", "scan_read", "scan_setup", "scan_summary",
                     "scan_destroy", "scan_strerror", "scan_autotune"):
        assert required in names, names


def test_every_declaration_cites_its_passage_and_errors():
    """Each entry point of include/*.h sits under a comment that cites the
    paper's passage (or says it is not in the paper) and states its errors."""
    bad = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        pat = r"(/\*(?:(?!\*/).)*\*/)\s*\n((?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\([^;]*\);)"
        for m in re.finditer(pat, text, flags=re.S):
            com, name = m.group(1), m.group(3)
            if not re.search(r"Sec\.|Eqs?\.|Table|Fig\.|not in the paper|Not in the paper", com):
                bad.append((name, "no citation"))
            if not re.search(r"Errors?|ERR_|Returns|returns|no error", com):
                bad.append((name, "no error behaviour"))
    assert not bad, bad


def test_library_exports_every_declared_symbol(pn):
    L = ctypes.CDLL(pn.library_path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_strerror_and_version(pn):
    assert pn.scan_strerror(0) == "ok"
    assert "argument" in pn.scan_strerror(-1)
    assert "sm_103a" in pn.scan_version()


def test_params_default_values(pn):
    p = pn.scan_params_default()
    assert (p.pn_order, p.use_so, p.use_ss, p.use_qm, p.correct) == (2, 1, 1, 0, 1)
    assert p.newton_tol == 1e-10 and p.newton_max == 50 and p.newton_det_min == 1e-5
    assert p.fli_d0 == 1e-9 and p.fli_renorm_steps == 100 and p.fli_thresh == 6.0
    assert p.r_merge == 6.0 and p.r_escape == 1e3
    assert (p.radiation_reaction, p.rr_gauge_a, p.rr_gauge_b) == (0, 4.0, 5.0)
    assert ctypes.sizeof(pn.ScanParams) == ctypes.sizeof(p)


def test_bad_arguments_are_rejected_before_any_device_work(pn):
    L = pn.lib()
    h = ctypes.c_void_p()
    assert L.scan_create(None, ctypes.byref(h)) == pn.ERR_ARG
    p = pn.scan_params_default()
    p.n = 4
    p.newton_tol = 0.0           # Newton tolerance must be positive
    assert L.scan_create(ctypes.byref(p), ctypes.byref(h)) == pn.ERR_ARG
    p = pn.scan_params_default()
    p.block_size = 96 + 256      # block size out of range
    assert L.scan_create(ctypes.byref(p), ctypes.byref(h)) == pn.ERR_ARG
    p = pn.scan_params_default()
    p.n = -1
    assert L.scan_create(ctypes.byref(p), ctypes.byref(h)) == pn.ERR_ARG
    p.n = 0
    p.pn_order = 3
    assert L.scan_create(ctypes.byref(p), ctypes.byref(h)) == pn.ERR_ARG
    for field, bad in (("schedule", 5), ("schedule", -1), ("correct", 4), ("rk_order", 3),
                       ("register_variant", 1), ("register_variant", 5), ("queue_wait_limit_ms", -1)):
        p = pn.scan_params_default()
        p.n = 4
        setattr(p, field, bad)
        assert L.scan_create(ctypes.byref(p), ctypes.byref(h)) == pn.ERR_ARG, (field, bad)
    # radiation reaction: a flag, finite gauge constants
    for fields in (dict(radiation_reaction=2),
                   dict(radiation_reaction=1, rr_gauge_a=float("nan")),
                   dict(radiation_reaction=1, rr_gauge_b=float("inf"))):
        p = pn.scan_params_default()
        p.n = 4
        for k, v in fields.items():
            setattr(p, k, v)
        assert L.scan_create(ctypes.byref(p), ctypes.byref(h)) == pn.ERR_ARG, fields
    assert h.value is None
    assert L.scan_run(None, None, 1.0, 1.0) == pn.ERR_ARG
    assert L.scan_read(None, None, None, None, None, None) == pn.ERR_ARG
    P3 = (ctypes.c_double * 3)(1.0, 0.0, 0.0)
    assert L.scan_waveform(None, 1.0, P3, P3, None, None) == pn.ERR_ARG
    assert L.scan_checkpoint_size(None) == 0
    buf = ctypes.create_string_buffer(64)
    assert L.scan_checkpoint(None, buf, 64) == pn.ERR_ARG
    assert L.scan_restore(None, buf, 64) == pn.ERR_ARG
    L.scan_destroy(None)


def test_no_device_is_reported(pn):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = pn.scan_params_default()
    beta = np.ones(3)
    p.n = 3
    p.beta_m = beta.ctypes.data
    h = ctypes.c_void_p()
    assert pn.lib().scan_create(ctypes.byref(p), ctypes.byref(h)) == pn.ERR_NODEVICE
