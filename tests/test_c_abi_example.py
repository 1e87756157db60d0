"""The C ABI used from plain C: tests/c_abi_example.c compiles against
include/pnscan.h alone, links libpnscan.so, and runs the whole call sequence
(create, set-up, two runs, read, summary, destroy).  Without a GPU it must
stop at the first call that needs one with PNSCAN_ERR_NODEVICE; on a GPU it
must finish with the energy of every finished orbit restored."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1802_00147_gb300")


def _compile(tmp_path):
    from paper_1802_00147_gb300 import build
    build.build()
    exe = str(tmp_path / "c_abi_example")
    cmd = ["gcc", "-O2", "-Wall", "-Wextra", "-Werror", "-std=c99", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_example.c"), "-o", exe, "-L", PKG, "-lpnscan",
           "-Wl,-rpath," + PKG, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_example_builds_and_reports_no_device(tmp_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present (the gpu test runs the example)")
    r = subprocess.run([_compile(tmp_path)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 77, (r.returncode, r.stdout, r.stderr)
    assert "no CUDA device" in r.stderr


@pytest.mark.gpu
def test_c_example_runs_on_the_gpu(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([_compile(tmp_path)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "summary:" in r.stdout and r.stdout.count("orbit ") == 8
