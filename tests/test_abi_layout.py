"""The ctypes mirrors of the C ABI's structs (scan_params, scan_summary_t)
have the same field order, offsets and size as the C compiler gives them
from include/pnscan.h (gcc, no GPU needed)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def c_layout(struct, fields):
    """Offsets of `fields` and sizeof(struct) compiled by gcc from the header."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = ['#include <stddef.h>', '#include <stdio.h>', '#include "pnscan.h"', "int main(void) {"]
    for f in fields:
        src.append('  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f))
    src.append('  printf("%%zu\\n", sizeof(%s));' % struct)
    src.append("  return 0; }")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        with open(c, "w") as fh:
            fh.write("\n".join(src))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    vals = [int(v) for v in out]
    return vals[:-1], vals[-1]


@pytest.mark.parametrize("cname, pyname", [("scan_params", "ScanParams"), ("scan_summary_t", "ScanSummary")])
def test_ctypes_struct_matches_c_layout(cname, pyname):
    import paper_1802_00147_gb300 as pn
    cls = getattr(pn, pyname)
    names = [f[0] for f in cls._fields_]
    offsets, size = c_layout(cname, names)
    assert [getattr(cls, n).offset for n in names] == offsets
    assert ctypes.sizeof(cls) == size
