"""Build step of the scan library: compiles csrc/*.cu for sm_103a with nvcc into
``libpnscan.so`` beside this file (in-tree, git-ignored).  Translation units
are compiled in parallel; the CUDA runtime is linked statically so the
library loads on a machine without a GPU driver.  ptxas's resource report
(registers per thread of every kernel) is kept in ``_build/registers.json``."""
import json
import os
import re
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libpnscan.so")
BUILD_DIR = os.path.join(HERE, "_build")
REGISTERS = os.path.join(BUILD_DIR, "registers.json")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    files = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return files


def _compile(src, extra):
    obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
    cmd = [NVCC] + ARCH + CFLAGS + ["-Xptxas", "-v"] + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def parse_registers(log):
    """{kernel symbol: registers per thread} from ptxas's -v report."""
    regs, entry = {}, None
    for line in log.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            entry = m.group(1)
            continue
        m = re.search(r"Used (\d+) registers", line)
        if m and entry:
            regs[entry] = int(m.group(1))
            entry = None
    return regs


def kernel_registers():
    """The registers-per-thread report of the last build ({} if absent)."""
    try:
        with open(REGISTERS) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def build(force: bool = False, verbose: bool = False, extra=None) -> str:
    """Compile the library if missing or stale; return the path of libpnscan.so."""
    newest = max(os.path.getmtime(f) for f in _deps())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    extra = list(extra or [])
    with ThreadPoolExecutor(max_workers=len(sources())) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), sources()))
    if verbose:
        for _, log in results:
            print(log)
    regs = {}
    for _, log in results:
        regs.update(parse_registers(log))
    tmpj = REGISTERS + ".tmp%d" % os.getpid()
    with open(tmpj, "w") as f:
        json.dump(regs, f, indent=0, sort_keys=True)
    os.replace(tmpj, REGISTERS)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
