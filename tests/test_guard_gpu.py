"""Out-of-bounds writes, caught without a sanitizer: every device buffer the
library allocates comes from a test allocator (the alloc_fn / free_fn hooks
of scan_params) that surrounds it with 4 KiB of canary bytes on each side.
After runs through every schedule (and, with the 2.5PN radiation reaction,
the static, compacting and paired ones) and every reading call, and at each
free, the canaries must be intact."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GUARD = 4096
CANARY = 0xA5


@pytest.fixture(scope="module")
def pn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00147_gb300 import build
    build.build()
    import paper_1802_00147_gb300 as pn
    pn.lib()
    return pn


class GuardedAllocator:
    def __init__(self, pn, torch):
        self.torch = torch
        self.live = {}
        self.bad = []
        self.count = 0

        def alloc(nbytes, ctx):
            t = torch.full((int(nbytes) + 2 * GUARD,), CANARY, dtype=torch.uint8, device="cuda")
            ptr = t.data_ptr() + GUARD
            assert ptr % 256 == 0
            self.live[ptr] = (t, int(nbytes))
            self.count += 1
            return ptr

        def free(ptr, ctx):
            if ptr in self.live:
                torch.cuda.synchronize()
                self.check_one(ptr)
                self.live.pop(ptr)

        self.cb = (pn._ALLOC_FN(alloc), pn._FREE_FN(free))

    def check_one(self, ptr):
        t, n = self.live[ptr]
        if not bool((t[:GUARD] == CANARY).all()) or not bool((t[GUARD + n:] == CANARY).all()):
            self.bad.append(n)

    def check_all(self):
        self.torch.cuda.synchronize()
        for ptr in list(self.live):
            self.check_one(ptr)


@pytest.mark.parametrize("schedule,rr", [(1, 0), (2, 0), (3, 0), (4, 0), (1, 1), (3, 1), (4, 1)])
def test_no_write_outside_the_library_buffers(pn, schedule, rr):
    import torch
    from paper_1802_00147_gb300 import workloads as W
    cells = W.uneven_batch(n=1000, seed=17)
    ga = GuardedAllocator(pn, torch)
    p = pn.scan_params_default()
    p.n = cells.shape[0]
    p.device_ptrs = 1
    p.cuda_stream = torch.cuda.current_stream().cuda_stream
    p.schedule = schedule
    p.chunk_steps = 40
    p.fli_cap = 12.0
    p.radiation_reaction = rr
    p.alloc_fn, p.free_fn = ga.cb
    h = pn.scan_create(p)
    try:
        cd = torch.as_tensor(np.ascontiguousarray(cells[:, :9]), device="cuda")
        pn.scan_setup(h, cd)
        pn.scan_run(h, None, 150.0, 1.0)
        pn.scan_run(h, None, 300.0, 1.0)                   # a second segment
        n = cells.shape[0]
        out = dict(states=torch.empty((n, 12), dtype=torch.float64, device="cuda"),
                   integrals=torch.empty((n, 6), dtype=torch.float64, device="cuda"),
                   fli=torch.empty(n, dtype=torch.float64, device="cuda"),
                   status=torch.empty(n, dtype=torch.int32, device="cuda"),
                   t_stop=torch.empty(n, dtype=torch.float64, device="cuda"))
        pn.scan_read(h, **out)
        pn.scan_read_diag(h, torch.empty((n, 12), dtype=torch.float64, device="cuda"),
                          torch.empty(n, dtype=torch.int32, device="cuda"),
                          torch.empty(n, dtype=torch.int32, device="cuda"),
                          torch.empty(n, dtype=torch.int32, device="cuda"))
        pn.scan_summary(h)
        hp = torch.empty(n, dtype=torch.float64, device="cuda")
        pn.scan_waveform(h, 1.0, (1, 0, 0), (0, 1, 0), hp, hp.clone())
        pn.scan_autotune(h, 50)
        pn.scan_run(h, None, 400.0, 1.0)
        ga.check_all()
        assert ga.count > 0
        assert not ga.bad, ga.bad
    finally:
        pn.scan_destroy(h)
    assert not ga.bad, ga.bad
    assert not ga.live
