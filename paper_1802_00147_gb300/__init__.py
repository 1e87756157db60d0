"""GB300 (sm_103a) batched scan of manifold-corrected post-Newtonian spinning
compact binaries (arXiv:1802.00147).

This module is a thin ctypes binding over ``libpnscan.so`` (C ABI in
``include/pnscan.h``): it marshals arguments and nothing else.  Every step of
the scan runs in the library's CUDA kernels; there is no CPU fallback, and
loading fails loudly if the library has not been built
(``python -m paper_1802_00147_gb300.build`` or ``__graft_entry__.build()``).

Functions keep the C names (``scan_create``, ``scan_setup``, ``scan_run``,
``scan_read``, ``scan_summary``, ...).  ``Scan`` bundles them for numpy host
arrays or torch CUDA tensors.
"""
import ctypes as _ct
import os as _os

import numpy as _np

__all__ = [
    "ScanParams", "ScanSummary", "ScanError", "lib", "library_path",
    "scan_params_default", "scan_create", "scan_setup", "scan_run", "scan_read",
    "scan_read_diag", "scan_summary", "scan_autotune", "scan_last_run_timing",
    "scan_fp64_peak", "scan_summary_noalloc", "scan_destroy", "scan_strerror", "scan_version", "Scan",
    "OK", "ORBIT_RUNNING", "ORBIT_DONE", "ORBIT_MERGED", "ORBIT_ESCAPED",
    "ORBIT_FLI_SATURATED", "ORBIT_NONFINITE", "SCHED_AUTO", "SCHED_STATIC", "SCHED_QUEUE", "SCHED_COMPACT", "SCHED_PAIR",
    "MLP_PARAMS", "MLP_BATCH", "Surrogate", "adaptive_features", "adaptive_select", "adaptive_merge",
]

_HERE = _os.path.dirname(_os.path.abspath(__file__))
library_path = _os.path.join(_HERE, "libpnscan.so")

OK = 0
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_STATE, ERR_KERNEL, ERR_NODEVICE = -1, -2, -3, -4, -5, -6, -7
ORBIT_RUNNING, ORBIT_DONE, ORBIT_MERGED, ORBIT_ESCAPED, ORBIT_FLI_SATURATED, ORBIT_NONFINITE = range(6)
SCHED_AUTO, SCHED_STATIC, SCHED_QUEUE, SCHED_COMPACT, SCHED_PAIR = 0, 1, 2, 3, 4

_ALLOC_FN = _ct.CFUNCTYPE(_ct.c_void_p, _ct.c_size_t, _ct.c_void_p)
_FREE_FN = _ct.CFUNCTYPE(None, _ct.c_void_p, _ct.c_void_p)


class ScanParams(_ct.Structure):
    _fields_ = [
        ("n", _ct.c_int64),
        ("beta_m", _ct.c_void_p), ("kappa1", _ct.c_void_p), ("kappa2", _ct.c_void_p),
        ("pn_order", _ct.c_int), ("use_so", _ct.c_int), ("use_ss", _ct.c_int), ("use_qm", _ct.c_int),
        ("correct", _ct.c_int), ("rk_order", _ct.c_int),
        ("newton_tol", _ct.c_double), ("newton_max", _ct.c_int), ("newton_det_min", _ct.c_double),
        ("newton_apply_small", _ct.c_int),
        ("fli_d0", _ct.c_double), ("fli_renorm_steps", _ct.c_int), ("fli_thresh", _ct.c_double),
        ("fli_cap", _ct.c_double), ("r_merge", _ct.c_double), ("r_escape", _ct.c_double),
        ("device_ptrs", _ct.c_int), ("cuda_stream", _ct.c_void_p),
        ("schedule", _ct.c_int), ("block_size", _ct.c_int), ("chunk_steps", _ct.c_int),
        ("epoch_steps", _ct.c_int),
        ("blocks_per_sm", _ct.c_int), ("register_variant", _ct.c_int), ("use_graph", _ct.c_int),
        ("sync_timeout_s", _ct.c_double),
        ("queue_wait_limit_ms", _ct.c_int),
        ("alloc_fn", _ALLOC_FN), ("free_fn", _FREE_FN), ("alloc_ctx", _ct.c_void_p),
        ("radiation_reaction", _ct.c_int), ("rr_gauge_a", _ct.c_double), ("rr_gauge_b", _ct.c_double),
        ("newton_split_min", _ct.c_double), ("newton_cond_switch", _ct.c_double),
    ]


class ScanSummary(_ct.Structure):
    _fields_ = [
        ("n", _ct.c_int64), ("n_chaotic", _ct.c_int64), ("status_count", _ct.c_int64 * 6),
        ("newton_iters", _ct.c_int64), ("n_skip", _ct.c_int64), ("orbit_steps", _ct.c_int64),
        ("max_dE", _ct.c_double), ("max_dJ", _ct.c_double), ("max_dJ_all", _ct.c_double),
        ("n_final_fallback", _ct.c_int64), ("max_dS", _ct.c_double),
        ("fli_max", _ct.c_double), ("fli_mean", _ct.c_double),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "status_count"}
        d["status_count"] = list(self.status_count)
        return d


class ScanError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, scan_strerror(code), code))


_lib = None


def lib():
    """Load libpnscan.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not _os.path.exists(library_path):
            raise ImportError("libpnscan.so is missing: build it with __graft_entry__.build() "
                              "or python -m paper_1802_00147_gb300.build (no CPU fallback exists)")
        L = _ct.CDLL(library_path)
        P, vp, i, d = _ct.POINTER, _ct.c_void_p, _ct.c_int, _ct.c_double
        L.scan_params_default.argtypes = [P(ScanParams)]
        L.scan_create.argtypes = [P(ScanParams), P(vp)]
        L.scan_setup.argtypes = [vp, vp]
        L.scan_run.argtypes = [vp, vp, d, d]
        L.scan_read.argtypes = [vp, vp, vp, vp, vp, vp]
        L.scan_read_diag.argtypes = [vp, vp, vp, vp, vp]
        L.scan_summary.argtypes = [vp, P(ScanSummary)]
        L.scan_autotune.argtypes = [vp, i, P(i), P(i), P(i), P(i), P(i)]
        L.scan_last_run_timing.argtypes = [vp, P(d), P(i)]
        L.scan_fp64_peak.argtypes = [vp, i, P(d)]
        L.scan_waveform.argtypes = [vp, d, P(d), P(d), vp, vp]
        L.scan_checkpoint_size.argtypes = [vp]
        L.scan_checkpoint_size.restype = _ct.c_size_t
        L.scan_checkpoint.argtypes = [vp, vp, _ct.c_size_t]
        L.scan_restore.argtypes = [vp, vp, _ct.c_size_t]
        L.scan_summary_noalloc.argtypes = [_ct.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, d, d, vp,
                                           P(ScanSummary)]
        f, u64, i64 = _ct.c_float, _ct.c_uint64, _ct.c_int64
        L.mlp_create.argtypes = [i, u64, P(f), P(f), vp, P(vp)]
        L.mlp_get_params.argtypes = [vp, vp]
        L.mlp_set_params.argtypes = [vp, vp]
        L.mlp_get_moments.argtypes = [vp, vp, vp]
        L.mlp_train.argtypes = [vp, vp, vp, i64, i, f, u64, vp]
        L.mlp_gradient.argtypes = [vp, vp, vp, vp, vp]
        L.mlp_predict.argtypes = [vp, vp, i64, vp, vp]
        L.mlp_destroy.argtypes = [vp]
        L.mlp_destroy.restype = None
        L.adaptive_features.argtypes = [vp, i64, vp, vp]
        L.adaptive_features.restype = i
        L.adaptive_features_fields.argtypes = [vp, i64, P(_ct.c_int32), vp, vp]
        L.adaptive_features_fields.restype = i
        L.adaptive_interp_grid.argtypes = [vp, vp, i64, i64, _ct.c_int32, vp, vp, vp]
        L.adaptive_interp_grid.restype = i
        L.adaptive_select_workspace.argtypes = [i64]
        L.adaptive_select_workspace.restype = _ct.c_size_t
        L.adaptive_select.argtypes = [vp, vp, i64, f, f, f, vp, vp, vp, P(i64), vp, vp]
        L.adaptive_merge.argtypes = [vp, i64, f, vp, i64, vp, vp, vp, vp]
        for name in ("mlp_create", "mlp_get_params", "mlp_get_moments", "mlp_set_params", "mlp_train", "mlp_gradient",
                     "mlp_predict", "adaptive_select", "adaptive_merge"):
            getattr(L, name).restype = i
        L.scan_destroy.argtypes = [vp]
        L.scan_destroy.restype = None
        L.scan_strerror.argtypes = [i]
        L.scan_strerror.restype = _ct.c_char_p
        L.scan_version.restype = _ct.c_char_p
        for name in ("scan_params_default", "scan_create", "scan_setup", "scan_run", "scan_read",
                     "scan_read_diag", "scan_summary", "scan_autotune", "scan_last_run_timing",
                     "scan_fp64_peak", "scan_summary_noalloc", "scan_waveform", "scan_checkpoint",
                     "scan_restore"):
            getattr(L, name).restype = i
        _lib = L
    return _lib


def _check(code, where):
    if code != OK:
        raise ScanError(code, where)


def _ptr(a):
    """Address of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, _np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


# ------------------------------------------------------------ raw C names
def scan_params_default():
    p = ScanParams()
    _check(lib().scan_params_default(_ct.byref(p)), "scan_params_default")
    return p


def scan_create(params):
    h = _ct.c_void_p()
    _check(lib().scan_create(_ct.byref(params), _ct.byref(h)), "scan_create")
    return h


def scan_setup(h, cells):
    _check(lib().scan_setup(h, _ptr(cells)), "scan_setup")


def scan_run(h, initial_states, t_end, h_step):
    _check(lib().scan_run(h, _ptr(initial_states), float(t_end), float(h_step)), "scan_run")


def scan_read(h, states=None, integrals=None, fli=None, status=None, t_stop=None):
    _check(lib().scan_read(h, _ptr(states), _ptr(integrals), _ptr(fli), _ptr(status), _ptr(t_stop)),
           "scan_read")


def scan_read_diag(h, shadow=None, newton_iters=None, n_skip=None, last_kind=None):
    _check(lib().scan_read_diag(h, _ptr(shadow), _ptr(newton_iters), _ptr(n_skip), _ptr(last_kind)),
           "scan_read_diag")


def scan_summary(h):
    s = ScanSummary()
    _check(lib().scan_summary(h, _ct.byref(s)), "scan_summary")
    return s


def scan_autotune(h, steps):
    out = [_ct.c_int() for _ in range(5)]
    _check(lib().scan_autotune(h, int(steps), *[_ct.byref(o) for o in out]), "scan_autotune")
    return dict(schedule=out[0].value, block_size=out[1].value, chunk_steps=out[2].value,
                blocks_per_sm=out[3].value, register_variant=out[4].value)


def scan_waveform(h, R, P, Q, hplus, hcross):
    Pv = (_ct.c_double * 3)(*[float(v) for v in P])
    Qv = (_ct.c_double * 3)(*[float(v) for v in Q])
    _check(lib().scan_waveform(h, float(R), Pv, Qv, _ptr(hplus), _ptr(hcross)), "scan_waveform")


def scan_checkpoint(h):
    """The handle's complete orbit state as bytes (host memory)."""
    n = int(lib().scan_checkpoint_size(h))
    buf = _ct.create_string_buffer(n)
    _check(lib().scan_checkpoint(h, buf, n), "scan_checkpoint")
    return buf.raw


def scan_restore(h, data):
    buf = _ct.create_string_buffer(bytes(data), len(data))
    _check(lib().scan_restore(h, buf, len(data)), "scan_restore")


def scan_last_run_timing(h):
    ms, n = _ct.c_double(), _ct.c_int()
    _check(lib().scan_last_run_timing(h, _ct.byref(ms), _ct.byref(n)), "scan_last_run_timing")
    return ms.value, n.value


def scan_fp64_peak(h, iters=200_000):
    t = _ct.c_double()
    _check(lib().scan_fp64_peak(h, int(iters), _ct.byref(t)), "scan_fp64_peak")
    return t.value


def scan_summary_noalloc(n, status, fli, integrals, spin_ref=None, newton_iters=None, n_skip=None,
                         last_kind=None, t_stop=None, h_step=1.0, fli_thresh=6.0, stream=None):
    """Scan reduction over caller-owned device arrays without any run-time
    allocation (see include/pnscan.h).  ``stream``: a torch stream or None."""
    s = ScanSummary()
    st = None if stream is None else stream.cuda_stream
    _check(lib().scan_summary_noalloc(int(n), _ptr(status), _ptr(fli), _ptr(integrals), _ptr(spin_ref),
                                      _ptr(newton_iters), _ptr(n_skip), _ptr(last_kind), _ptr(t_stop),
                                      float(h_step), float(fli_thresh), st, _ct.byref(s)),
           "scan_summary_noalloc")
    return s


def scan_destroy(h):
    if h:
        lib().scan_destroy(h)


def scan_strerror(code):
    return lib().scan_strerror(int(code)).decode()


def scan_version():
    return lib().scan_version().decode()


# --------------------------------------------------------------- wrapper
class Scan:
    """One scan handle over n orbits.

    ``device=False``: host numpy arrays in and out (copies inside the calls).
    ``device=True``: torch CUDA tensors in and out; the handle's device
    buffers come from PyTorch's caching allocator and work runs on the current
    torch stream.
    """

    def __init__(self, beta, kappa1=None, kappa2=None, device=False, stream=None, n=None, **opts):
        """beta None: mass ratios come from the cells given to setup() (n required)."""
        p = scan_params_default()
        self.device = bool(device)
        self._keep = {}
        if self.device:
            import torch
            self._torch = torch
            dev = torch.device("cuda", torch.cuda.current_device())
            beta = None if beta is None else torch.as_tensor(beta, dtype=torch.float64, device=dev).contiguous()
            kappa1 = None if kappa1 is None else torch.as_tensor(kappa1, dtype=torch.float64, device=dev).contiguous()
            kappa2 = None if kappa2 is None else torch.as_tensor(kappa2, dtype=torch.float64, device=dev).contiguous()
            st = stream if stream is not None else torch.cuda.current_stream()
            p.cuda_stream = st.cuda_stream
            p.device_ptrs = 1
            blocks = self._keep

            def _alloc(nbytes, ctx):
                t = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
                blocks[t.data_ptr()] = t
                return t.data_ptr()

            def _free(ptr, ctx):
                blocks.pop(ptr, None)

            self._cb = (_ALLOC_FN(_alloc), _FREE_FN(_free))
            p.alloc_fn, p.free_fn = self._cb
        else:
            beta = None if beta is None else _np.ascontiguousarray(beta, dtype=_np.float64)
            kappa1 = None if kappa1 is None else _np.ascontiguousarray(kappa1, dtype=_np.float64)
            kappa2 = None if kappa2 is None else _np.ascontiguousarray(kappa2, dtype=_np.float64)
        self.n = int(beta.shape[0]) if beta is not None else int(n)
        p.n = self.n
        p.beta_m, p.kappa1, p.kappa2 = _ptr(beta), _ptr(kappa1), _ptr(kappa2)
        for k, v in opts.items():
            if not hasattr(p, k):
                raise TypeError("unknown scan parameter %r" % k)
            setattr(p, k, v)
        self.params = p
        self._args = (beta, kappa1, kappa2)
        self.h = scan_create(p)

    def close(self):
        if getattr(self, "h", None):
            scan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _arr(self, a, cols):
        if self.device:
            t = self._torch.as_tensor(a, dtype=self._torch.float64, device="cuda").contiguous()
            assert t.numel() == self.n * cols
            return t
        a = _np.ascontiguousarray(a, dtype=_np.float64)
        assert a.size == self.n * cols
        return a

    def setup(self, cells):
        """cells: n x 9 (x0, pfac, theta1, phi1, theta2, phi2, beta, chi1, chi2)."""
        c = self._arr(cells[:, :9], 9)
        scan_setup(self.h, c)
        self._cells = c

    def run(self, t_end, h_step, initial_states=None):
        s = None if initial_states is None else self._arr(initial_states, 12)
        scan_run(self.h, s, t_end, h_step)
        self._init = s

    def _out(self, shape, dtype):
        if self.device:
            tdt = {_np.float64: self._torch.float64, _np.int32: self._torch.int32}[dtype]
            return self._torch.empty(shape, dtype=tdt, device="cuda")
        return _np.empty(shape, dtype=dtype)

    def read(self):
        n = self.n
        out = dict(states=self._out((n, 12), _np.float64), integrals=self._out((n, 6), _np.float64),
                   fli=self._out((n,), _np.float64), status=self._out((n,), _np.int32),
                   t_stop=self._out((n,), _np.float64))
        scan_read(self.h, out["states"], out["integrals"], out["fli"], out["status"], out["t_stop"])
        return out

    def read_diag(self):
        n = self.n
        out = dict(shadow=self._out((n, 12), _np.float64), newton_iters=self._out((n,), _np.int32),
                   n_skip=self._out((n,), _np.int32), last_kind=self._out((n,), _np.int32))
        scan_read_diag(self.h, out["shadow"], out["newton_iters"], out["n_skip"], out["last_kind"])
        return out

    def summary(self):
        return scan_summary(self.h).as_dict()

    def checkpoint(self):
        """Bytes of the complete orbit state (scan_checkpoint)."""
        return scan_checkpoint(self.h)

    def restore(self, data):
        """Continue from a checkpoint of a handle with the same n and configuration."""
        scan_restore(self.h, data)

    def waveform(self, R=1.0, P=(1.0, 0.0, 0.0), Q=(0.0, 1.0, 0.0)):
        """(h_plus, h_cross) of every orbit at its current state (scan_waveform)."""
        hp, hc = self._out((self.n,), _np.float64), self._out((self.n,), _np.float64)
        scan_waveform(self.h, R, P, Q, hp, hc)
        return hp, hc

    def autotune(self, steps):
        return scan_autotune(self.h, steps)

    def last_run_timing(self):
        return scan_last_run_timing(self.h)

    def fp64_peak(self, iters=200_000):
        return scan_fp64_peak(self.h, iters)


# ----------------------------------------------------- surrogate (mlp_*)
MLP_PARAMS = 4545
MLP_BATCH = 128


class Surrogate:
    """Ensemble of small networks mapping (x0, theta, beta, chi) to the FLI
    (mlp_* of the C ABI).  Arrays are torch CUDA tensors (float32)."""

    def __init__(self, members=5, seed=1, center=(30.0, 1.5707963267948966, 0.5, 0.5),
                 scale=(20.0, 1.5707963267948966, 0.5, 0.5), stream=None):
        import torch
        self._torch = torch
        self.members = int(members)
        c = (_ct.c_float * 4)(*center)
        sc = (_ct.c_float * 4)(*scale)
        st = (stream or torch.cuda.current_stream()).cuda_stream
        self.h = _ct.c_void_p()
        _check(lib().mlp_create(self.members, int(seed), c, sc, st, _ct.byref(self.h)), "mlp_create")

    def close(self):
        if getattr(self, "h", None):
            lib().mlp_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f32(self, a, shape=None):
        t = self._torch.as_tensor(a, dtype=self._torch.float32, device="cuda").contiguous()
        if shape is not None:
            assert tuple(t.shape) == tuple(shape), (t.shape, shape)
        return t

    def get_params(self):
        out = self._torch.empty((self.members, MLP_PARAMS), dtype=self._torch.float32, device="cuda")
        _check(lib().mlp_get_params(self.h, _ptr(out)), "mlp_get_params")
        return out

    def get_moments(self):
        """The Adam moments (m, v), each (members, MLP_PARAMS) float32."""
        m = self._torch.empty((self.members, MLP_PARAMS), dtype=self._torch.float32, device="cuda")
        v = self._torch.empty_like(m)
        _check(lib().mlp_get_moments(self.h, _ptr(m), _ptr(v)), "mlp_get_moments")
        return m, v

    def set_params(self, params):
        p = self._f32(params, (self.members, MLP_PARAMS))
        _check(lib().mlp_set_params(self.h, _ptr(p)), "mlp_set_params")

    def train(self, X, y, steps, lr=1e-3, seed=7, record_loss=True):
        X = self._f32(X)
        y = self._f32(y)
        n = int(X.shape[0])
        hist = self._torch.empty((self.members, steps), dtype=self._torch.float32,
                                 device="cuda") if record_loss else None
        _check(lib().mlp_train(self.h, _ptr(X), _ptr(y), n, int(steps), float(lr), int(seed), _ptr(hist)),
               "mlp_train")
        return hist

    def gradient(self, X, y):
        X = self._f32(X, (MLP_BATCH, 4))
        y = self._f32(y, (MLP_BATCH,))
        g = self._torch.empty((self.members, MLP_PARAMS), dtype=self._torch.float32, device="cuda")
        loss = self._torch.empty(self.members, dtype=self._torch.float32, device="cuda")
        _check(lib().mlp_gradient(self.h, _ptr(X), _ptr(y), _ptr(g), _ptr(loss)), "mlp_gradient")
        return g, loss

    def predict(self, X):
        X = self._f32(X)
        n = int(X.shape[0])
        mean = self._torch.empty(n, dtype=self._torch.float32, device="cuda")
        spread = self._torch.empty(n, dtype=self._torch.float32, device="cuda")
        _check(lib().mlp_predict(self.h, _ptr(X), n, _ptr(mean), _ptr(spread)), "mlp_predict")
        return mean, spread


def adaptive_features(cells, stream=None):
    """Surrogate inputs (x0, theta1, beta, chi1) as float32 of cells (n x 9 float64, CUDA)."""
    import torch
    cells = cells.contiguous()
    n = int(cells.shape[0])
    X = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib().adaptive_features(_ptr(cells), n, _ptr(X), st), "adaptive_features")
    return X


def adaptive_features_fields(cells, fields, stream=None):
    """Surrogate inputs from four chosen cell fields (indices 0..8) of cells
    (n x 9 float64, CUDA), as float32 (n x 4)."""
    import torch
    cells = cells.contiguous()
    n = int(cells.shape[0])
    X = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    f = (_ct.c_int32 * 4)(*[int(k) for k in fields])
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib().adaptive_features_fields(_ptr(cells), n, f, _ptr(X), st), "adaptive_features_fields")
    return X


def adaptive_interp_grid(fli_nodes, status_nodes, n1, n2, stride, stream=None):
    """Mean and spread (float32, n1*n2, CUDA) of a row-major n1 x n2 grid
    interpolated from its integrated coarse grid of every stride-th cell."""
    import torch
    fli_nodes = fli_nodes.contiguous()
    status_nodes = status_nodes.contiguous()
    mean = torch.empty(n1 * n2, dtype=torch.float32, device="cuda")
    spread = torch.empty(n1 * n2, dtype=torch.float32, device="cuda")
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib().adaptive_interp_grid(_ptr(fli_nodes), _ptr(status_nodes), int(n1), int(n2), int(stride),
                                      _ptr(mean), _ptr(spread), st), "adaptive_interp_grid")
    return mean, spread


def adaptive_select(mean, spread, thr=6.0, band=1.0, spread_max=0.5, cells=None, stream=None):
    """Indices (ascending, int32) of the cells to integrate, and their gathered
    scan parameters (n x 9 float64) when cells is given.  Torch CUDA tensors."""
    import torch
    n = int(mean.shape[0])
    ws = torch.empty(max(1, int(lib().adaptive_select_workspace(n))), dtype=torch.uint8, device="cuda")
    idx = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    cells_out = None
    if cells is not None:
        cells = cells.contiguous()
        cells_out = torch.empty((max(n, 1), 9), dtype=torch.float64, device="cuda")
    count = _ct.c_int64()
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib().adaptive_select(_ptr(mean), _ptr(spread), n, float(thr), float(band), float(spread_max),
                                 _ptr(cells), _ptr(idx), _ptr(cells_out), _ct.byref(count), _ptr(ws), st),
           "adaptive_select")
    k = count.value
    return idx[:k], (None if cells_out is None else cells_out[:k])


def adaptive_merge(mean, thr, idx, fli_sel, status_sel, stream=None):
    """Class map (int8, 1 chaotic) of all cells: integrator results on idx, surrogate elsewhere."""
    import torch
    n = int(mean.shape[0])
    cls = torch.empty(n, dtype=torch.int8, device="cuda")
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib().adaptive_merge(_ptr(mean), n, float(thr), _ptr(idx), int(idx.shape[0]), _ptr(fli_sel),
                                _ptr(status_sel), _ptr(cls), st), "adaptive_merge")
    return cls
