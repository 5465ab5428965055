"""ctypes declarations of libdsanls and a small handle class (argument marshalling only)."""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_PKG, "libdsanls.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ENUMERIC, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
GAUSSIAN, SUBSAMPLE, IDENTITY, RADEMACHER, COUNT, SRHT = 0, 1, 2, 3, 4, 5
PGD, RCD = 0, 1
FP32, BF16, FP8 = 0, 1, 2
ORDER_PAPER, ORDER_REASSOCIATED = 0, 1
STREAM_SKETCH_U, STREAM_SKETCH_V, STREAM_INIT_U, STREAM_INIT_V = 0, 1, 2, 3

_NAMES = {OK: "OK", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ESTATE: "ESTATE",
          ENUMERIC: "ENUMERIC", ETIMEOUT: "ETIMEOUT"}

EXPORTED_SYMBOLS = [
    "dsanls_default_options", "dsanls_create", "dsanls_get_options", "dsanls_set_options",
    "dsanls_set_dense", "dsanls_set_csr", "dsanls_set_factors", "dsanls_step", "dsanls_half_step",
    "dsanls_rel_error", "dsanls_get_factors", "dsanls_get_gram", "dsanls_sync", "dsanls_last_error",
    "dsanls_destroy", "dsanls_philox_field", "dsanls_gaussian_field", "dsanls_rademacher_field", "dsanls_count_field", "dsanls_srht_field",
    "dsanls_uniform_field",
    "dsanls_subsample_indices", "dsanls_profile_half_step", "dsanls_kernel_launches", "dsanls_gram_noalloc",
    "dsanls_batch_create", "dsanls_batch_set_options", "dsanls_batch_set_dense", "dsanls_batch_set_factors",
    "dsanls_batch_step", "dsanls_batch_get_factors", "dsanls_batch_rel_error", "dsanls_batch_tuned_blocks", "dsanls_batch_tuned_tile", "dsanls_batch_set_tile", "dsanls_batch_profile",
    "dsanls_batch_last_error", "dsanls_batch_destroy",
    "dsanls_mlp_create", "dsanls_mlp_param_count", "dsanls_mlp_get_params", "dsanls_mlp_set_params",
    "dsanls_mlp_predict", "dsanls_mlp_train_step", "dsanls_mlp_destroy", "dsanls_set_mlp", "dsanls_mlp_kept",
    "dsanls_harvest", "dsanls_debug_fail_alloc_after", "dsanls_debug_tc_wait", "dsanls_debug_bounds_report",
]
NPHASES = 7
PHASES = ["sketch", "B", "product", "rhs", "gram", "step_size", "update"]


class DSANLSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_NAMES.get(code, "?"), code, msg))
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [
        ("solver", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("d_v", ctypes.c_int32),
        ("power_iters", ctypes.c_int32),
        ("alpha", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("t", ctypes.c_int64),
        ("bound_clamp", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("order", ctypes.c_int32),
        ("inner_iters", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("regen_sketch", ctypes.c_int32),
    ]


_lib = None


def lib():
    """Load libdsanls.so (ImportError if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(lib_path):
            raise ImportError("libdsanls.so is not built; run paper_2009_02845_gb300.build.build()")
        L = ctypes.CDLL(lib_path)
        vp, i32, i64, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
        dbl_p = ctypes.POINTER(ctypes.c_double)
        sig = {
            "dsanls_default_options": ([ctypes.POINTER(Options)], ctypes.c_int),
            "dsanls_create": ([i64, i64, i32, i32, i32, u64, ctypes.POINTER(vp)], ctypes.c_int),
            "dsanls_get_options": ([vp, ctypes.POINTER(Options)], ctypes.c_int),
            "dsanls_set_options": ([vp, ctypes.POINTER(Options)], ctypes.c_int),
            "dsanls_set_dense": ([vp, vp, i64, i32], ctypes.c_int),
            "dsanls_set_csr": ([vp, vp, vp, vp, i64, vp, vp, vp, i32], ctypes.c_int),
            "dsanls_set_factors": ([vp, vp, vp, i32], ctypes.c_int),
            "dsanls_step": ([vp, i32], ctypes.c_int),
            "dsanls_half_step": ([vp, i32], ctypes.c_int),
            "dsanls_rel_error": ([vp, dbl_p], ctypes.c_int),
            "dsanls_get_factors": ([vp, vp, vp, i32], ctypes.c_int),
            "dsanls_get_gram": ([vp, i32, vp, vp], ctypes.c_int),
            "dsanls_sync": ([vp], ctypes.c_int),
            "dsanls_last_error": ([vp], ctypes.c_char_p),
            "dsanls_destroy": ([vp], None),
            "dsanls_philox_field": ([u64, u32, u64, i64, i64, vp, vp], ctypes.c_int),
            "dsanls_gaussian_field": ([u64, u32, u64, i64, i64, ctypes.c_float, i32, vp, vp], ctypes.c_int),
            "dsanls_rademacher_field": ([u64, u32, u64, i64, i64, ctypes.c_float, i32, vp, vp], ctypes.c_int),
            "dsanls_count_field": ([u64, u32, u64, i64, i64, i32, vp, vp], ctypes.c_int),
            "dsanls_srht_field": ([u64, u32, u64, i64, i64, ctypes.c_float, i32, vp, vp], ctypes.c_int),
            "dsanls_uniform_field": ([u64, u32, u64, i64, i64, vp, vp], ctypes.c_int),
            "dsanls_subsample_indices": ([u64, u32, u64, i64, i32, vp, vp], ctypes.c_int),
            "dsanls_profile_half_step": ([vp, i32, i32, vp], ctypes.c_int),
            "dsanls_kernel_launches": ([ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
            "dsanls_gram_noalloc": ([vp, i32, i64, vp, vp], ctypes.c_int),
            "dsanls_batch_create": ([i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(vp)], ctypes.c_int),
            "dsanls_batch_set_options": ([vp, ctypes.POINTER(Options)], ctypes.c_int),
            "dsanls_batch_set_dense": ([vp, i32, vp, i64, i32], ctypes.c_int),
            "dsanls_batch_set_factors": ([vp, i32, vp, vp, i32], ctypes.c_int),
            "dsanls_batch_step": ([vp, i32], ctypes.c_int),
            "dsanls_batch_get_factors": ([vp, i32, vp, vp, i32], ctypes.c_int),
            "dsanls_batch_rel_error": ([vp, vp], ctypes.c_int),
            "dsanls_batch_tuned_blocks": ([vp, ctypes.POINTER(i32)], ctypes.c_int),
            "dsanls_batch_tuned_tile": ([vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                         ctypes.POINTER(i32)],
                                        ctypes.c_int),
            "dsanls_batch_set_tile": ([vp, i32, i32, i32, i32, i32], ctypes.c_int),
            "dsanls_batch_profile": ([vp, vp], ctypes.c_int),
            "dsanls_batch_last_error": ([vp], ctypes.c_char_p),
            "dsanls_batch_destroy": ([vp], None),
            "dsanls_mlp_create": ([i32, i32, i64, i32, u64, ctypes.POINTER(vp)], ctypes.c_int),
            "dsanls_mlp_param_count": ([vp, ctypes.POINTER(i64)], ctypes.c_int),
            "dsanls_mlp_get_params": ([vp, vp], ctypes.c_int),
            "dsanls_mlp_set_params": ([vp, vp], ctypes.c_int),
            "dsanls_mlp_predict": ([vp, vp, vp, vp, i32, vp, i64, vp, vp], ctypes.c_int),
            "dsanls_mlp_train_step": ([vp, vp, vp, vp, i32, vp, vp, i64, ctypes.c_float, dbl_p, vp, vp],
                                      ctypes.c_int),
            "dsanls_mlp_destroy": ([vp], None),
            "dsanls_set_mlp": ([vp, vp, i32], ctypes.c_int),
            "dsanls_mlp_kept": ([vp, ctypes.POINTER(i64)], ctypes.c_int),
            "dsanls_harvest": ([vp, i32, i32, vp, vp, vp, vp], ctypes.c_int),
            "dsanls_debug_fail_alloc_after": ([i64], ctypes.c_int),
            "dsanls_debug_tc_wait": ([u64, i32], ctypes.c_int),
            "dsanls_debug_bounds_report": ([i32, ctypes.POINTER(i64)], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(code, what="", handle=None):
    if code != OK:
        m = lib().dsanls_last_error(handle)
        detail = m.decode() if m else ""
        raise DSANLSError(code, "%s: %s" % (what, detail) if detail else what)


def _dev_ptr(t):
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# stateless primitives (outputs are torch CUDA tensors)
# ---------------------------------------------------------------------------

def kernel_launches():
    """Cumulative kernel launches issued by libdsanls in this process."""
    v = ctypes.c_uint64()
    _check(lib().dsanls_kernel_launches(ctypes.byref(v)), "kernel_launches")
    return v.value


def debug_fail_alloc_after(n):
    """Test switch: the next n device allocations of handles succeed, the one
    after fails as out of memory (n < 0: off)."""
    _check(lib().dsanls_debug_fail_alloc_after(int(n)), "debug_fail_alloc_after")


def debug_tc_wait(wait_ns=0, starve=False):
    """Test switch of the tensor-core kernels' bounded waits on the current
    device: a limit of wait_ns (0: the default 2 s) and, with starve, a GEMM
    producer that issues no copy so the waits run out."""
    _check(lib().dsanls_debug_tc_wait(int(wait_ns), int(bool(starve))), "debug_tc_wait")


def use_bounds_build():
    """Load libdsanls_bounds.so (the index-checking debug build) instead of
    libdsanls.so; call before anything else loads the library."""
    global lib_path
    if _lib is not None:
        raise RuntimeError("the library is already loaded")
    lib_path = os.path.join(_PKG, "libdsanls_bounds.so")


def debug_bounds_report(reset=False):
    """(checking build?, failed index checks, site of the first, its index)."""
    out = (ctypes.c_int64 * 3)()
    rc = lib().dsanls_debug_bounds_report(int(bool(reset)), out)
    if rc < 0:
        _check(rc, "debug_bounds_report")
    return bool(rc), int(out[0]), int(out[1]), int(out[2])


def gram_noalloc(B, G=None):
    """G = B B^T (FP64) through the allocation-free entry point.  B: k x d
    float32 CUDA tensor; G: optional k x k float64 CUDA tensor to fill (the
    binding allocates it with torch when not given)."""
    torch = _torch()
    k, d = B.shape
    if G is None:
        G = torch.empty((k, k), dtype=torch.float64, device=B.device)
    _check(lib().dsanls_gram_noalloc(_dev_ptr(B), int(k), int(d), _dev_ptr(G), _stream_ptr()), "gram_noalloc")
    return G


def philox_field(seed, stream_id, t, rows, cols, device="cuda"):
    torch = _torch()
    out = torch.empty((rows, cols), dtype=torch.int32, device=device)
    _check(lib().dsanls_philox_field(seed, stream_id, t, rows, cols, _dev_ptr(out), _stream_ptr()), "philox_field")
    return out


def gaussian_field(seed, stream_id, t, rows, cols, scale, transposed=False, device="cuda"):
    torch = _torch()
    shape = (cols, rows) if transposed else (rows, cols)
    out = torch.empty(shape, dtype=torch.float32, device=device)
    _check(lib().dsanls_gaussian_field(seed, stream_id, t, rows, cols, float(scale), int(bool(transposed)),
                                       _dev_ptr(out), _stream_ptr()), "gaussian_field")
    return out


def rademacher_field(seed, stream_id, t, rows, cols, scale, transposed=False, device="cuda"):
    torch = _torch()
    shape = (cols, rows) if transposed else (rows, cols)
    out = torch.empty(shape, dtype=torch.float32, device=device)
    _check(lib().dsanls_rademacher_field(seed, stream_id, t, rows, cols, float(scale), int(bool(transposed)),
                                         _dev_ptr(out), _stream_ptr()), "rademacher_field")
    return out


def count_field(seed, side, t, rows, cols, transposed=False, device="cuda"):
    torch = _torch()
    shape = (cols, rows) if transposed else (rows, cols)
    out = torch.empty(shape, dtype=torch.float32, device=device)
    _check(lib().dsanls_count_field(seed, side, t, rows, cols, int(bool(transposed)), _dev_ptr(out), _stream_ptr()),
           "count_field")
    return out


def srht_field(seed, side, t, rows, cols, scale, transposed=False, device="cuda"):
    torch = _torch()
    shape = (cols, rows) if transposed else (rows, cols)
    out = torch.empty(shape, dtype=torch.float32, device=device)
    _check(lib().dsanls_srht_field(seed, side, t, rows, cols, float(scale), int(bool(transposed)), _dev_ptr(out),
                                   _stream_ptr()), "srht_field")
    return out


def uniform_field(seed, stream_id, t, rows, cols, device="cuda"):
    torch = _torch()
    out = torch.empty((rows, cols), dtype=torch.float32, device=device)
    _check(lib().dsanls_uniform_field(seed, stream_id, t, rows, cols, _dev_ptr(out), _stream_ptr()), "uniform_field")
    return out


def subsample_indices(seed, side, t, n, d, device="cuda"):
    torch = _torch()
    out = torch.empty((d,), dtype=torch.int32, device=device)
    _check(lib().dsanls_subsample_indices(seed, side, t, n, d, _dev_ptr(out), _stream_ptr()), "subsample_indices")
    return out


# ---------------------------------------------------------------------------
# handle
# ---------------------------------------------------------------------------

def _host_or_device(a, dtype):
    """Returns (pointer, on_device, keepalive) for a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != dtype[1]:
                raise TypeError("expected %s" % dtype[1])
            a = a.contiguous()
            if a.is_cuda:
                return ctypes.c_void_p(a.data_ptr()), 1, a
            return ctypes.c_void_p(a.data_ptr()), 0, a
    except ImportError:
        pass
    a = np.ascontiguousarray(a, dtype=dtype[0])
    return a.ctypes.data_as(ctypes.c_void_p), 0, a


def _dt(kind):
    torch = _torch()
    return {"f32": (np.float32, torch.float32), "i32": (np.int32, torch.int32), "i64": (np.int64, torch.int64)}[kind]


class DSANLS:
    """One factorisation problem M (m x n) ~ U V^T of rank k on the current CUDA device."""

    def __init__(self, m, n, k, d, sketch=GAUSSIAN, seed=0, **options):
        h = ctypes.c_void_p()
        _check(lib().dsanls_create(m, n, k, d, sketch, seed, ctypes.byref(h)), "dsanls_create(%d,%d,%d,%d)" % (m, n, k, d))
        self._h = h
        self.m, self.n, self.k, self.d, self.sketch, self.seed = m, n, k, d, sketch, seed
        if options:
            self.set_options(**options)

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            lib().dsanls_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- options
    def options(self):
        o = Options()
        _check(lib().dsanls_get_options(self._h, ctypes.byref(o)), "get_options", self._h)
        return o

    def set_options(self, stream="current", **kw):
        """Apply options.  stream="current" hands the library torch's current
        stream; torch's legacy default stream (handle 0) maps to the handle's
        own stream, so synchronise with the handle (sync / factors) there."""
        o = self.options()
        for key, v in kw.items():
            if not hasattr(o, key) or key == "stream":
                raise TypeError("unknown option %r" % key)
            setattr(o, key, v)
        if stream == "current":
            o.stream = _stream_ptr().value
        elif stream is None:
            o.stream = None
        else:
            o.stream = stream.cuda_stream
        _check(lib().dsanls_set_options(self._h, ctypes.byref(o)), "set_options", self._h)

    # -- data
    def set_dense(self, M):
        p, on_dev, keep = _host_or_device(M, _dt("f32"))
        if tuple(keep.shape) != (self.m, self.n):
            raise ValueError("M must be %d x %d" % (self.m, self.n))
        _check(lib().dsanls_set_dense(self._h, p, self.n, on_dev), "set_dense", self._h)

    def set_csr(self, rowptr, col, val, t_rowptr=None, t_col=None, t_val=None):
        rp, dev, k1 = _host_or_device(rowptr, _dt("i64"))
        cp, _, k2 = _host_or_device(col, _dt("i32"))
        vp, _, k3 = _host_or_device(val, _dt("f32"))
        nnz = int(k2.shape[0])
        if t_rowptr is not None:
            trp, _, k4 = _host_or_device(t_rowptr, _dt("i64"))
            tcp, _, k5 = _host_or_device(t_col, _dt("i32"))
            tvp, _, k6 = _host_or_device(t_val, _dt("f32"))
        else:
            trp = tcp = tvp = None
        _check(lib().dsanls_set_csr(self._h, rp, cp, vp, nnz, trp, tcp, tvp, dev), "set_csr", self._h)

    def set_factors(self, U=None, V=None):
        up, udev, ku = _host_or_device(U, _dt("f32")) if U is not None else (None, 0, None)
        vp, vdev, kv = _host_or_device(V, _dt("f32")) if V is not None else (None, 0, None)
        if U is not None and V is not None and udev != vdev:
            raise ValueError("U and V must both be host or both device arrays")
        _check(lib().dsanls_set_factors(self._h, up, vp, udev or vdev), "set_factors", self._h)

    # -- iteration
    def step(self, iters=1):
        _check(lib().dsanls_step(self._h, int(iters)), "step", self._h)

    def half_step(self, side):
        _check(lib().dsanls_half_step(self._h, int(side)), "half_step", self._h)

    def sync(self):
        _check(lib().dsanls_sync(self._h), "sync", self._h)

    def rel_error(self):
        v = ctypes.c_double()
        _check(lib().dsanls_rel_error(self._h, ctypes.byref(v)), "rel_error", self._h)
        return v.value

    def factors(self, out_U=None, out_V=None):
        """Returns (U, V) as numpy arrays, or fills the given torch CUDA tensors."""
        if out_U is not None or out_V is not None:
            _check(lib().dsanls_get_factors(self._h, _dev_ptr(out_U) if out_U is not None else None,
                                            _dev_ptr(out_V) if out_V is not None else None, 1), "get_factors", self._h)
            return out_U, out_V
        U = np.empty((self.m, self.k), dtype=np.float32)
        V = np.empty((self.n, self.k), dtype=np.float32)
        _check(lib().dsanls_get_factors(self._h, U.ctypes.data_as(ctypes.c_void_p),
                                        V.ctypes.data_as(ctypes.c_void_p), 0), "get_factors", self._h)
        return U, V

    def profile_half_step(self, side, reps=1):
        """Mean milliseconds per phase (dict) of `reps` half-steps of `side`."""
        ms = np.zeros(NPHASES, dtype=np.float64)
        _check(lib().dsanls_profile_half_step(self._h, int(side), int(reps), ms.ctypes.data_as(ctypes.c_void_p)),
               "profile_half_step", self._h)
        return dict(zip(PHASES, ms.tolist()))

    def set_mlp(self, mlp, pg_iters=4):
        """Use the learned warm start `mlp` (an MLP; None for the plain solver)."""
        self._mlp = mlp
        _check(lib().dsanls_set_mlp(self._h, mlp._h if mlp is not None else None, int(pg_iters)), "set_mlp", self._h)

    def mlp_kept(self):
        v = ctypes.c_int64()
        _check(lib().dsanls_mlp_kept(self._h, ctypes.byref(v)), "mlp_kept", self._h)
        return v.value

    def harvest(self, side, iters=300):
        """(G, mu, b, x*) of the current state's `side` half-step as CUDA tensors (no update)."""
        torch = _torch()
        rows = self.m if side == 0 else self.n
        G = torch.empty((self.k, self.k), dtype=torch.float32, device="cuda")
        mu = torch.empty((1,), dtype=torch.float32, device="cuda")
        b = torch.empty((rows, self.k), dtype=torch.float32, device="cuda")
        x = torch.empty((rows, self.k), dtype=torch.float32, device="cuda")
        _check(lib().dsanls_harvest(self._h, int(side), int(iters), _dev_ptr(G), _dev_ptr(mu), _dev_ptr(b),
                                    _dev_ptr(x)), "harvest", self._h)
        return G, mu, b, x

    def gram(self, side):
        G = np.empty((self.k, self.k), dtype=np.float64)
        eta = ctypes.c_double()
        _check(lib().dsanls_get_gram(self._h, int(side), G.ctypes.data_as(ctypes.c_void_p), ctypes.byref(eta)),
               "get_gram", self._h)
        return G, eta.value


class Batch:
    """Many independent dense problems advanced together (binary32)."""

    def __init__(self, shapes, **options):
        """shapes: list of dicts with m, n, k, d, d_v, seed."""
        self.shapes = list(shapes)
        c = len(self.shapes)
        arr = lambda key, dt: np.ascontiguousarray([s[key] for s in self.shapes], dtype=dt)
        self._keep = [arr("m", np.int64), arr("n", np.int64), arr("k", np.int32), arr("d", np.int32),
                      arr("d_v", np.int32), arr("seed", np.uint64)]
        ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in self._keep]
        h = ctypes.c_void_p()
        _check(lib().dsanls_batch_create(c, *ptrs, ctypes.byref(h)), "dsanls_batch_create")
        self._h = h
        if options:
            self.set_options(**options)

    def _err(self, code, what):
        if code != OK:
            m = lib().dsanls_batch_last_error(self._h)
            raise DSANLSError(code, "%s: %s" % (what, m.decode() if m else ""))

    def set_options(self, stream="current", **kw):
        o = Options()
        lib().dsanls_default_options(ctypes.byref(o))
        for key, v in kw.items():
            if not hasattr(o, key) or key == "stream":
                raise TypeError("unknown option %r" % key)
            setattr(o, key, v)
        o.stream = _stream_ptr().value if stream == "current" else (None if stream is None else stream.cuda_stream)
        self._err(lib().dsanls_batch_set_options(self._h, ctypes.byref(o)), "batch_set_options")

    def set_dense(self, i, M):
        p, dev, keep = _host_or_device(M, _dt("f32"))
        self._err(lib().dsanls_batch_set_dense(self._h, int(i), p, int(keep.shape[1]), dev), "batch_set_dense")

    def set_factors(self, i, U=None, V=None):
        up, udev, ku = _host_or_device(U, _dt("f32")) if U is not None else (None, 0, None)
        vp, vdev, kv = _host_or_device(V, _dt("f32")) if V is not None else (None, 0, None)
        self._err(lib().dsanls_batch_set_factors(self._h, int(i), up, vp, udev or vdev), "batch_set_factors")

    def step(self, iters=1):
        self._err(lib().dsanls_batch_step(self._h, int(iters)), "batch_step")

    def factors(self, i):
        sh = self.shapes[i]
        U = np.empty((sh["m"], sh["k"]), np.float32)
        V = np.empty((sh["n"], sh["k"]), np.float32)
        self._err(lib().dsanls_batch_get_factors(self._h, int(i), U.ctypes.data_as(ctypes.c_void_p),
                                                 V.ctypes.data_as(ctypes.c_void_p), 0), "batch_get_factors")
        return U, V

    def rel_errors(self):
        out = np.empty(len(self.shapes), np.float64)
        self._err(lib().dsanls_batch_rel_error(self._h, out.ctypes.data_as(ctypes.c_void_p)), "batch_rel_error")
        return out

    def profile(self):
        """Milliseconds per phase of one eager outer iteration: {side: {phase: ms}}."""
        ms = np.zeros(10, np.float64)
        self._err(lib().dsanls_batch_profile(self._h, ms.ctypes.data_as(ctypes.c_void_p)), "batch_profile")
        names = ["sketch", "B", "AR", "gram", "update"]
        return {side: dict(zip(names, ms[5 * i:5 * i + 5].tolist())) for i, side in enumerate(("U", "V"))}

    def tuned_blocks(self):
        v = ctypes.c_int32()
        self._err(lib().dsanls_batch_tuned_blocks(self._h, ctypes.byref(v)), "batch_tuned_blocks")
        return v.value

    def set_tile(self, chunk, stages, row_tiles, pipeline=1, side=-1):
        """Pin the tensor-core tile (bf16 paper order) of one half-step (side 0 or
        1) or both (-1) instead of autotuning it; pipeline 0: cp.async ring, 1: TMA
        ring, 2: TMA ring with the chunk epilogue off the copy path; (0, 0, 0)
        returns to the autotuner."""
        self._err(lib().dsanls_batch_set_tile(self._h, int(side), int(chunk), int(stages), int(row_tiles),
                                              int(pipeline)), "batch_set_tile")

    def tuned_tile(self, side=0):
        """(chunk, ctas, row tiles per item, pipeline) of the tensor-core product of
        half-step `side` chosen by the autotuner (bf16 paper order; zeros otherwise
        or before the first step)."""
        c, n, r, t = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        self._err(lib().dsanls_batch_tuned_tile(self._h, int(side), ctypes.byref(c), ctypes.byref(n), ctypes.byref(r),
                                                ctypes.byref(t)), "batch_tuned_tile")
        return c.value, n.value, r.value, t.value

    def close(self):
        if getattr(self, "_h", None):
            lib().dsanls_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The learned warm start's network (k <= 32, hidden <= 256)."""

    def __init__(self, k, hidden=256, max_rows=1 << 16, max_groups=64, seed=0):
        h = ctypes.c_void_p()
        _check(lib().dsanls_mlp_create(int(k), int(hidden), int(max_rows), int(max_groups), int(seed),
                                       ctypes.byref(h)), "dsanls_mlp_create")
        self._h = h
        self.k, self.hidden = k, hidden
        c = ctypes.c_int64()
        _check(lib().dsanls_mlp_param_count(self._h, ctypes.byref(c)), "mlp_param_count")
        self.n_params = c.value

    def params(self):
        out = np.empty(self.n_params, np.float32)
        _check(lib().dsanls_mlp_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p)), "mlp_get_params")
        return out

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        assert theta.size == self.n_params
        _check(lib().dsanls_mlp_set_params(self._h, theta.ctypes.data_as(ctypes.c_void_p)), "mlp_set_params")

    def predict(self, G, mu, off, b):
        """G (groups x k x k), mu (groups), off (groups + 1, int64), b (rows x k): CUDA tensors."""
        torch = _torch()
        x = torch.empty_like(b)
        _check(lib().dsanls_mlp_predict(self._h, _dev_ptr(G), _dev_ptr(mu), _dev_ptr(off), int(mu.numel()),
                                        _dev_ptr(b), int(b.shape[0]), _dev_ptr(x), _stream_ptr()), "mlp_predict")
        return x

    def train_step(self, G, mu, off, b, xstar, lr, want_grad=False):
        loss = ctypes.c_double()
        grad = np.empty(self.n_params, np.float32) if want_grad else None
        _check(lib().dsanls_mlp_train_step(self._h, _dev_ptr(G), _dev_ptr(mu), _dev_ptr(off), int(mu.numel()),
                                           _dev_ptr(b), _dev_ptr(xstar), int(b.shape[0]), float(lr),
                                           ctypes.byref(loss),
                                           grad.ctypes.data_as(ctypes.c_void_p) if want_grad else None,
                                           _stream_ptr()), "mlp_train_step")
        return (loss.value, grad) if want_grad else loss.value

    def close(self):
        if getattr(self, "_h", None):
            lib().dsanls_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
