"""ctypes binding of libcld's C ABI (include/cld.h), one function per entry point.

Argument marshalling only: every step of the estimator runs in the library's
CUDA kernels.  Device pointers are plain integers (``tensor.data_ptr()``);
streams are ``torch.cuda.Stream.cuda_stream`` integers or 0.  A non-zero
status raises ``CldError`` carrying the status and ``cld_last_error()``.
If libcld.so is missing the import fails: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcld.so")

CLD_OK, CLD_ERR_INVALID, CLD_ERR_INTERVAL, CLD_ERR_SPECTRUM = 0, 1, 2, 3
CLD_ERR_NOMEM, CLD_ERR_CUDA, CLD_ERR_TIMEOUT, CLD_ERR_UNSUPPORTED = 4, 5, 6, 7
CLD_F32, CLD_BF16, CLD_F64 = 0, 1, 2
CLD_SPD, CLD_GENERAL = 0, 1
STATUS_NAMES = {0: "CLD_OK", 1: "CLD_ERR_INVALID", 2: "CLD_ERR_INTERVAL", 3: "CLD_ERR_SPECTRUM",
                4: "CLD_ERR_NOMEM", 5: "CLD_ERR_CUDA", 6: "CLD_ERR_TIMEOUT", 7: "CLD_ERR_UNSUPPORTED"}

# (name, restype, argtypes) for every exported entry point of include/cld.h
_vp, _i64, _i32, _u64, _f64, _sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t
_P = ctypes.POINTER
SIGNATURES = [
    ("cld_create_csr", _i32, [_P(_vp), _i64, _i64, _vp, _vp, _vp, _i32, _i32, _vp]),
    ("cld_create_dense", _i32, [_P(_vp), _i64, _i64, _vp, _i32, _i32, _vp]),
    ("cld_workspace_size", _i32, [_vp, _i32, _i32, _i32, _P(_sz)]),
    ("cld_set_workspace", _i32, [_vp, _vp, _sz]),
    ("cld_set_interval", _i32, [_vp, _f64, _f64]),
    ("cld_auto_interval", _i32, [_vp, _i32, _P(_f64), _P(_f64)]),
    ("cld_estimate", _i32, [_vp, _i32, _i32, _u64, _P(_f64), _P(_f64), _vp]),
    ("cld_last_details", _i32, [_vp, _vp, _vp]),
    ("cld_grad", _i32, [_vp, _i32, _i32, _u64, _P(_f64), _vp]),
    ("cld_host_workspace_size", _i32, [_i64, _i64, _i32, _i32, _i32, _P(_sz)]),
    ("cld_logdet_csr_host", _i32, [_i64, _i64, _vp, _vp, _vp, _i32, _i32, _f64, _f64, _i32, _i32, _u64,
                                   _vp, _sz, _vp, _P(_f64), _P(_f64)]),
    ("cld_estimate_static", _i32, [_i64, _i64, _vp, _vp, _vp, _i32, _f64, _f64, _i32, _i32, _u64, _vp,
                                   _P(_f64), _P(_f64)]),
    ("cld_create_batch", _i32, [_P(_vp), _i32, _vp, _i64, _vp, _vp, _vp, _i32, _i32, _vp]),
    ("cld_batch_set_tile_rows", _i32, [_vp, _i32]),
    ("cld_batch_get_tile_rows", _i32, [_vp, _P(_i32)]),
    ("cld_batch_set_intervals", _i32, [_vp, _vp, _vp]),
    ("cld_batch_auto_intervals", _i32, [_vp, _vp, _vp]),
    ("cld_batch_estimate", _i32, [_vp, _i32, _i32, _u64, _vp, _vp]),
    ("cld_set_graph", _i32, [_vp, _i32]),
    ("cld_set_kernel_variant", _i32, [_vp, _i32]),
    ("cld_set_grad_checkpoint", _i32, [_vp, _i32]),
    ("cld_autotune", _i32, [_vp, _i32, _i32, _P(_i32), _P(ctypes.c_float)]),
    ("cld_debug_withhold_tile", _i32, [_vp, _i64]),
    ("cld_set_profiling", _i32, [_vp, _i32]),
    ("cld_last_timing", _i32, [_vp, _P(ctypes.c_float), _P(_i32), _P(_i32)]),
    ("cld_launch_config", _i32, [_vp, _i32, _P(_i32), _P(_i32), _P(_i32), _P(_i32)]),
    ("cld_destroy", None, [_vp]),
    ("cld_last_error", ctypes.c_char_p, []),
    ("cld_version", ctypes.c_char_p, []),
]


class CldError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status
        self.message = message


_lib = None


def load(path: str = LIB_PATH):
    """Loads libcld.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("libcld.so not found at %s: run `python -c 'import __graft_entry__ as g; "
                              "g.build()'` (needs nvcc)" % path)
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(st: int):
    if st != CLD_OK:
        raise CldError(st, load().cld_last_error().decode())


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError("cannot take a pointer of %r" % type(x))


def cld_version() -> str:
    return load().cld_version().decode()


def cld_last_error() -> str:
    return load().cld_last_error().decode()


def cld_create_csr(d, nnz, rowptr, col, val, val_dtype, kind, stream=0):
    h = ctypes.c_void_p()
    _check(load().cld_create_csr(ctypes.byref(h), d, nnz, _ptr(rowptr), _ptr(col), _ptr(val),
                                 val_dtype, kind, stream or None))
    return h.value


def cld_create_dense(d, ld, val, val_dtype, kind, stream=0):
    h = ctypes.c_void_p()
    _check(load().cld_create_dense(ctypes.byref(h), d, ld, _ptr(val), val_dtype, kind, stream or None))
    return h.value


def cld_workspace_size(h, n, M, with_grad=0) -> int:
    out = ctypes.c_size_t()
    _check(load().cld_workspace_size(h, n, M, with_grad, ctypes.byref(out)))
    return out.value


def cld_set_workspace(h, dev_ptr, nbytes):
    _check(load().cld_set_workspace(h, _ptr(dev_ptr), nbytes))


def cld_set_interval(h, a, b):
    _check(load().cld_set_interval(h, a, b))


def cld_auto_interval(h, lanczos_iters=0):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().cld_auto_interval(h, lanczos_iters, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def cld_estimate(h, n, M, seed, moments=False, raise_on_spectrum=True):
    """Returns (logdet, stderr, moments or None, status)."""
    g, se = ctypes.c_double(), ctypes.c_double()
    t = np.zeros((n + 1, M), dtype=np.float64) if moments else None
    st = load().cld_estimate(h, n, M, seed, ctypes.byref(g), ctypes.byref(se), _ptr(t) or None)
    if st != CLD_OK and (raise_on_spectrum or st != CLD_ERR_SPECTRUM):
        _check(st)
    return g.value, se.value, t, st


def cld_last_details(h, n, M):
    c = np.zeros(n + 1, dtype=np.float64)
    gp = np.zeros(M, dtype=np.float64)
    _check(load().cld_last_details(h, _ptr(c), _ptr(gp)))
    return c, gp


def cld_grad(h, n, M, seed, dvalues_dev):
    g = ctypes.c_double()
    _check(load().cld_grad(h, n, M, seed, ctypes.byref(g), _ptr(dvalues_dev)))
    return g.value


def cld_host_workspace_size(d, nnz, val_dtype, n, M) -> int:
    out = ctypes.c_size_t()
    _check(load().cld_host_workspace_size(d, nnz, val_dtype, n, M, ctypes.byref(out)))
    return out.value


def cld_logdet_csr_host(d, nnz, rowptr_host, col_host, val_host, val_dtype, kind, a, b, n, M, seed,
                        workspace_dev, workspace_bytes, stream=0):
    g, se = ctypes.c_double(), ctypes.c_double()
    _check(load().cld_logdet_csr_host(d, nnz, _ptr(rowptr_host), _ptr(col_host), _ptr(val_host), val_dtype,
                                      kind, a, b, n, M, seed, _ptr(workspace_dev), workspace_bytes,
                                      stream or None, ctypes.byref(g), ctypes.byref(se)))
    return g.value, se.value


def cld_estimate_static(d, nnz, rowptr, col, val, val_dtype, a, b, n, M, seed, stream=0):
    """Estimate with the library's built-in device scratch (no allocation);
    returns (logdet, stderr)."""
    g, se = ctypes.c_double(), ctypes.c_double()
    _check(load().cld_estimate_static(d, nnz, _ptr(rowptr), _ptr(col), _ptr(val), val_dtype, a, b, n, M, seed,
                                      stream or None, ctypes.byref(g), ctypes.byref(se)))
    return g.value, se.value


def cld_create_batch(blk_rows, nnz, rowptr, col, val, val_dtype, kind, stream=0):
    br = np.ascontiguousarray(blk_rows, dtype=np.int64)
    h = ctypes.c_void_p()
    _check(load().cld_create_batch(ctypes.byref(h), br.shape[0] - 1, _ptr(br), nnz, _ptr(rowptr), _ptr(col),
                                   _ptr(val), val_dtype, kind, stream or None))
    return h.value


def cld_batch_get_tile_rows(h):
    r = ctypes.c_int32()
    _check(load().cld_batch_get_tile_rows(h, ctypes.byref(r)))
    return r.value


def cld_batch_set_tile_rows(h, rows):
    _check(load().cld_batch_set_tile_rows(h, rows))


def cld_batch_set_intervals(h, a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    _check(load().cld_batch_set_intervals(h, _ptr(a), _ptr(b)))


def cld_batch_auto_intervals(h, nb):
    a = np.zeros(nb, dtype=np.float64)
    b = np.zeros(nb, dtype=np.float64)
    _check(load().cld_batch_auto_intervals(h, _ptr(a), _ptr(b)))
    return a, b


def cld_batch_estimate(h, nb, n, M, seed):
    g = np.zeros(nb, dtype=np.float64)
    se = np.zeros(nb, dtype=np.float64)
    _check(load().cld_batch_estimate(h, n, M, seed, _ptr(g), _ptr(se)))
    return g, se


def cld_set_graph(h, on):
    _check(load().cld_set_graph(h, 1 if on else 0))


def cld_set_kernel_variant(h, variant):
    _check(load().cld_set_kernel_variant(h, variant))


def cld_set_grad_checkpoint(h, interval):
    _check(load().cld_set_grad_checkpoint(h, interval))


def cld_autotune(h, M, reps=3):
    """Times every step-kernel variant on this matrix and keeps the fastest;
    returns (variant, ms per step)."""
    v, ms = ctypes.c_int(), ctypes.c_float()
    _check(load().cld_autotune(h, M, reps, ctypes.byref(v), ctypes.byref(ms)))
    return v.value, ms.value


def cld_debug_withhold_tile(h, tile):
    """Testing aid of the staged step kernel (variant 6): tile > 0 withholds
    row tile `tile - 1`, so its bounded waits run out; 0 turns it off."""
    _check(load().cld_debug_withhold_tile(h, int(tile)))


def cld_set_profiling(h, on):
    _check(load().cld_set_profiling(h, 1 if on else 0))


def cld_last_timing(h):
    ms, sl, tl = ctypes.c_float(), ctypes.c_int(), ctypes.c_int()
    _check(load().cld_last_timing(h, ctypes.byref(ms), ctypes.byref(sl), ctypes.byref(tl)))
    return ms.value, sl.value, tl.value


def cld_launch_config(h, M):
    v = [ctypes.c_int() for _ in range(4)]
    _check(load().cld_launch_config(h, M, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def cld_destroy(h):
    if h:
        load().cld_destroy(h)
