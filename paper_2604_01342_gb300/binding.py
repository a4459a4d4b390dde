"""ctypes binding of the C ABI declared in ``include/hawkes_gb300.h``.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libhawkes_gb300.so``.  Tensors are passed as raw device pointers
(``torch.Tensor.data_ptr()``) together with the current CUDA stream.  The
library is loaded on first use; if it is missing the call raises, there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_NAME = "libhawkes_gb300.so"
_lock = threading.Lock()
_lib = None

STATUS_NAMES = {
    0: "HAWKES_OK", 1: "HAWKES_ERR_INVALID_ARG", 2: "HAWKES_ERR_UNSORTED",
    3: "HAWKES_ERR_MARK_RANGE", 4: "HAWKES_ERR_TIME_RANGE", 5: "HAWKES_ERR_PARAM_DOMAIN",
    6: "HAWKES_ERR_NONPOS_INTENSITY", 7: "HAWKES_ERR_WORKSPACE", 8: "HAWKES_ERR_UNSUPPORTED",
    9: "HAWKES_ERR_CUDA",
}

# every symbol include/hawkes_gb300.h declares
EXPORTED = (
    "hawkes_default_opts", "hawkes_workspace_size", "hawkes_loglik", "hawkes_loglik_grad",
    "hawkes_loglik_varlen", "hawkes_loglik_grad_varlen", "hawkes_workspace_size_host",
    "hawkes_loglik_grad_host", "hawkes_last_device_status", "hawkes_mark_counts",
    "hawkes_status_str", "hawkes_last_launch_count", "hawkes_profile_enable",
    "hawkes_profile_read", "hawkes_static_scratch_bytes", "hawkes_loglik_grad_static",
    "hawkes_slice_aggregate", "hawkes_loglik_grad_slice", "hawkes_integer_tables",
)


class HawkesOpts(ctypes.Structure):
    _fields_ = [("beta_shared", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("validate", ctypes.c_int32), ("path", ctypes.c_int32),
                ("kernels", ctypes.c_int32), ("support", ctypes.c_int32),
                ("reduce", ctypes.c_int32), ("fp32_times", ctypes.c_int32),
                ("walk_lanes", ctypes.c_int32)]


class HawkesTables(ctypes.Structure):
    _fields_ = [("mark_counts", ctypes.c_void_p), ("chunk_base", ctypes.c_void_p),
                ("chunk_seq", ctypes.c_void_p), ("bucket_start", ctypes.c_void_p),
                ("bucket_slots", ctypes.c_void_p), ("chunk", ctypes.c_int32),
                ("mark_blocks", ctypes.c_int32), ("support_row_ptr", ctypes.c_void_p),
                ("support_col", ctypes.c_void_p), ("mark_start", ctypes.c_void_p),
                ("mark_slots", ctypes.c_void_p), ("segment_events", ctypes.c_int64),
                ("segments", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class HawkesError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        name = STATUS_NAMES.get(code, str(code))
        super().__init__(f"{where}: {name}" if where else name)
        self.code = code
        self.name = name


def library_path() -> str:
    return os.path.join(_HERE, "_build", _LIB_NAME)


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{_LIB_NAME} is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        p, i32, i64, d, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                              ctypes.c_size_t)
        op = ctypes.POINTER(HawkesOpts)
        L.hawkes_default_opts.argtypes = []
        L.hawkes_default_opts.restype = HawkesOpts
        L.hawkes_workspace_size.argtypes = [i64, i32, i32, i32, op]
        L.hawkes_workspace_size.restype = sz
        L.hawkes_loglik.argtypes = [p, p, i64, d, i32, p, p, p, op, p, sz, p, p]
        L.hawkes_loglik_grad.argtypes = [p, p, i64, d, i32, p, p, p, op, p, sz, p, p, p, p, p]
        L.hawkes_loglik_varlen.argtypes = [p, p, p, i32, i64, p, i32, p, p, p, op, p, sz, p, p]
        L.hawkes_loglik_grad_varlen.argtypes = [p, p, p, i32, i64, p, i32, p, p, p, op, p, sz,
                                                p, p, p, p, p]
        L.hawkes_workspace_size_host.argtypes = [i64, i32, op]
        L.hawkes_workspace_size_host.restype = sz
        L.hawkes_loglik_grad_host.argtypes = [p, p, i64, d, i32, p, p, p, op, p, sz, p, p, p,
                                              p, p]
        L.hawkes_last_device_status.argtypes = [p, p]
        L.hawkes_mark_counts.argtypes = [p]
        L.hawkes_mark_counts.restype = p
        L.hawkes_status_str.argtypes = [ctypes.c_int]
        L.hawkes_status_str.restype = ctypes.c_char_p
        L.hawkes_last_launch_count.argtypes = []
        L.hawkes_last_launch_count.restype = i32
        L.hawkes_profile_enable.argtypes = [i32]
        L.hawkes_profile_enable.restype = i32
        L.hawkes_profile_read.argtypes = [ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_char_p), i32]
        L.hawkes_profile_read.restype = i32
        L.hawkes_slice_aggregate.argtypes = [p, p, i64, i32, p, op, d, p, sz, p, p, p]
        L.hawkes_loglik_grad_slice.argtypes = [p, p, i64, d, i32, p, p, p, op, p, p, i32, p, sz,
                                               p, p, p, p, p]
        L.hawkes_static_scratch_bytes.argtypes = []
        L.hawkes_static_scratch_bytes.restype = sz
        L.hawkes_loglik_grad_static.argtypes = [p, p, i64, d, i32, p, p, p, op, p, p, p, p, p]
        L.hawkes_integer_tables.argtypes = [p, i64, i32, i32, i32, op,
                                            ctypes.POINTER(HawkesTables)]
        for name in ("hawkes_integer_tables", "hawkes_slice_aggregate", "hawkes_loglik_grad_slice",
                     "hawkes_loglik_grad_static", "hawkes_loglik", "hawkes_loglik_grad",
                     "hawkes_loglik_varlen",
                     "hawkes_loglik_grad_varlen", "hawkes_loglik_grad_host",
                     "hawkes_last_device_status"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def make_opts(beta_shared: bool, chunk: int = 0, validate: bool = True, path: int = 0,
              kernels: int = 1, support: bool = False, reduce: int = 0,
              fp32_times: bool = False, walk_lanes: int = 0):
    return HawkesOpts(int(bool(beta_shared)), int(chunk), int(bool(validate)), int(path),
                      int(kernels), int(bool(support)), int(reduce), int(bool(fp32_times)),
                      int(walk_lanes))


def _check(rc: int, where: str):
    if rc != 0:
        raise HawkesError(rc, where)


def hawkes_status_str(code: int) -> str:
    return lib().hawkes_status_str(int(code)).decode()


def hawkes_workspace_size(N: int, M: int, B: int, grad: bool, opts: HawkesOpts) -> int:
    n = lib().hawkes_workspace_size(int(N), int(M), int(B), int(bool(grad)), ctypes.byref(opts))
    if n == 0:
        raise HawkesError(8, "hawkes_workspace_size")
    return int(n)


def hawkes_loglik(t, c, N, T, M, mu, alpha, beta, opts, ws, ws_bytes, out_ll, stream):
    _check(lib().hawkes_loglik(t, c, int(N), float(T), int(M), mu, alpha, beta,
                               ctypes.byref(opts), ws, int(ws_bytes), out_ll, stream),
           "hawkes_loglik")


def hawkes_loglik_grad(t, c, N, T, M, mu, alpha, beta, opts, ws, ws_bytes, out_ll, d_mu,
                       d_alpha, d_beta, stream):
    _check(lib().hawkes_loglik_grad(t, c, int(N), float(T), int(M), mu, alpha, beta,
                                    ctypes.byref(opts), ws, int(ws_bytes), out_ll, d_mu,
                                    d_alpha, d_beta, stream), "hawkes_loglik_grad")


def hawkes_loglik_varlen(t, c, offsets, B, N, T, M, mu, alpha, beta, opts, ws, ws_bytes,
                         out_ll, stream):
    _check(lib().hawkes_loglik_varlen(t, c, offsets, int(B), int(N), T, int(M), mu, alpha,
                                      beta, ctypes.byref(opts), ws, int(ws_bytes), out_ll,
                                      stream), "hawkes_loglik_varlen")


def hawkes_loglik_grad_varlen(t, c, offsets, B, N, T, M, mu, alpha, beta, opts, ws, ws_bytes,
                              out_ll, d_mu, d_alpha, d_beta, stream):
    _check(lib().hawkes_loglik_grad_varlen(t, c, offsets, int(B), int(N), T, int(M), mu,
                                           alpha, beta, ctypes.byref(opts), ws, int(ws_bytes),
                                           out_ll, d_mu, d_alpha, d_beta, stream),
           "hawkes_loglik_grad_varlen")


def hawkes_workspace_size_host(N: int, M: int, opts: HawkesOpts) -> int:
    n = lib().hawkes_workspace_size_host(int(N), int(M), ctypes.byref(opts))
    if n == 0:
        raise HawkesError(8, "hawkes_workspace_size_host")
    return int(n)


def hawkes_loglik_grad_host(t, c, N, T, M, mu, alpha, beta, opts, ws, ws_bytes, out_ll, d_mu,
                            d_alpha, d_beta, stream):
    _check(lib().hawkes_loglik_grad_host(t, c, int(N), float(T), int(M), mu, alpha, beta,
                                         ctypes.byref(opts), ws, int(ws_bytes), out_ll, d_mu,
                                         d_alpha, d_beta, stream), "hawkes_loglik_grad_host")


def hawkes_last_device_status(ws, stream) -> int:
    return int(lib().hawkes_last_device_status(ws, stream))


def hawkes_mark_counts_ptr(ws) -> int:
    return lib().hawkes_mark_counts(ws) or 0


def hawkes_last_launch_count() -> int:
    return int(lib().hawkes_last_launch_count())


def hawkes_profile_enable(on: bool) -> None:
    rc = lib().hawkes_profile_enable(int(bool(on)))
    if rc:
        raise HawkesError(rc, "hawkes_profile_enable")


def hawkes_profile_read(cap: int = 64):
    """[(kernel name, milliseconds)] of the last call, in launch order."""
    ms = (ctypes.c_float * cap)()
    names = (ctypes.c_char_p * cap)()
    n = lib().hawkes_profile_read(ms, names, cap)
    if n < 0:
        raise HawkesError(-n, "hawkes_profile_read")
    return [(names[i].decode(), float(ms[i])) for i in range(n)]


def hawkes_integer_tables(ws, N, M, B, grad, opts) -> HawkesTables:
    """Device pointers of the integer tables of the last call on ``ws``."""
    out = HawkesTables()
    _check(lib().hawkes_integer_tables(ws, int(N), int(M), int(B), int(bool(grad)),
                                       ctypes.byref(opts), ctypes.byref(out)),
           "hawkes_integer_tables")
    return out


def hawkes_static_scratch_bytes() -> int:
    return int(lib().hawkes_static_scratch_bytes())


def hawkes_loglik_grad_static(t, c, N, T, M, mu, alpha, beta, opts, out_ll, d_mu, d_alpha,
                              d_beta, stream):
    """hawkes_loglik_grad on the library's built-in scratch array (no workspace)."""
    _check(lib().hawkes_loglik_grad_static(t, c, int(N), float(T), int(M), mu, alpha, beta,
                                           ctypes.byref(opts), out_ll, d_mu, d_alpha, d_beta,
                                           stream), "hawkes_loglik_grad_static")


def hawkes_slice_aggregate(t, c, N, M, beta, opts, t_next, ws, ws_bytes, agg_S, agg_G, stream):
    _check(lib().hawkes_slice_aggregate(t, c, int(N), int(M), beta, ctypes.byref(opts),
                                        float(t_next), ws, int(ws_bytes), agg_S, agg_G, stream),
           "hawkes_slice_aggregate")


def hawkes_loglik_grad_slice(t, c, N, T, M, mu, alpha, beta, opts, carry_S, carry_G, base_term,
                             ws, ws_bytes, out_ll, d_mu, d_alpha, d_beta, stream):
    _check(lib().hawkes_loglik_grad_slice(t, c, int(N), float(T), int(M), mu, alpha, beta,
                                          ctypes.byref(opts), carry_S, carry_G,
                                          int(bool(base_term)), ws, int(ws_bytes), out_ll, d_mu,
                                          d_alpha, d_beta, stream), "hawkes_loglik_grad_slice")
