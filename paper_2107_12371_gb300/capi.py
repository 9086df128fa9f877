"""ctypes binding of include/spmv.h -- argument marshalling only.

Every function here has the name of the C entry point it calls and does nothing but convert
arguments (torch tensors -> device pointers, numpy arrays -> host pointers, Python numbers ->
C types) and raise :class:`SpmvError` on a non-OK status.  All arithmetic runs in the CUDA
library.  If the library is missing or cannot be loaded, importing the binding raises: there
is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# ---- status codes and option constants (mirror include/spmv.h) ------------------------
SPMV_OK = 0
SPMV_ERR_INVALID_ARG = 1
SPMV_ERR_INVALID_CSR = 2
SPMV_ERR_OOM = 3
SPMV_ERR_BUDGET = 4
SPMV_ERR_CUDA = 5
SPMV_ERR_NOT_CONVERGED = 6
SPMV_ERR_TIMEOUT = 7
SPMV_ERR_PENDING = 8
SPMV_ERR_UNSUPPORTED = 9
SPMV_ERR_CANCELLED = 10

SPMV_REORDER_NONE, SPMV_REORDER_RCM, SPMV_REORDER_CM = 0, 1, 2
SPMV_PREC_FP64, SPMV_PREC_FP32, SPMV_PREC_DUAL = 0, 1, 2
SPMV_VARIANT_AUTO, SPMV_VARIANT_CSR, SPMV_VARIANT_SELL, SPMV_VARIANT_SELL_WINDOW = 0, 1, 2, 3
SPMV_VARIANT_SELL_BULK = 4
SPMV_SPMM_AUTO, SPMV_SPMM_WIDE, SPMV_SPMM_WIDE_PIPE, SPMV_SPMM_WIDE_GS4, SPMV_SPMM_WIDE_GS6 = \
    0, 1, 2, 3, 4
SPMV_SPMM_UNROLLED = 5
SPMV_CHAIN_AUTO, SPMV_CHAIN_FUSED, SPMV_CHAIN_TWO = 0, 1, 2


class spmv_options_t(ctypes.Structure):
    _fields_ = [("slice_height", ctypes.c_int), ("block", ctypes.c_int),
                ("variant", ctypes.c_int), ("reorder", ctypes.c_int),
                ("precision", ctypes.c_int), ("autotune", ctypes.c_int),
                ("peripheral", ctypes.c_int), ("window_words", ctypes.c_int),
                ("index_bits", ctypes.c_int), ("sigma", ctypes.c_int),
                ("checks", ctypes.c_int), ("spmm_form", ctypes.c_int),
                ("pq_ctas", ctypes.c_int), ("pq_unroll", ctypes.c_int),
                ("gather_bytes", ctypes.c_int), ("chain_form", ctypes.c_int)]


class spmv_info_t(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("slice_height", ctypes.c_int32), ("block", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("reorder", ctypes.c_int32), ("n_slices", ctypes.c_int32),
                ("sell_entries", ctypes.c_int64), ("bandwidth", ctypes.c_int32),
                ("max_slice_span", ctypes.c_int32), ("window_words", ctypes.c_int32),
                ("device_bytes", ctypes.c_size_t), ("index_bits", ctypes.c_int32),
                ("n_cols", ctypes.c_int32), ("spmm_form", (ctypes.c_int32 * 4) * 2),
                ("pq_ctas", ctypes.c_int32), ("pq_unroll", ctypes.c_int32),
                ("gather_bytes", ctypes.c_int32), ("chain_form", ctypes.c_int32 * 2)]


class spmv_part_info_t(ctypes.Structure):
    _fields_ = [("n_parts", ctypes.c_int32), ("part", ctypes.c_int32),
                ("row_begin", ctypes.c_int32), ("row_end", ctypes.c_int32),
                ("n_local", ctypes.c_int32), ("n_halo_lo", ctypes.c_int32),
                ("n_halo_hi", ctypes.c_int32), ("n_ext", ctypes.c_int32),
                ("nnz_local", ctypes.c_int64), ("send_total", ctypes.c_int32),
                ("recv_total", ctypes.c_int32), ("device_bytes", ctypes.c_size_t)]


class cg_options_t(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mixed", ctypes.c_int),
                ("inner_rtol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("use_x0", ctypes.c_int), ("persistent", ctypes.c_int),
                ("check_every", ctypes.c_int), ("timeout_s", ctypes.c_double),
                ("adaptive_inner", ctypes.c_int)]


class cg_result_t(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("status", ctypes.c_int)]


class spmv_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("active_slots", ctypes.c_int),
                ("queued", ctypes.c_int), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("p50_latency_s", ctypes.c_double),
                ("p99_latency_s", ctypes.c_double), ("cancelled", ctypes.c_uint64),
                ("setup_s", ctypes.c_double), ("solve_s", ctypes.c_double),
                ("teardown_s", ctypes.c_double)]


class SpmvError(RuntimeError):
    def __init__(self, status, where):
        self.status = int(status)
        msg = _lib.spmv_status_string(int(status)).decode() if _lib else str(status)
        super().__init__("%s: %s (status %d)" % (where, msg, int(status)))


_P = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_int = ctypes.c_int

# (name, argtypes); every entry point returns spmv_status_t (int) except the string lookup
_SIGS = {
    "spmv_default_options": [ctypes.POINTER(spmv_options_t)],
    "spmv_create": [_i32, _i32, _i64, _P, _P, _P, _int, ctypes.POINTER(spmv_options_t), _P,
                    ctypes.POINTER(_P)],
    "spmv_destroy": [_P],
    "spmv_get_info": [_P, ctypes.POINTER(spmv_info_t)],
    "spmv_get_permutation": [_P, _P],
    "spmv_export_csr": [_P, _P, _P, _P],
    "spmv_export_sell": [_P, _P, _P, _P, _P, _P],
    "spmv_apply": [_P, _P, _P, _P],
    "spmv_apply_f32": [_P, _P, _P, _P],
    "spmv_apply_axpby": [_P, ctypes.c_double, _P, ctypes.c_double, _P, _P],
    "spmv_apply_axpby_f32": [_P, ctypes.c_float, _P, ctypes.c_float, _P, _P],
    "spmv_apply_csr": [_P, _P, _P, _P],
    "spmv_apply_chain": [_P, _P, _P, _P, _P],
    "spmv_apply_multi": [_P, _int, _P, _P, _P],
    "spmv_apply_multi_f32": [_P, _int, _P, _P, _P],
    "spmv_permute": [_P, _int, _int, _P, _P, _P],
    "cg_default_options": [ctypes.POINTER(cg_options_t)],
    "cg_solve": [_P, _P, _P, ctypes.POINTER(cg_options_t), ctypes.POINTER(cg_result_t), _P],
    "cg_solve_multi": [_P, _int, _P, _P, ctypes.POINTER(cg_options_t),
                       ctypes.POINTER(cg_result_t), _P],
    "spmv_diag_barrier_timeout": [_int, ctypes.c_double, _P],
    "spmv_diag_cg_timing": [_P, _int, _P, _P],
    "cg_solve_csr_noalloc": [_i32, _i64, _P, _P, _P, _P, _P, ctypes.POINTER(cg_options_t),
                             ctypes.POINTER(cg_result_t), _P],
    "spmv_server_create": [ctypes.c_size_t, _int, ctypes.POINTER(_P)],
    "spmv_server_submit": [_P, _i32, _i64, _P, _P, _P, _P, ctypes.POINTER(cg_options_t),
                           ctypes.POINTER(ctypes.c_uint64)],
    "spmv_server_poll": [_P, ctypes.c_uint64, _P, ctypes.POINTER(cg_result_t)],
    "spmv_server_get_stats": [_P, ctypes.POINTER(spmv_server_stats_t)],
    "spmv_server_set_priority_bytes": [_P, ctypes.c_size_t],
    "spmv_server_destroy": [_P],
    "spmv_server_cancel": [_P, ctypes.c_uint64],
    "spmv_apply_host": [_P, _P, _P, _P],
    "spmv_apply_chain_f32": [_P, _P, _P, _P, _P],
    "spmv_apply_host_async": [_P, _P, _P, _P],
    "spmv_verify": [_P, ctypes.POINTER(_int), _P],
    "spmv_device_status": [_P, _P],
    "spmv_diag_bulk_timeout": [_P, _P],
    "spmv_diag_checks": [_P, ctypes.POINTER(_int), ctypes.POINTER(_int), _P],
    "spmv_partition_create": [_i32, _i64, _P, _P, _P, _int, _P, _int, _int,
                              ctypes.POINTER(spmv_options_t), _P, ctypes.POINTER(_P)],
    "spmv_partition_destroy": [_P],
    "spmv_partition_info": [_P, ctypes.POINTER(spmv_part_info_t)],
    "spmv_partition_lists": [_P, _P, _P, _P, _P],
    "spmv_partition_local_csr": [_P, _P, _P, _P],
    "spmv_partition_pack": [_P, _P, _P, _P],
    "spmv_partition_apply": [_P, _P, _P, _P],
    "cg_solve_partitioned": [_P, _P, _P, ctypes.POINTER(cg_options_t),
                             ctypes.POINTER(cg_result_t), _P, _P, _P, _P],
}

# transport callbacks of cg_solve_partitioned
EXCHANGE_FN = ctypes.CFUNCTYPE(_int, _P, _P, _P)
ALLREDUCE_FN = ctypes.CFUNCTYPE(_int, ctypes.POINTER(ctypes.c_double), _int, _P)

_lib = None


def load(path: str | None = None):
    """Load (building first if needed) the CUDA library.  Raises if it is unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB_PATH
    if not os.path.exists(path):
        path = _build.build()
    lib = ctypes.CDLL(path)
    lib.spmv_status_string.argtypes = [_int]
    lib.spmv_status_string.restype = ctypes.c_char_p
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = _int
    _lib = lib
    return lib


def library_path() -> str:
    return _build.LIB_PATH


def _check(status, where):
    if status != SPMV_OK:
        raise SpmvError(status, where)
    return status


def _ptr(t):
    """Device/host pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def spmv_status_string(status):
    return load().spmv_status_string(int(status)).decode()


def spmv_default_options(**overrides):
    o = spmv_options_t()
    _check(load().spmv_default_options(ctypes.byref(o)), "spmv_default_options")
    for k, v in overrides.items():
        setattr(o, k, int(v))
    return o


def cg_default_options(**overrides):
    o = cg_options_t()
    _check(load().cg_default_options(ctypes.byref(o)), "cg_default_options")
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def spmv_create(n, row_ptr, col_idx, values, options=None, stream=None, raw_status=False,
                n_cols=None):
    """Create a handle from CSR given as numpy host arrays or torch device tensors
    (int32 row_ptr/col_idx, float64 values); n rows, n_cols columns (default n).
    Returns the handle (an int)."""
    L = load()
    on_dev = not isinstance(row_ptr, np.ndarray)
    if not on_dev:
        row_ptr = np.ascontiguousarray(row_ptr, np.int32)
        col_idx = np.ascontiguousarray(col_idx, np.int32)
        values = np.ascontiguousarray(values, np.float64)
        nnz = int(col_idx.size)
    else:
        nnz = int(col_idx.numel())
    h = _P()
    st = L.spmv_create(int(n), int(n if n_cols is None else n_cols), nnz, _ptr(row_ptr),
                       _ptr(col_idx), _ptr(values),
                       int(on_dev), ctypes.byref(options) if options is not None else None,
                       _stream(stream), ctypes.byref(h))
    if raw_status:
        return st, h.value
    _check(st, "spmv_create")
    return h.value


def spmv_destroy(h):
    _check(load().spmv_destroy(h), "spmv_destroy")


def spmv_get_info(h):
    info = spmv_info_t()
    _check(load().spmv_get_info(h, ctypes.byref(info)), "spmv_get_info")
    out = {}
    for f, _ in spmv_info_t._fields_:
        v = getattr(info, f)
        out[f] = ([list(r) for r in v] if f == "spmm_form" else
                  list(v) if f == "chain_form" else v)
    return out


def spmv_verify(h, stream=None):
    """Run the structure checks on a handle; returns the SPMV_CHECK_* bits violated (0 = none)."""
    v = _int(0)
    st = load().spmv_verify(h, ctypes.byref(v), _stream(stream))
    if st not in (SPMV_OK, SPMV_ERR_INVALID_CSR):
        raise SpmvError(st, "spmv_verify")
    return v.value


def spmv_device_status(h, stream=None):
    """SPMV_ERR_TIMEOUT when a kernel on the handle gave up a bounded wait since the last call,
    else SPMV_OK (the record is cleared)."""
    st = load().spmv_device_status(h, _stream(stream))
    if st not in (SPMV_OK, SPMV_ERR_TIMEOUT):
        raise SpmvError(st, "spmv_device_status")
    return st


def spmv_diag_bulk_timeout(h, stream=None):
    """Self-test of the staged product's bounded wait; returns the status (SPMV_ERR_TIMEOUT is
    the expected outcome)."""
    return load().spmv_diag_bulk_timeout(h, _stream(stream))


def spmv_diag_cg_timing(h, iters, stream=None):
    """Per-iteration times (ms) of an FP64 CG iteration: graph batch, direct launches, the three
    kernels each alone, and a scalar read-back (spmv_diag_cg_timing)."""
    out = np.zeros(6)
    _check(load().spmv_diag_cg_timing(h, int(iters), out.ctypes.data, _stream(stream)),
           "spmv_diag_cg_timing")
    return dict(zip(("graph_per_iter", "direct_per_iter", "product", "update_xr", "update_p",
                     "scalar_readback"), out.tolist()))


def spmv_diag_checks(h, stream=None):
    """Self-test of the checks: returns (planted, detected) fault bits."""
    p, d = _int(0), _int(0)
    _check(load().spmv_diag_checks(h, ctypes.byref(p), ctypes.byref(d), _stream(stream)),
           "spmv_diag_checks")
    return p.value, d.value


def spmv_get_permutation(h, n):
    perm = np.empty(n, np.int32)
    _check(load().spmv_get_permutation(h, perm.ctypes.data), "spmv_get_permutation")
    return perm


def spmv_export_csr(h, n, nnz, with_values=True):
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(nnz, np.int32)
    v = np.empty(nnz, np.float64) if with_values else None
    _check(load().spmv_export_csr(h, rp.ctypes.data, ci.ctypes.data, _ptr(v)), "spmv_export_csr")
    return rp, ci, v


def spmv_export_sell(h, with_values=True):
    info = spmv_get_info(h)
    ns, ne = info["n_slices"], info["sell_entries"]
    sp = np.empty(ns + 1, np.int64)
    col = np.empty(ne, np.int32)
    val = np.empty(ne, np.float64) if with_values else None
    cs = np.empty(ns, np.int32)
    ce = np.empty(ns, np.int32)
    _check(load().spmv_export_sell(h, sp.ctypes.data, col.ctypes.data, _ptr(val), cs.ctypes.data,
                                   ce.ctypes.data), "spmv_export_sell")
    return sp, col, val, cs, ce


def spmv_apply(h, x, y, stream=None):
    _check(load().spmv_apply(h, _ptr(x), _ptr(y), _stream(stream)), "spmv_apply")


def _host_ptr(a):
    """Address of a host array: a C-contiguous float64 numpy array or a CPU torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host vectors must be C-contiguous float64")
        return a.ctypes.data
    if a.device.type != "cpu" or a.dtype != torch_float64() or not a.is_contiguous():
        raise ValueError("host vectors must be contiguous float64 CPU tensors")
    return a.data_ptr()


def torch_float64():
    import torch
    return torch.float64


def spmv_apply_host(h, x_host, y_host, stream=None):
    """y = A x with x and y in host memory (copies pipelined with the product)."""
    _check(load().spmv_apply_host(h, _host_ptr(x_host), _host_ptr(y_host), _stream(stream)),
           "spmv_apply_host")


def spmv_apply_host_async(h, x_host, y_host, stream=None):
    """The same, enqueued on `stream` without waiting (y_host valid once the stream is done)."""
    _check(load().spmv_apply_host_async(h, _host_ptr(x_host), _host_ptr(y_host),
                                        _stream(stream)), "spmv_apply_host_async")


def spmv_apply_axpby(h, alpha, x, beta, y, stream=None):
    _check(load().spmv_apply_axpby(h, float(alpha), _ptr(x), float(beta), _ptr(y),
                                   _stream(stream)), "spmv_apply_axpby")


def spmv_apply_axpby_f32(h, alpha, x, beta, y, stream=None):
    _check(load().spmv_apply_axpby_f32(h, float(alpha), _ptr(x), float(beta), _ptr(y),
                                       _stream(stream)), "spmv_apply_axpby_f32")


def spmv_apply_f32(h, x, y, stream=None):
    _check(load().spmv_apply_f32(h, _ptr(x), _ptr(y), _stream(stream)), "spmv_apply_f32")


def spmv_apply_chain(hb, hc, x, y, stream=None):
    """y = B (C x) without materialising C x."""
    _check(load().spmv_apply_chain(hb, hc, _ptr(x), _ptr(y), _stream(stream)), "spmv_apply_chain")


def spmv_apply_chain_f32(hb, hc, x, y, stream=None):
    """y = B (C x) in FP32 without writing C x (see spmv_apply_chain)."""
    _check(load().spmv_apply_chain_f32(hb, hc, _ptr(x), _ptr(y), _stream(stream)),
           "spmv_apply_chain_f32")


def spmv_apply_csr(h, x, y, stream=None):
    _check(load().spmv_apply_csr(h, _ptr(x), _ptr(y), _stream(stream)), "spmv_apply_csr")


def spmv_apply_multi(h, k, X, Y, stream=None):
    _check(load().spmv_apply_multi(h, int(k), _ptr(X), _ptr(Y), _stream(stream)),
           "spmv_apply_multi")


def spmv_apply_multi_f32(h, k, X, Y, stream=None):
    _check(load().spmv_apply_multi_f32(h, int(k), _ptr(X), _ptr(Y), _stream(stream)),
           "spmv_apply_multi_f32")


def spmv_permute(h, direction, x_in, x_out, stream=None):
    eb = x_in.element_size()
    _check(load().spmv_permute(h, int(direction), eb, _ptr(x_in), _ptr(x_out), _stream(stream)),
           "spmv_permute")


def cg_solve(h, b, x, options=None, stream=None, raise_on_error=True):
    """Returns the cg_result_t as a dict (status included)."""
    opt = options if options is not None else cg_default_options()
    res = cg_result_t()
    st = load().cg_solve(h, _ptr(b), _ptr(x), ctypes.byref(opt), ctypes.byref(res),
                         _stream(stream))
    out = dict(iterations=res.iterations, outer_iterations=res.outer_iterations,
               rel_residual=res.rel_residual, status=st)
    if raise_on_error and st not in (SPMV_OK,):
        raise SpmvError(st, "cg_solve")
    return out


def cg_solve_multi(h, k, B, X, options=None, stream=None):
    """k right-hand sides in lock-step; B, X row-major n x k device tensors.  Returns
    (status, [per-column result dicts])."""
    opt = options if options is not None else cg_default_options()
    res = (cg_result_t * int(k))()
    st = load().cg_solve_multi(h, int(k), _ptr(B), _ptr(X), ctypes.byref(opt), res,
                               _stream(stream))
    cols = [dict(iterations=r.iterations, outer_iterations=r.outer_iterations,
                 rel_residual=r.rel_residual, status=r.status) for r in res]
    return st, cols


class Partition:
    """One part of a row-block partition (spmv_partition_*): the host plan (halo, send lists,
    the part's CSR) and, with on_device, its device handle."""

    def __init__(self, n, row_ptr, col_idx, values, row_begin, part, on_device=True,
                 stream=None, **options):
        row_ptr = np.ascontiguousarray(row_ptr, np.int32)
        col_idx = np.ascontiguousarray(col_idx, np.int32)
        values = np.ascontiguousarray(values, np.float64)
        rb = np.ascontiguousarray(row_begin, np.int32)
        h = _P()
        opt = spmv_default_options(**options)
        _check(load().spmv_partition_create(int(n), int(col_idx.size), row_ptr.ctypes.data,
                                            col_idx.ctypes.data, values.ctypes.data,
                                            int(rb.size - 1), rb.ctypes.data, int(part),
                                            int(bool(on_device)), ctypes.byref(opt),
                                            _stream(stream) if on_device else None,
                                            ctypes.byref(h)), "spmv_partition_create")
        self.handle = h.value
        self.n_parts = int(rb.size - 1)
        info = spmv_part_info_t()
        _check(load().spmv_partition_info(self.handle, ctypes.byref(info)), "spmv_partition_info")
        self.info = {f: getattr(info, f) for f, _ in spmv_part_info_t._fields_}
        sc = np.zeros(self.n_parts, np.int32)
        rc = np.zeros(self.n_parts, np.int32)
        sr = np.zeros(max(1, self.info["send_total"]), np.int32)
        hc = np.zeros(max(1, self.info["recv_total"]), np.int32)
        _check(load().spmv_partition_lists(self.handle, sc.ctypes.data, rc.ctypes.data,
                                           sr.ctypes.data, hc.ctypes.data),
               "spmv_partition_lists")
        self.send_counts, self.recv_counts = sc, rc
        self.send_rows = sr[:self.info["send_total"]]
        self.halo_cols = hc[:self.info["recv_total"]]

    def local_csr(self):
        nl, nz = self.info["n_local"], self.info["nnz_local"]
        rp = np.zeros(nl + 1, np.int32)
        ci = np.zeros(max(1, nz), np.int32)
        v = np.zeros(max(1, nz), np.float64)
        _check(load().spmv_partition_local_csr(self.handle, rp.ctypes.data, ci.ctypes.data,
                                               v.ctypes.data), "spmv_partition_local_csr")
        return rp, ci[:nz], v[:nz]

    def pack(self, x_own, send, stream=None):
        _check(load().spmv_partition_pack(self.handle, _ptr(x_own), _ptr(send), _stream(stream)),
               "spmv_partition_pack")

    def apply(self, x_ext, y, stream=None):
        _check(load().spmv_partition_apply(self.handle, _ptr(x_ext), _ptr(y), _stream(stream)),
               "spmv_partition_apply")

    def solve(self, b, x, exchange, allreduce, stream=None, **cg_opts):
        """cg_solve_partitioned with Python transport callbacks exchange(send_ptr, recv_ptr)
        and allreduce(values: numpy view) (each returns nothing; an exception fails the
        solve)."""
        def ex(send_p, recv_p, _ctx):
            try:
                exchange(send_p, recv_p)
                return 0
            except Exception:  # reported to the C side as a failed transport
                return 1

        def ar(vals, count, _ctx):
            try:
                allreduce(np.ctypeslib.as_array(vals, shape=(count,)))
                return 0
            except Exception:
                return 1
        ex_c, ar_c = EXCHANGE_FN(ex), ALLREDUCE_FN(ar)
        res = cg_result_t()
        st = load().cg_solve_partitioned(self.handle, _ptr(b), _ptr(x),
                                         ctypes.byref(cg_default_options(**cg_opts)),
                                         ctypes.byref(res), ex_c, ar_c, None, _stream(stream))
        return dict(iterations=res.iterations, outer_iterations=res.outer_iterations,
                    rel_residual=res.rel_residual, status=st)

    def close(self):
        if getattr(self, "handle", None):
            load().spmv_partition_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SPMV_NOALLOC_MAX_ROWS = 65536


def cg_solve_csr_noalloc(n, row_ptr, col_idx, values, b, x, options=None, stream=None):
    """Allocation-free CG on device CSR tensors; returns the result dict (status included)."""
    opt = options if options is not None else cg_default_options()
    res = cg_result_t()
    nnz = int(col_idx.numel()) if col_idx is not None else 0
    st = load().cg_solve_csr_noalloc(int(n), nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(values),
                                     _ptr(b), _ptr(x), ctypes.byref(opt), ctypes.byref(res),
                                     _stream(stream))
    return dict(iterations=res.iterations, outer_iterations=res.outer_iterations,
                rel_residual=res.rel_residual, status=st)


def spmv_server_create(budget_bytes, max_slots):
    s = _P()
    _check(load().spmv_server_create(int(budget_bytes), int(max_slots), ctypes.byref(s)),
           "spmv_server_create")
    return s.value


def spmv_server_submit(s, n, row_ptr, col_idx, values, b, options=None):
    row_ptr = np.ascontiguousarray(row_ptr, np.int32)
    col_idx = np.ascontiguousarray(col_idx, np.int32)
    values = np.ascontiguousarray(values, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    opt = options if options is not None else cg_default_options()
    t = ctypes.c_uint64()
    _check(load().spmv_server_submit(s, int(n), int(col_idx.size), row_ptr.ctypes.data,
                                     col_idx.ctypes.data, values.ctypes.data, b.ctypes.data,
                                     ctypes.byref(opt), ctypes.byref(t)), "spmv_server_submit")
    return t.value


def spmv_server_poll(s, ticket, x_out):
    """Returns None while pending, else the result dict (x_out filled)."""
    res = cg_result_t()
    st = load().spmv_server_poll(s, ctypes.c_uint64(ticket), x_out.ctypes.data, ctypes.byref(res))
    if st == SPMV_ERR_PENDING:
        return None
    return dict(iterations=res.iterations, outer_iterations=res.outer_iterations,
                rel_residual=res.rel_residual, status=st)


def spmv_server_get_stats(s):
    stt = spmv_server_stats_t()
    _check(load().spmv_server_get_stats(s, ctypes.byref(stt)), "spmv_server_get_stats")
    return {f: getattr(stt, f) for f, _ in spmv_server_stats_t._fields_}


def spmv_server_set_priority_bytes(s, nbytes):
    _check(load().spmv_server_set_priority_bytes(s, int(nbytes)), "spmv_server_set_priority_bytes")


def spmv_server_cancel(s, ticket):
    """Cancel a queued or running request; its poll then reports SPMV_ERR_CANCELLED."""
    _check(load().spmv_server_cancel(s, ctypes.c_uint64(ticket)), "spmv_server_cancel")


def spmv_server_destroy(s):
    _check(load().spmv_server_destroy(s), "spmv_server_destroy")


class Matrix:
    """Owning wrapper of a matrix handle (destroyed with the object)."""

    def __init__(self, n, row_ptr, col_idx, values, stream=None, n_cols=None, **options):
        self.n = int(n)
        self.n_cols = int(n if n_cols is None else n_cols)
        self.nnz = int(col_idx.size if isinstance(col_idx, np.ndarray) else col_idx.numel())
        self.options = spmv_default_options(**options)
        self.handle = spmv_create(self.n, row_ptr, col_idx, values, self.options, stream,
                                  n_cols=self.n_cols)

    def info(self):
        return spmv_get_info(self.handle)

    def apply(self, x, y, stream=None):
        spmv_apply(self.handle, x, y, stream)

    def apply_host(self, x_host, y_host, stream=None):
        spmv_apply_host(self.handle, x_host, y_host, stream)

    def apply_host_async(self, x_host, y_host, stream=None):
        spmv_apply_host_async(self.handle, x_host, y_host, stream)

    def apply_f32(self, x, y, stream=None):
        spmv_apply_f32(self.handle, x, y, stream)

    def apply_axpby(self, alpha, x, beta, y, stream=None):
        if x.dtype.itemsize == 4:
            spmv_apply_axpby_f32(self.handle, alpha, x, beta, y, stream)
        else:
            spmv_apply_axpby(self.handle, alpha, x, beta, y, stream)

    def apply_csr(self, x, y, stream=None):
        spmv_apply_csr(self.handle, x, y, stream)

    def apply_multi(self, X, Y, stream=None):
        if X.dtype.itemsize == 4:
            spmv_apply_multi_f32(self.handle, X.shape[1], X, Y, stream)
        else:
            spmv_apply_multi(self.handle, X.shape[1], X, Y, stream)

    def permutation(self):
        return spmv_get_permutation(self.handle, self.n)

    def permute(self, direction, x_in, x_out, stream=None):
        spmv_permute(self.handle, direction, x_in, x_out, stream)

    def solve(self, b, x, stream=None, raise_on_error=True, **cg_opts):
        return cg_solve(self.handle, b, x, cg_default_options(**cg_opts), stream, raise_on_error)

    def solve_multi(self, B, X, stream=None, **cg_opts):
        """B, X: n x k row-major device tensors; returns (status, per-column results)."""
        return cg_solve_multi(self.handle, B.shape[1], B, X, cg_default_options(**cg_opts),
                              stream)

    def close(self):
        if getattr(self, "handle", None):
            spmv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
