"""CPU oracle for the SpMV / CG path -- TEST INFRASTRUCTURE ONLY.

Plain, sequential FP64 C code (``oracle.c``) behind thin ctypes wrappers.  Only the test
suite, the package smoke check and the benchmark's CPU-baseline leg may import this
package.  It shares no code with the CUDA library and never imports it.

Pinned by tests/test_oracle_*.py against dense brute force, closed-form eigenpairs,
invariants of the matrices, hand-worked orderings and textbook special cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_i32 = ctypes.c_int32
_int = ctypes.c_int
_f64 = ctypes.c_double
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PF64 = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, no FP contraction) into liboracle.so."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cc = os.environ.get("CC", "gcc")
    subprocess.check_call([cc, "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _configure(L):
    """Argument and result types of the oracle's C functions on a loaded library."""
    L.oracle_csr_spmv.argtypes = [_i32, _i32p, _i32p, _f64p, _f64p, _f64p, _int]
    L.oracle_csr_spmv.restype = None
    L.oracle_csr_spmv_f32.argtypes = [_i32, _i32p, _i32p, _f32p, _f32p, _f32p, _int]
    L.oracle_csr_spmv_f32.restype = None
    L.oracle_csr_spmv_axpby.argtypes = [_i32, _i32p, _i32p, _f64p, _f64, _f64p, _f64, _f64p]
    L.oracle_csr_spmv_axpby.restype = None
    L.oracle_spmm.argtypes = [_i32, _i32p, _i32p, _f64p, _i32, _f64p, _f64p, _int]
    L.oracle_spmm.restype = None
    L.oracle_spmm_f32.argtypes = [_i32, _i32p, _i32p, _f32p, _i32, _f32p, _f32p, _int]
    L.oracle_spmm_f32.restype = None
    L.oracle_cm_order.argtypes = [_i32, _i32p, _i32p, _int, _int, _i32p]
    L.oracle_cm_order.restype = _int
    L.oracle_sigma_sort.argtypes = [_i32, _i32p, ctypes.c_void_p, _i32, _i32p]
    L.oracle_sigma_sort.restype = _int
    L.oracle_permute_csr.argtypes = [_i32, _i32p, _i32p, _f64p, _i32p, _i32p, _i32p, _f64p]
    L.oracle_permute_csr.restype = _int
    L.oracle_sell_slice_ptr.argtypes = [_i32, _i32p, _i32, _i64p]
    L.oracle_sell_slice_ptr.restype = ctypes.c_int64
    L.oracle_sell_fill.argtypes = [_i32, _i32p, _i32p, _f64p, _i32, _i64p, _i32p, _f64p]
    L.oracle_sell_fill.restype = None
    L.oracle_window_meta.argtypes = [_i32, _i32, _i64p, _i32p, _i32p, _i32p]
    L.oracle_window_meta.restype = None
    L.oracle_jacobi_pcg.argtypes = [_i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64, _i32,
                                    _i32, _PI32, _PF64, _PF64]
    L.oracle_jacobi_pcg.restype = _int
    L.oracle_mixed_ir.argtypes = [_i32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64, _f64, _i32,
                                  _i32, _int, _PI32, _PI32, _PF64]
    L.oracle_mixed_ir.restype = _int
    return L


def _csr(row_ptr, col_idx):
    return (np.ascontiguousarray(row_ptr, dtype=np.int32),
            np.ascontiguousarray(col_idx, dtype=np.int32))


def spmv(row_ptr, col_idx, values, x, use_fma=False):
    """y = A x, FP64, CSR order."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    y = np.empty(n)
    lib().oracle_csr_spmv(n, rp, ci, np.ascontiguousarray(values, np.float64),
                          np.ascontiguousarray(x, np.float64), y, int(use_fma))
    return y


def spmv_axpby(row_ptr, col_idx, values, alpha, x, beta, y):
    """y = alpha (A x) + beta y (returns a new array; beta == 0 ignores y)."""
    rp, ci = _csr(row_ptr, col_idx)
    out = np.array(y, dtype=np.float64, copy=True)
    lib().oracle_csr_spmv_axpby(rp.size - 1, rp, ci, np.ascontiguousarray(values, np.float64),
                                float(alpha), np.ascontiguousarray(x, np.float64), float(beta),
                                out)
    return out


def spmv_f32(row_ptr, col_idx, values32, x32, use_fma=True):
    """y = A x with FP32 values, vector and accumulator."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    y = np.empty(n, np.float32)
    lib().oracle_csr_spmv_f32(n, rp, ci, np.ascontiguousarray(values32, np.float32),
                              np.ascontiguousarray(x32, np.float32), y, int(use_fma))
    return y


def spmm(row_ptr, col_idx, values, X, use_fma=False):
    """Y = A X for a row-major block X (n_cols x k), as k independent SpMVs."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    X = np.ascontiguousarray(X)
    k = X.shape[1]
    if X.dtype == np.float32:
        Y = np.empty((n, k), np.float32)
        lib().oracle_spmm_f32(n, rp, ci, np.ascontiguousarray(values, np.float32), k, X, Y,
                              int(use_fma))
    else:
        Y = np.empty((n, k))
        lib().oracle_spmm(n, rp, ci, np.ascontiguousarray(values, np.float64), k,
                          np.ascontiguousarray(X, np.float64), Y, int(use_fma))
    return Y


def cm_order(row_ptr, col_idx, reverse=True, peripheral=True):
    """Cuthill-McKee (reverse=False) or reverse Cuthill-McKee order; perm[new] = old."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    perm = np.empty(n, np.int32)
    rc = lib().oracle_cm_order(n, rp, ci, int(reverse), int(peripheral), perm)
    if rc != 0:
        raise RuntimeError("oracle_cm_order failed: %d" % rc)
    return perm


def sigma_sort(row_ptr, sigma, perm_in=None):
    """Rows (in the order perm_in, default identity) sorted by decreasing length inside windows
    of sigma positions, ties kept in order; returns perm[new] = old."""
    rp = np.ascontiguousarray(row_ptr, np.int32)
    n = rp.size - 1
    out = np.empty(n, np.int32)
    pin = None if perm_in is None else np.ascontiguousarray(perm_in, np.int32)
    rc = lib().oracle_sigma_sort(n, rp, None if pin is None else pin.ctypes.data, int(sigma), out)
    if rc != 0:
        raise RuntimeError("oracle_sigma_sort failed: %d" % rc)
    return out


def permute_csr(row_ptr, col_idx, values, perm):
    """B = P A P^T with perm[new] = old; rows sorted by new column."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    rpo = np.empty(n + 1, np.int32)
    cio = np.empty(ci.size, np.int32)
    vo = np.empty(ci.size)
    rc = lib().oracle_permute_csr(n, rp, ci, np.ascontiguousarray(values, np.float64),
                                  np.ascontiguousarray(perm, np.int32), rpo, cio, vo)
    if rc != 0:
        raise RuntimeError("oracle_permute_csr failed: %d" % rc)
    return rpo, cio, vo


def sell(row_ptr, col_idx, values, S):
    """Sliced ELLPACK arrays (slice_ptr int64[n_slices+1], col int32, val float64)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    n_slices = (n + S - 1) // S
    sp = np.empty(n_slices + 1, np.int64)
    total = lib().oracle_sell_slice_ptr(n, rp, S, sp)
    scol = np.empty(total, np.int32)
    sval = np.empty(total)
    lib().oracle_sell_fill(n, rp, ci, np.ascontiguousarray(values, np.float64), S, sp, scol, sval)
    return sp, scol, sval


def window_meta(n, S, slice_ptr, sell_col):
    """Per-slice (col_start, col_end) of the multiplying vector."""
    n_slices = (n + S - 1) // S
    cs = np.empty(n_slices, np.int32)
    ce = np.empty(n_slices, np.int32)
    lib().oracle_window_meta(n, S, np.ascontiguousarray(slice_ptr, np.int64),
                             np.ascontiguousarray(sell_col, np.int32), cs, ce)
    return cs, ce


def jacobi_pcg(row_ptr, col_idx, values, b, x0=None, rtol=1e-10, max_iter=100000,
               max_restarts=2):
    """Jacobi-preconditioned CG in FP64.  Returns (x, info dict)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    tr = ctypes.c_double(0.0)
    rc = lib().oracle_jacobi_pcg(n, rp, ci, np.ascontiguousarray(values, np.float64),
                                 np.ascontiguousarray(b, np.float64), x, rtol, max_iter,
                                 max_restarts, ctypes.byref(it), ctypes.byref(rr),
                                 ctypes.byref(tr))
    if rc < 0:
        raise RuntimeError("oracle_jacobi_pcg failed: %d" % rc)
    return x, dict(converged=(rc == 0), iterations=it.value, rel_residual=rr.value,
                   true_rel_residual=tr.value)


def mixed_ir(row_ptr, col_idx, values, b, rtol=1e-10, inner_rtol=1e-4, inner_max_iter=1000,
             max_outer=20, adaptive=True):
    """FP32 inner Jacobi-PCG with FP64 iterative refinement.  Returns (x, info dict)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    x = np.zeros(n)
    outer = ctypes.c_int32(0)
    inner = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    rc = lib().oracle_mixed_ir(n, rp, ci, np.ascontiguousarray(values, np.float64),
                               np.ascontiguousarray(b, np.float64), x, rtol, inner_rtol,
                               inner_max_iter, max_outer, int(adaptive), ctypes.byref(outer),
                               ctypes.byref(inner), ctypes.byref(rr))
    if rc < 0:
        raise RuntimeError("oracle_mixed_ir failed: %d" % rc)
    return x, dict(converged=(rc == 0), outer_iterations=outer.value,
                   inner_iterations=inner.value, rel_residual=rr.value)
