"""CPU oracle for the msRep SpMV hot path (arXiv 2209.07552).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package entry module's
``smoke()`` check and the benchmark's CPU-baseline leg may import this
package.  The product library never loads it and shares no code with it.

The arithmetic lives in ``msrep_oracle.c`` (plain single-threaded C11, FP64,
``-ffp-contract=off``), compiled on first use with gcc into ``oracle/_build``.
This module only marshals numpy arrays into it.  Each wrapper names the
passage of the paper that the C function follows; the readings of garbled or
silent passages are listed at the top of ``msrep_oracle.c``.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(dense matvec, closed forms, brute force, invariants) except where the
function's docstring says "parity unpinned".
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msrep_oracle.c")
_LOCK = threading.Lock()
_LIB = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)


def build() -> str:
    """Compile msrep_oracle.c into oracle/_build and return the .so path."""
    with open(_SRC, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, f"libmsrep_oracle_{tag}.so")
    if not os.path.exists(so):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            lib.ref_partition_compressed.argtypes = [
                ctypes.c_int32, ctypes.c_int64, _i32p, ctypes.c_int32,
                _i32p, _i32p, _i32p, _i32p, _u8p]
            lib.ref_partition_compressed.restype = ctypes.c_int
            lib.ref_partition_merge_path.argtypes = [
                ctypes.c_int32, ctypes.c_int64, _i32p, ctypes.c_int32,
                _i32p, _i32p, _i32p, _i32p, _u8p, _i32p]
            lib.ref_partition_merge_path.restype = ctypes.c_int
            lib.ref_partition_row_block.argtypes = [
                ctypes.c_int32, ctypes.c_int64, _i32p, ctypes.c_int32,
                _i32p, _i32p, _i32p, _i32p, _u8p]
            lib.ref_partition_row_block.restype = ctypes.c_int
            lib.ref_partition_coo_row_block.argtypes = [
                ctypes.c_int64, _i32p, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                _i32p, _i32p, _u8p]
            lib.ref_partition_coo_row_block.restype = ctypes.c_int
            lib.ref_local_offsets.argtypes = [ctypes.c_int32, _i32p, _i32p, _i64p]
            lib.ref_local_offsets.restype = ctypes.c_int64
            lib.ref_partition_local_compressed.argtypes = [
                _i32p, ctypes.c_int32, _i32p, _i32p, _i32p, _i32p, _i64p, _i32p]
            lib.ref_partition_coo.argtypes = [
                ctypes.c_int64, _i32p, ctypes.c_int32, _i32p, _i32p, _i32p,
                _i32p, _u8p]
            lib.ref_partition_coo.restype = ctypes.c_int
            lib.ref_partition_coo_unsorted.argtypes = [
                ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                _i32p, _i32p, _u8p]
            lib.ref_partition_coo_unsorted.restype = ctypes.c_int
            lib.ref_pspmv_coo_scatter.argtypes = [
                ctypes.c_int32, _i32p, _i32p, _f64p, ctypes.c_int32, _i32p,
                _i32p, ctypes.c_double, _f64p, ctypes.c_double, _f64p]
            lib.ref_pspmv_coo_scatter.restype = ctypes.c_int
            lib.ref_partition_local_coo.argtypes = [
                _i32p, ctypes.c_int32, _i32p, _i32p, _i32p, _i32p]
            lib.ref_spmv_csr.argtypes = [
                ctypes.c_int32, _i32p, _i32p, _f64p, ctypes.c_double, _f64p,
                ctypes.c_double, _f64p]
            lib.ref_spmv_csr.restype = None
            lib.ref_spmv_csc.argtypes = [
                ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _f64p,
                ctypes.c_double, _f64p, ctypes.c_double, _f64p]
            lib.ref_spmv_csc.restype = None
            lib.ref_spmv_coo.argtypes = [
                ctypes.c_int32, ctypes.c_int64, _i32p, _i32p, _f64p,
                ctypes.c_double, _f64p, ctypes.c_double, _f64p]
            lib.ref_spmv_coo.restype = None
            lib.ref_spmm_csr.argtypes = [
                ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _f64p,
                ctypes.c_double, _f64p, ctypes.c_double, _f64p]
            lib.ref_spmm_csr.restype = None
            for name in ("ref_pspmv_csr", "ref_pspmv_csc", "ref_pspmv_coo"):
                getattr(lib, name).argtypes = [
                    ctypes.c_int32, _i32p, _i32p, _f64p, ctypes.c_int32,
                    _i32p, _i32p, _i32p, _i32p, ctypes.c_double, _f64p,
                    ctypes.c_double, _f64p]
                getattr(lib, name).restype = ctypes.c_int
            lib.ref_two_sum_f32.argtypes = [ctypes.c_float, ctypes.c_float,
                                            _f32p, _f32p]
            lib.ref_two_sum_f32.restype = None
            lib.ref_sum_f32.argtypes = [_f32p, ctypes.c_int64]
            lib.ref_sum_f32.restype = ctypes.c_float
            lib.ref_sum2_f32.argtypes = [_f32p, ctypes.c_int64]
            lib.ref_sum2_f32.restype = ctypes.c_float
            _LIB = lib
    return _LIB


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


# --------------------------------------------------------------------------
# Partitioning: Alg. 2 (pCSR), Alg. 4 (pCSC), Alg. 6 (pCOO).
# --------------------------------------------------------------------------

def _partition_compressed(ptr, nnz: int, np_: int, with_local: bool,
                          merge_path: bool = False, row_block: bool = False):
    ptr = _c(ptr, np.int32)
    n_major = ptr.shape[0] - 1
    out = {k: np.empty(np_, np.int32) for k in
           ("start_idx", "end_idx", "start_major", "end_major")}
    out["start_flag"] = np.empty(np_, np.uint8)
    if merge_path:
        out["cut_row"] = np.empty(np_ + 1, np.int32)
        rc = _lib().ref_partition_merge_path(
            n_major, nnz, _p(ptr, _i32p), np_, _p(out["start_idx"], _i32p),
            _p(out["end_idx"], _i32p), _p(out["start_major"], _i32p),
            _p(out["end_major"], _i32p), _p(out["start_flag"], _u8p),
            _p(out["cut_row"], _i32p))
    elif row_block:
        rc = _lib().ref_partition_row_block(
            n_major, nnz, _p(ptr, _i32p), np_, _p(out["start_idx"], _i32p),
            _p(out["end_idx"], _i32p), _p(out["start_major"], _i32p),
            _p(out["end_major"], _i32p), _p(out["start_flag"], _u8p))
    else:
        rc = _lib().ref_partition_compressed(
            n_major, nnz, _p(ptr, _i32p), np_, _p(out["start_idx"], _i32p),
            _p(out["end_idx"], _i32p), _p(out["start_major"], _i32p),
            _p(out["end_major"], _i32p), _p(out["start_flag"], _u8p))
    if rc != 0:
        raise ValueError("invalid partition arguments")
    if with_local:
        off = np.empty(np_ + 1, np.int64)
        total = _lib().ref_local_offsets(
            np_, _p(out["start_major"], _i32p), _p(out["end_major"], _i32p),
            _p(off, _i64p))
        local = np.empty(max(total, 1), np.int32)
        _lib().ref_partition_local_compressed(
            _p(ptr, _i32p), np_, _p(out["start_idx"], _i32p),
            _p(out["end_idx"], _i32p), _p(out["start_major"], _i32p),
            _p(out["end_major"], _i32p), _p(off, _i64p), _p(local, _i32p))
        out["local_off"] = off
        out["local"] = local[:total]
    return out


def partition_csr(row_ptr, nnz: int, np_: int, with_local: bool = False):
    """CSR -> pCSR metadata, Alg. 2 (Sec. 3.2.1) under readings R2-R5.

    Returns start_idx, end_idx (inclusive), start_major (= start_row),
    end_major (= end_row), start_flag and, with ``with_local``, the
    concatenated local row pointers and their np+1 offsets."""
    return _partition_compressed(row_ptr, nnz, np_, with_local)


def partition_csc(col_ptr, nnz: int, np_: int, with_local: bool = False):
    """CSC -> pCSC metadata, Alg. 4 (Sec. 3.2.2): Alg. 2 over col_ptr."""
    return _partition_compressed(col_ptr, nnz, np_, with_local)


def partition_merge_path(ptr, nnz: int, np_: int, with_local: bool = False):
    """Row+nonzero merge-path partitioning of CSR (row_ptr) or CSC (col_ptr),
    reading R10: cuts at equal steps of the merged sequence of row ends and
    nonzeros, metadata as Alg. 2 for each cut's nonzero range.  Also returns
    ``cut_row``, the row coordinate of each of the np+1 cuts."""
    return _partition_compressed(ptr, nnz, np_, with_local, merge_path=True)


def partition_row_block(ptr, nnz: int, np_: int, with_local: bool = False):
    """The Baseline row-block partitioning of Sec. 5.1 (reading R11) of CSR
    (row_ptr) or CSC (col_ptr): np blocks of equal row (column) count, each
    with all of its nonzeros; metadata as Alg. 2 gives them for each block's
    nonzero range."""
    return _partition_compressed(ptr, nnz, np_, with_local, row_block=True)


def partition_coo_row_block(row_idx, m: int, np_: int, with_local: bool = False):
    """The Baseline row-block partitioning (reading R11) of row-sorted COO:
    block i holds the nonzeros of rows floor(i*m/np) .. floor((i+1)*m/np)-1,
    found by scanning row_idx."""
    row_idx = _c(row_idx, np.int32)
    nnz = row_idx.shape[0]
    out = {k: np.empty(np_, np.int32) for k in
           ("start_idx", "end_idx", "start_major", "end_major")}
    out["start_flag"] = np.empty(np_, np.uint8)
    rc = _lib().ref_partition_coo_row_block(
        nnz, _p(row_idx, _i32p), m, np_, _p(out["start_idx"], _i32p),
        _p(out["end_idx"], _i32p), _p(out["start_major"], _i32p),
        _p(out["end_major"], _i32p), _p(out["start_flag"], _u8p))
    if rc != 0:
        raise ValueError("invalid partition arguments")
    if with_local:
        lrow = np.empty(max(nnz, 1), np.int32)
        _lib().ref_partition_local_coo(
            _p(row_idx, _i32p), np_, _p(out["start_idx"], _i32p),
            _p(out["end_idx"], _i32p), _p(out["start_major"], _i32p),
            _p(lrow, _i32p))
        out["local"] = lrow[:nnz]
    return out


def partition_coo(row_idx, np_: int, with_local: bool = False):
    """Row-sorted COO -> pCOO metadata, Alg. 6 (Sec. 3.2.3), reading R8.

    With ``with_local`` also the local row-index array of Sec. 4.1
    (``local``, length nnz; partition i starts at ``start_idx[i]``)."""
    row_idx = _c(row_idx, np.int32)
    nnz = row_idx.shape[0]
    out = {k: np.empty(np_, np.int32) for k in
           ("start_idx", "end_idx", "start_major", "end_major")}
    out["start_flag"] = np.empty(np_, np.uint8)
    rc = _lib().ref_partition_coo(
        nnz, _p(row_idx, _i32p), np_, _p(out["start_idx"], _i32p),
        _p(out["end_idx"], _i32p), _p(out["start_major"], _i32p),
        _p(out["end_major"], _i32p), _p(out["start_flag"], _u8p))
    if rc != 0:
        raise ValueError("invalid partition arguments")
    if with_local:
        lrow = np.empty(max(nnz, 1), np.int32)
        _lib().ref_partition_local_coo(
            _p(row_idx, _i32p), np_, _p(out["start_idx"], _i32p),
            _p(out["end_idx"], _i32p), _p(out["start_major"], _i32p),
            _p(lrow, _i32p))
        out["local"] = lrow[:nnz]
    return out


def partition_coo_by_col(col_idx, np_: int, with_local: bool = False):
    """pCOO of a COO matrix sorted by (col, row), reading R9: Alg. 6 with
    the column index as the major index (start/end column, split-column
    flag; with ``with_local`` the local column index col - start_col)."""
    return partition_coo(col_idx, np_, with_local)


def partition_coo_unsorted(row_idx, m: int, np_: int, with_local: bool = False):
    """pCOO of a COO matrix in no particular order, reading R9: the
    nonzero ranges of Alg. 6; every non-empty partition spans rows
    0..m-1, flags 0.  With ``with_local``, the local row index relative to
    start_row = 0, i.e. the row index itself."""
    row_idx = _c(row_idx, np.int32)
    nnz = row_idx.shape[0]
    out = {k: np.empty(np_, np.int32) for k in
           ("start_idx", "end_idx", "start_major", "end_major")}
    out["start_flag"] = np.empty(np_, np.uint8)
    rc = _lib().ref_partition_coo_unsorted(
        nnz, m, np_, _p(out["start_idx"], _i32p), _p(out["end_idx"], _i32p),
        _p(out["start_major"], _i32p), _p(out["end_major"], _i32p),
        _p(out["start_flag"], _u8p))
    if rc != 0:
        raise ValueError("invalid partition arguments")
    if with_local:
        lrow = np.empty(max(nnz, 1), np.int32)
        _lib().ref_partition_local_coo(
            _p(row_idx, _i32p), np_, _p(out["start_idx"], _i32p),
            _p(out["end_idx"], _i32p), _p(out["start_major"], _i32p),
            _p(lrow, _i32p))
        out["local"] = lrow[:nnz]
    return out


# --------------------------------------------------------------------------
# Plain SpMV (Sec. 2.2, Alg. 1 reading R1).
# --------------------------------------------------------------------------

def _yin(y, m):
    if y is None:
        return np.zeros(m, np.float64)
    return _c(y, np.float64).copy()


def spmv_csr(m, row_ptr, col_idx, val, x, alpha=1.0, beta=0.0, y=None):
    """y = alpha*A*x + beta*y for CSR A: Alg. 1 (reading R1), FP64."""
    row_ptr = _c(row_ptr, np.int32)
    col_idx = _c(col_idx, np.int32)
    val = _c(val, np.float64)
    x = _c(x, np.float64)
    out = _yin(y, m)
    _lib().ref_spmv_csr(m, _p(row_ptr, _i32p), _p(col_idx, _i32p),
                        _p(val, _f64p), alpha, _p(x, _f64p), beta,
                        _p(out, _f64p))
    return out


def spmv_csc(m, n, col_ptr, row_idx, val, x, alpha=1.0, beta=0.0, y=None):
    """CSC SpMV: Alg. 1 with the roles of x and y switched (Sec. 2.2)."""
    col_ptr = _c(col_ptr, np.int32)
    row_idx = _c(row_idx, np.int32)
    val = _c(val, np.float64)
    x = _c(x, np.float64)
    out = _yin(y, m)
    _lib().ref_spmv_csc(m, n, _p(col_ptr, _i32p), _p(row_idx, _i32p),
                        _p(val, _f64p), alpha, _p(x, _f64p), beta,
                        _p(out, _f64p))
    return out


def spmv_coo(m, row_idx, col_idx, val, x, alpha=1.0, beta=0.0, y=None):
    """COO SpMV: one loop over the nonzeros (Sec. 2.2)."""
    row_idx = _c(row_idx, np.int32)
    col_idx = _c(col_idx, np.int32)
    val = _c(val, np.float64)
    x = _c(x, np.float64)
    out = _yin(y, m)
    _lib().ref_spmv_coo(m, row_idx.shape[0], _p(row_idx, _i32p),
                        _p(col_idx, _i32p), _p(val, _f64p), alpha,
                        _p(x, _f64p), beta, _p(out, _f64p))
    return out


def spmm_csr(m, row_ptr, col_idx, val, X, alpha=1.0, beta=0.0, Y=None):
    """Y = alpha*A*X + beta*Y for an n x k row-major block X: k applications
    of Alg. 1 (the multi-vector case Sec. 2.3 says behaves like SpMV)."""
    row_ptr = _c(row_ptr, np.int32)
    col_idx = _c(col_idx, np.int32)
    val = _c(val, np.float64)
    X = _c(X, np.float64)
    k = X.shape[1]
    out = np.zeros((m, k), np.float64) if Y is None else _c(Y, np.float64).copy()
    _lib().ref_spmm_csr(m, k, _p(row_ptr, _i32p), _p(col_idx, _i32p),
                        _p(val, _f64p), alpha, _p(X, _f64p), beta,
                        _p(out, _f64p))
    return out


# --------------------------------------------------------------------------
# The partitioned method with the paper's merge (Alg. 3, 5, 7).
# --------------------------------------------------------------------------

def _pspmv(fn, m, ptr_or_row, idx, val, part, x, alpha, beta, y):
    a = _c(ptr_or_row, np.int32)
    idx = _c(idx, np.int32)
    val = _c(val, np.float64)
    x = _c(x, np.float64)
    out = _yin(y, m)
    np_ = part["start_idx"].shape[0]
    pp = {k: _c(part[k], np.int32) for k in
          ("start_idx", "end_idx", "start_major", "end_major")}
    rc = fn(m, _p(a, _i32p), _p(idx, _i32p), _p(val, _f64p), np_,
            _p(pp["start_idx"], _i32p), _p(pp["end_idx"], _i32p),
            _p(pp["start_major"], _i32p), _p(pp["end_major"], _i32p),
            alpha, _p(x, _f64p), beta, _p(out, _f64p))
    assert rc == 0
    return out


def pspmv_csr(m, row_ptr, col_idx, val, part, x, alpha=1.0, beta=0.0, y=None):
    """Alg. 3: per-partition partial results, then the row merge (R6)."""
    return _pspmv(_lib().ref_pspmv_csr, m, row_ptr, col_idx, val, part, x,
                  alpha, beta, y)


def pspmv_csc(m, col_ptr, row_idx, val, part, x, alpha=1.0, beta=0.0, y=None):
    """Alg. 5: per-partition full partial vectors, summed (R7)."""
    return _pspmv(_lib().ref_pspmv_csc, m, col_ptr, row_idx, val, part, x,
                  alpha, beta, y)


def pspmv_coo(m, row_idx, col_idx, val, part, x, alpha=1.0, beta=0.0, y=None):
    """Alg. 7: the COO analogue of Alg. 3 on row-sorted input."""
    return _pspmv(_lib().ref_pspmv_coo, m, row_idx, col_idx, val, part, x,
                  alpha, beta, y)


def pspmv_coo_scatter(m, row_idx, col_idx, val, part, x, alpha=1.0, beta=0.0,
                      y=None):
    """Partitioned SpMV of a COO matrix sorted by column or in no order
    (reading R9): a full m-vector of partials per partition, summed in
    partition order."""
    row_idx = _c(row_idx, np.int32)
    col_idx = _c(col_idx, np.int32)
    val = _c(val, np.float64)
    x = _c(x, np.float64)
    out = _yin(y, m)
    np_ = part["start_idx"].shape[0]
    s = _c(part["start_idx"], np.int32)
    e = _c(part["end_idx"], np.int32)
    rc = _lib().ref_pspmv_coo_scatter(
        m, _p(row_idx, _i32p), _p(col_idx, _i32p), _p(val, _f64p), np_,
        _p(s, _i32p), _p(e, _i32p), alpha, _p(x, _f64p), beta, _p(out, _f64p))
    assert rc == 0
    return out


# --------------------------------------------------------------------------
# Binary32 summation helpers for the low-precision form.
# --------------------------------------------------------------------------

def two_sum_f32(a: float, b: float):
    """Knuth's TwoSum in binary32: (s, e) with a + b = s + e exactly."""
    s = ctypes.c_float()
    e = ctypes.c_float()
    _lib().ref_two_sum_f32(a, b, ctypes.byref(s), ctypes.byref(e))
    return s.value, e.value


def sum_f32(v) -> float:
    """Plain recursive binary32 summation."""
    v = _c(v, np.float32)
    return _lib().ref_sum_f32(_p(v, _f32p), v.shape[0])


def sum2_f32(v) -> float:
    """Compensated binary32 summation (cascaded TwoSum, 'Sum2' of Ogita,
    Rump and Oishi 2005)."""
    v = _c(v, np.float32)
    return _lib().ref_sum2_f32(_p(v, _f32p), v.shape[0])
