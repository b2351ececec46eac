"""All-core CPU baseline of the benchmark (``cpu_baseline.c``).

MEASUREMENT INFRASTRUCTURE ONLY, and not the oracle: bench.py times it
beside the single-threaded oracle so that the GPU numbers also stand next
to a CPU SpMV that uses every host core.  Nonzero-balanced partitions, one
OpenMP thread per partition, the partial sums of split rows (CSR, COO) or
the partial vectors (CSC) merged afterwards.  Built with gcc -fopenmp into
``oracle/_build``; the product library never loads it.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_baseline.c")
_LOCK = threading.Lock()
_LIB = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build() -> str:
    with open(_SRC, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, f"libcpu_baseline_{tag}.so")
    if not os.path.exists(so):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            lib.cpu_threads.restype = ctypes.c_int
            lib.cpu_spmv_csr.argtypes = [ctypes.c_int32, ctypes.c_int64, _i32p, _i32p, _f64p,
                                         _f64p, ctypes.c_double, _f64p]
            lib.cpu_spmv_coo.argtypes = lib.cpu_spmv_csr.argtypes
            lib.cpu_spmv_csc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _i32p,
                                         _i32p, _f64p, _f64p, ctypes.c_double, _f64p, _f64p]
            for f in (lib.cpu_spmv_csr, lib.cpu_spmv_coo, lib.cpu_spmv_csc):
                f.restype = ctypes.c_int
            _LIB = lib
    return _LIB


def threads() -> int:
    """Threads (= partitions) the baseline runs with (OMP_NUM_THREADS, else
    every host core)."""
    return _lib().cpu_threads()


def _p(a, t):
    return a.ctypes.data_as(t)


class Prepared:
    """One (matrix, format) pair with its arrays made contiguous, ready to
    be timed: ``run(x, y)`` computes y = A x."""

    def __init__(self, fmt: str, m: int, n: int, ptr, idx, val, row_idx=None):
        self.fmt, self.m, self.n = fmt, int(m), int(n)
        self.ptr = None if ptr is None else np.ascontiguousarray(ptr, np.int32)
        self.idx = np.ascontiguousarray(idx, np.int32)
        self.val = np.ascontiguousarray(val, np.float64)
        self.row_idx = None if row_idx is None else np.ascontiguousarray(row_idx, np.int32)
        self.nnz = int(self.idx.shape[0])
        self.part = (np.empty(threads() * self.m, np.float64) if fmt == "csc" else None)

    def run(self, x: np.ndarray, y: np.ndarray):
        L = _lib()
        if self.fmt == "csr":
            rc = L.cpu_spmv_csr(self.m, self.nnz, _p(self.ptr, _i32p), _p(self.idx, _i32p),
                                _p(self.val, _f64p), _p(x, _f64p), 1.0, _p(y, _f64p))
        elif self.fmt == "coo":
            rc = L.cpu_spmv_coo(self.m, self.nnz, _p(self.row_idx, _i32p), _p(self.idx, _i32p),
                                _p(self.val, _f64p), _p(x, _f64p), 1.0, _p(y, _f64p))
        else:
            rc = L.cpu_spmv_csc(self.m, self.n, self.nnz, _p(self.ptr, _i32p),
                                _p(self.idx, _i32p), _p(self.val, _f64p), _p(x, _f64p), 1.0,
                                _p(y, _f64p), _p(self.part, _f64p))
        if rc != 0:
            raise MemoryError("cpu_baseline: allocation failed")
