"""Python binding of libmsrep.so (the C ABI declared in include/msrep.h).

Argument marshalling only: every step of the SpMV path runs in the CUDA
kernels of libmsrep.so.  PyTorch supplies device memory and streams.  The
functions keep the C names (msrep_partition_csr, msrep_spmv, ...); the small
classes DeviceMatrix / DevicePartition own the torch tensors that back the
C structs.  If libmsrep.so has not been built, every call raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("MSREP_LIB_PATH") or os.path.join(_HERE, "libmsrep.so")
_LOCK = threading.Lock()
_LIB = None

MSREP_CSR, MSREP_CSC, MSREP_COO, MSREP_COO_BY_COL, MSREP_COO_UNSORTED = 0, 1, 2, 3, 4
COO_FORMATS = (MSREP_COO, MSREP_COO_BY_COL, MSREP_COO_UNSORTED)
MSREP_F64, MSREP_F32, MSREP_BF16 = 0, 1, 2
MSREP_VALIDATE = 0x1
MSREP_PART_MERGE_PATH = 0x2
MSREP_PART_ROW_BLOCK = 0x4
MSREP_COMP_ALL = 0x10
MSREP_COMP_NONE = 0x20
MSREP_STREAM_TMA = 0x40
MSREP_SCHED_PER_PARTITION = 0x80
MSREP_SPMM_MAX_K = 8

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "BAD_MATRIX", 3: "OOM", 4: "CUDA",
          5: "TIMEOUT", 6: "BUDGET", 7: "NOT_FOUND", 8: "SHUTDOWN",
          9: "WORKSPACE"}

_DTYPE_CODES = {"f64": MSREP_F64, "f32": MSREP_F32, "bf16": MSREP_BF16}


class MsrepError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"msrep {STATUS.get(status, status)}: {msg}")
        self.status = status


class c_msrep_matrix(ctypes.Structure):
    _fields_ = [("fmt", ctypes.c_int32), ("val_dtype", ctypes.c_int32),
                ("m", ctypes.c_int32), ("n", ctypes.c_int32),
                ("nnz", ctypes.c_int64), ("ptr", ctypes.c_void_p),
                ("idx", ctypes.c_void_p), ("idx2", ctypes.c_void_p),
                ("val", ctypes.c_void_p)]


class c_msrep_partition(ctypes.Structure):
    _fields_ = [("np", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("start_idx", ctypes.c_void_p), ("end_idx", ctypes.c_void_p),
                ("start_major", ctypes.c_void_p), ("end_major", ctypes.c_void_p),
                ("start_flag", ctypes.c_void_p), ("local_off", ctypes.c_void_p),
                ("local", ctypes.c_void_p), ("plan", ctypes.c_void_p),
                ("plan_bytes", ctypes.c_int64)]


class c_msrep_tune_table(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32 * 32), ("part_nnz", ctypes.c_int64 * 32),
                ("cta_threads", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class c_msrep_batch(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("val_dtype", ctypes.c_int32),
                ("total_tiles", ctypes.c_int64), ("ws_bytes", ctypes.c_int64),
                ("dev", ctypes.c_void_p), ("dev_bytes", ctypes.c_int64),
                ("items_off", ctypes.c_int64), ("toff_off", ctypes.c_int64),
                ("cta_threads", ctypes.c_int32), ("max_tile", ctypes.c_int32)]


class c_msrep_serve_config(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("arena_bytes", ctypes.c_int64),
                ("contexts", ctypes.c_int32), ("max_items", ctypes.c_int32),
                ("max_k", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("max_tiles", ctypes.c_int64), ("device", ctypes.c_int32)]


class c_msrep_serve_counters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double),
                ("gbs", ctypes.c_double), ("mean_items", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("resident_bytes", ctypes.c_int64),
                ("wait_p50_us", ctypes.c_double), ("wait_p99_us", ctypes.c_double),
                ("device_p50_us", ctypes.c_double), ("device_p99_us", ctypes.c_double),
                ("kernel_mean_us", ctypes.c_double), ("host_launch_p50_us", ctypes.c_double),
                ("host_launch_p99_us", ctypes.c_double)]


_M = ctypes.POINTER(c_msrep_matrix)
_P = ctypes.POINTER(c_msrep_partition)
_vp = ctypes.c_void_p

# name -> (restype, argtypes); mirrors include/msrep.h
SIGNATURES = {
    "msrep_version": (ctypes.c_char_p, []),
    "msrep_last_error": (ctypes.c_char_p, []),
    "msrep_partition_local_bound": (ctypes.c_int, [_M, ctypes.c_int32,
                                                   ctypes.POINTER(ctypes.c_int64)]),
    "msrep_tile_supported": (ctypes.c_int, [ctypes.c_int32]),
    "msrep_plan_size": (ctypes.c_int, [_M, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int64)]),
    "msrep_partition_csr": (ctypes.c_int, [_M, _P, ctypes.c_uint, _vp]),
    "msrep_partition_csc": (ctypes.c_int, [_M, _P, ctypes.c_uint, _vp]),
    "msrep_partition_coo": (ctypes.c_int, [_M, _P, ctypes.c_uint, _vp]),
    "msrep_spmv_workspace_size": (ctypes.c_int, [_M, _P,
                                                 ctypes.POINTER(ctypes.c_size_t)]),
    "msrep_spmv": (ctypes.c_int, [_M, _P, ctypes.c_double, _vp, ctypes.c_double,
                                  _vp, ctypes.c_int32, ctypes.c_uint, _vp, _vp]),
    "msrep_profile_events": (ctypes.c_int, [_vp, _vp]),
    "msrep_access_floor": (ctypes.c_int, [ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.c_int64,
                                          ctypes.c_int64, _vp, _vp]),
    "msrep_spmm_workspace_size": (ctypes.c_int, [_M, _P, ctypes.c_int32,
                                                 ctypes.POINTER(ctypes.c_size_t)]),
    "msrep_spmm": (ctypes.c_int, [_M, _P, ctypes.c_int32, ctypes.c_double, _vp, ctypes.c_int64,
                                  ctypes.c_double, _vp, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_uint, _vp, _vp]),
    "msrep_spmv_noalloc": (ctypes.c_int, [_M, _P, ctypes.c_double, _vp, ctypes.c_double,
                                          _vp, ctypes.c_int32, ctypes.c_uint, _vp]),
    "msrep_device_status": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "msrep_wait_selftest": (ctypes.c_int, [ctypes.c_int64, _vp, _vp]),
    "msrep_tune_default": (ctypes.c_int, [ctypes.POINTER(c_msrep_tune_table)]),
    "msrep_batch_plan_size": (ctypes.c_int, [ctypes.c_int32, _M,
                                             ctypes.POINTER(c_msrep_tune_table),
                                             ctypes.POINTER(ctypes.c_int64)]),
    "msrep_batch_prepare": (ctypes.c_int, [ctypes.c_int32, _M,
                                           ctypes.POINTER(c_msrep_tune_table), _vp,
                                           ctypes.c_int64, ctypes.POINTER(c_msrep_batch),
                                           _vp]),
    "msrep_spmv_batched": (ctypes.c_int, [ctypes.POINTER(c_msrep_batch), _vp, _vp,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_uint,
                                          _vp, _vp]),
    "msrep_autotune_scratch_size": (ctypes.c_int, [ctypes.c_int32, _M,
                                                   ctypes.POINTER(ctypes.c_int64)]),
    "msrep_serve_config_default": (ctypes.c_int, [ctypes.POINTER(c_msrep_serve_config)]),
    "msrep_serve_create": (ctypes.c_int, [ctypes.POINTER(c_msrep_serve_config),
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "msrep_serve_register": (ctypes.c_int, [_vp, _M, ctypes.POINTER(ctypes.c_int64)]),
    "msrep_serve_unregister": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "msrep_serve_submit": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int32, _vp, _vp,
                                          ctypes.POINTER(ctypes.c_uint64)]),
    "msrep_serve_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_int64]),
    "msrep_serve_stats": (ctypes.c_int, [_vp, ctypes.POINTER(c_msrep_serve_counters),
                                         ctypes.c_int32]),
    "msrep_serve_destroy": (ctypes.c_int, [_vp]),
    "msrep_serve_replay": (ctypes.c_int, [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp,
                                          ctypes.c_double, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_double)]),
    "msrep_autotune": (ctypes.c_int, [ctypes.c_int32, _M, ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_void_p), _vp, ctypes.c_int64,
                                      ctypes.POINTER(c_msrep_tune_table), _vp]),
}


def lib(path: str | None = None):
    """Load libmsrep.so (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    "libmsrep.so is not built: run "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            so = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(so, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = so
    return _LIB


def _check(status: int):
    if status != 0:
        msg = lib().msrep_last_error()
        raise MsrepError(status, msg.decode() if msg else "")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream")
                           else int(stream))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# --------------------------------------------------------------------------
# device-side containers
# --------------------------------------------------------------------------

def _val_tensor(val: np.ndarray, val_dtype: str, device):
    import torch

    from . import inputs as I
    if val_dtype == "f64":
        return torch.from_numpy(np.ascontiguousarray(val, np.float64)).to(device)
    if val_dtype == "f32":
        return torch.from_numpy(I.to_f32(val)).to(device)
    if val_dtype == "bf16":
        bits = I.bf16_bits(val).view(np.int16)
        return torch.from_numpy(bits).to(device).view(torch.bfloat16)
    raise ValueError(val_dtype)


class DeviceMatrix:
    """A matrix resident in device memory plus its msrep_matrix struct."""

    def __init__(self, fmt, m, n, nnz, ptr, idx, idx2, val, val_dtype: str):
        self.fmt, self.m, self.n, self.nnz = fmt, int(m), int(n), int(nnz)
        self.ptr, self.idx, self.idx2, self.val = ptr, idx, idx2, val
        self.val_dtype = val_dtype
        self.c = c_msrep_matrix(fmt, _DTYPE_CODES[val_dtype], self.m, self.n,
                              self.nnz, _ptr(ptr), _ptr(idx), _ptr(idx2),
                              _ptr(val))

    @property
    def format_name(self):
        return {MSREP_CSR: "csr", MSREP_CSC: "csc", MSREP_COO: "coo",
                MSREP_COO_BY_COL: "coo_col", MSREP_COO_UNSORTED: "coo_any"}[self.fmt]

    @classmethod
    def from_host(cls, a, fmt: str = "csr", val_dtype: str = "f64",
                  device="cuda", order_seed=None):
        """Upload an inputs.CSR (converted to `fmt`) to the device.  `fmt`:
        "csr", "csc", "coo" (sorted by row), "coo_col" (sorted by column) or
        "coo_any" (the nonzeros in a seeded random order, `order_seed`)."""
        import torch

        from . import inputs as I

        def t32(v):
            return torch.from_numpy(np.ascontiguousarray(v, np.int32)).to(device)
        if fmt == "csr":
            return cls(MSREP_CSR, a.m, a.n, a.nnz, t32(a.row_ptr), t32(a.col_idx),
                       None, _val_tensor(a.val, val_dtype, device), val_dtype)
        if fmt == "csc":
            c = I.csr_to_csc(a)
            return cls(MSREP_CSC, a.m, a.n, a.nnz, t32(c.col_ptr), t32(c.row_idx),
                       None, _val_tensor(c.val, val_dtype, device), val_dtype)
        if fmt in ("coo", "coo_col", "coo_any"):
            if fmt == "coo":
                q, code = I.csr_to_coo(a), MSREP_COO
            elif fmt == "coo_col":
                q, code = I.csr_to_coo_by_col(a), MSREP_COO_BY_COL
            else:
                q = (I.csr_to_coo_unsorted(a) if order_seed is None
                     else I.csr_to_coo_unsorted(a, order_seed))
                code = MSREP_COO_UNSORTED
            return cls(code, a.m, a.n, a.nnz, None, t32(q.col_idx),
                       t32(q.row_idx), _val_tensor(q.val, val_dtype, device),
                       val_dtype)
        raise ValueError(fmt)

    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size()
                   for t in (self.ptr, self.idx, self.idx2, self.val)
                   if t is not None)


class DevicePartition:
    """Caller-allocated pCSR/pCSC/pCOO metadata (+ optional local pointers
    and tile plan) for one matrix, plus its msrep_partition struct."""

    def __init__(self, A: DeviceMatrix, np_: int, tile: int = 0,
                 local: bool = False, plan: bool = True, device="cuda"):
        import torch
        self.np, self.tile = int(np_), int(tile)
        self.nnz = A.nnz
        i32 = dict(dtype=torch.int32, device=device)
        self.start_idx = torch.empty(self.np, **i32)
        self.end_idx = torch.empty(self.np, **i32)
        self.start_major = torch.empty(self.np, **i32)
        self.end_major = torch.empty(self.np, **i32)
        self.start_flag = torch.empty(self.np, dtype=torch.uint8, device=device)
        self.local_off = self.local = None
        if local:
            if A.fmt not in COO_FORMATS:
                self.local_off = torch.empty(self.np + 1, dtype=torch.int64,
                                             device=device)
            self.local = torch.empty(max(1, msrep_partition_local_bound(A, self.np)),
                                     **i32)
        self.plan = None
        pb = 0
        if plan and A.fmt != MSREP_COO:
            pb = msrep_plan_size(A, self.np, self.tile)
            self.plan = torch.empty(max(pb, 256), dtype=torch.uint8, device=device)
        self.c = c_msrep_partition(
            self.np, self.tile, _ptr(self.start_idx), _ptr(self.end_idx),
            _ptr(self.start_major), _ptr(self.end_major), _ptr(self.start_flag),
            _ptr(self.local_off), _ptr(self.local), _ptr(self.plan), pb)

    def to_host(self) -> dict:
        out = {k: getattr(self, k).cpu().numpy() for k in
               ("start_idx", "end_idx", "start_major", "end_major", "start_flag")}
        if self.local_off is not None:
            out["local_off"] = self.local_off.cpu().numpy()
            out["local"] = self.local.cpu().numpy()[: int(out["local_off"][-1])]
        elif self.local is not None:
            out["local"] = self.local.cpu().numpy()[: self.nnz]
        return out


# --------------------------------------------------------------------------
# the C entry points
# --------------------------------------------------------------------------

def msrep_version() -> str:
    return lib().msrep_version().decode()


def msrep_partition_local_bound(A: DeviceMatrix, np_: int) -> int:
    out = ctypes.c_int64()
    _check(lib().msrep_partition_local_bound(ctypes.byref(A.c), np_,
                                             ctypes.byref(out)))
    return out.value


def msrep_tile_supported(tile: int) -> bool:
    return bool(lib().msrep_tile_supported(tile))


def msrep_plan_size(A: DeviceMatrix, np_: int, tile: int = 0) -> int:
    out = ctypes.c_int64()
    _check(lib().msrep_plan_size(ctypes.byref(A.c), np_, tile, ctypes.byref(out)))
    return out.value


def msrep_partition_csr(A: DeviceMatrix, part: DevicePartition, flags: int = 0,
                        stream=None):
    _check(lib().msrep_partition_csr(ctypes.byref(A.c), ctypes.byref(part.c),
                                     flags, _stream(stream)))


def msrep_partition_csc(A: DeviceMatrix, part: DevicePartition, flags: int = 0,
                        stream=None):
    _check(lib().msrep_partition_csc(ctypes.byref(A.c), ctypes.byref(part.c),
                                     flags, _stream(stream)))


def msrep_partition_coo(A: DeviceMatrix, part: DevicePartition, flags: int = 0,
                        stream=None):
    _check(lib().msrep_partition_coo(ctypes.byref(A.c), ctypes.byref(part.c),
                                     flags, _stream(stream)))


def msrep_partition(A: DeviceMatrix, part: DevicePartition, flags: int = 0,
                    stream=None):
    """Dispatch to msrep_partition_{csr,csc,coo} by the matrix format."""
    {MSREP_CSR: msrep_partition_csr, MSREP_CSC: msrep_partition_csc,
     MSREP_COO: msrep_partition_coo, MSREP_COO_BY_COL: msrep_partition_coo,
     MSREP_COO_UNSORTED: msrep_partition_coo}[A.fmt](A, part, flags, stream)


def msrep_spmv_workspace_size(A: DeviceMatrix, part: DevicePartition) -> int:
    out = ctypes.c_size_t()
    _check(lib().msrep_spmv_workspace_size(ctypes.byref(A.c), ctypes.byref(part.c),
                                           ctypes.byref(out)))
    return out.value


def alloc_workspace(A: DeviceMatrix, part: DevicePartition, device="cuda"):
    import torch
    return torch.empty(max(256, msrep_spmv_workspace_size(A, part)),
                       dtype=torch.uint8, device=device)


def msrep_spmv(A: DeviceMatrix, part: DevicePartition, alpha: float, x,
               beta: float, y, flags: int = 0, workspace=None, stream=None):
    """y = alpha*A*x + beta*y.  x, y are device tensors (float64 for an FP64
    matrix, float32 for FP32/BF16 values)."""
    import torch
    xy = MSREP_F64 if y.dtype == torch.float64 else MSREP_F32
    _check(lib().msrep_spmv(ctypes.byref(A.c), ctypes.byref(part.c),
                            float(alpha), _ptr(x), float(beta), _ptr(y), xy,
                            flags, _ptr(workspace), _stream(stream)))


def msrep_access_floor(mode: int, idx, val, vec, idx2=None, sink=None, stream=None):
    """The access-pattern floor kernel (see include/msrep.h): mode 0 gather,
    1 gather plus a second index stream, 2 scatter-add, 3 scatter-add to the
    permuted slot, 4 and 5 as 0 and 1 with lane-interleaved steps.
    vec.numel() must be a power of two."""
    import torch
    if sink is None:
        sink = torch.zeros(1, dtype=torch.float64, device=vec.device)
    _check(lib().msrep_access_floor(int(mode), _ptr(idx), _ptr(idx2) if idx2 is not None else None,
                                    _ptr(val), _ptr(vec), int(val.numel()), int(vec.numel()),
                                    _ptr(sink), _stream(stream)))


def msrep_spmm_workspace_size(A: DeviceMatrix, part: DevicePartition, k: int) -> int:
    out = ctypes.c_size_t()
    _check(lib().msrep_spmm_workspace_size(ctypes.byref(A.c), ctypes.byref(part.c), int(k),
                                           ctypes.byref(out)))
    return out.value


def msrep_spmm(A: DeviceMatrix, part: DevicePartition, alpha: float, X, beta: float, Y,
               flags: int = 0, workspace=None, stream=None):
    """Y = alpha*A*X + beta*Y for k vectors (passes of up to 8): X is a
    (k, n) and Y a (k, m) device tensor (row v = vector v, rows contiguous).
    A must be CSR."""
    import torch
    k = X.shape[0]
    if workspace is None:
        workspace = torch.empty(max(256, msrep_spmm_workspace_size(A, part, k)),
                                dtype=torch.uint8, device=X.device)
    xy = MSREP_F64 if Y.dtype == torch.float64 else MSREP_F32
    _check(lib().msrep_spmm(ctypes.byref(A.c), ctypes.byref(part.c), int(k), float(alpha),
                            _ptr(X), int(X.stride(0)), float(beta), _ptr(Y), int(Y.stride(0)),
                            xy, flags, _ptr(workspace), _stream(stream)))


def msrep_spmv_noalloc(A: DeviceMatrix, part: DevicePartition, alpha: float, x,
                       beta: float, y, flags: int = 0, stream=None):
    """msrep_spmv without a workspace: the library's built-in scratch array
    is used instead, so nothing is allocated (see include/msrep.h for the
    size limit and the rule that such calls must not overlap)."""
    import torch
    xy = MSREP_F64 if y.dtype == torch.float64 else MSREP_F32
    _check(lib().msrep_spmv_noalloc(ctypes.byref(A.c), ctypes.byref(part.c), float(alpha),
                                    _ptr(x), float(beta), _ptr(y), xy, flags,
                                    _stream(stream)))


def msrep_profile_events(start=None, stop=None):
    """Record torch.cuda.Event `start`/`stop` around the main kernel of every
    following msrep_spmv call on this thread (None, None to stop)."""
    if start is not None:
        # torch only reports elapsed time for events it has seen recorded;
        # the library re-records the same CUDA events on every call
        start.record()
        stop.record()
    sp = ctypes.c_void_p(start.cuda_event) if start is not None else None
    ep = ctypes.c_void_p(stop.cuda_event) if stop is not None else None
    _check(lib().msrep_profile_events(sp, ep))


def msrep_device_status(stream=None) -> int:
    """Read and clear the device error word (syncs); raises MsrepError with
    status TIMEOUT if a kernel gave up on a bounded wait."""
    st = ctypes.c_int()
    _check(lib().msrep_device_status(_stream(stream), ctypes.byref(st)))
    return st.value


def msrep_wait_selftest(max_cycles: int, gave_up, stream=None):
    """Queue the bounded-wait self-test kernel; gave_up: a device int32
    tensor of one element (1 after the wait gave up)."""
    _check(lib().msrep_wait_selftest(int(max_cycles), _ptr(gave_up), _stream(stream)))


# --------------------------------------------------------------------------
# batched form
# --------------------------------------------------------------------------

def msrep_tune_default() -> c_msrep_tune_table:
    t = c_msrep_tune_table()
    _check(lib().msrep_tune_default(ctypes.byref(t)))
    return t


def _mat_array(mats):
    arr = (c_msrep_matrix * len(mats))()
    for i, A in enumerate(mats):
        arr[i] = A.c
    return arr


def msrep_batch_plan_size(mats, tune=None) -> int:
    out = ctypes.c_int64()
    arr = _mat_array(mats)
    _check(lib().msrep_batch_plan_size(len(mats), arr,
                                       ctypes.byref(tune) if tune is not None else None,
                                       ctypes.byref(out)))
    return out.value


class DeviceBatch:
    """A prepared batch of CSR DeviceMatrix objects (msrep_batch_prepare),
    with device pointer arrays for x and y and the workspace."""

    def __init__(self, mats, xs, ys, tune=None, device="cuda", stream=None):
        import torch
        self.mats, self.xs, self.ys = list(mats), list(xs), list(ys)
        self.tune = tune
        arr = _mat_array(self.mats)
        self._arr = arr
        need = msrep_batch_plan_size(self.mats, tune)
        self.dev = torch.empty(max(need, 256), dtype=torch.uint8, device=device)
        self.c = c_msrep_batch()
        _check(lib().msrep_batch_prepare(
            len(self.mats), arr, ctypes.byref(tune) if tune is not None else None,
            _ptr(self.dev), need, ctypes.byref(self.c), _stream(stream)))
        self.ws = torch.empty(max(int(self.c.ws_bytes), 256), dtype=torch.uint8,
                              device=device)
        self.xptr = torch.tensor([t.data_ptr() for t in self.xs], dtype=torch.int64,
                                 device=device)
        self.yptr = torch.tensor([t.data_ptr() for t in self.ys], dtype=torch.int64,
                                 device=device)

    @property
    def total_tiles(self) -> int:
        return int(self.c.total_tiles)

    def run(self, alpha=1.0, beta=0.0, flags=0, stream=None):
        msrep_spmv_batched(self, alpha, beta, flags, stream)


def msrep_spmv_batched(batch: DeviceBatch, alpha=1.0, beta=0.0, flags=0, stream=None):
    """One persistent launch (plus fix-up) over every matrix of the batch."""
    _check(lib().msrep_spmv_batched(ctypes.byref(batch.c), _ptr(batch.xptr),
                                    _ptr(batch.yptr), float(alpha), float(beta), flags,
                                    _ptr(batch.ws), _stream(stream)))


def msrep_autotune(mats, xs, ys, device="cuda", stream=None) -> c_msrep_tune_table:
    """Run the autotuner over the batch's size buckets; returns the table."""
    import torch
    arr = _mat_array(mats)
    need = ctypes.c_int64()
    _check(lib().msrep_autotune_scratch_size(len(mats), arr, ctypes.byref(need)))
    scratch = torch.empty(max(need.value, 256), dtype=torch.uint8, device=device)
    xp = (ctypes.c_void_p * len(mats))(*[t.data_ptr() for t in xs])
    yp = (ctypes.c_void_p * len(mats))(*[t.data_ptr() for t in ys])
    out = c_msrep_tune_table()
    _check(lib().msrep_autotune(len(mats), arr, xp, yp, _ptr(scratch), need.value,
                                ctypes.byref(out), _stream(stream)))
    return out


# --------------------------------------------------------------------------
# serving
# --------------------------------------------------------------------------

def msrep_serve_config_default() -> c_msrep_serve_config:
    c = c_msrep_serve_config()
    _check(lib().msrep_serve_config_default(ctypes.byref(c)))
    return c


class ServeTicket:
    """A submitted request: keeps the host x and y buffers alive."""

    def __init__(self, req_id, x, y, k, m):
        self.id, self.x, self.y, self.k, self.m = req_id, x, y, k, m

    @property
    def result(self) -> np.ndarray:
        return self.y[: self.k * self.m].reshape(self.k, self.m)


def pinned_empty(shape, dtype=np.float32) -> np.ndarray:
    """A page-locked host numpy array (the server DMAs these directly)."""
    import torch
    t = torch.empty(int(np.prod(shape)), dtype=torch.from_numpy(np.empty(0, dtype)).dtype,
                    pin_memory=True)
    return t.numpy().reshape(shape)


class Server:
    """msrep_serve_* around host numpy buffers."""

    def __init__(self, **cfg):
        self.cfg = msrep_serve_config_default()
        for k, v in cfg.items():
            setattr(self.cfg, k, v)
        h = ctypes.c_void_p()
        _check(lib().msrep_serve_create(ctypes.byref(self.cfg), ctypes.byref(h)))
        self.h = h
        self.shapes = {}

    def register(self, a) -> int:
        """Register an inputs.CSR (host arrays); values are stored as FP32."""
        ptr = np.ascontiguousarray(a.row_ptr, np.int32)
        col = np.ascontiguousarray(a.col_idx, np.int32)
        if a.val.dtype == np.float64:
            val, dt = np.ascontiguousarray(a.val), MSREP_F64
        else:
            val, dt = np.ascontiguousarray(a.val, np.float32), MSREP_F32
        c = c_msrep_matrix(MSREP_CSR, dt, a.m, a.n, a.nnz, ptr.ctypes.data,
                           col.ctypes.data, None, val.ctypes.data)
        out = ctypes.c_int64()
        _check(lib().msrep_serve_register(self.h, ctypes.byref(c), ctypes.byref(out)))
        self.shapes[out.value] = (a.m, a.n)
        return out.value

    def unregister(self, mid: int):
        # the shape stays known so that later calls reach the library and
        # get its NOT_FOUND status
        _check(lib().msrep_serve_unregister(self.h, mid))

    def submit(self, mid: int, X: np.ndarray, y: np.ndarray | None = None) -> ServeTicket:
        """X: (k, n) float32 (or (n,)); returns a ticket whose .result is (k, m)."""
        X = np.ascontiguousarray(np.atleast_2d(X), np.float32)
        k = X.shape[0]
        m, n = self.shapes.get(mid, (0, X.shape[1]))
        if X.shape[1] != n:
            raise ValueError(f"x has {X.shape[1]} entries, matrix has {n} columns")
        if y is None:
            y = np.empty(max(k * m, 1), np.float32)
        rid = ctypes.c_uint64()
        _check(lib().msrep_serve_submit(self.h, mid, k, X.ctypes.data, y.ctypes.data,
                                        ctypes.byref(rid)))
        return ServeTicket(rid.value, X, y, k, m)

    def wait(self, t: ServeTicket, timeout_us: int = -1) -> np.ndarray:
        _check(lib().msrep_serve_wait(self.h, t.id, timeout_us))
        return t.result

    def replay(self, t_us, mids, ks, xs, ys, reuse, reset_after_us=-1.0):
        """Native open-loop driver (msrep_serve_replay): request i arrives
        t_us[i] us after the call starts, names matrix mids[i] with ks[i]
        vectors from the host array xs[i] into ys[i]; reuse[i] is the
        earlier request whose y buffer request i reuses (-1: none).
        Returns (late submissions, largest submission lag in us)."""
        n = len(t_us)
        t = np.ascontiguousarray(t_us, np.float64)
        mi = np.ascontiguousarray(mids, np.int64)
        kk = np.ascontiguousarray(ks, np.int32)
        ru = np.ascontiguousarray(reuse, np.int64)
        if not (len(mi) == len(kk) == len(ru) == len(xs) == len(ys) == n):
            raise ValueError("replay: per-request arrays differ in length")
        for i in range(n):
            # the native driver reads and writes these buffers in place
            m, nc = self.shapes.get(int(mi[i]), (0, 0))
            for a, need in ((xs[i], int(kk[i]) * nc), (ys[i], int(kk[i]) * m)):
                if a.dtype != np.float32 or not a.flags.c_contiguous or a.size < need:
                    raise ValueError(f"replay: request {i} needs C-contiguous float32 "
                                     f"buffers of {need} values")
        xp = (ctypes.c_void_p * n)(*[a.ctypes.data for a in xs])
        yp = (ctypes.c_void_p * n)(*[a.ctypes.data for a in ys])
        late, lag = ctypes.c_int64(), ctypes.c_double()
        _check(lib().msrep_serve_replay(self.h, n, t.ctypes.data, mi.ctypes.data, kk.ctypes.data,
                                        xp, yp, ru.ctypes.data, float(reset_after_us),
                                        ctypes.byref(late), ctypes.byref(lag)))
        return late.value, lag.value

    def stats(self, reset: bool = False) -> dict:
        c = c_msrep_serve_counters()
        _check(lib().msrep_serve_stats(self.h, ctypes.byref(c), 1 if reset else 0))
        return {f: getattr(c, f) for f, _ in c._fields_}

    def close(self):
        if self.h:
            _check(lib().msrep_serve_destroy(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
