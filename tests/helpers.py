"""Shared helpers of the GPU parity tests: run the CUDA path through the C
ABI binding and the oracle on the same seeded inputs."""
import numpy as np

import oracle as O
from paper_2209_07552_gb300 import inputs as I

FORMATS = ("csr", "csc", "coo")
# COO sorted by column and in no order (the scatter forms of pCOO)
SCATTER_COO = ("coo_col", "coo_any")


def normwise(y, yref):
    """||y - yref||_2 / ||yref||_2 (absolute when yref == 0)."""
    y = np.asarray(y, np.float64)
    yref = np.asarray(yref, np.float64)
    d = np.linalg.norm(y - yref)
    n = np.linalg.norm(yref)
    return d / n if n > 0 else d


def oracle_spmv(a: I.CSR, fmt: str, x, alpha=1.0, beta=0.0, y=None):
    if fmt == "csr":
        return O.spmv_csr(a.m, a.row_ptr, a.col_idx, a.val, x, alpha, beta, y)
    if fmt == "csc":
        c = I.csr_to_csc(a)
        return O.spmv_csc(a.m, a.n, c.col_ptr, c.row_idx, c.val, x, alpha, beta, y)
    q = coo_of(a, fmt)
    return O.spmv_coo(a.m, q.row_idx, q.col_idx, q.val, x, alpha, beta, y)


def coo_of(a: I.CSR, fmt: str) -> I.COO:
    """The COO arrays the binding uploads for "coo", "coo_col" and
    "coo_any" (default order seed)."""
    if fmt == "coo_col":
        return I.csr_to_coo_by_col(a)
    if fmt == "coo_any":
        return I.csr_to_coo_unsorted(a)
    return I.csr_to_coo(a)


def oracle_partition(a: I.CSR, fmt: str, P: int, with_local=False):
    if fmt == "csr":
        return O.partition_csr(a.row_ptr, a.nnz, P, with_local)
    if fmt == "csc":
        c = I.csr_to_csc(a)
        return O.partition_csc(c.col_ptr, c.nnz, P, with_local)
    q = coo_of(a, fmt)
    if fmt == "coo_col":
        return O.partition_coo_by_col(q.col_idx, P, with_local)
    if fmt == "coo_any":
        return O.partition_coo_unsorted(q.row_idx, a.m, P, with_local)
    return O.partition_coo(q.row_idx, P, with_local)


def gpu_spmv(a: I.CSR, fmt: str, P: int, x, alpha=1.0, beta=0.0, y0=None,
             tile=0, val_dtype="f64", flags=0, repeat=1, part_flags=0):
    """Partition and run msrep_spmv on the GPU; returns y as numpy."""
    import torch

    import paper_2209_07552_gb300 as M
    A = M.DeviceMatrix.from_host(a, fmt, val_dtype)
    part = M.DevicePartition(A, P, tile=tile)
    M.msrep_partition(A, part, part_flags)
    xt = torch.float64 if val_dtype == "f64" else torch.float32
    xd = torch.from_numpy(np.asarray(x)).to("cuda", xt)
    if y0 is None:
        yd = torch.full((a.m,), float("nan"), dtype=xt, device="cuda")
    else:
        yd = torch.from_numpy(np.asarray(y0)).to("cuda", xt)
    ws = M.alloc_workspace(A, part)
    outs = []
    for _ in range(repeat):
        yy = yd.clone()
        M.msrep_spmv(A, part, alpha, xd, beta, yy, flags=flags, workspace=ws)
        outs.append(yy.cpu().numpy().astype(np.float64))
    torch.cuda.synchronize()
    return outs[0] if repeat == 1 else outs


U32 = 2.0 ** -24


def f32_row_bound(a_stored: I.CSR, x, yref):
    """Element-wise error bound of a binary32 SpMV row against the FP64
    product of the stored values and x: recursive summation of L_r products
    (Higham, "Accuracy and Stability of Numerical Algorithms", Sec. 3.1)
    gives |y_r - yref_r| <= (L_r + 2) u (|A| |x|)_r + u |yref_r|, u = 2^-24;
    compensated rows are well inside it."""
    absa = I.CSR(a_stored.m, a_stored.n, a_stored.row_ptr, a_stored.col_idx,
                 np.abs(a_stored.val))
    ax = O.spmv_csr(absa.m, absa.row_ptr, absa.col_idx, absa.val, np.abs(x))
    L = np.diff(a_stored.row_ptr.astype(np.int64)).astype(np.float64)
    return (L + 2) * U32 * ax + U32 * np.abs(yref)
