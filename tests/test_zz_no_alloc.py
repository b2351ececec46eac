"""msrep_spmv_noalloc: the SpMV entry point that allocates nothing.

Some callers cannot allocate device memory: code that only receives the
matrix and vector buffers from a host framework that owns all device memory,
or a loop where a cudaMalloc is not acceptable.  For them the library offers
msrep_spmv_noalloc, which takes its scratch from an array compiled into the
library instead of a caller workspace.  These tests call it through the C ABI
and check it against msrep_spmv (with an allocated workspace) on the same
inputs, on two calls in a row, since the calls share and reuse that array.
The file is named to be collected last."""
import numpy as np
import pytest

from helpers import normwise
from paper_2209_07552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.mark.parametrize("fmt", ["csr", "coo"])
def test_noalloc_matches_workspace_entry_point_twice(fmt):
    import torch

    import paper_2209_07552_gb300 as M
    a = I.rmat(scale=14, nnz=200_000, seed=61)
    A = M.DeviceMatrix.from_host(a, fmt, "f64")
    part = M.DevicePartition(A, 148)
    M.msrep_partition(A, part)
    ws = M.alloc_workspace(A, part)
    for call in range(2):
        x = torch.from_numpy(I.vector(a.n, 62 + call)).cuda()
        y_ref = torch.empty(a.m, dtype=torch.float64, device="cuda")
        M.msrep_spmv(A, part, 1.0, x, 0.0, y_ref, workspace=ws)
        y = torch.full((a.m,), float("nan"), dtype=torch.float64, device="cuda")
        M.native.msrep_spmv_noalloc(A, part, 1.0, x, 0.0, y)
        torch.cuda.synchronize()
        assert normwise(y.cpu().numpy(), y_ref.cpu().numpy()) <= TOL64


def test_noalloc_rejects_problems_larger_than_its_scratch():
    import torch

    import paper_2209_07552_gb300 as M
    a = I.laplace_full()                   # 25.2 million rows + nonzeros
    A = M.DeviceMatrix.from_host(a, "csr", "f64")
    part = M.DevicePartition(A, 148, tile=256)  # about 98,000 tiles
    x = torch.zeros(a.n, dtype=torch.float64, device="cuda")
    y = torch.zeros(a.m, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MsrepError) as e:
        M.native.msrep_spmv_noalloc(A, part, 1.0, x, 0.0, y)
    assert e.value.status == 9             # MSREP_ERR_WORKSPACE
    assert "scratch" in str(e.value)


@pytest.mark.parametrize("fmt", ["csc", "coo_col", "coo_any"])
@pytest.mark.parametrize("scale", [14, 18])
def test_noalloc_csc_with_and_without_the_permuted_accumulator(scale, fmt):
    """CSC, and COO sorted by column or in no order, which scatter the same
    way, on a power-law matrix (hub rows found): at 2^14 rows the permuted
    accumulator fits in the scratch array, at 2^18 rows (2 MiB) it does not
    and the call scatters into y directly.  Integer-valued data make every
    sum exact, so both entry points must match the oracle bit for bit, with
    beta != 0 applied once."""
    import torch

    import paper_2209_07552_gb300 as M
    from helpers import oracle_spmv
    a0 = I.rmat(scale=scale, nnz=16 * (1 << scale), seed=63)
    a, x = I.integer_twin(a0, seed=64)
    y0 = np.round(I.y_vector(a.m, 65) * 4)
    want = oracle_spmv(a, "csc", x, 1.0, 2.0, y0)
    A = M.DeviceMatrix.from_host(a, fmt, "f64")
    part = M.DevicePartition(A, 148)
    M.msrep_partition(A, part)
    ws = M.alloc_workspace(A, part)
    xd = torch.from_numpy(x).cuda()
    for call in range(2):
        y_ref = torch.from_numpy(y0).cuda()
        M.msrep_spmv(A, part, 1.0, xd, 2.0, y_ref, workspace=ws)
        y = torch.from_numpy(y0).cuda()
        M.native.msrep_spmv_noalloc(A, part, 1.0, xd, 2.0, y)
        torch.cuda.synchronize()
        assert np.array_equal(y_ref.cpu().numpy(), want), call
        assert np.array_equal(y.cpu().numpy(), want), call


@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("fmt", ["csc", "coo_col"])
def test_noalloc_low_precision_scatter_row_ordered_accumulator(fmt, dt):
    """Low-precision CSC and column-sorted COO at 100,000 rows: the permuted
    accumulator (2^17 doubles, 1 MiB) does not fit in the scratch array but
    m doubles do, so the call accumulates in FP64 in row order in the
    scratch and rounds to FP32 once.  Checked against msrep_spmv and against
    the FP64 oracle on the original values (1e-5 FP32, 1e-2 BF16 values),
    on two calls in a row."""
    import torch

    import paper_2209_07552_gb300 as M
    from helpers import oracle_spmv
    tol = {"f32": 1e-5, "bf16": 1e-2}[dt]
    a = I.geometric_matrix(100_000, 8.0, 66, np.float64)
    A = M.DeviceMatrix.from_host(a, fmt, dt)
    part = M.DevicePartition(A, 148)
    M.msrep_partition(A, part)
    ws = M.alloc_workspace(A, part)
    for call in range(2):
        x64 = I.vector(a.n, 67 + call)
        x = torch.from_numpy(I.to_f32(x64)).cuda()
        y_ref = torch.empty(a.m, dtype=torch.float32, device="cuda")
        M.msrep_spmv(A, part, 1.0, x, 0.0, y_ref, workspace=ws)
        y = torch.full((a.m,), float("nan"), dtype=torch.float32, device="cuda")
        M.native.msrep_spmv_noalloc(A, part, 1.0, x, 0.0, y)
        torch.cuda.synchronize()
        yh = y.cpu().numpy().astype(np.float64)
        assert normwise(yh, y_ref.cpu().numpy().astype(np.float64)) <= 1e-6, call
        assert normwise(yh, oracle_spmv(a, "csr", x64)) <= tol, call
