"""pCOO of COO matrices sorted by column or in no order (Sec. 3.2.3) on the
GPU against the oracle: the partition metadata bit-exact, the scatter SpMV
within the FP64 tolerance (bit-exact on integer-valued data), low precision
within its tolerances, and validation of the two orders."""
import numpy as np
import pytest

import oracle as O
from helpers import SCATTER_COO, coo_of, gpu_spmv, normwise, oracle_partition
from paper_2209_07552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KEYS = ("start_idx", "end_idx", "start_major", "end_major", "start_flag")
TOL64 = 1e-12


def _adversarial():
    yield I.csr_from_triplets(7, 5, [], [], [])
    yield I.csr_from_triplets(1, 9, [0] * 9, list(range(9)), np.arange(1.0, 10.0))
    yield I.csr_from_triplets(12, 40, [5] * 40, list(range(40)), np.ones(40))
    rows = [0, 0, 3, 3, 3, 9, 9, 9, 9, 9, 9, 14]
    cols = [1, 4, 0, 2, 7, 0, 1, 2, 3, 5, 6, 7]
    yield I.csr_from_triplets(20, 8, rows, cols, np.arange(1.0, 13.0))
    yield I.rmat(scale=8, nnz=1500, seed=5)
    yield I.uniform_rows()


def _gpu_partition(a, fmt, P):
    import paper_2209_07552_gb300 as M
    A = M.DeviceMatrix.from_host(a, fmt, "f64")
    part = M.DevicePartition(A, P, local=True)
    M.msrep_partition(A, part)
    return part.to_host()


@pytest.mark.parametrize("fmt", SCATTER_COO)
def test_partition_bit_exact(fmt):
    for a in _adversarial():
        for P in sorted({1, 2, 3, 7, 148, max(1, a.nnz), a.nnz + 5}):
            got = _gpu_partition(a, fmt, P)
            want = oracle_partition(a, fmt, P, with_local=True)
            for k in KEYS:
                assert np.array_equal(got[k], want[k]), (k, P)
            assert np.array_equal(got["local"], want["local"]), P


def test_column_sorted_partition_equals_pcsc():
    a = I.rmat(scale=12, nnz=60_000, seed=71)
    for P in (5, 148, 2368):
        q = _gpu_partition(a, "coo_col", P)
        c = oracle_partition(a, "csc", P)
        for k in KEYS:
            assert np.array_equal(q[k], c[k]), k


@pytest.mark.parametrize("fmt", SCATTER_COO)
@pytest.mark.parametrize("P", [1, 7, 148, 2368])
def test_spmv_fp64_vs_oracle(fmt, P):
    """R-MAT (hub rows: the permuted accumulator path) and the 2D Laplacian
    (none), with alpha and beta, against the oracle's partitioned SpMV and
    its plain COO product."""
    for a in (I.rmat(scale=14, nnz=200_000, seed=72), I.laplace5(200)):
        q = coo_of(a, fmt)
        x = I.vector(a.n, 73)
        y0 = I.y_vector(a.m, 74)
        got = gpu_spmv(a, fmt, P, x, 1.25, -0.5, y0)
        part = oracle_partition(a, fmt, P)
        want = O.pspmv_coo_scatter(a.m, q.row_idx, q.col_idx, q.val, part, x, 1.25, -0.5, y0)
        plain = O.spmv_coo(a.m, q.row_idx, q.col_idx, q.val, x, 1.25, -0.5, y0)
        assert normwise(got, want) <= TOL64
        assert normwise(got, plain) <= TOL64


@pytest.mark.parametrize("fmt", SCATTER_COO)
def test_spmv_integer_data_bit_exact_and_beta_zero_ignores_nan(fmt):
    a0 = I.rmat(scale=13, nnz=120_000, seed=75)
    a, x = I.integer_twin(a0, seed=76)
    want = O.spmv_csr(a.m, a.row_ptr, a.col_idx, a.val, x)
    for P in (3, 148, 4096):
        got = gpu_spmv(a, fmt, P, x)  # y starts as NaN, beta = 0
        assert np.array_equal(got, want), P
    y0 = np.round(I.y_vector(a.m, 77) * 8)
    want_b = O.spmv_csr(a.m, a.row_ptr, a.col_idx, a.val, x, 2.0, 3.0, y0)
    assert np.array_equal(gpu_spmv(a, fmt, 148, x, 2.0, 3.0, y0), want_b)


@pytest.mark.parametrize("fmt", SCATTER_COO)
def test_spmv_hub_row_and_edge_cases(fmt):
    """One row holding every nonzero (every partition adds to it), an empty
    matrix, a single nonzero, and nnz not a multiple of 8 (ragged tail)."""
    n = 5000
    g = I.rng(78, 1)
    a = I.csr_from_triplets(6, n, [4] * n, list(range(n)),
                            g.integers(-3, 4, n).astype(float))
    x = g.integers(-4, 5, n).astype(float)
    exact = float(sum(int(v) * int(w) for v, w in zip(a.val, x)))
    for P in (1, 9, 5000, 6000):
        assert gpu_spmv(a, fmt, P, x).tolist() == [0.0] * 4 + [exact, 0.0]
    e = I.csr_from_triplets(7, 5, [], [], [])
    assert np.array_equal(gpu_spmv(e, fmt, 3, np.ones(5), 1.0, 0.5, np.full(7, 2.0)),
                          np.full(7, 1.0))
    one = I.csr_from_triplets(3, 3, [2], [1], [2.5])
    assert gpu_spmv(one, fmt, 4, np.array([0.0, 4.0, 0.0])).tolist() == [0.0, 0.0, 10.0]
    r = I.rmat(scale=10, nnz=12_345, seed=79)
    xr = I.vector(r.n, 80)
    q = coo_of(r, fmt)
    want = O.spmv_coo(r.m, q.row_idx, q.col_idx, q.val, xr)
    assert normwise(gpu_spmv(r, fmt, 37, xr), want) <= TOL64


@pytest.mark.parametrize("fmt", SCATTER_COO)
@pytest.mark.parametrize("val_dtype,tol", [("f32", 1e-5), ("bf16", 1e-2)])
def test_low_precision_vs_fp64_oracle(fmt, val_dtype, tol):
    a = I.rmat(scale=14, nnz=200_000, seed=81)
    x = I.vector(a.n, 82)
    want = O.spmv_csr(a.m, a.row_ptr, a.col_idx, a.val, x)
    got = gpu_spmv(a, fmt, 148, x, val_dtype=val_dtype)
    assert normwise(got, want) <= tol


def test_validation_checks_each_order():
    import torch

    import paper_2209_07552_gb300 as M
    a = I.rmat(scale=8, nnz=1500, seed=83)
    for fmt in SCATTER_COO:
        A = M.DeviceMatrix.from_host(a, fmt, "f64")
        part = M.DevicePartition(A, 7)
        M.msrep_partition(A, part, M.MSREP_VALIDATE)  # a good matrix passes
        bad = A.idx2.clone()
        bad[5] = a.m + 2                                # row out of range
        B = M.DeviceMatrix(A.fmt, A.m, A.n, A.nnz, None, A.idx, bad, A.val, "f64")
        with pytest.raises(M.MsrepError) as e:
            M.msrep_partition(B, M.DevicePartition(B, 7), M.MSREP_VALIDATE)
        assert e.value.status == 2
    # row-sorted arrays are not sorted by column: rejected as COO_BY_COL,
    # accepted as COO_UNSORTED
    q = I.csr_to_coo(a)
    rows = torch.from_numpy(q.row_idx).cuda()
    cols = torch.from_numpy(q.col_idx).cuda()
    vals = torch.from_numpy(q.val).cuda()
    C = M.DeviceMatrix(M.MSREP_COO_BY_COL, a.m, a.n, a.nnz, None, cols, rows, vals, "f64")
    with pytest.raises(M.MsrepError):
        M.msrep_partition(C, M.DevicePartition(C, 7), M.MSREP_VALIDATE)
    U = M.DeviceMatrix(M.MSREP_COO_UNSORTED, a.m, a.n, a.nnz, None, cols, rows, vals, "f64")
    M.msrep_partition(U, M.DevicePartition(U, 7), M.MSREP_VALIDATE)


def test_spmv_needs_the_plan():
    import torch

    import paper_2209_07552_gb300 as M
    a = I.rmat(scale=8, nnz=1500, seed=84)
    A = M.DeviceMatrix.from_host(a, "coo_any", "f64")
    part = M.DevicePartition(A, 7, plan=False)
    M.msrep_partition(A, part)
    x = torch.ones(a.n, dtype=torch.float64, device="cuda")
    y = torch.zeros(a.m, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MsrepError) as e:
        M.msrep_spmv(A, part, 1.0, x, 0.0, y, workspace=M.alloc_workspace(A, part))
    assert e.value.status == 9


def test_hub_rows_found_for_power_law_only():
    """The plan's first word counts the hub rows the partitioner found: some
    on R-MAT, none on a Laplacian whose 160,000 rows each hold at most five
    of its 800,000 nonzeros.  (The search samples 4096 nonzeros; on a much
    smaller matrix in random order a row can reach the threshold of four
    samples by chance, which changes only where its sums are kept.)"""
    import torch

    import paper_2209_07552_gb300 as M
    for a, hub in ((I.rmat(scale=14, nnz=200_000, seed=85), True), (I.laplace5(400), False)):
        for fmt in SCATTER_COO:
            A = M.DeviceMatrix.from_host(a, fmt, "f64")
            part = M.DevicePartition(A, 148)
            M.msrep_partition(A, part)
            count = int(part.plan[:4].view(torch.int32).cpu().item())
            assert (count > 0) == hub, (fmt, count)


@pytest.mark.slow
@pytest.mark.parametrize("fmt", SCATTER_COO)
def test_full_size_rmat_vs_oracle(fmt, rmat_full):
    a = rmat_full
    q = coo_of(a, fmt)
    x = I.vector(a.n, I.SEED_BASE + 1)
    want = O.spmv_coo(a.m, q.row_idx, q.col_idx, q.val, x)
    got = gpu_spmv(a, fmt, 2368, x)
    assert normwise(got, want) <= TOL64
