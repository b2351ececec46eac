"""Row+nonzero merge-path partitioning (MSREP_PART_MERGE_PATH) on the GPU
against the oracle: the metadata and local pointers bit-exact, and the
SpMV over such partitions within the FP64 tolerance (bit-exact on
integer-valued data)."""
import numpy as np
import pytest

import oracle as O
from helpers import gpu_spmv, normwise, oracle_spmv
from paper_2209_07552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KEYS = ("start_idx", "end_idx", "start_major", "end_major", "start_flag")
TOL64 = 1e-12


def _ptr(a, fmt):
    return a.row_ptr if fmt == "csr" else I.csr_to_csc(a).col_ptr


def _gpu_partition(a, fmt, P, tile=0):
    import paper_2209_07552_gb300 as M
    A = M.DeviceMatrix.from_host(a, fmt, "f64")
    part = M.DevicePartition(A, P, tile=tile, local=True)
    M.msrep_partition(A, part, M.MSREP_PART_MERGE_PATH)
    return part.to_host()


def _mats():
    yield I.csr_from_triplets(7, 5, [], [], [])
    yield I.csr_from_triplets(1, 9, [0] * 9, list(range(9)), np.arange(1.0, 10.0))
    yield I.csr_from_triplets(12, 40, [5] * 40, list(range(40)), np.ones(40))
    rows = [0, 0, 3, 3, 3, 9, 9, 9, 9, 9, 9, 14]
    cols = [1, 4, 0, 2, 7, 0, 1, 2, 3, 5, 6, 7]
    yield I.csr_from_triplets(20, 8, rows, cols, np.arange(1.0, 13.0))
    yield I.csr_from_triplets(1000, 1000, [999] * 1000, list(range(1000)), np.ones(1000))
    yield I.rmat(scale=10, nnz=8000, seed=91)


@pytest.mark.parametrize("fmt", ["csr", "csc"])
def test_metadata_and_local_pointers_bit_exact(fmt):
    for a in _mats():
        tot = (a.m if fmt == "csr" else a.n) + a.nnz
        for P in sorted({1, 2, 3, 7, 148, tot, tot + 5}):
            got = _gpu_partition(a, fmt, P)
            want = O.partition_merge_path(_ptr(a, fmt), a.nnz, P, with_local=True)
            for k in KEYS:
                assert np.array_equal(got[k], want[k]), (k, P)
            assert np.array_equal(got["local_off"], want["local_off"]), P
            assert np.array_equal(got["local"], want["local"]), P


@pytest.mark.parametrize("fmt", ["csr", "csc"])
@pytest.mark.parametrize("tile", [256, 512, 1024])
def test_spmv_over_merge_path_partitions(fmt, tile):
    for a in (I.rmat(scale=14, nnz=200_000, seed=92), I.laplace5(150),
              I.csr_from_triplets(1000, 1000, [999] * 1000, list(range(1000)),
                                  I.rng(93, 1).uniform(-1, 1, 1000))):
        x = I.vector(a.n, 94)
        y0 = I.y_vector(a.m, 95)
        want = oracle_spmv(a, fmt, x, 0.75, -1.25, y0)
        for P in (1, 2, 148, 2368):
            got = gpu_spmv(a, fmt, P, x, 0.75, -1.25, y0, tile=tile, part_flags=2)
            assert normwise(got, want) <= TOL64, (P, tile)


@pytest.mark.parametrize("fmt", ["csr", "csc"])
def test_integer_data_bit_exact(fmt):
    a0 = I.rmat(scale=13, nnz=120_000, seed=96)
    a, x = I.integer_twin(a0, seed=97)
    want = O.spmv_csr(a.m, a.row_ptr, a.col_idx, a.val, x)
    for P in (3, 148, 9472):
        assert np.array_equal(gpu_spmv(a, fmt, P, x, part_flags=2), want), P


def test_low_precision_over_merge_path_partitions():
    a = I.rmat(scale=14, nnz=200_000, seed=98)
    x = I.vector(a.n, 99)
    want = O.spmv_csr(a.m, a.row_ptr, a.col_idx, a.val, x)
    for vd, tol in (("f32", 1e-5), ("bf16", 1e-2)):
        assert normwise(gpu_spmv(a, "csr", 148, x, val_dtype=vd, part_flags=2), want) <= tol


def test_coo_rejects_the_flag():
    import paper_2209_07552_gb300 as M
    a = I.rmat(scale=8, nnz=1500, seed=100)
    A = M.DeviceMatrix.from_host(a, "coo", "f64")
    part = M.DevicePartition(A, 7)
    with pytest.raises(M.MsrepError) as e:
        M.msrep_partition(A, part, M.MSREP_PART_MERGE_PATH)
    assert e.value.status == 1


@pytest.mark.slow
def test_full_size_rmat(rmat_full):
    a = rmat_full
    got = _gpu_partition(a, "csr", 2368)
    want = O.partition_merge_path(a.row_ptr, a.nnz, 2368, with_local=True)
    for k in KEYS:
        assert np.array_equal(got[k], want[k]), k
    assert np.array_equal(got["local"], want["local"])
    x = I.vector(a.n, I.SEED_BASE + 1)
    y = gpu_spmv(a, "csr", 2368, x, part_flags=2)
    assert normwise(y, oracle_spmv(a, "csr", x)) <= TOL64
