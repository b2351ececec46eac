"""CUDA SpMV over pCSR / pCSC / pCOO (Alg. 3, 5, 7) against the oracle.

FP64 tolerance: normwise relative error <= 1e-12.  The GPU sums each row
in a different order (tile tree, carry chain, atomics for CSC) than the
oracle's sequential order; with n terms per row the difference is bounded
by about n * 2^-53 * sum|a_k x_k| per row, far below 1e-12 relative for the
row lengths here.  Integer-valued inputs (values in [-3, 3], x in [-4, 4])
make every partial sum an exact integer below 2^53, so there the results
must match bit for bit in every format and partitioning.
"""
import numpy as np
import pytest

from helpers import FORMATS, gpu_spmv, normwise, oracle_spmv
from paper_2209_07552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TILES = (256, 512, 1024)


def _small_set():
    yield "uniform", I.uniform_rows()
    yield "rmat12", I.rmat(scale=12, nnz=40_000, seed=12)
    yield "hub", I.csr_from_triplets(
        9, 6000, [4] * 6000, list(range(6000)), I.rng(4, 4).uniform(-1, 1, 6000))
    rows = [0, 0, 3, 3, 3, 9, 9, 9, 9, 9, 9, 14]
    cols = [1, 4, 0, 2, 7, 0, 1, 2, 3, 5, 6, 7]
    yield "gaps", I.csr_from_triplets(20, 8, rows, cols,
                                      I.rng(5, 5).uniform(-1, 1, len(rows)))
    lead = I.rmat(scale=10, nnz=8000, seed=6)
    # shift rows down by 300 and pad: long runs of empty leading/trailing rows
    rp = np.concatenate([np.zeros(300, np.int32), lead.row_ptr,
                         np.full(500, lead.row_ptr[-1], np.int32)])
    yield "padded", I.CSR(lead.m + 800, lead.n, rp, lead.col_idx, lead.val)


@pytest.mark.parametrize("fmt", FORMATS)
def test_uniform_2k_all_p_and_tiles(fmt):
    a = I.uniform_rows()
    x = I.vector(a.n, I.SEED_BASE)
    want = oracle_spmv(a, fmt, x)
    for P in (3, 4, 7):
        for tile in TILES:
            y = gpu_spmv(a, fmt, P, x, tile=tile)
            assert normwise(y, want) <= TOL64, (P, tile)


@pytest.mark.parametrize("fmt", FORMATS)
def test_small_set_alpha_beta(fmt):
    for name, a in _small_set():
        x = I.vector(a.n, 7)
        y0 = I.y_vector(a.m, 8)
        for alpha, beta in ((1.0, 0.0), (-1.5, 0.75), (2.0, 1.0)):
            want = oracle_spmv(a, fmt, x, alpha, beta, y0)
            for P in (1, 5, 148, a.nnz + 5):
                y = gpu_spmv(a, fmt, P, x, alpha, beta, y0 if beta else None,
                             tile=256)
                assert normwise(y, want) <= TOL64, (name, alpha, beta, P)


@pytest.mark.parametrize("fmt", FORMATS)
def test_integer_valued_bit_exact(fmt):
    for name, a0 in _small_set():
        a, x = I.integer_twin(a0, seed=9)
        want = oracle_spmv(a, fmt, x)
        for P in (1, 2, 7, 148, 4096):
            for tile in (256, 1024):
                y = gpu_spmv(a, fmt, P, x, tile=tile)
                assert np.array_equal(y, want), (name, P, tile)


@pytest.mark.parametrize("fmt", FORMATS)
def test_empty_matrix_and_beta(fmt):
    a = I.csr_from_triplets(37, 11, [], [], [])
    x = I.vector(11, 1)
    y0 = I.y_vector(37, 2)
    assert np.array_equal(gpu_spmv(a, fmt, 4, x), np.zeros(37))
    assert np.array_equal(gpu_spmv(a, fmt, 4, x, 1.0, 2.0, y0), 2.0 * y0)


@pytest.mark.parametrize("fmt", FORMATS)
def test_hub_row_spanning_all_partitions(fmt):
    n = 50_000
    a0 = I.csr_from_triplets(3, n, [1] * n, list(range(n)), np.ones(n))
    a, x = I.integer_twin(a0, seed=3)
    want = oracle_spmv(a, fmt, x)
    for P in (2, 148, 9472):
        assert np.array_equal(gpu_spmv(a, fmt, P, x), want)


@pytest.mark.parametrize("fmt", FORMATS)
def test_direct_loads_match_streaming(fmt):
    """The direct-load (default) and bulk-copy staging (MSREP_STREAM_TMA)
    kernels run the same arithmetic: identical results for CSR and COO, and
    for CSC within atomic-add reordering."""
    a = I.rmat(scale=12, nnz=40_000, seed=13)
    x = I.vector(a.n, 4)
    for tile in (256, 512):
        y0 = gpu_spmv(a, fmt, 37, x, tile=tile)
        y1 = gpu_spmv(a, fmt, 37, x, tile=tile, flags=0x40)
        if fmt == "csc":
            assert normwise(y1, y0) <= TOL64
        else:
            assert np.array_equal(y0, y1)


def test_no_kernel_gave_up_a_wait():
    import paper_2209_07552_gb300 as M
    a = I.uniform_rows()
    gpu_spmv(a, "csr", 4, I.vector(a.n, 1))
    assert M.native.msrep_device_status() == 0


@pytest.mark.parametrize("fmt", ("csr", "coo"))
def test_atomic_free_formats_are_deterministic(fmt):
    a = I.rmat(scale=12, nnz=40_000, seed=12)
    x = I.vector(a.n, 3)
    ys = gpu_spmv(a, fmt, 148, x, repeat=3)
    assert all(np.array_equal(ys[0], v) for v in ys[1:])


# --------------------------------------------------------------------------
# full-size workloads
# --------------------------------------------------------------------------

@pytest.mark.slow
@pytest.mark.parametrize("fmt", FORMATS)
def test_rmat_full_size(fmt, rmat_full):
    a = rmat_full
    x = I.vector(a.n, I.SEED_BASE + 1)
    want = oracle_spmv(a, fmt, x)
    for P in (148, 148 * 16, 148 * 64):
        y = gpu_spmv(a, fmt, P, x)
        assert normwise(y, want) <= TOL64, P


@pytest.mark.slow
@pytest.mark.parametrize("fmt", FORMATS)
def test_laplacian_full_size(fmt, laplace_full):
    a = laplace_full
    g = 2048
    i, j = np.divmod(np.arange(a.m), g)
    # closed form with x = 1: number of off-grid neighbours, bit-exact
    off = ((i == 0).astype(int) + (i == g - 1) + (j == 0) + (j == g - 1))
    assert np.array_equal(gpu_spmv(a, fmt, 148 * 16, np.ones(a.n)), off.astype(float))
    x = I.vector(a.n, I.SEED_BASE + 1)
    y = gpu_spmv(a, fmt, 148 * 16, x)
    assert normwise(y, oracle_spmv(a, fmt, x)) <= TOL64


@pytest.mark.slow
def test_rmat_integer_twin_full_size_bit_exact(rmat_full):
    a, x = I.integer_twin(rmat_full, seed=11)
    want = oracle_spmv(a, "csr", x)
    for fmt in FORMATS:
        assert np.array_equal(gpu_spmv(a, fmt, 148 * 64, x), want), fmt
