"""Low-precision form: FP32 / BF16 values, FP32 x and y, FP32 accumulation
with TwoSum compensation, FP64 merge of split rows.

Errors are stated two ways:
 (i)  against the FP64 oracle on the original FP64 values and x, with the
      tolerances 1e-5 (FP32 values) and 1e-2 (BF16 values), normwise;
 (ii) against the FP64 oracle on the values and x as stored (dequantised),
      which isolates the arithmetic.  The bound is the classical one for
      recursive summation of a row of L products in binary32 (Higham,
      "Accuracy and Stability of Numerical Algorithms", Sec. 3.1):
      |err_r| <= (L_r + 2) u (|A| |x|)_r + u |y_r|, u = 2^-24, which also
      covers compensated rows (their error is about u |y_r|); the test
      requires ||y - y_stored|| <= ||bound|| over all rows.
"""
import numpy as np
import pytest

from helpers import FORMATS, gpu_spmv, normwise, oracle_spmv
from paper_2209_07552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "bf16": 1e-2}
U32 = 2.0 ** -24


def _stored(a, dt):
    v = I.to_f32(a.val).astype(np.float64) if dt == "f32" else \
        I.bf16_to_f32(I.bf16_bits(a.val)).astype(np.float64)
    return I.CSR(a.m, a.n, a.row_ptr, a.col_idx, v)


def _row_bound(a, x, yref, fmt):
    absa = I.CSR(a.m, a.n, a.row_ptr, a.col_idx, np.abs(a.val))
    ax = oracle_spmv(absa, fmt, np.abs(x))
    L = np.diff(a.row_ptr.astype(np.int64)).astype(np.float64)
    return (L + 2) * U32 * ax + U32 * np.abs(yref)


def _check(a, fmt, P, dt, x64, flags=0, tile=0):
    """Returns (normwise error vs original FP64 inputs,
    ||y - y_stored||, ||bound||)."""
    x32 = I.to_f32(x64).astype(np.float64)
    y = gpu_spmv(a, fmt, P, x32, val_dtype=dt, flags=flags, tile=tile)
    e_orig = normwise(y, oracle_spmv(a, fmt, x64))
    st = _stored(a, dt)
    ys = oracle_spmv(st, fmt, x32)
    return e_orig, np.linalg.norm(y - ys), np.linalg.norm(_row_bound(st, x32, ys, fmt))


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_precision_small(fmt, dt):
    a = I.rmat(scale=13, nnz=100_000, seed=21)
    x = I.vector(a.n, 22)
    for P in (7, 148, 2048):
        e_orig, e_arith, bound = _check(a, fmt, P, dt, x)
        assert e_orig <= TOL[dt], (P, e_orig)
        assert e_arith <= bound, (P, e_arith, bound)


@pytest.mark.slow
@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("fmt", FORMATS)
def test_precision_rmat_full_size(fmt, dt, rmat_full):
    x = I.vector(rmat_full.n, I.SEED_BASE + 1)
    e_orig, e_arith, bound = _check(rmat_full, fmt, 148 * 16, dt, x)
    assert e_orig <= TOL[dt]
    assert e_arith <= bound


def _cancel_matrix(L, rows):
    """Each row: (2^24, 1, -2^24) repeated L/3 times; with x = 1 the exact
    row sum is L/3, while plain binary32 accumulation loses every 1."""
    pat = np.tile(np.array([2.0**24, 1.0, -(2.0**24)]), L // 3)
    r = np.repeat(np.arange(rows), pat.shape[0])
    c = np.tile(np.arange(pat.shape[0]), rows)
    v = np.tile(pat, rows)
    return I.csr_from_triplets(rows, pat.shape[0], r, c, v), L // 3


@pytest.mark.parametrize("fmt", ("csr", "coo"))
def test_compensation_long_rows_exact(fmt):
    a, exact = _cancel_matrix(900, 4)   # rows of 900 > 256 nonzeros
    x = np.ones(a.n)
    for P in (1, 3, 17):                # also split rows across partitions
        y = gpu_spmv(a, fmt, P, x, val_dtype="f32", tile=256)
        assert np.array_equal(y, np.full(4, float(exact))), (P, y)
    y_plain = gpu_spmv(a, fmt, 1, x, val_dtype="f32", tile=512,
                       flags=0x20)   # MSREP_COMP_NONE
    assert np.all(y_plain != exact)


@pytest.mark.parametrize("fmt", ("csr", "coo"))
def test_compensation_split_short_rows(fmt):
    """Rows of 60 nonzeros (short) cut by many partitions are compensated
    because they are split."""
    a, exact = _cancel_matrix(60, 40)
    x = np.ones(a.n)
    y = gpu_spmv(a, fmt, 97, x, val_dtype="f32", tile=256)
    assert np.array_equal(y, np.full(40, float(exact)))


def test_csc_low_precision_merges_in_fp64():
    a, exact = _cancel_matrix(900, 4)
    y = gpu_spmv(a, "csc", 5, np.ones(a.n), val_dtype="f32", tile=256)
    assert np.array_equal(y, np.full(4, float(exact)))


@pytest.mark.parametrize("fmt", ["csc", "coo_col"])
def test_low_precision_scatter_widening_special_values(fmt):
    """The scatter forms widen FP32 values and x to FP64 by integer
    operations (and the hardware conversion for zero, subnormal, infinite
    and NaN inputs).  Each row here holds one product, so the FP64
    accumulator holds it exactly and y must be the oracle's product rounded
    to binary32, bit for bit: values and x cover +-0, binary32 subnormals,
    the smallest and largest normal exponents and ordinary numbers."""
    g = np.random.default_rng(5)
    specials = np.array([0.0, -0.0, 1e-40, -3e-39, 1.401298464324817e-45,
                         1.1754943508222875e-38, -1.1754943508222875e-38, 2.0**-126, 2.0**127,
                         -(2.0**127) * 1.5, 1.0, -1.0, 0.5, 3.0, 1e30, -1e-30])
    n = 600
    v = np.concatenate([specials, g.standard_normal(n - specials.size)]).astype(np.float32)
    xv = np.concatenate([specials[::-1], g.standard_normal(n - specials.size)]).astype(np.float32)
    perm = g.permutation(n)
    # column c holds one nonzero, at row perm[c]: row r's only product
    a = I.csr_from_triplets(n, n, perm, np.arange(n), v.astype(np.float64))
    x = xv.astype(np.float64)
    y = gpu_spmv(a, fmt, 7, x, val_dtype="f32", tile=256)
    want = oracle_spmv(a, "csr", x)           # exact products in FP64
    w32 = want.astype(np.float32)
    assert np.isfinite(w32).all()
    assert np.array_equal(y.astype(np.float32).view(np.uint32), w32.view(np.uint32))
