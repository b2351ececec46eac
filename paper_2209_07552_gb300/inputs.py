"""Seeded synthetic inputs for the msRep SpMV path.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It holds input synthesis and storage-format bookkeeping only
(which nonzero sits where, in which storage type); none of the method's
arithmetic (partitioning, products, sums, merges) is here.

Every array is drawn from its own counter-based Philox stream, keyed by
(seed, stream id), so that any array can be regenerated alone.  The default
seeds are ``20220915 + workload index`` (workload 0: the 2,000 x 2,000
uniform matrix; 1: R-MAT and 2D Laplacian; 3: the batched set; 4: the served
set).

The paper evaluates on SuiteSparse power-law matrices (Table 2), which are
not available here; the R-MAT generator supplies the same skewed
degree structure (Sec. 5.2 selects matrices with power-law exponent R in
[1, 4]).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20220915

# stream ids
_S_COLS, _S_VALS, _S_X, _S_Y, _S_RMAT_BITS, _S_RMAT_VALS, _S_SIZES, _S_ORDER = range(8)


def rng(seed: int, stream: int) -> np.random.Generator:
    """Counter-based Philox stream ``stream`` of ``seed``."""
    return np.random.Generator(np.random.Philox(key=(int(seed) << 32) | int(stream)))


@dataclass
class CSR:
    """CSR matrix (Sec. 2.1.2): row_ptr int32[m+1], col_idx int32[nnz], val."""
    m: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])


@dataclass
class CSC:
    """CSC matrix (Sec. 2.1.3): col_ptr int32[n+1], row_idx int32[nnz], val."""
    m: int
    n: int
    col_ptr: np.ndarray
    row_idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_idx.shape[0])


@dataclass
class COO:
    """COO matrix (Sec. 2.1.1): sorted by (row, col) unless made by
    csr_to_coo_by_col or csr_to_coo_unsorted."""
    m: int
    n: int
    row_idx: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_idx.shape[0])


# --------------------------------------------------------------------------
# format bookkeeping (integer permutations only)
# --------------------------------------------------------------------------

def row_ptr_from_counts(counts: np.ndarray) -> np.ndarray:
    ptr = np.zeros(counts.shape[0] + 1, np.int64)
    np.cumsum(counts, out=ptr[1:])
    if ptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 offsets")
    return ptr.astype(np.int32)


def csr_to_coo(a: CSR) -> COO:
    counts = np.diff(a.row_ptr.astype(np.int64))
    rows = np.repeat(np.arange(a.m, dtype=np.int32), counts)
    return COO(a.m, a.n, rows, a.col_idx.copy(), a.val.copy())


def csr_to_csc(a: CSR) -> CSC:
    """Stable reorder of the nonzeros by column; rows stay ascending inside
    each column because the CSR rows are visited in order."""
    rows = np.repeat(np.arange(a.m, dtype=np.int32),
                     np.diff(a.row_ptr.astype(np.int64)))
    order = np.argsort(a.col_idx, kind="stable")
    counts = np.bincount(a.col_idx, minlength=a.n)
    return CSC(a.m, a.n, row_ptr_from_counts(counts),
               rows[order].astype(np.int32), a.val[order].copy())


def csr_to_coo_by_col(a: CSR) -> COO:
    """COO sorted by (col, row): the nonzeros in CSC order."""
    c = csr_to_csc(a)
    cols = np.repeat(np.arange(a.n, dtype=np.int32), np.diff(c.col_ptr.astype(np.int64)))
    return COO(a.m, a.n, c.row_idx.copy(), cols, c.val.copy())


def csr_to_coo_unsorted(a: CSR, seed: int = SEED_BASE + 1) -> COO:
    """COO in no particular order: the nonzeros under a seeded random
    permutation (Philox stream _S_ORDER of ``seed``)."""
    q = csr_to_coo(a)
    order = rng(seed, _S_ORDER).permutation(q.nnz)
    return COO(a.m, a.n, q.row_idx[order].copy(), q.col_idx[order].copy(),
               q.val[order].copy())


def transpose_csr(a: CSR) -> CSR:
    """CSR of A^T; its arrays equal those of CSC(A) (Sec. 2.1.3)."""
    c = csr_to_csc(a)
    return CSR(a.n, a.m, c.col_ptr, c.row_idx, c.val)


def csr_from_triplets(m, n, rows, cols, vals) -> CSR:
    """Sort triplets by (row, col); duplicates must already be merged."""
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    order = np.lexsort((cols, rows))
    counts = np.bincount(rows, minlength=m) if rows.size else np.zeros(m, np.int64)
    return CSR(m, n, row_ptr_from_counts(counts), cols[order].astype(np.int32),
               np.asarray(vals)[order])


def dense_of(a: CSR) -> np.ndarray:
    d = np.zeros((a.m, a.n), np.float64)
    rows = np.repeat(np.arange(a.m), np.diff(a.row_ptr.astype(np.int64)))
    np.add.at(d, (rows, a.col_idx), a.val.astype(np.float64))
    return d


# --------------------------------------------------------------------------
# storage precisions of the low-precision form
# --------------------------------------------------------------------------

def to_f32(v: np.ndarray) -> np.ndarray:
    """Round to binary32 (round-to-nearest-even)."""
    return np.asarray(v, np.float64).astype(np.float32)


def bf16_bits(v: np.ndarray) -> np.ndarray:
    """bfloat16 storage bits of v: v is first rounded to binary32, then the
    binary32 pattern is rounded to its top 16 bits, nearest-even.  (NaN is
    not produced by the generators.)"""
    f = to_f32(v)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) >> 16
    return r.astype(np.uint16)


def bf16_to_f32(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, np.uint16).astype(np.uint32) << 16).view(np.float32)


# --------------------------------------------------------------------------
# workload 0: 2,000 x 2,000, exactly 10 distinct uniform columns per row
# --------------------------------------------------------------------------

def uniform_rows(m: int = 2000, n: int = 2000, per_row: int = 10,
                 seed: int = SEED_BASE + 0) -> CSR:
    gc = rng(seed, _S_COLS)
    cols = np.empty((m, per_row), np.int32)
    for r in range(m):
        cols[r] = np.sort(gc.choice(n, size=per_row, replace=False))
    val = rng(seed, _S_VALS).uniform(-1.0, 1.0, m * per_row)
    ptr = np.arange(0, m * per_row + 1, per_row, dtype=np.int32)
    return CSR(m, n, ptr, cols.reshape(-1), val,
               meta={"kind": "uniform", "per_row": per_row, "seed": seed})


def vector(n: int, seed: int, stream: int = _S_X, lo=-1.0, hi=1.0) -> np.ndarray:
    """Dense FP64 vector ~ U(lo, hi)."""
    return rng(seed, stream).uniform(lo, hi, n)


def y_vector(m: int, seed: int) -> np.ndarray:
    return rng(seed, _S_Y).uniform(-1.0, 1.0, m)


# --------------------------------------------------------------------------
# workload 1a: R-MAT power-law matrix
# --------------------------------------------------------------------------

def rmat(scale: int = 20, nnz: int = 1 << 24, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = SEED_BASE + 1) -> CSR:
    """R-MAT (Chakrabarti, Zhan, Faloutsos 2004) on 2^scale x 2^scale.

    Edges are drawn one after another; each edge descends `scale` quadrant
    levels (a: top-left, b: top-right, c: bottom-left, d: bottom-right, most
    significant bit first), with no noise and no vertex permutation.  Level l
    of edge j uses the 32-bit uniform word j of draw block l of the Philox
    stream; quadrant thresholds are a, a+b, a+b+c scaled to 2^32.  Each
    occurrence of an edge adds one N(0,1) draw (stream position = edge index)
    to that entry, summed in edge order.  Sampling stops at the edge that
    makes the count of distinct entries exactly `nnz`; later edges are
    discarded.  The result is sorted by (row, col)."""
    n_side = 1 << scale
    ta = np.uint32(int(a * 2**32))
    tab = np.uint32(int((a + b) * 2**32))
    tabc = np.uint32(int((a + b + c) * 2**32))
    draw = int(nnz * 1.08) + 1024
    while True:
        bits = rng(seed, _S_RMAT_BITS)
        rows = np.zeros(draw, np.uint32)
        cols = np.zeros(draw, np.uint32)
        t1 = np.empty(draw, bool)
        t2 = np.empty(draw, bool)
        for _ in range(scale):
            u = bits.integers(0, 2**32, draw, dtype=np.uint32)
            np.left_shift(rows, 1, out=rows)
            np.left_shift(cols, 1, out=cols)
            np.greater_equal(u, tab, out=t1)          # bottom half: c or d
            rows |= t1
            np.greater_equal(u, ta, out=t2)           # b, c or d
            np.logical_xor(t2, t1, out=t2)            # b
            np.greater_equal(u, tabc, out=t1)         # d
            np.logical_xor(t2, t1, out=t2)            # b or d: right half
            cols |= t2
        del u, t1, t2
        keys = (rows.astype(np.int64) << scale) | cols
        del rows, cols
        order = np.argsort(keys)
        sk = keys[order]
        head = np.empty(draw, bool)
        head[0] = True
        np.not_equal(sk[1:], sk[:-1], out=head[1:])
        starts = np.flatnonzero(head)
        if starts.shape[0] < nnz:
            draw = int(draw * 1.1)
            continue
        first = np.minimum.reduceat(order, starts)
        cut = int(np.partition(first, nnz - 1)[nnz - 1])
        run_id = np.cumsum(head) - 1
        inv = np.empty(draw, np.int64)
        inv[order] = run_id
        vals = rng(seed, _S_RMAT_VALS).standard_normal(cut + 1)
        summed = np.bincount(inv[: cut + 1], weights=vals,
                             minlength=starts.shape[0])
        keep = first <= cut
        ukeys = sk[starts][keep]
        rows = ukeys >> scale
        cols = (ukeys & (n_side - 1)).astype(np.int32)
        counts = np.bincount(rows, minlength=n_side)
        return CSR(n_side, n_side, row_ptr_from_counts(counts), cols,
                   summed[keep],
                   meta={"kind": "rmat", "scale": scale, "a": a, "b": b,
                         "c": c, "edges_drawn": cut + 1, "seed": seed})


def power_law_exponent(a: CSR) -> float:
    """Fitted exponent R of P(k) ~ k^-R over nonzeros per column (Sec. 5.2),
    by the discrete maximum-likelihood estimate over columns with k >= 1
    (Clauset, Shalizi, Newman 2009, Eq. 3.7 with k_min = 1)."""
    k = np.bincount(a.col_idx, minlength=a.n)
    k = k[k >= 1].astype(np.float64)
    return float(1.0 + k.size / np.sum(np.log(k / 0.5)))


# --------------------------------------------------------------------------
# workload 1b: 2D 5-point Laplacian
# --------------------------------------------------------------------------

def laplace5(g: int = 2048) -> CSR:
    """5-point Laplacian on a g x g grid, natural (row-major) ordering,
    Dirichlet boundary (neighbours off the grid are dropped), diagonal 4,
    off-diagonals -1.  Node (i, j) is row i*g + j."""
    N = g * g
    idx = np.arange(N, dtype=np.int64)
    gi, gj = idx // g, idx % g
    # per row, in ascending column order: north, west, centre, east, south
    offs = [(-g, gi > 0), (-1, gj > 0), (0, np.ones(N, bool)), (1, gj < g - 1),
            (g, gi < g - 1)]
    counts = sum(mask.astype(np.int64) for _, mask in offs)
    ptr = row_ptr_from_counts(counts)
    nnz = int(ptr[-1])
    cols = np.empty(nnz, np.int32)
    vals = np.empty(nnz, np.float64)
    pos = ptr[:-1].astype(np.int64).copy()
    for off, mask in offs:
        r = idx[mask]
        cols[pos[r]] = (r + off).astype(np.int32)
        vals[pos[r]] = 4.0 if off == 0 else -1.0
        pos[r] += 1
    return CSR(N, N, ptr, cols, vals, meta={"kind": "laplace5", "grid": g})


# --------------------------------------------------------------------------
# integer-valued twin: every partial sum is an exact integer
# --------------------------------------------------------------------------

def integer_twin(a: CSR, seed: int, vmax: int = 3, xmax: int = 4):
    """Same pattern as `a`, values in {-vmax..vmax}, x in {-xmax..xmax}."""
    v = rng(seed, 101).integers(-vmax, vmax + 1, a.nnz).astype(np.float64)
    x = rng(seed, 102).integers(-xmax, xmax + 1, a.n).astype(np.float64)
    return CSR(a.m, a.n, a.row_ptr, a.col_idx, v, meta=dict(a.meta)), x


# --------------------------------------------------------------------------
# workload 3: batch of uneven CSR matrices
# --------------------------------------------------------------------------

def batched_sizes(count: int = 512, seed: int = SEED_BASE + 3,
                  m_lo: float = 1e3, m_hi: float = 2e5,
                  mu_lo: float = 4.0, mu_hi: float = 64.0):
    """Per matrix: m = floor(exp(U(ln m_lo, ln m_hi))) and mean row length
    mu ~ U(mu_lo, mu_hi)."""
    g = rng(seed, _S_SIZES)
    m = np.floor(np.exp(g.uniform(math.log(m_lo), math.log(m_hi), count)))
    mu = g.uniform(mu_lo, mu_hi, count)
    return m.astype(np.int64), mu


def geometric_matrix(m: int, mu: float, seed: int, dtype=np.float32) -> CSR:
    """Square m x m matrix; row lengths ~ Geometric(p = 1/mu) on {1, 2, ...}
    clamped to m; columns distinct and sorted within a row.  A row of
    length L takes the order statistics of L uniforms on [0, 1) (normalised
    cumulative sums of L+1 exponential gaps), maps them to draws in
    {0..m-L} and adds 0..L-1, which gives L distinct sorted columns.
    Values ~ U(-1, 1)."""
    g = rng(seed, _S_COLS)
    lens = np.minimum(g.geometric(1.0 / mu, m), m).astype(np.int64)
    return _rows_of_lengths(m, lens, g, seed, dtype, {"kind": "geometric", "mu": mu,
                                                      "seed": seed})


def block_imbalance_matrix(m: int, blocks: int, heavy_len: int, ratio: float, seed: int,
                           dtype=np.float64) -> CSR:
    """The two-level nonzero distribution of the paper's imbalance experiment
    (Sec. 2.3, Fig. 5): the m rows fall in `blocks` equal row blocks; rows
    of the first half of the blocks hold heavy_len nonzeros each, rows of
    the other half round(heavy_len / ratio) (at least 1), so that an equal
    split of the rows gives half the blocks 1/ratio of the others' nonzeros.
    Columns distinct, sorted and uniform over the m columns; values
    U(-1, 1)."""
    light = max(1, int(round(heavy_len / ratio)))
    r = np.arange(m, dtype=np.int64)
    blk = (r * blocks) // m  # the row block of each row, as floor(i m / blocks) cuts it
    lens = np.where(blk < blocks // 2, heavy_len, light).astype(np.int64)
    g = rng(seed, _S_COLS)
    return _rows_of_lengths(m, lens, g, seed, dtype,
                            {"kind": "block_imbalance", "blocks": blocks,
                             "heavy_len": heavy_len, "light_len": light, "ratio": ratio,
                             "seed": seed})


def _rows_of_lengths(m, lens, g, seed, dtype, meta) -> CSR:
    """Square m x m CSR whose row r has lens[r] distinct sorted uniform
    columns (the order-statistics construction of geometric_matrix)."""
    ptr = row_ptr_from_counts(lens)
    nnz = int(ptr[-1])
    starts = ptr[:-1].astype(np.int64)
    # L+1 gaps per row; cumulative sums inside each row, normalised by the
    # row's total, are L sorted uniforms
    gaps = g.standard_exponential(nnz + m)
    cs = np.cumsum(gaps)
    gap_starts = starts + np.arange(m, dtype=np.int64)        # row r's gaps start here
    before = np.where(gap_starts > 0, cs[np.maximum(gap_starts - 1, 0)], 0.0)
    row_total = cs[gap_starts + lens] - before                 # sum of the row's L+1 gaps
    rows = np.repeat(np.arange(m, dtype=np.int64), lens)
    within = np.arange(nnz, dtype=np.int64) - starts[rows]
    u = (cs[gap_starts[rows] + within] - before[rows]) / row_total[rows]
    span = (m - lens + 1)[rows]
    draw = np.minimum(np.floor(u * span).astype(np.int64), span - 1)
    cols = (draw + within).astype(np.int32)
    val = rng(seed, _S_VALS).uniform(-1.0, 1.0, nnz).astype(dtype)
    return CSR(m, m, ptr, cols, val, meta=meta)


def _batched_one(job):
    i, m, mu, seed, dtype = job
    s = seed * 1000 + i
    a = geometric_matrix(int(m), float(mu), s, dtype)
    return a, vector(int(m), s).astype(dtype)


def batched_set_parallel(count: int = 512, seed: int = SEED_BASE + 3, dtype=np.float32,
                         workers: int = 0, **size_kw):
    """batched_set computed by a pool of spawned worker processes (same
    result, element for element)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    ms, mus = batched_sizes(count, seed, **size_kw)
    jobs = [(i, int(m), float(mu), seed, dtype) for i, (m, mu) in enumerate(zip(ms, mus))]
    workers = workers or min(16, os.cpu_count() or 1)
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        out = list(ex.map(_batched_one, jobs, chunksize=4))
    return [a for a, _ in out], [x for _, x in out]


def batched_set(count: int = 512, seed: int = SEED_BASE + 3, dtype=np.float32,
                **size_kw):
    """The batched workload: `count` independent square CSR matrices and one
    x per matrix (FP32 by default)."""
    ms, mus = batched_sizes(count, seed, **size_kw)
    mats, xs = [], []
    for i, (m, mu) in enumerate(zip(ms, mus)):
        s = seed * 1000 + i
        mats.append(geometric_matrix(int(m), float(mu), s, dtype))
        xs.append(vector(int(m), s).astype(dtype))
    return mats, xs


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int):
    """Arrival times (s) of a Poisson stream: exponential gaps."""
    g = rng(seed, 201)
    n = int(rate_hz * duration_s * 1.2) + 16
    t = np.cumsum(g.exponential(1.0 / rate_hz, n))
    return t[t < duration_s]


# --------------------------------------------------------------------------
# on-disk cache of the large generated matrices (regenerated when absent)
# --------------------------------------------------------------------------

def _cache_dir() -> str:
    d = os.environ.get("MSREP_INPUT_CACHE")
    if not d:
        d = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                         ".input_cache")
    return d


def cached_csr(key: str, make) -> CSR:
    """make() once, then reload from an .npz under the cache directory."""
    path = os.path.join(_cache_dir(), key + ".npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        return CSR(int(z["m"]), int(z["n"]), z["row_ptr"], z["col_idx"], z["val"],
                   meta={"cached": key})
    a = make()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez(tmp, m=a.m, n=a.n, row_ptr=a.row_ptr, col_idx=a.col_idx, val=a.val)
        os.replace(tmp, path)
    except OSError:
        pass
    return a


def rmat_full(seed: int = SEED_BASE + 1) -> CSR:
    """The 2^20 x 2^20, 2^24-nonzero R-MAT matrix (a,b,c,d = .57/.19/.19/.05)."""
    return cached_csr(f"rmat20_{seed}", lambda: rmat(seed=seed))


def laplace_full() -> CSR:
    """The 2048 x 2048 grid 5-point Laplacian (4,194,304 rows)."""
    return cached_csr("laplace2048", lambda: laplace5(2048))
