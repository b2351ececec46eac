"""Pins of the CPU oracle against facts it does not compute itself.

Each test checks the oracle against the paper's definitions restated by hand
(the hand-worked fixture), closed forms, a library routine that implements a
special case independently (numpy dense products, np.searchsorted), brute
force on tiny inputs, or exact integer arithmetic.  None re-types the
oracle's own loops.  No GPU is used.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2209_07552_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _hand():
    with open(os.path.join(GOLD, "hand_6x6.json")) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Hand-worked example (Alg. 1-7 applied by hand)
# --------------------------------------------------------------------------

def test_hand_example_pcsr():
    g = _hand()
    p = O.partition_csr(g["csr"]["row_ptr"], 9, g["np"], with_local=True)
    e = g["pcsr"]
    assert p["start_idx"].tolist() == e["start_idx"]
    assert p["end_idx"].tolist() == e["end_idx"]
    assert p["start_major"].tolist() == e["start_row"]
    assert p["end_major"].tolist() == e["end_row"]
    assert p["start_flag"].tolist() == e["start_flag"]
    flat = [v for part in e["local_row_ptr"] for v in part]
    assert p["local"].tolist() == flat
    assert np.diff(p["local_off"]).tolist() == [len(v) for v in e["local_row_ptr"]]


def test_hand_example_pcsc_pcoo():
    g = _hand()
    c = O.partition_csc(g["csc"]["col_ptr"], 9, g["np"], with_local=True)
    e = g["pcsc"]
    assert c["start_idx"].tolist() == e["start_idx"]
    assert c["start_major"].tolist() == e["start_col"]
    assert c["end_major"].tolist() == e["end_col"]
    assert c["start_flag"].tolist() == e["start_flag"]
    assert c["local"].tolist() == [v for part in e["local_col_ptr"] for v in part]
    q = O.partition_coo(g["coo"]["row_idx"], g["np"], with_local=True)
    e = g["pcoo"]
    assert q["start_major"].tolist() == e["start_row"]
    assert q["end_major"].tolist() == e["end_row"]
    assert q["start_flag"].tolist() == e["start_flag"]
    assert q["local"].tolist() == e["local_row_idx"]


def test_hand_example_merge_path_and_other_coo_orders():
    g = _hand()
    p = O.partition_merge_path(g["csr"]["row_ptr"], 9, g["np"], with_local=True)
    e = g["pcsr_merge_path"]
    assert p["cut_row"].tolist() == e["cut_row"]
    assert p["start_idx"].tolist() == e["start_idx"]
    assert p["end_idx"].tolist() == e["end_idx"]
    assert p["start_major"].tolist() == e["start_row"]
    assert p["end_major"].tolist() == e["end_row"]
    assert p["start_flag"].tolist() == e["start_flag"]
    assert p["local"].tolist() == [v for part in e["local_row_ptr"] for v in part]
    x, yin, a, b = g["x"], g["y_in"], g["alpha"], g["beta"]
    assert O.pspmv_csr(6, g["csr"]["row_ptr"], g["csr"]["col_idx"], g["csr"]["val"], p,
                       x, a, b, yin).tolist() == g["y"]
    e = g["pcoo_by_col"]
    q = O.partition_coo_by_col(e["col_idx"], g["np"], with_local=True)
    assert q["start_major"].tolist() == e["start_col"]
    assert q["end_major"].tolist() == e["end_col"]
    assert q["start_flag"].tolist() == e["start_flag"]
    assert q["local"].tolist() == e["local_col_idx"]
    assert O.pspmv_coo_scatter(6, e["row_idx"], e["col_idx"], g["csc"]["val"], q, x, a, b,
                               yin).tolist() == g["y"]
    e = g["pcoo_unsorted"]
    u = O.partition_coo_unsorted(g["coo"]["row_idx"], 6, g["np"])
    for key, name in (("start_idx", "start_idx"), ("end_idx", "end_idx"),
                      ("start_major", "start_row"), ("end_major", "end_row"),
                      ("start_flag", "start_flag")):
        assert u[key].tolist() == e[name]


def test_hand_example_spmv_all_formats():
    g = _hand()
    x, yin = g["x"], g["y_in"]
    a, b = g["alpha"], g["beta"]
    ys = [
        O.spmv_csr(6, g["csr"]["row_ptr"], g["csr"]["col_idx"], g["csr"]["val"],
                   x, a, b, yin),
        O.spmv_csc(6, 6, g["csc"]["col_ptr"], g["csc"]["row_idx"],
                   g["csc"]["val"], x, a, b, yin),
        O.spmv_coo(6, g["coo"]["row_idx"], g["coo"]["col_idx"], g["coo"]["val"],
                   x, a, b, yin),
    ]
    p = O.partition_csr(g["csr"]["row_ptr"], 9, 4)
    ys.append(O.pspmv_csr(6, g["csr"]["row_ptr"], g["csr"]["col_idx"],
                          g["csr"]["val"], p, x, a, b, yin))
    pc = O.partition_csc(g["csc"]["col_ptr"], 9, 4)
    ys.append(O.pspmv_csc(6, g["csc"]["col_ptr"], g["csc"]["row_idx"],
                          g["csc"]["val"], pc, x, a, b, yin))
    pq = O.partition_coo(g["coo"]["row_idx"], 4)
    ys.append(O.pspmv_coo(6, g["coo"]["row_idx"], g["coo"]["col_idx"],
                          g["coo"]["val"], pq, x, a, b, yin))
    for y in ys:
        assert y.tolist() == g["y"]
    assert O.spmv_csr(6, g["csr"]["row_ptr"], g["csr"]["col_idx"],
                      g["csr"]["val"], x).tolist() == g["Ax"]


# --------------------------------------------------------------------------
# Small random matrices against numpy's dense product
# --------------------------------------------------------------------------

def _tiny(seed, m, n, density):
    g = I.rng(seed, 0)
    d = np.where(g.random((m, n)) < density, g.uniform(-1, 1, (m, n)), 0.0)
    if m > 2:
        d[m // 2] = 0.0          # an empty row in the middle
        d[0] = 0.0               # and a leading one
    if n > 2:
        d[:, n - 1] = 0.0        # an empty trailing column
    r, c = np.nonzero(d)
    a = I.csr_from_triplets(m, n, r, c, d[r, c])
    return d, a


@pytest.mark.parametrize("seed", range(12))
def test_dense_matvec_all_formats(seed):
    g = I.rng(seed, 9)
    m, n = int(g.integers(1, 17)), int(g.integers(1, 17))
    d, a = _tiny(seed, m, n, float(g.uniform(0.05, 0.9)))
    x = g.uniform(-1, 1, n)
    yin = g.uniform(-1, 1, m)
    alpha, beta = float(g.uniform(-2, 2)), float(g.uniform(-2, 2))
    want = alpha * (d @ x) + beta * yin
    c = I.csr_to_csc(a)
    q = I.csr_to_coo(a)
    got = [
        O.spmv_csr(m, a.row_ptr, a.col_idx, a.val, x, alpha, beta, yin),
        O.spmv_csc(m, n, c.col_ptr, c.row_idx, c.val, x, alpha, beta, yin),
        O.spmv_coo(m, q.row_idx, q.col_idx, q.val, x, alpha, beta, yin),
    ]
    for y in got:
        np.testing.assert_allclose(y, want, rtol=1e-13, atol=1e-13)
    for P in (1, 2, 3, 5, max(1, a.nnz), a.nnz + 3):
        p = O.partition_csr(a.row_ptr, a.nnz, P)
        np.testing.assert_allclose(
            O.pspmv_csr(m, a.row_ptr, a.col_idx, a.val, p, x, alpha, beta, yin),
            want, rtol=1e-13, atol=1e-13)
        pc = O.partition_csc(c.col_ptr, c.nnz, P)
        np.testing.assert_allclose(
            O.pspmv_csc(m, c.col_ptr, c.row_idx, c.val, pc, x, alpha, beta, yin),
            want, rtol=1e-13, atol=1e-13)
        pq = O.partition_coo(q.row_idx, P)
        np.testing.assert_allclose(
            O.pspmv_coo(m, q.row_idx, q.col_idx, q.val, pq, x, alpha, beta, yin),
            want, rtol=1e-13, atol=1e-13)


def test_dense_spmm():
    d, a = _tiny(3, 13, 11, 0.4)
    g = I.rng(3, 10)
    X = g.uniform(-1, 1, (11, 5))
    Y0 = g.uniform(-1, 1, (13, 5))
    np.testing.assert_allclose(
        O.spmm_csr(13, a.row_ptr, a.col_idx, a.val, X, 0.5, 2.0, Y0),
        0.5 * (d @ X) + 2.0 * Y0, rtol=1e-13, atol=1e-13)


def test_beta_zero_ignores_nan_y():
    d, a = _tiny(5, 9, 7, 0.5)
    x = np.ones(7)
    y = O.spmv_csr(9, a.row_ptr, a.col_idx, a.val, x, 1.0, 0.0,
                   np.full(9, np.nan))
    assert np.all(np.isfinite(y))
    np.testing.assert_allclose(y, d.sum(axis=1), rtol=1e-14, atol=1e-14)


# --------------------------------------------------------------------------
# Exact special cases
# --------------------------------------------------------------------------

def test_identity_and_permutation_bit_exact():
    m = 1000
    g = I.rng(11, 0)
    x = g.uniform(-1, 1, m)
    eye = I.CSR(m, m, np.arange(m + 1, dtype=np.int32),
                np.arange(m, dtype=np.int32), np.ones(m))
    assert np.array_equal(O.spmv_csr(m, eye.row_ptr, eye.col_idx, eye.val, x), x)
    pi = g.permutation(m).astype(np.int32)
    perm = I.CSR(m, m, np.arange(m + 1, dtype=np.int32), pi, np.ones(m))
    assert np.array_equal(O.spmv_csr(m, perm.row_ptr, perm.col_idx, perm.val, x),
                          x[pi])
    c = I.csr_to_csc(perm)
    assert np.array_equal(O.spmv_csc(m, m, c.col_ptr, c.row_idx, c.val, x), x[pi])
    q = I.csr_to_coo(perm)
    assert np.array_equal(O.spmv_coo(m, q.row_idx, q.col_idx, q.val, x), x[pi])


def test_integer_valued_exact_against_python_ints():
    a0 = I.rmat(scale=9, nnz=3000, seed=77)
    a, x = I.integer_twin(a0, seed=78)
    rows = np.repeat(np.arange(a.m), np.diff(a.row_ptr))
    want = [0] * a.m
    for r, c, v in zip(rows.tolist(), a.col_idx.tolist(), a.val.tolist()):
        want[r] += int(v) * int(x[c])
    y = O.spmv_csr(a.m, a.row_ptr, a.col_idx, a.val, x)
    assert y.tolist() == [float(w) for w in want]
    q = I.csr_to_coo(a)
    assert O.spmv_coo(a.m, q.row_idx, q.col_idx, q.val, x).tolist() == y.tolist()
    c = I.csr_to_csc(a)
    assert O.spmv_csc(a.m, a.n, c.col_ptr, c.row_idx, c.val, x).tolist() == y.tolist()


def test_ones_gives_row_sums_integer():
    a0 = I.rmat(scale=10, nnz=6000, seed=79)
    a, _ = I.integer_twin(a0, seed=80)
    y = O.spmv_csr(a.m, a.row_ptr, a.col_idx, a.val, np.ones(a.n))
    sums = np.zeros(a.m)
    rows = np.repeat(np.arange(a.m), np.diff(a.row_ptr))
    np.add.at(sums, rows, a.val)      # integer sums: exact in any order
    assert np.array_equal(y, sums)


@pytest.mark.slow
def test_laplacian_closed_forms_full_size():
    g = 2048
    a = I.laplace5(g)
    assert a.nnz == 5 * g * g - 4 * g
    # x = 1: 4 minus the number of on-grid neighbours = number of off-grid ones
    y = O.spmv_csr(a.m, a.row_ptr, a.col_idx, a.val, np.ones(a.n))
    i, j = np.divmod(np.arange(a.m), g)
    off = ((i == 0).astype(int) + (i == g - 1) + (j == 0) + (j == g - 1))
    assert np.array_equal(y, off.astype(np.float64))
    # x = i + 2j (affine): y is the sum of x extended to the off-grid neighbours
    x = (i + 2.0 * j)
    y = O.spmv_csr(a.m, a.row_ptr, a.col_idx, a.val, x)
    want = np.zeros(a.m)
    want += np.where(i == 0, (i - 1) + 2.0 * j, 0.0)
    want += np.where(i == g - 1, (i + 1) + 2.0 * j, 0.0)
    want += np.where(j == 0, i + 2.0 * (j - 1), 0.0)
    want += np.where(j == g - 1, i + 2.0 * (j + 1), 0.0)
    assert np.array_equal(y, want)
    assert np.count_nonzero(y[(i > 0) & (i < g - 1) & (j > 0) & (j < g - 1)]) == 0


# --------------------------------------------------------------------------
# Partitioning: brute force, closed forms and invariants
# --------------------------------------------------------------------------

def _brute_partition(ptr, nnz, P):
    """Alg. 2 read literally, with the owner row from np.searchsorted."""
    ptr = np.asarray(ptr, np.int64)
    m = ptr.shape[0] - 1
    out = {"start_idx": [], "end_idx": [], "start_major": [], "end_major": [],
           "start_flag": []}
    for i in range(P):
        s = (i * nnz) // P
        e = ((i + 1) * nnz) // P - 1
        out["start_idx"].append(s)
        out["end_idx"].append(e)
        if e < s:
            out["start_major"].append(0)
            out["end_major"].append(-1)
            out["start_flag"].append(0)
            continue
        sr = int(np.searchsorted(ptr[:m], s, side="right") - 1)
        er = int(np.searchsorted(ptr[:m], e, side="right") - 1)
        out["start_major"].append(sr)
        out["end_major"].append(er)
        out["start_flag"].append(int(s > ptr[sr]))
    return out


def _adversarial():
    mats = []
    mats.append(I.csr_from_triplets(7, 5, [], [], []))                 # nnz = 0
    mats.append(I.csr_from_triplets(1, 9, [0] * 9, list(range(9)),
                                    np.arange(1.0, 10.0)))               # m = 1
    r = [5] * 40                                                        # one hub row
    mats.append(I.csr_from_triplets(12, 40, r, list(range(40)),
                                    np.ones(40)))
    rows = [0, 0, 3, 3, 3, 9, 9, 9, 9, 9, 9, 14]                         # gaps + tail
    cols = [1, 4, 0, 2, 7, 0, 1, 2, 3, 5, 6, 7]
    mats.append(I.csr_from_triplets(20, 8, rows, cols, np.ones(len(rows))))
    d, a = _tiny(21, 16, 16, 0.3)
    mats.append(a)
    mats.append(I.rmat(scale=8, nnz=1500, seed=5))
    return mats


@pytest.mark.parametrize("k", range(6))
def test_partition_brute_force(k):
    a = _adversarial()[k]
    nnz = a.nnz
    for P in sorted({1, 2, 3, 4, 7, 16, max(1, nnz - 1), max(1, nnz),
                     nnz + 5}):
        got = O.partition_csr(a.row_ptr, nnz, P, with_local=True)
        want = _brute_partition(a.row_ptr, nnz, P)
        for key in want:
            assert got[key].tolist() == want[key], (key, P)
        # local pointers: slice of row_ptr shifted and clamped (Alg. 2 loop)
        for i in range(P):
            sl = got["local"][got["local_off"][i]:got["local_off"][i + 1]]
            s, e = want["start_idx"][i], want["end_idx"][i]
            sr, er = want["start_major"][i], want["end_major"][i]
            exp = [0] + [int(a.row_ptr[r]) - s for r in range(sr + 1, er + 1)]
            if e >= s:
                exp.append(e - s + 1)
            assert sl.tolist() == exp


def _check_invariants(ptr, nnz, P, p):
    s, e = p["start_idx"].astype(np.int64), p["end_idx"].astype(np.int64)
    ln = e - s + 1
    # the nnz ranges tile [0, nnz) exactly once, in order
    assert s[0] == 0 and e[-1] == nnz - 1
    assert np.all(s[1:] == e[:-1] + 1)
    # balanced: every length is floor or ceil of nnz/P
    assert set(np.unique(ln).tolist()) <= {nnz // P, -(-nnz // P)}
    ne = ln > 0
    sr, er = p["start_major"][ne], p["end_major"][ne]
    assert np.all(sr <= er)
    assert np.all(np.diff(sr) >= 0)
    ptr = np.asarray(ptr, np.int64)
    # row_ptr[start_row] <= start_idx < row_ptr[start_row + 1]
    assert np.all(ptr[sr] <= s[ne]) and np.all(s[ne] < ptr[sr + 1])
    assert np.all(ptr[er] <= e[ne]) and np.all(e[ne] < ptr[er + 1])
    # the flag says whether the previous non-empty partition ends in that row
    fl = p["start_flag"][ne].astype(bool)
    prev_end = np.concatenate(([-1], er[:-1]))
    assert np.array_equal(fl, prev_end == sr)


@pytest.mark.parametrize("P", [148, 1184, 9472])
def test_partition_invariants_rmat(P):
    a = I.rmat(scale=14, nnz=200_000, seed=31)
    p = O.partition_csr(a.row_ptr, a.nnz, P, with_local=True)
    _check_invariants(a.row_ptr, a.nnz, P, p)
    loc = p["local"]
    for i in range(0, P, max(1, P // 50)):
        sl = loc[p["local_off"][i]:p["local_off"][i + 1]]
        assert np.all(np.diff(sl) >= 0)
        assert sl[-1] == p["end_idx"][i] - p["start_idx"][i] + 1


def test_partition_uniform_closed_form():
    """2,000 rows of exactly 10 nonzeros, P = 4: 5,000 nonzeros per part,
    cuts exactly at rows 500, 1000, 1500, so no row is split."""
    a = I.uniform_rows()
    p = O.partition_csr(a.row_ptr, a.nnz, 4)
    assert p["start_idx"].tolist() == [0, 5000, 10000, 15000]
    assert p["end_idx"].tolist() == [4999, 9999, 14999, 19999]
    assert p["start_major"].tolist() == [0, 500, 1000, 1500]
    assert p["end_major"].tolist() == [499, 999, 1499, 1999]
    assert p["start_flag"].tolist() == [0, 0, 0, 0]
    # P = 3: cuts at nnz 6666 (row 666, 6th nonzero) and 13333 (row 1333)
    p = O.partition_csr(a.row_ptr, a.nnz, 3)
    assert p["start_idx"].tolist() == [0, 6666, 13333]
    assert p["start_major"].tolist() == [0, 666, 1333]
    assert p["start_flag"].tolist() == [0, 1, 1]


def test_pcsc_is_pcsr_of_transpose_and_pcoo_is_pcsr():
    a = I.rmat(scale=11, nnz=20_000, seed=41)
    c = I.csr_to_csc(a)
    t = I.transpose_csr(a)
    q = I.csr_to_coo(a)
    for P in (3, 148, 4096):
        pc = O.partition_csc(c.col_ptr, c.nnz, P, with_local=True)
        pt = O.partition_csr(t.row_ptr, t.nnz, P, with_local=True)
        for key in pc:
            assert np.array_equal(pc[key], pt[key])
        pr = O.partition_csr(a.row_ptr, a.nnz, P)
        pq = O.partition_coo(q.row_idx, P)
        for key in ("start_idx", "end_idx", "start_major", "end_major",
                    "start_flag"):
            assert np.array_equal(pq[key], pr[key]), key


def test_partition_rejects_bad_np():
    with pytest.raises(ValueError):
        O.partition_csr([0, 1], 1, 0)
    with pytest.raises(ValueError):
        O.partition_coo([0], 0)


def test_hub_row_spanning_every_partition_merges_exactly():
    """One row holds every nonzero: each of the P partitions gets a piece,
    all but the first flagged, and the merge must restore the full row."""
    n = 4096
    a = I.csr_from_triplets(3, n, [1] * n, list(range(n)),
                            I.rng(3, 3).integers(-3, 4, n).astype(float))
    x = I.rng(3, 4).integers(-4, 5, n).astype(float)
    exact = float(sum(int(v) * int(w) for v, w in zip(a.val, x)))
    for P in (2, 7, 148, 4096, 5000):
        p = O.partition_csr(a.row_ptr, a.nnz, P)
        ne = p["end_idx"] >= p["start_idx"]
        assert np.all(p["start_major"][ne] == 1)
        assert p["start_flag"][ne].tolist() == [0] + [1] * (int(ne.sum()) - 1)
        y = O.pspmv_csr(3, a.row_ptr, a.col_idx, a.val, p, x, 1.0, 0.0)
        assert y.tolist() == [0.0, exact, 0.0]


# --------------------------------------------------------------------------
# Row+nonzero merge-path partitioning (reading R10)
# --------------------------------------------------------------------------

def _brute_merge_cuts(ptr, nnz, P):
    """Cut (row, nonzero) coordinates by a library search: the row
    coordinate of item d is the last r with ptr[r] + r <= d."""
    ptr = np.asarray(ptr, np.int64)
    m = ptr.shape[0] - 1
    d = (np.arange(P + 1, dtype=np.int64) * (m + nnz)) // P
    r = np.searchsorted(ptr + np.arange(m + 1), d, side="right") - 1
    return r, d - r


def _brute_meta(ptr, s, e):
    ptr = np.asarray(ptr, np.int64)
    m = ptr.shape[0] - 1
    if e < s:
        return 0, -1, 0
    sr = int(np.searchsorted(ptr[:m], s, side="right") - 1)
    er = int(np.searchsorted(ptr[:m], e, side="right") - 1)
    return sr, er, int(s > ptr[sr])


@pytest.mark.parametrize("k", range(6))
def test_merge_path_partition_brute_force(k):
    a = _adversarial()[k]
    nnz = a.nnz
    for P in sorted({1, 2, 3, 4, 7, 16, a.m + nnz, a.m + nnz + 3}):
        got = O.partition_merge_path(a.row_ptr, nnz, P, with_local=True)
        r, kk = _brute_merge_cuts(a.row_ptr, nnz, P)
        assert got["cut_row"].tolist() == r.tolist(), P
        assert got["start_idx"].tolist() == kk[:-1].tolist()
        assert got["end_idx"].tolist() == (kk[1:] - 1).tolist()
        for i in range(P):
            want = _brute_meta(a.row_ptr, int(kk[i]), int(kk[i + 1]) - 1)
            assert (got["start_major"][i], got["end_major"][i], got["start_flag"][i]) == want
        # every partition holds floor or ceil of (m + nnz) / P merged items
        items = np.diff(r + kk)
        assert set(items.tolist()) <= {(a.m + nnz) // P, -(-(a.m + nnz) // P)}


def test_merge_path_closed_forms():
    """Uniform rows (10 nonzeros + 1 row end each): the merge-path split at
    P = 4 equals the nonzero split, cutting at rows 500/1000/1500.  One full
    row after 999 empty ones, P = 2: the first cut comes after the 999 empty
    rows' ends and the full row's first nonzero."""
    a = I.uniform_rows()
    p = O.partition_merge_path(a.row_ptr, a.nnz, 4)
    q = O.partition_csr(a.row_ptr, a.nnz, 4)
    for key in ("start_idx", "end_idx", "start_major", "end_major", "start_flag"):
        assert np.array_equal(p[key], q[key])
    assert p["cut_row"].tolist() == [0, 500, 1000, 1500, 2000]
    b = I.csr_from_triplets(1000, 1000, [999] * 1000, list(range(1000)), np.ones(1000))
    p = O.partition_merge_path(b.row_ptr, b.nnz, 2)
    assert p["cut_row"].tolist() == [0, 999, 1000]
    assert p["start_idx"].tolist() == [0, 1] and p["end_idx"].tolist() == [0, 999]
    assert p["start_flag"].tolist() == [0, 1]


@pytest.mark.parametrize("seed", range(6))
def test_merge_path_partitioned_spmv_dense(seed):
    g = I.rng(seed, 29)
    m, n = int(g.integers(1, 17)), int(g.integers(1, 17))
    d, a = _tiny(seed + 200, m, n, float(g.uniform(0.05, 0.9)))
    x = g.uniform(-1, 1, n)
    yin = g.uniform(-1, 1, m)
    for P in sorted({1, 2, 3, 5, m + a.nnz, m + a.nnz + 4}):
        p = O.partition_merge_path(a.row_ptr, a.nnz, P)
        y = O.pspmv_csr(m, a.row_ptr, a.col_idx, a.val, p, x, 0.5, 2.0, yin)
        assert np.allclose(y, 0.5 * (d @ x) + 2.0 * yin, rtol=0, atol=1e-13)


# --------------------------------------------------------------------------
# pCOO sorted by column and in no order (reading R9)
# --------------------------------------------------------------------------

def test_pcoo_by_col_is_pcsc():
    """Column-sorted pCOO is Alg. 6 over the column index: its metadata
    equals pCSC's (itself pinned as pCSR of the transpose), and the local
    column index is col - start_col of the owning partition."""
    for a in _adversarial() + [I.rmat(scale=11, nnz=20_000, seed=41)]:
        c = I.csr_to_csc(a)
        q = I.csr_to_coo_by_col(a)
        nnz = a.nnz
        for P in sorted({1, 3, 7, 148, max(1, nnz), nnz + 5}):
            pq = O.partition_coo_by_col(q.col_idx, P, with_local=True)
            pc = O.partition_csc(c.col_ptr, nnz, P)
            for key in ("start_idx", "end_idx", "start_major", "end_major",
                        "start_flag"):
                assert np.array_equal(pq[key], pc[key]), (key, P)
            if nnz:
                owner = np.searchsorted(pc["start_idx"], np.arange(nnz), side="right") - 1
                # the owner search lands on the last partition starting at or
                # before k, which is the non-empty one holding k
                assert np.array_equal(pq["local"], q.col_idx - pc["start_major"][owner])


def test_pcoo_unsorted_ranges_and_whole_row_span():
    a = I.rmat(scale=10, nnz=9_000, seed=43)
    q = I.csr_to_coo_unsorted(a, seed=7)
    s = I.csr_to_coo(a)
    for P in (1, 5, 148, a.nnz, a.nnz + 3):
        pu = O.partition_coo_unsorted(q.row_idx, a.m, P, with_local=True)
        ps = O.partition_coo(s.row_idx, P)
        assert np.array_equal(pu["start_idx"], ps["start_idx"])
        assert np.array_equal(pu["end_idx"], ps["end_idx"])
        ne = pu["end_idx"] >= pu["start_idx"]
        assert np.all(pu["start_major"] == 0)
        assert np.all(pu["end_major"][ne] == a.m - 1)
        assert np.all(pu["end_major"][~ne] == -1)
        assert not pu["start_flag"].any()
        assert np.array_equal(pu["local"], q.row_idx)


def test_unsorted_coo_is_a_permutation_of_the_sorted_one():
    a = I.rmat(scale=9, nnz=3_000, seed=44)
    q, s = I.csr_to_coo_unsorted(a, seed=9), I.csr_to_coo(a)
    assert not np.array_equal(q.row_idx, s.row_idx)
    key_q = np.lexsort((q.col_idx, q.row_idx))
    assert np.array_equal(q.row_idx[key_q], s.row_idx)
    assert np.array_equal(q.col_idx[key_q], s.col_idx)
    assert np.array_equal(q.val[key_q], s.val)


@pytest.mark.parametrize("seed", range(8))
def test_pspmv_coo_scatter_dense(seed):
    """Partitioned SpMV of column-sorted and unsorted COO against numpy's
    dense product, for P from 1 to beyond nnz, with alpha and beta."""
    g = I.rng(seed, 19)
    m, n = int(g.integers(1, 17)), int(g.integers(1, 17))
    d, a = _tiny(seed + 100, m, n, float(g.uniform(0.05, 0.9)))
    x = g.uniform(-1, 1, n)
    yin = g.uniform(-1, 1, m)
    want = 0.75 * (d @ x) - 1.5 * yin
    for by_col, q in ((True, I.csr_to_coo_by_col(a)),
                      (False, I.csr_to_coo_unsorted(a, seed=seed))):
        for P in sorted({1, 2, 5, max(1, a.nnz), a.nnz + 2}):
            p = (O.partition_coo_by_col(q.col_idx, P) if by_col
                 else O.partition_coo_unsorted(q.row_idx, m, P))
            y = O.pspmv_coo_scatter(m, q.row_idx, q.col_idx, q.val, p, x, 0.75, -1.5, yin)
            assert np.allclose(y, want, rtol=0, atol=1e-13)
            nan = np.full(m, np.nan)
            y0 = O.pspmv_coo_scatter(m, q.row_idx, q.col_idx, q.val, p, x, 1.0, 0.0, nan)
            assert np.allclose(y0, d @ x, rtol=0, atol=1e-13)


def test_pspmv_coo_scatter_hub_row_exact():
    """One row holds every nonzero, in shuffled order: every partition adds
    to it, and the integer-valued sum is exact."""
    n = 3000
    a = I.csr_from_triplets(4, n, [2] * n, list(range(n)),
                            I.rng(5, 5).integers(-3, 4, n).astype(float))
    x = I.rng(5, 6).integers(-4, 5, n).astype(float)
    exact = float(sum(int(v) * int(w) for v, w in zip(a.val, x)))
    for q in (I.csr_to_coo_by_col(a), I.csr_to_coo_unsorted(a, seed=3)):
        for P in (1, 7, 148, 3000, 4000):
            p = O.partition_coo_unsorted(q.row_idx, 4, P)
            y = O.pspmv_coo_scatter(4, q.row_idx, q.col_idx, q.val, p, x)
            assert y.tolist() == [0.0, 0.0, exact, 0.0]


# --------------------------------------------------------------------------
# binary32 TwoSum and compensated summation
# --------------------------------------------------------------------------

def test_two_sum_is_error_free():
    g = I.rng(1, 1)
    a = (g.standard_normal(2000) * np.exp2(g.integers(-30, 30, 2000))).astype(np.float32)
    b = (g.standard_normal(2000) * np.exp2(g.integers(-30, 30, 2000))).astype(np.float32)
    for x, y in zip(a.tolist(), b.tolist()):
        s, e = O.two_sum_f32(x, y)
        assert np.float32(s) == np.float32(np.float32(x) + np.float32(y))
        assert Fraction(x) + Fraction(y) == Fraction(s) + Fraction(e)


def test_compensated_sum_recovers_small_terms():
    """(2^24, 1, -2^24) repeated: plain binary32 loses every 1 (2^24 + 1
    rounds to 2^24), the compensated sum returns the exact count."""
    v = np.tile(np.array([2.0**24, 1.0, -2.0**24], np.float32), 300)
    assert O.sum_f32(v) == 0.0
    assert O.sum2_f32(v) == 300.0
    g = I.rng(2, 2)
    w = (g.standard_normal(5000) * np.exp2(g.integers(-20, 20, 5000))).astype(np.float32)
    exact = sum(Fraction(t) for t in w.tolist())
    got = Fraction(O.sum2_f32(w))
    # Sum2 error bound: |res - s| <= eps|s| + gamma_{n-1}^2 sum|w| (eps = 2^-24)
    eps = Fraction(1, 2**24)
    gam = (len(w) - 1) * eps / (1 - (len(w) - 1) * eps)
    bound = eps * abs(exact) + gam * gam * sum(abs(Fraction(t)) for t in w.tolist())
    assert abs(got - exact) <= bound


# --------------------------------------------------------------------------
# Baseline row-block partitioning (Sec. 5.1, reading R11)
# --------------------------------------------------------------------------

def test_hand_example_row_block():
    g = _hand()
    e = g["pcsr_row_block"]
    p = O.partition_row_block(g["csr"]["row_ptr"], 9, e["np"], with_local=True)
    assert p["start_idx"].tolist() == e["start_idx"]
    assert p["end_idx"].tolist() == e["end_idx"]
    assert p["start_major"].tolist() == e["start_row"]
    assert p["end_major"].tolist() == e["end_row"]
    assert p["start_flag"].tolist() == e["start_flag"]
    assert p["local"].tolist() == [v for part in e["local_row_ptr"] for v in part]
    q = O.partition_coo_row_block(g["coo"]["row_idx"], g["m"], e["np"], with_local=True)
    assert q["start_idx"].tolist() == e["start_idx"]
    assert q["start_major"].tolist() == e["start_row"]
    assert q["end_major"].tolist() == e["end_row"]
    assert q["local"].tolist() == e["pcoo_local_row_idx"]
    c = g["pcsc_row_block"]
    r = O.partition_row_block(g["csc"]["col_ptr"], 9, c["np"], with_local=True)
    assert r["start_idx"].tolist() == c["start_idx"]
    assert r["end_idx"].tolist() == c["end_idx"]
    assert r["start_major"].tolist() == c["start_col"]
    assert r["end_major"].tolist() == c["end_col"]
    assert r["start_flag"].tolist() == c["start_flag"]
    assert r["local"].tolist() == [v for part in c["local_col_ptr"] for v in part]


def _brute_row_block(row_ptr, m, P):
    """Block i = rows [floor(i m / P), floor((i+1) m / P)); its nonzero range
    read off row_ptr, its first and last owning row by numpy's
    searchsorted (the last r with row_ptr[r] <= k)."""
    ptr = np.asarray(row_ptr, np.int64)
    out = {"start_idx": [], "end_idx": [], "start_major": [], "end_major": [],
           "start_flag": []}
    for i in range(P):
        r0, r1 = (i * m) // P, ((i + 1) * m) // P
        s, e = int(ptr[r0]), int(ptr[r1]) - 1
        out["start_idx"].append(s)
        out["end_idx"].append(e)
        if e < s:
            out["start_major"].append(0)
            out["end_major"].append(-1)
            out["start_flag"].append(0)
            continue
        sr = int(np.searchsorted(ptr[:m], s, side="right")) - 1
        er = int(np.searchsorted(ptr[:m], e, side="right")) - 1
        out["start_major"].append(sr)
        out["end_major"].append(er)
        out["start_flag"].append(int(s > ptr[sr]))
    return out


@pytest.mark.parametrize("k", range(6))
def test_row_block_partition_brute_force(k):
    a = _adversarial()[k]
    coo = I.csr_to_coo(a)
    for P in sorted({1, 2, 3, 4, 7, 16, max(1, a.m - 1), a.m, a.m + 5}):
        want = _brute_row_block(a.row_ptr, a.m, P)
        got = O.partition_row_block(a.row_ptr, a.nnz, P, with_local=True)
        for key in want:
            assert got[key].tolist() == want[key], (key, P)
        # row blocks never split a row, and the ranges tile [0, nnz) in order
        assert not got["start_flag"].any()
        assert got["start_idx"][0] == 0 and got["end_idx"][-1] == a.nnz - 1
        assert np.all(got["start_idx"][1:] == got["end_idx"][:-1] + 1)
        # pCOO's row blocks (found by scanning row_idx) equal pCSR's
        q = O.partition_coo_row_block(coo.row_idx, a.m, P, with_local=True)
        for key in want:
            assert q[key].tolist() == want[key], (key, P)
        if a.nnz:
            owner = np.repeat(np.arange(P), got["end_idx"] - got["start_idx"] + 1)
            sm = got["start_major"][owner]
            assert np.array_equal(q["local"], coo.row_idx - sm)


def test_row_block_csc_is_row_block_of_transpose():
    a = I.rmat(scale=9, nnz=3000, seed=17)
    c = I.csr_to_csc(a)
    t = I.transpose_csr(a)
    for P in (1, 5, 64, 600):
        p = O.partition_row_block(c.col_ptr, a.nnz, P)
        q = O.partition_row_block(t.row_ptr, a.nnz, P)
        for key in p:
            assert np.array_equal(p[key], q[key]), (key, P)


def test_row_block_partitioned_spmv_equals_dense():
    """The partitioned SpMV of Alg. 3 over row blocks (no row is split, so
    the merge only writes each block's rows) gives the dense product."""
    for seed in (3, 4):
        d, a = _tiny(seed, 16, 13, 0.25)
        x = I.vector(a.n, seed + 100)
        for P in (1, 3, 7, 16, 20):
            part = O.partition_row_block(a.row_ptr, a.nnz, P)
            y = O.pspmv_csr(a.m, a.row_ptr, a.col_idx, a.val, part, x)
            assert np.allclose(y, d @ x, rtol=0, atol=1e-13)
