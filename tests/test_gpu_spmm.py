"""msrep_spmm: k right-hand sides over the CSR tiles, against the oracle's
k-vector product (k applications of Alg. 1) and against msrep_spmv.

The k-vector kernel performs, for every vector, exactly the operations the
SpMV kernel performs (same lane order, warp scan and tile merge), so each
column of Y must equal msrep_spmv of that x bit for bit; against the oracle
the FP64 bound is the SpMV's normwise 1e-12."""
import numpy as np
import pytest

from helpers import normwise
from paper_2209_07552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _mats():
    yield "uniform", I.uniform_rows()
    yield "rmat12", I.rmat(scale=12, nnz=40_000, seed=21)
    rows = [0, 0, 3, 3, 3, 9, 9, 9, 9, 9, 9, 14]
    cols = [1, 4, 0, 2, 7, 0, 1, 2, 3, 5, 6, 7]
    yield "gaps", I.csr_from_triplets(20, 8, rows, cols, I.rng(5, 5).uniform(-1, 1, len(rows)))
    yield "hub", I.csr_from_triplets(9, 6000, [4] * 6000, list(range(6000)),
                                     I.rng(4, 4).uniform(-1, 1, 6000))


def _setup(a, dtype, P, tile=0):
    import paper_2209_07552_gb300 as M
    A = M.DeviceMatrix.from_host(a, "csr", dtype)
    part = M.DevicePartition(A, P, tile=tile)
    M.msrep_partition(A, part)
    return A, part


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 9, 21])
def test_fp64_matches_oracle(k):
    import torch

    import oracle as O
    import paper_2209_07552_gb300 as M
    for name, a in _mats():
        X = np.stack([I.vector(a.n, 100 + v) for v in range(k)])          # (k, n)
        Y0 = np.stack([I.y_vector(a.m, 200 + v) for v in range(k)])       # (k, m)
        for P, tile in ((4, 256), (148, 512), (a.nnz + 3, 1024)):
            A, part = _setup(a, "f64", P, tile)
            for alpha, beta in ((1.0, 0.0), (-0.5, 1.5)):
                Y = torch.from_numpy(Y0.copy()).cuda()
                M.msrep_spmm(A, part, alpha, torch.from_numpy(X).cuda(), beta, Y)
                want = O.spmm_csr(a.m, a.row_ptr, a.col_idx, a.val, X.T.copy(), alpha, beta,
                                  Y0.T.copy()).T
                got = Y.cpu().numpy()
                for v in range(k):
                    assert normwise(got[v], want[v]) <= TOL64, (name, k, P, alpha, v)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_columns_equal_spmv_bit_for_bit(dtype):
    import torch

    import paper_2209_07552_gb300 as M
    a = I.rmat(scale=13, nnz=120_000, seed=22)
    xt = torch.float64 if dtype == "f64" else torch.float32
    A, part = _setup(a, dtype, 148)
    k = 6
    X = torch.from_numpy(np.stack([I.vector(a.n, 300 + v) for v in range(k)])).to("cuda", xt)
    Y0 = torch.from_numpy(np.stack([I.y_vector(a.m, 400 + v) for v in range(k)])).to("cuda", xt)
    ws = M.alloc_workspace(A, part)
    # alpha = 2, beta = 0.5 scale exactly; 1.5 and -0.3 round, so the merged
    # rows' finishing must round alike in both kernels too
    for alpha, beta in ((2.0, 0.5), (1.5, -0.3), (0.7, 0.0)):
        Y = Y0.clone()
        M.msrep_spmm(A, part, alpha, X, beta, Y)
        for v in range(k):
            y = Y0[v].clone()
            M.msrep_spmv(A, part, alpha, X[v], beta, y, workspace=ws)
            assert torch.equal(Y[v], y), (alpha, beta, v)


@pytest.mark.parametrize("k", [9, 16, 21])
def test_more_than_eight_vectors_in_passes(k):
    """k > 8 vectors run in passes of up to 8 through one workspace: every
    column still equals msrep_spmv of its x bit for bit."""
    import torch

    import paper_2209_07552_gb300 as M
    a = I.rmat(scale=12, nnz=50_000, seed=25)
    A, part = _setup(a, "f64", 148)
    X = torch.from_numpy(np.stack([I.vector(a.n, 700 + v) for v in range(k)])).cuda()
    Y0 = torch.from_numpy(np.stack([I.y_vector(a.m, 800 + v) for v in range(k)])).cuda()
    Y = Y0.clone()
    ws = torch.empty(M.msrep_spmm_workspace_size(A, part, k), dtype=torch.uint8, device="cuda")
    assert ws.numel() == M.msrep_spmm_workspace_size(A, part, 8)
    M.msrep_spmm(A, part, 1.5, X, -0.25, Y, workspace=ws)
    wsv = M.alloc_workspace(A, part)
    for v in range(k):
        y = Y0[v].clone()
        M.msrep_spmv(A, part, 1.5, X[v], -0.25, y, workspace=wsv)
        assert torch.equal(Y[v], y), v


def test_strided_x_and_y():
    """ldx > n and ldy > m: the vectors are rows of wider tensors."""
    import torch

    import oracle as O
    import paper_2209_07552_gb300 as M
    a = I.rmat(scale=11, nnz=20_000, seed=23)
    A, part = _setup(a, "f64", 37)
    k = 4
    Xw = torch.zeros((k, a.n + 7), dtype=torch.float64, device="cuda")
    X = np.stack([I.vector(a.n, 500 + v) for v in range(k)])
    Xw[:, :a.n] = torch.from_numpy(X).cuda()
    Yw = torch.full((k, a.m + 5), 7.0, dtype=torch.float64, device="cuda")
    M.msrep_spmm(A, part, 1.0, Xw[:, :a.n], 0.0, Yw[:, :a.m])
    want = O.spmm_csr(a.m, a.row_ptr, a.col_idx, a.val, X.T.copy()).T
    got = Yw.cpu().numpy()
    for v in range(k):
        assert normwise(got[v, :a.m], want[v]) <= TOL64
    assert np.all(got[:, a.m:] == 7.0)        # nothing written past m


def test_low_precision_error_vs_fp64_oracle():
    import torch

    import oracle as O
    import paper_2209_07552_gb300 as M
    a = I.rmat(scale=13, nnz=120_000, seed=24)
    k = 8
    X = np.stack([I.vector(a.n, 600 + v) for v in range(k)])
    want = O.spmm_csr(a.m, a.row_ptr, a.col_idx, a.val, X.T.copy()).T
    for dtype, tol in (("f32", 1e-5), ("bf16", 1e-2)):
        A, part = _setup(a, dtype, 148)
        Y = torch.empty((k, a.m), dtype=torch.float32, device="cuda")
        M.msrep_spmm(A, part, 1.0, torch.from_numpy(X).to("cuda", torch.float32), 0.0, Y)
        got = Y.cpu().numpy().astype(np.float64)
        for v in range(k):
            assert normwise(got[v], want[v]) <= tol, (dtype, v)


def test_rejects_bad_arguments():
    import ctypes

    import torch

    import paper_2209_07552_gb300 as M
    a = I.uniform_rows()
    A, part = _setup(a, "f64", 4)
    X = torch.zeros((9, a.n), dtype=torch.float64, device="cuda")
    Y = torch.zeros((9, a.m), dtype=torch.float64, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    lib = M.native.lib()
    for ldx, ldy in ((a.n, a.m - 1), (a.n - 1, a.m)):   # ldy < m, ldx < n
        rc = lib.msrep_spmm(ctypes.byref(A.c), ctypes.byref(part.c), 2, 1.0,
                            ctypes.c_void_p(X.data_ptr()), ldx, 0.0,
                            ctypes.c_void_p(Y.data_ptr()), ldy, M.MSREP_F64, 0,
                            ctypes.c_void_p(ws.data_ptr()), None)
        assert rc == 1
    with pytest.raises(M.MsrepError) as e:     # k = 0
        M.msrep_spmm(A, part, 1.0, X[:0], 0.0, Y[:0], workspace=ws)
    assert e.value.status == 1
    C = M.DeviceMatrix.from_host(a, "csc", "f64")
    cpart = M.DevicePartition(C, 4)
    M.msrep_partition(C, cpart)
    with pytest.raises(M.MsrepError):
        M.msrep_spmm(C, cpart, 1.0, X[:2], 0.0, Y[:2],
                     workspace=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("k", [1, 3, 8])
def test_empty_matrix_and_empty_rows(k):
    """No nonzeros: Y = beta * Y for every vector; a matrix whose rows are
    mostly empty: the oracle's product, exactly (integer data)."""
    import torch

    import oracle as O
    import paper_2209_07552_gb300 as M
    a = I.csr_from_triplets(37, 11, [], [], [])
    A, part = _setup(a, "f64", 4)
    Y0 = np.stack([I.y_vector(a.m, 700 + v) for v in range(k)])
    Y = torch.from_numpy(Y0.copy()).cuda()
    M.msrep_spmm(A, part, 1.0, torch.zeros((k, a.n), dtype=torch.float64, device="cuda"), 2.0, Y)
    assert np.array_equal(Y.cpu().numpy(), 2.0 * Y0)
    rows = [3, 3, 40, 41, 41, 41, 900]
    cols = [0, 5, 2, 2, 3, 9, 1]
    b, _ = I.integer_twin(I.csr_from_triplets(1000, 10, rows, cols, np.ones(len(rows))), seed=3)
    B, bpart = _setup(b, "f64", 3, 256)
    X = np.stack([I.integer_twin(b, seed=10 + v)[1] for v in range(k)])
    Yb = torch.full((k, b.m), float("nan"), dtype=torch.float64, device="cuda")
    M.msrep_spmm(B, bpart, 1.0, torch.from_numpy(X).cuda(), 0.0, Yb)
    want = O.spmm_csr(b.m, b.row_ptr, b.col_idx, b.val, X.T.copy()).T
    assert np.array_equal(Yb.cpu().numpy(), want)


@pytest.mark.parametrize("k", [2, 4, 8])
def test_full_size_rmat_columns_equal_spmv(k, rmat_full):
    """The bench's k-vector case at full size (R-MAT 2^20, 2^24 nonzeros,
    FP32, P = 2368, default tile): every column equals msrep_spmv of that
    x bit for bit, for each width the kernel has (KP 2, 4 with one thread
    per lane, 8 with two), and the spot rows match the FP64 oracle's dot
    products within the binary32 row bound ((L + 2) u (|A||x|)_r + u |y_r|,
    recursive summation)."""
    import torch

    import paper_2209_07552_gb300 as M
    a = rmat_full
    A, part = _setup(a, "f32", 2368)
    g = I.rng(77, k)
    X = torch.from_numpy(g.uniform(-1, 1, (k, a.n)).astype(np.float32)).cuda()
    Y = torch.empty((k, a.m), dtype=torch.float32, device="cuda")
    M.msrep_spmm(A, part, 1.0, X, 0.0, Y)
    ws = M.alloc_workspace(A, part)
    y = torch.empty(a.m, dtype=torch.float32, device="cuda")
    stored = I.CSR(a.m, a.n, a.row_ptr, a.col_idx, a.val.astype(np.float32).astype(np.float64))
    rows = np.concatenate([np.arange(16), g.integers(0, a.m, 200)])   # hub rows and a sample
    for v in range(k):
        M.msrep_spmv(A, part, 1.0, X[v], 0.0, y, workspace=ws)
        assert torch.equal(Y[v], y), v
        xv = X[v].cpu().numpy().astype(np.float64)
        got = Y[v].cpu().numpy()
        for r in rows:
            s, e = stored.row_ptr[r], stored.row_ptr[r + 1]
            want = float(np.dot(stored.val[s:e], xv[stored.col_idx[s:e]]))
            bound = (e - s + 2) * 2.0**-24 * float(np.dot(np.abs(stored.val[s:e]),
                                                           np.abs(xv[stored.col_idx[s:e]])))
            assert abs(float(got[r]) - want) <= bound + 2.0**-24 * abs(want), (v, r)
