"""Batched form: many uneven CSR matrices in one persistent launch.

Each matrix's y must equal, bit for bit, what msrep_spmv gives for the same
matrix with the same partition count and tile (the two share the tile
code), and must match the FP64 oracle on the stored values (FP32 within the
summation bound of the low-precision tests, FP64 within 1e-12)."""
import numpy as np
import pytest

from helpers import normwise, oracle_spmv
from paper_2209_07552_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _small_batch(count, dtype, seed=77):
    ms, mus = I.batched_sizes(count, seed, m_lo=300, m_hi=20000)
    mats, xs = [], []
    for i, (m, mu) in enumerate(zip(ms, mus)):
        a = I.geometric_matrix(int(m), float(mu), seed * 100 + i, np.float64)
        mats.append(a)
        xs.append(I.vector(a.n, seed * 100 + i))
    # one hub-heavy and one empty-row matrix at the ends
    mats.append(I.rmat(scale=11, nnz=30_000, seed=seed))
    xs.append(I.vector(mats[-1].n, seed + 5))
    mats.append(I.csr_from_triplets(50, 40, [3, 3, 49], [0, 39, 7], [1.0, 2.0, 3.0]))
    xs.append(I.vector(40, seed + 6))
    return mats, xs


def _solo(M, a, dt, x, np_, tile):
    import torch
    A = M.DeviceMatrix.from_host(a, "csr", dt)
    part = M.DevicePartition(A, np_, tile=tile)
    M.msrep_partition(A, part)
    xt = torch.float64 if dt == "f64" else torch.float32
    y = torch.empty(a.m, dtype=xt, device="cuda")
    M.msrep_spmv(A, part, 1.0, torch.from_numpy(x).to("cuda", xt), 0.0, y,
                 workspace=M.alloc_workspace(A, part))
    return y.cpu().numpy()


def _tuned(tune, nnz):
    b = 0
    while b + 1 < 32 and (1 << (b + 1)) <= nnz:
        b += 1
    tile = tune.tile[b] or 512
    pn = tune.part_nnz[b]
    return (max(1, -(-nnz // pn)) if pn > 0 else 1), tile


@pytest.mark.parametrize("cta", [128, 256, 512])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_batched_equals_solo_and_oracle(dt, cta):
    import torch

    import paper_2209_07552_gb300 as M
    mats, xs = _small_batch(20, dt)
    xt = torch.float64 if dt == "f64" else torch.float32
    D = [M.DeviceMatrix.from_host(a, "csr", dt) for a in mats]
    X = [torch.from_numpy(x).to("cuda", xt) for x in xs]
    Y = [torch.full((a.m,), float("nan"), dtype=xt, device="cuda") for a in mats]
    tune = M.msrep_tune_default()
    for b in range(8, 20):            # vary partitions and tiles across buckets
        tune.tile[b] = (256, 512, 1024)[b % 3]
        tune.part_nnz[b] = (0, 1 << 12, 1 << 15)[b % 3]
    tune.cta_threads = cta            # thread-block shape of the launch
    B = M.DeviceBatch(D, X, Y, tune)
    assert B.c.cta_threads == cta and B.c.max_tile == 1024
    B.run()
    torch.cuda.synchronize()
    for a, x, y in zip(mats, xs, Y):
        np_, tile = _tuned(tune, a.nnz)
        got = y.cpu().numpy()
        assert np.array_equal(got, _solo(M, a, dt, x, np_, tile))
        if dt == "f64":
            assert normwise(got, oracle_spmv(a, "csr", x)) <= 1e-12
        else:
            st = I.CSR(a.m, a.n, a.row_ptr, a.col_idx, I.to_f32(a.val).astype(np.float64))
            x32 = I.to_f32(x).astype(np.float64)
            assert normwise(got, oracle_spmv(st, "csr", x32)) <= 1e-6


def test_autotune_then_batch():
    import torch

    import paper_2209_07552_gb300 as M
    mats, xs = _small_batch(12, "f32", seed=91)
    D = [M.DeviceMatrix.from_host(a, "csr", "f32") for a in mats]
    X = [torch.from_numpy(x).to("cuda", torch.float32) for x in xs]
    Y = [torch.empty(a.m, dtype=torch.float32, device="cuda") for a in mats]
    tune = M.msrep_autotune(D, X, Y)
    for b in range(32):
        assert tune.tile[b] in (256, 512, 1024)
        assert tune.part_nnz[b] in (0, 1 << 14, 1 << 18)
    assert tune.cta_threads in (128, 256, 512)
    B = M.DeviceBatch(D, X, Y, tune)
    B.run()
    torch.cuda.synchronize()
    for a, x, y in zip(mats, xs, Y):
        np_, tile = _tuned(tune, a.nnz)
        assert np.array_equal(y.cpu().numpy(), _solo(M, a, "f32", x, np_, tile))


def test_batched_graph_capture_replay():
    """The batched call captures into a CUDA graph; replays after new x
    values are copied into the same buffers give the new results."""
    import torch

    import paper_2209_07552_gb300 as M
    mats, xs = _small_batch(10, "f32", seed=55)
    D = [M.DeviceMatrix.from_host(a, "csr", "f32") for a in mats]
    X = [torch.from_numpy(x).to("cuda", torch.float32) for x in xs]
    Y = [torch.empty(a.m, dtype=torch.float32, device="cuda") for a in mats]
    B = M.DeviceBatch(D, X, Y)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        B.run(stream=s)                 # warm up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        B.run(stream=s)
    for trial in range(2):
        new = [I.vector(a.n, 1000 + 10 * trial + i) for i, a in enumerate(mats)]
        for t, v in zip(X, new):
            t.copy_(torch.from_numpy(v).to(torch.float32))
        g.replay()
        torch.cuda.synchronize()
        for a, v, y in zip(mats, new, Y):
            want = _solo(M, a, "f32", v, 1, 512)
            assert np.array_equal(y.cpu().numpy(), want)
