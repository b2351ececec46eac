"""Serving: device-resident matrices, budget admission, continuous batching.

Every result must equal, bit for bit, msrep_spmv of the same matrix (FP32
values, one partition per 2^20 nonzeros, the default tile) on the same x,
whether the request ran alone or inside a mixed batch of requests for other
matrices; and it must match the FP64 oracle on the stored values."""
import threading

import numpy as np
import pytest

import oracle as O
from helpers import f32_row_bound, normwise, oracle_spmv
from paper_2209_07552_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _mats(seed=5):
    out = []
    ms, mus = I.batched_sizes(6, seed, m_lo=500, m_hi=30000)
    for i, (m, mu) in enumerate(zip(ms, mus)):
        out.append(I.geometric_matrix(int(m), float(mu), seed * 10 + i, np.float32))
    out.append(I.rmat(scale=12, nnz=50_000, seed=seed))
    return out


def _solo(M, a, X):
    import torch
    A = M.DeviceMatrix.from_host(a, "csr", "f32")
    np_ = max(1, -(-a.nnz // (1 << 20)))
    part = M.DevicePartition(A, np_)
    M.msrep_partition(A, part)
    ws = M.alloc_workspace(A, part)
    ys = []
    for x in X:
        y = torch.empty(a.m, dtype=torch.float32, device="cuda")
        M.msrep_spmv(A, part, 1.0, torch.from_numpy(np.ascontiguousarray(x)).cuda(), 0.0, y,
                     workspace=ws)
        ys.append(y.cpu().numpy())
    return np.stack(ys)


def _stored(a):
    return I.CSR(a.m, a.n, a.row_ptr, a.col_idx, a.val.astype(np.float32).astype(np.float64))


def test_serve_results_alone_and_in_the_mix():
    """Every one of the 8 columns a request can carry: alone (one request
    of 8 vectors, the batched k-vector kernel) it equals msrep_spmv of that
    column bit for bit and the FP64 oracle on the stored values within the
    binary32 bound; in the mix (requests of 1..8 vectors for all matrices,
    from several threads, so launches hold both batched kernels) each of its
    k columns equals the alone result bit for bit."""
    import paper_2209_07552_gb300 as M
    mats = _mats()
    with M.Server(budget_bytes=4 << 30, arena_bytes=16 << 20, contexts=3) as S:
        ids = [S.register(a) for a in mats]
        rng = I.rng(9, 9)
        X = [rng.uniform(-1, 1, (8, a.n)).astype(np.float32) for a in mats]
        # alone: one request at a time, all eight vectors
        alone = []
        for mid, x in zip(ids, X):
            alone.append(S.wait(S.submit(mid, x)).copy())
        # in the mix: many requests of every matrix from several threads
        tickets, lock = [], threading.Lock()

        def client(tid):
            g = I.rng(100 + tid, 1)
            for _ in range(25):
                j = int(g.integers(len(ids)))
                k = int(g.integers(1, 9))
                t = S.submit(ids[j], X[j][:k])
                with lock:
                    tickets.append((j, k, t))

        th = [threading.Thread(target=client, args=(t,)) for t in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        ks = set()
        for j, k, t in tickets:
            y = S.wait(t, 60_000_000)
            assert y.shape[0] == k
            assert np.array_equal(y, alone[j][:k]), (j, k)
            ks.add(k)
        assert ks == set(range(1, 9))
        st = S.stats()
        assert st["completed"] >= len(tickets) + len(ids)
        assert st["launches"] >= 1 and st["p99_us"] >= st["p50_us"] > 0
        # where the latency goes: queue wait (host) and per-launch device time
        assert st["wait_p99_us"] >= st["wait_p50_us"] >= 0
        assert st["device_p99_us"] >= st["device_p50_us"] > 0
        assert 0 < st["kernel_mean_us"] <= st["device_p99_us"]
        assert st["host_launch_p99_us"] >= st["host_launch_p50_us"] > 0
        assert st["device_p50_us"] <= st["p99_us"]
    for a, x, y in zip(mats, X, alone):
        assert y.shape == (8, a.m)
        assert np.array_equal(y, _solo(M, a, x))
        st = _stored(a)
        want = O.spmm_csr(a.m, a.row_ptr, a.col_idx, st.val, x.astype(np.float64).T)
        for v in range(8):
            assert normwise(y[v], want[:, v]) <= 1e-6, v
            assert np.all(np.abs(y[v] - want[:, v]) <= f32_row_bound(st, x[v], want[:, v])), v


@pytest.mark.parametrize("k", [2, 3, 4, 5, 8])
def test_serve_k_vector_kernel_columns(k):
    """The server's batched k-vector kernel (and its interleaving of X) on
    uneven matrices in one launch: requests of k vectors for every matrix
    are queued while the server is held busy, so they share launches.
    Every column is checked element-wise against the oracle's k-vector
    product on the stored values (binary32 bound) and bit for bit against
    msrep_spmv of that column."""
    import paper_2209_07552_gb300 as M
    mats = _mats(seed=7)
    with M.Server(budget_bytes=4 << 30, arena_bytes=32 << 20, contexts=1) as S:
        ids = [S.register(a) for a in mats]
        g = I.rng(31, k)
        X = [g.uniform(-1, 1, (k, a.n)).astype(np.float32) for a in mats]
        # a large request first keeps the single context busy while the
        # others queue, so they are packed into one launch
        big = I.rmat(scale=16, nnz=1_500_000, seed=33)
        bid = S.register(big)
        hold = S.submit(bid, np.ones((8, big.n), np.float32))
        tickets = [S.submit(mid, x) for mid, x in zip(ids, X)]
        S.wait(hold)
        ys = [S.wait(t) for t in tickets]
        st = S.stats()
        assert st["launches"] <= 2 + len(ids)
    for a, x, y in zip(mats, X, ys):
        assert y.shape == (k, a.m)
        s = _stored(a)
        want = O.spmm_csr(a.m, a.row_ptr, a.col_idx, s.val, x.astype(np.float64).T)
        solo = _solo(M, a, x)
        for v in range(k):
            assert np.all(np.abs(y[v] - want[:, v]) <= f32_row_bound(s, x[v], want[:, v])), v
            assert np.array_equal(y[v], solo[v]), v


def test_serve_budget_admission_and_unregister():
    import paper_2209_07552_gb300 as M
    big = I.rmat(scale=14, nnz=400_000, seed=3)
    small = I.geometric_matrix(2000, 8.0, 4, np.float32)
    cfg = dict(arena_bytes=1 << 20, contexts=3, max_tiles=1 << 16, max_items=64)
    with M.Server(budget_bytes=1 << 30, **cfg) as S0:
        ctx = S0.stats()["resident_bytes"]        # the launch contexts alone
    with M.Server(budget_bytes=ctx + 2_000_000, **cfg) as S:
        sid = S.register(small)
        with pytest.raises(M.MsrepError) as e:
            S.register(big)               # about 3.3 MB does not fit
        assert e.value.status == 6        # MSREP_ERR_BUDGET
        assert S.stats()["rejected"] == 1
        S.unregister(sid)
        with pytest.raises(M.MsrepError) as e:
            S.submit(sid, np.zeros((1, small.n), np.float32))
        assert e.value.status == 7        # NOT_FOUND after unregister


def test_serve_wait_timeout_then_complete():
    import paper_2209_07552_gb300 as M
    a = I.rmat(scale=16, nnz=1_000_000, seed=8)
    with M.Server(budget_bytes=2 << 30) as S:
        mid = S.register(a)
        t = S.submit(mid, np.ones((8, a.n), np.float32))
        with pytest.raises(M.MsrepError) as e:
            S.wait(t, 0)
        assert e.value.status == 5        # MSREP_ERR_TIMEOUT: not done after 0 us
        y = S.wait(t, -1)
        ones = I.CSR(a.m, a.n, a.row_ptr, a.col_idx,
                     I.to_f32(a.val).astype(np.float64))
        assert normwise(y[0], oracle_spmv(ones, "csr", np.ones(a.n))) <= 1e-6
        with pytest.raises(M.MsrepError) as e:
            S.wait(t, 0)
        assert e.value.status == 7        # collected already


def test_serve_replay_driver():
    """The native open-loop driver: requests submitted at their arrival
    times from one native thread, some writing into the y buffer of an
    earlier request for the same matrix (the driver waits for that request
    first).  Every buffer ends up holding the result of its last request,
    equal bit for bit to msrep_spmv of that request's columns; a reuse
    index that does not point back is refused before anything is
    submitted."""
    import paper_2209_07552_gb300 as M
    mats = _mats(seed=11)
    g = I.rng(41, 2)
    X = [g.uniform(-1, 1, (8, a.n)).astype(np.float32) for a in mats]
    solo = [_solo(M, a, x) for a, x in zip(mats, X)]
    with M.Server(budget_bytes=4 << 30, arena_bytes=16 << 20, contexts=2) as S:
        ids = [S.register(a) for a in mats]
        n = 60
        t_us = np.cumsum(g.exponential(200.0, n))
        pick = g.integers(0, len(mats), n)
        ks = g.integers(1, 9, n).astype(np.int32)
        bufs, ys, reuse, last = {}, [], np.full(n, -1, np.int64), {}
        for i in range(n):
            j = int(pick[i])
            slot = i % 3 if i >= 30 else i          # later requests share 3 buffers a matrix
            key = (j, slot)
            if key not in bufs:
                bufs[key] = np.full((8, mats[j].m), np.nan, np.float32)
            ys.append(bufs[key])
            reuse[i] = last.get(key, -1)
            last[key] = i
        xs = [X[int(pick[i])][:int(ks[i])] for i in range(n)]
        late, lag = S.replay(t_us, [ids[int(p)] for p in pick], ks, xs, ys, reuse)
        assert late >= 0 and lag >= 0.0
        assert S.stats()["completed"] == n
        for key, i in last.items():
            j, k = key[0], int(ks[i])
            assert np.array_equal(bufs[key][:k], solo[j][:k]), (key, i, k)
        bad = reuse.copy()
        bad[5] = 5
        with pytest.raises(M.MsrepError) as e:
            S.replay(t_us, [ids[int(p)] for p in pick], ks, xs, ys, bad)
        assert e.value.status == 1        # MSREP_ERR_INVALID_ARG
        assert S.stats()["completed"] == n


def test_serve_mapped_page_locked_buffers():
    """Page-locked x and y are read and written by the launch's kernels
    directly (one-vector x through the copy kernel, k-vector x by the
    interleaving kernel, y by the copy-out kernel); mixed in one stream with
    pageable buffers, every result equals msrep_spmv bit for bit."""
    import paper_2209_07552_gb300 as M
    mats = _mats(seed=13)
    g = I.rng(43, 1)
    X = [g.uniform(-1, 1, (8, a.n)).astype(np.float32) for a in mats]
    solo = [_solo(M, a, x) for a, x in zip(mats, X)]
    with M.Server(budget_bytes=4 << 30, arena_bytes=16 << 20, contexts=2) as S:
        ids = [S.register(a) for a in mats]
        pending = []
        for rep in range(3):
            for j, (mid, a) in enumerate(zip(ids, mats)):
                for k in (1, 2, 3, 8):
                    pinned = (rep + j + k) % 2 == 0
                    if pinned:
                        xb = M.native.pinned_empty((k, a.n))
                        xb[:] = X[j][:k]
                        yb = M.native.pinned_empty((k * a.m,))
                        yb[:] = np.nan
                    else:
                        xb, yb = X[j][:k].copy(), None
                    pending.append((j, k, xb, S.submit(mid, xb, yb)))
        for j, k, xb, t in pending:
            y = S.wait(t).reshape(k, -1)
            assert np.array_equal(y, solo[j][:k]), (j, k)


def test_serve_full_size_rmat(rmat_full):
    """The served R-MAT of the bench (2^20 rows, 2^24 nonzeros) at each
    width, through mapped page-locked buffers: every column equals
    msrep_spmv of that x bit for bit."""
    import paper_2209_07552_gb300 as M
    a = rmat_full
    g = I.rng(45, 3)
    X = g.uniform(-1, 1, (8, a.n)).astype(np.float32)
    solo = _solo(M, a, X)
    with M.Server(budget_bytes=8 << 30, arena_bytes=64 << 20, contexts=2) as S:
        mid = S.register(a)
        for k in (1, 2, 3, 8):
            xb = M.native.pinned_empty((k, a.n))
            xb[:] = X[:k]
            yb = M.native.pinned_empty((k * a.m,))
            y = S.wait(S.submit(mid, xb, yb)).reshape(k, -1)
            assert np.array_equal(y, solo[:k]), k
