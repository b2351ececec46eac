"""Device partitioner (Alg. 2, 4, 6) against the oracle: bit-exact."""
import numpy as np
import pytest

from helpers import FORMATS, oracle_partition
from paper_2209_07552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KEYS = ("start_idx", "end_idx", "start_major", "end_major", "start_flag")


def _gpu_partition(a, fmt, P, local=True, tile=0, flags=0):
    import paper_2209_07552_gb300 as M
    A = M.DeviceMatrix.from_host(a, fmt, "f64")
    part = M.DevicePartition(A, P, tile=tile, local=local)
    M.msrep_partition(A, part, flags)
    return part.to_host()


def _assert_same(got, want, local=True):
    for k in KEYS:
        assert np.array_equal(got[k], want[k]), k
    if local:
        assert np.array_equal(got["local"], want["local"])
        if "local_off" in want:
            assert np.array_equal(got["local_off"], want["local_off"])


def _adversarial():
    yield "empty", I.csr_from_triplets(7, 5, [], [], [])
    yield "one_row", I.csr_from_triplets(1, 9, [0] * 9, list(range(9)), np.ones(9))
    yield "hub", I.csr_from_triplets(12, 40, [5] * 40, list(range(40)), np.ones(40))
    rows = [0, 0, 3, 3, 3, 9, 9, 9, 9, 9, 9, 14]
    cols = [1, 4, 0, 2, 7, 0, 1, 2, 3, 5, 6, 7]
    yield "gaps", I.csr_from_triplets(20, 8, rows, cols, np.ones(len(rows)))
    yield "rmat_small", I.rmat(scale=8, nnz=1500, seed=5)
    yield "uniform", I.uniform_rows()


@pytest.mark.parametrize("fmt", FORMATS)
def test_partition_adversarial_sweep(fmt):
    for name, a in _adversarial():
        nnz = a.nnz
        for P in sorted({1, 2, 3, 4, 7, 148, max(1, nnz - 1), max(1, nnz), nnz + 5}):
            got = _gpu_partition(a, fmt, P)
            want = oracle_partition(a, fmt, P, with_local=True)
            _assert_same(got, want)


@pytest.mark.parametrize("fmt", FORMATS)
def test_partition_uniform_p4_closed_form(fmt):
    a = I.uniform_rows()
    got = _gpu_partition(a, fmt, 4)
    if fmt != "csc":
        assert got["start_major"].tolist() == [0, 500, 1000, 1500]
        assert got["start_flag"].tolist() == [0, 0, 0, 0]
    _assert_same(got, oracle_partition(a, fmt, 4, with_local=True))


@pytest.mark.slow
@pytest.mark.parametrize("fmt", FORMATS)
def test_partition_rmat_full_size_p_sweep(fmt, rmat_full):
    a = rmat_full
    for k in range(0, 7):
        P = 148 << k
        got = _gpu_partition(a, fmt, P, local=(k in (0, 6)))
        want = oracle_partition(a, fmt, P, with_local=(k in (0, 6)))
        _assert_same(got, want, local=(k in (0, 6)))


def test_partition_validate_flags_bad_matrix():
    import torch

    import paper_2209_07552_gb300 as M
    a = I.rmat(scale=8, nnz=1500, seed=5)
    A = M.DeviceMatrix.from_host(a, "csr")
    part = M.DevicePartition(A, 7)
    M.msrep_partition(A, part, M.MSREP_VALIDATE)  # a good matrix passes
    bad = A.idx.clone()
    bad[10] = a.n + 3  # column out of range: caught on the device, no access
    B = M.DeviceMatrix(A.fmt, A.m, A.n, A.nnz, A.ptr, bad, None, A.val, "f64")
    with pytest.raises(M.MsrepError) as e:
        M.msrep_partition(B, part, M.MSREP_VALIDATE)
    assert e.value.status == 2
    q = I.csr_to_coo(a)
    rows = torch.from_numpy(q.row_idx[::-1].copy()).cuda()
    C = M.DeviceMatrix(M.MSREP_COO, a.m, a.n, a.nnz, None,
                       torch.from_numpy(q.col_idx).cuda(), rows, A.val, "f64")
    pc = M.DevicePartition(C, 7)
    with pytest.raises(M.MsrepError):
        M.msrep_partition(C, pc, M.MSREP_VALIDATE)


def test_partition_rejects_bad_arguments():
    import paper_2209_07552_gb300 as M
    a = I.uniform_rows(m=50, n=50, per_row=3)
    A = M.DeviceMatrix.from_host(a, "csr")
    part = M.DevicePartition(A, 4)
    part.c.np = 0
    with pytest.raises(M.MsrepError) as e:
        M.msrep_partition(A, part)
    assert e.value.status == 1
    part = M.DevicePartition(A, 4)
    with pytest.raises(M.MsrepError):
        M.msrep_partition_csc(A, part)  # wrong format for the call


@pytest.mark.parametrize("fmt", FORMATS)
def test_partition_local_unaligned_output(fmt):
    """Local pointers into a buffer that is not 16-byte aligned (the scalar
    store path) equal the oracle's, as do those into an aligned one."""
    import ctypes

    import torch

    import paper_2209_07552_gb300 as M
    a = I.rmat(scale=12, nnz=60_000, seed=11)
    A = M.DeviceMatrix.from_host(a, fmt, "f64")
    for P in (3, 148, 4099):
        want = oracle_partition(a, fmt, P, with_local=True)
        part = M.DevicePartition(A, P, local=True)
        buf = torch.full((part.local.numel() + 1,), -7, dtype=torch.int32, device="cuda")
        part.local = buf[1:]
        part.c.local = ctypes.c_void_p(part.local.data_ptr())
        M.msrep_partition(A, part)
        got = part.to_host()
        _assert_same(got, want)
        assert int(buf[0].item()) == -7  # nothing written before the array


@pytest.mark.parametrize("fmt", FORMATS)
def test_partition_local_many_strides(fmt):
    """Local arrays longer than one pass of the fill kernels' grid
    (8 x 152 blocks x 256 threads x 8 entries = 2.49M)."""
    a = I.laplace5(1600)   # 12.8M nonzeros, 2.56M rows
    for P in (1, 2368):
        got = _gpu_partition(a, fmt, P)
        want = oracle_partition(a, fmt, P, with_local=True)
        _assert_same(got, want)
