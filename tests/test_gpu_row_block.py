"""The Baseline row-block partitioning (Sec. 5.1; MSREP_PART_ROW_BLOCK) and
the one-block-per-partition schedule (MSREP_SCHED_PER_PARTITION).

Row-block metadata must equal the oracle's bit for bit (CSR, CSC's column
blocks, row-sorted COO, and COO sorted by column, whose column blocks equal
CSC's).  The SpMV over row blocks, and over Alg. 2's nonzero cuts with one
thread block per partition, must give the oracle's y (normwise 1e-12, and
bit for bit on integer-valued data)."""
import numpy as np
import pytest

import oracle as O
from helpers import FORMATS, coo_of, normwise, oracle_spmv
from paper_2209_07552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KEYS = ("start_idx", "end_idx", "start_major", "end_major", "start_flag")


def _mats():
    out = [I.csr_from_triplets(7, 5, [], [], []),
           I.csr_from_triplets(20, 8, [0, 0, 3, 3, 3, 9, 9, 9, 9, 9, 9, 14],
                               [1, 4, 0, 2, 7, 0, 1, 2, 3, 5, 6, 7], np.ones(12)),
           I.rmat(scale=12, nnz=60_000, seed=41),
           I.block_imbalance_matrix(4096, 16, 24, 10, 42)]
    return out


def _oracle_row_block(a, fmt, P, with_local):
    if fmt == "csr":
        return O.partition_row_block(a.row_ptr, a.nnz, P, with_local)
    if fmt == "csc":
        return O.partition_row_block(I.csr_to_csc(a).col_ptr, a.nnz, P, with_local)
    if fmt == "coo":
        return O.partition_coo_row_block(I.csr_to_coo(a).row_idx, a.m, P, with_local)
    q = I.csr_to_coo_by_col(a)           # column blocks over the column index
    return O.partition_coo_row_block(q.col_idx, a.n, P, with_local)


@pytest.mark.parametrize("fmt", FORMATS + ("coo_col",))
def test_row_block_metadata_bit_exact(fmt):
    import paper_2209_07552_gb300 as M
    for a in _mats():
        A = M.DeviceMatrix.from_host(a, fmt, "f64")
        for P in sorted({1, 3, 16, 148, max(1, a.m - 1), a.m + 7}):
            part = M.DevicePartition(A, P, local=True)
            M.msrep_partition(A, part, M.MSREP_PART_ROW_BLOCK)
            got = part.to_host()
            want = _oracle_row_block(a, fmt, P, True)
            for k in KEYS:
                assert np.array_equal(got[k], want[k]), (fmt, a.m, P, k)
            if fmt in ("csr", "csc"):
                assert np.array_equal(got["local_off"], want["local_off"])
            assert np.array_equal(got["local"], want["local"]), (fmt, P)


@pytest.mark.parametrize("fmt", FORMATS)
def test_row_block_and_per_partition_spmv(fmt):
    import torch

    import paper_2209_07552_gb300 as M
    for a in _mats()[1:]:
        x = I.vector(a.n, 43)
        want = oracle_spmv(a, fmt, x, 1.5, -0.5, I.y_vector(a.m, 44))
        ai, xi = I.integer_twin(a, seed=45)
        want_i = oracle_spmv(ai, fmt, xi)
        for pflags in (M.MSREP_PART_ROW_BLOCK, 0):
            for flags in (0, M.MSREP_SCHED_PER_PARTITION):
                for P in (1, 7, 152):
                    for tile in (256, 1024):
                        A = M.DeviceMatrix.from_host(a, fmt, "f64")
                        part = M.DevicePartition(A, P, tile=tile)
                        M.msrep_partition(A, part, pflags)
                        ws = M.alloc_workspace(A, part)
                        y = torch.from_numpy(I.y_vector(a.m, 44)).cuda()
                        M.msrep_spmv(A, part, 1.5, torch.from_numpy(x).cuda(), -0.5, y,
                                     flags=flags, workspace=ws)
                        assert normwise(y.cpu().numpy(), want) <= 1e-12, (pflags, flags, P)
                        Ai = M.DeviceMatrix.from_host(ai, fmt, "f64")
                        pi = M.DevicePartition(Ai, P, tile=tile)
                        M.msrep_partition(Ai, pi, pflags)
                        yi = torch.empty(a.m, dtype=torch.float64, device="cuda")
                        M.msrep_spmv(Ai, pi, 1.0, torch.from_numpy(xi).cuda(), 0.0, yi,
                                     flags=flags, workspace=M.alloc_workspace(Ai, pi))
                        assert np.array_equal(yi.cpu().numpy(), want_i), (pflags, flags, P)


def test_row_block_flag_errors():
    import paper_2209_07552_gb300 as M
    a = _mats()[2]
    A = M.DeviceMatrix.from_host(a, "csr", "f64")
    part = M.DevicePartition(A, 8)
    with pytest.raises(M.MsrepError) as e:
        M.msrep_partition(A, part, M.MSREP_PART_ROW_BLOCK | M.MSREP_PART_MERGE_PATH)
    assert e.value.status == 1
    U = M.DeviceMatrix.from_host(a, "coo_any", "f64")
    with pytest.raises(M.MsrepError) as e:
        M.msrep_partition(U, M.DevicePartition(U, 8), M.MSREP_PART_ROW_BLOCK)
    assert e.value.status == 1
