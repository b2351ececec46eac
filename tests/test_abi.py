"""The C ABI library builds, loads without a GPU and exports every symbol
that include/msrep.h declares; host-only entry points answer without a GPU.
No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "msrep.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(msrep_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def so():
    from paper_2209_07552_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(so):
    names = _declared()
    assert "msrep_spmv" in names and "msrep_partition_csr" in names
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2209_07552_gb300 import native
    missing = [n for n in _declared() if n not in native.SIGNATURES]
    assert not missing, missing


def test_host_only_entry_points(so):
    from paper_2209_07552_gb300 import native as N
    N.lib(so._name)
    assert N.msrep_version().startswith("msrep")
    assert N.msrep_tile_supported(256) and not N.msrep_tile_supported(100)
    A = N.DeviceMatrix.__new__(N.DeviceMatrix)
    A.c = N.c_msrep_matrix(N.MSREP_CSR, N.MSREP_F64, 1000, 1000, 5000, 1, 1, None, 1)
    A.fmt = N.MSREP_CSR
    assert N.msrep_partition_local_bound(A, 10) == 1000 + 20
    assert N.msrep_plan_size(A, 10, 0) > 0
    with pytest.raises(N.MsrepError) as e:
        N.msrep_plan_size(A, 0, 0)
    assert e.value.status == 1
    A.c.fmt = 7
    with pytest.raises(N.MsrepError):
        N.msrep_plan_size(A, 4, 0)


def test_spmm_workspace_size_host_checks(so):
    from paper_2209_07552_gb300 import native as N
    N.lib(so._name)
    A = N.DeviceMatrix.__new__(N.DeviceMatrix)
    A.c = N.c_msrep_matrix(N.MSREP_CSR, N.MSREP_F32, 1000, 800, 5000, 1, 1, None, 1)
    A.fmt = N.MSREP_CSR
    P = N.DevicePartition.__new__(N.DevicePartition)
    P.c = N.c_msrep_partition()
    P.c.np = 4
    sizes = [N.msrep_spmm_workspace_size(A, P, k) for k in (1, 2, 3, 4, 8, 9, 40)]
    # the interleaved copy of X grows with k rounded up to 1, 2, 4, 8; more
    # than 8 vectors go in passes of 8 through the same workspace
    assert sizes[0] < sizes[1] < sizes[2] == sizes[3] < sizes[4] == sizes[5] == sizes[6]
    for bad in (0, -3):
        with pytest.raises(N.MsrepError) as e:
            N.msrep_spmm_workspace_size(A, P, bad)
        assert e.value.status == 1
    A.c.fmt = N.MSREP_CSC
    with pytest.raises(N.MsrepError):
        N.msrep_spmm_workspace_size(A, P, 2)


def test_plan_sizes_per_format(so):
    """CSC plans also hold the frequent-row table and its 1 MB search
    scratch; row-sorted COO needs no plan; column-sorted and unsorted COO
    need a fixed-size one (hub rows, frequent-row table, scratch)."""
    from paper_2209_07552_gb300 import native as N
    N.lib(so._name)
    A = N.DeviceMatrix.__new__(N.DeviceMatrix)
    A.c = N.c_msrep_matrix(N.MSREP_CSR, N.MSREP_F64, 1000, 1000, 5000, 1, 1, None, 1)
    csr = N.msrep_plan_size(A, 10, 0)
    A.c.fmt = N.MSREP_CSC
    csc = N.msrep_plan_size(A, 10, 0)
    assert csc - csr >= (1 << 20)
    A.c.fmt = N.MSREP_COO
    A.c.ptr = None
    A.c.idx2 = 1
    assert N.msrep_plan_size(A, 10, 0) == 0
    sizes = set()
    for fmt in (N.MSREP_COO_BY_COL, N.MSREP_COO_UNSORTED):
        A.c.fmt = fmt
        for np_, nnz in ((10, 5000), (4096, 1 << 24)):
            A.c.nnz = nnz
            sizes.add(N.msrep_plan_size(A, np_, 0))
    assert len(sizes) == 1 and sizes.pop() >= (1 << 20)


def test_partition_argument_errors_before_any_device_work(so):
    """Errors the partitioners report from their arguments alone, before
    touching the device: the merge-path flag on COO, and plans smaller than
    msrep_plan_size (CSC: it holds the frequent-row table; COO sorted by
    column: its fixed-size plan).  The pointers are never dereferenced."""
    import ctypes

    from paper_2209_07552_gb300 import native as N
    N.lib(so._name)
    fake = ctypes.c_void_p(256)

    def part(plan_bytes):
        p = N.c_msrep_partition()
        p.np = 4
        p.start_idx = p.end_idx = p.start_major = p.end_major = p.start_flag = fake
        p.plan = fake if plan_bytes else None
        p.plan_bytes = plan_bytes
        return p

    A = N.c_msrep_matrix(N.MSREP_COO, N.MSREP_F64, 100, 100, 500, None, 256, 256, 256)
    rc = N.lib().msrep_partition_coo(ctypes.byref(A), ctypes.byref(part(0)),
                                     N.MSREP_PART_MERGE_PATH, None)
    assert rc == 1
    A.fmt = N.MSREP_COO_BY_COL
    rc = N.lib().msrep_partition_coo(ctypes.byref(A), ctypes.byref(part(1024)), 0, None)
    assert rc == 9                                       # plan too small
    C = N.c_msrep_matrix(N.MSREP_CSC, N.MSREP_F64, 100, 100, 500, 256, 256, None, 256)
    M = N.DeviceMatrix.__new__(N.DeviceMatrix)
    M.c = C
    need = N.msrep_plan_size(M, 4, 0)
    rc = N.lib().msrep_partition_csc(ctypes.byref(C), ctypes.byref(part(need - 256)), 0, None)
    assert rc == 9
