"""msrep_access_floor, the measurement kernel of the bench's access-pattern
floor: its scatter modes really perform the adds (checked against numpy on
integer values, exact in any order), and every mode accepts any index
(indices are reduced modulo the power-of-two vector length)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _slot(r, mask):
    return (r.astype(np.uint64) * 0x9E3779B1) & mask


def test_scatter_modes_add_every_value():
    import torch

    import paper_2209_07552_gb300 as M
    rng = np.random.default_rng(5)
    nnz, n = 100_003, 1 << 12          # ragged tail: nnz not a multiple of 8
    idx = rng.integers(0, 3 * n, nnz).astype(np.int32)   # beyond n too: masked
    val = rng.integers(-3, 4, nnz).astype(np.float64)
    di, dv = torch.from_numpy(idx).cuda(), torch.from_numpy(val).cuda()
    for mode, slots in ((2, idx.astype(np.uint64) & (n - 1)), (3, _slot(idx, n - 1))):
        vec = torch.zeros(n, dtype=torch.float64, device="cuda")
        M.native.msrep_access_floor(mode, di, dv, vec)
        want = np.bincount(slots.astype(np.int64), weights=val, minlength=n)
        assert np.array_equal(vec.cpu().numpy(), want), mode


def test_gather_modes_run_and_reject_bad_lengths():
    import torch

    import paper_2209_07552_gb300 as M
    idx = torch.arange(0, 4096, dtype=torch.int32, device="cuda") * 7
    val = torch.ones(4096, dtype=torch.float64, device="cuda")
    x = torch.ones(1024, dtype=torch.float64, device="cuda")
    M.native.msrep_access_floor(0, idx, val, x)
    M.native.msrep_access_floor(1, idx, val, x, idx2=idx)
    # lane-interleaved modes, also on a ragged length (not a multiple of 256)
    M.native.msrep_access_floor(4, idx, val, x)
    M.native.msrep_access_floor(5, idx, val, x, idx2=idx)
    M.native.msrep_access_floor(4, idx[:4000], val[:4000], x)
    M.native.msrep_access_floor(5, idx[:4000], val[:4000], x, idx2=idx[:4000])
    torch.cuda.synchronize()
    for bad in (-1, 6):
        with pytest.raises(M.MsrepError) as e:
            M.native.msrep_access_floor(bad, idx, val, x, idx2=idx)
        assert e.value.status == 1
    with pytest.raises(M.MsrepError) as e:
        M.native.msrep_access_floor(0, idx, val, torch.ones(1000, dtype=torch.float64,
                                                            device="cuda"))
    assert e.value.status == 1
