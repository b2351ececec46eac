"""Failure detection on the device: a bounded wait that runs out.

The streaming kernels wait on mbarriers for their bulk copies, each wait
bounded; when one gives up, the kernel records a timeout in the device error
word and returns, and msrep_device_status reports MSREP_ERR_TIMEOUT.  Here
the wait is made to run out without any fault: msrep_wait_selftest waits on
a barrier that can never complete (it expects two arrivals and gets one), so
the wait must give up after its cycle limit, the kernel must return, the
status must read TIMEOUT once, and the context must stay usable."""
import numpy as np
import pytest

from helpers import gpu_spmv, normwise, oracle_spmv
from paper_2209_07552_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_is_reported():
    import torch

    import paper_2209_07552_gb300 as M
    assert M.msrep_device_status() == 0          # nothing pending
    gave_up = torch.zeros(1, dtype=torch.int32, device="cuda")
    M.msrep_wait_selftest(20_000, gave_up)       # about 10 us at 2 GHz
    torch.cuda.synchronize()                     # the kernel returned
    assert int(gave_up.item()) == 1
    with pytest.raises(M.MsrepError) as e:
        M.msrep_device_status()
    assert e.value.status == 5                   # MSREP_ERR_TIMEOUT
    assert M.msrep_device_status() == 0          # read once, then cleared
    # the context is still usable: an SpMV right after is correct
    a = I.uniform_rows(m=2000, n=2000, per_row=10)
    x = I.vector(a.n, I.SEED_BASE)
    y = gpu_spmv(a, "csr", 4, x)
    assert normwise(y, oracle_spmv(a, "csr", x)) <= 1e-12


def test_wait_selftest_rejects_bad_limits():
    import torch

    import paper_2209_07552_gb300 as M
    g = torch.zeros(1, dtype=torch.int32, device="cuda")
    for bad in (0, -5, 3_000_000_000):
        with pytest.raises(M.MsrepError) as e:
            M.msrep_wait_selftest(bad, g)
        assert e.value.status == 1               # INVALID_ARG, nothing queued
    assert M.msrep_device_status() == 0
