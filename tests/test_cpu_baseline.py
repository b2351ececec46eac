"""The all-core CPU baseline the benchmark times (oracle/cpu_baseline.c)
computes the same SpMV as the oracle.  It is a timed program, not a
reference: this only guards the baseline numbers against a wrong program."""
import numpy as np
import pytest

from helpers import normwise, oracle_spmv
from paper_2209_07552_gb300 import inputs as I


@pytest.mark.parametrize("fmt", ["csr", "csc", "coo"])
def test_cpu_baseline_matches_oracle(fmt):
    from oracle import cpu_baseline as C
    for a in (I.rmat(scale=12, nnz=40_000, seed=71), I.laplace5(64),
              I.csr_from_triplets(9, 4, [2, 2, 7], [0, 3, 1], [1.0, 2.0, 3.0])):
        x = I.vector(a.n, 72)
        if fmt == "csr":
            P = C.Prepared("csr", a.m, a.n, a.row_ptr, a.col_idx, a.val)
        elif fmt == "csc":
            c = I.csr_to_csc(a)
            P = C.Prepared("csc", a.m, a.n, c.col_ptr, c.row_idx, c.val)
        else:
            q = I.csr_to_coo(a)
            P = C.Prepared("coo", a.m, a.n, None, q.col_idx, q.val, row_idx=q.row_idx)
        y = np.full(a.m, np.nan)
        P.run(x, y)
        assert normwise(y, oracle_spmv(a, fmt, x)) <= 1e-12
    assert C.threads() >= 1
