"""Debug mode of the solver (environment PDLP_DEBUG_CHECKS=1 at create): the
sliced-ELL copies of K and K' that the step and check kernels read without
bounds checks of their own are checked on the device -- every stored column
index inside [-1, columns), padding with value 0 (also in the FP32 copy),
every work item inside the storage, every row covered exactly once.  The
layouts of the test LPs pass, and the debug create changes nothing else."""

import numpy as np
import pytest

import lpgen
from paper_2311_12180_gb300 import pdlp as P

pytestmark = pytest.mark.gpu


def _ragged():
    rng = np.random.default_rng(5)
    m, n = 40, 12000
    lens = np.array([1, 2, 5000, 3, 2500, 1] + [40] * (m - 6))
    row_ptr, cols = lpgen._sample_rows(rng, lens, n)
    row_ptr, cols = lpgen._cover_columns(rng, row_ptr, cols, m, n)
    return lpgen.plant(rng, m, n, 20, row_ptr, cols, rng.standard_normal(cols.size), np.zeros(n), np.full(n, 10.0))


@pytest.mark.parametrize("case,bits", [("tiny", 64), ("tiny", 32), ("powerlaw", 64), ("powerlaw", 32),
                                       ("long_rows", 64)])
def test_debug_checks_pass_and_change_nothing(monkeypatch, case, bits):
    lp = {"tiny": lambda: lpgen.tiny_lp(7), "powerlaw": lambda: lpgen.large_lp(4, m=20000, n=40000, nnz=400000),
          "long_rows": _ragged}[case]()
    with P.Solver(lp, value_bits=bits) as s:
        ref = s.solve(tol=1e-14, max_iter=200)
    monkeypatch.setenv("PDLP_DEBUG_CHECKS", "1")
    with P.Solver(lp, value_bits=bits) as s:
        got = s.solve(tol=1e-14, max_iter=200)
    assert got[2] == ref[2] and got[3] == ref[3]
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
