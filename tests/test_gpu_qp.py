"""QP extension (diagonal Hessian) on the GPU against the FP64 oracle: the
same planted QPs, element by element over a short horizon and to a tight
tolerance; an LP after the Hessian is cleared is unchanged bit for bit."""

import numpy as np
import pytest

import lpgen
import oracle
from paper_2311_12180_gb300 import pdlp as P

pytestmark = pytest.mark.gpu


def _qp(case):
    base = {"tiny": lambda: lpgen.tiny_lp(5),
            "powerlaw": lambda: lpgen.large_lp(4, m=20000, n=40000, nnz=400000),
            # small enough for the oracle to reach 1e-8 in seconds
            "powerlaw_small": lambda: lpgen.large_lp(2, m=1000, n=2000, nnz=20000)}[case]()
    return lpgen.planted_qp(base, seed=2)


@pytest.mark.parametrize("case,P_,N", [("tiny", 8, 96), ("powerlaw", 64, 30)])
def test_qp_iterates_match_oracle(case, P_, N):
    # a horizon over which the two FP64 paths (different summation orders)
    # stay within 1e-9; they separate later, as LPs do (reading 24)
    qp = _qp(case)
    with P.Solver(qp, check_period=P_) as s:
        x, y, st, it = s.solve(tol=1e-14, max_iter=N)
        tr = s.trace()
        info = s.info()
    r = oracle.solve(qp, tol=1e-14, max_iter=N, check_period=P_)
    assert st == P.ITER_LIMIT == r.status and it == N == r.iters
    assert info["attempts"] == r.attempts and info["restarts"] == r.restarts
    np.testing.assert_array_equal(tr["restart"], r.trace["restart"])
    for f in ("kkt_cur", "kkt_avg", "kkt_start", "omega", "eta_hat"):
        np.testing.assert_allclose(tr[f], r.trace[f], rtol=1e-9, err_msg=f)
    np.testing.assert_allclose(x, r.x, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.x).max()))
    np.testing.assert_allclose(y, r.y, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.y).max()))


@pytest.mark.parametrize("case", ["tiny", "powerlaw_small"])
def test_qp_solution_matches_oracle_and_planted_optimum(case):
    qp = _qp(case)
    with P.Solver(qp) as s:
        x, y, st, it = s.solve(tol=1e-8, max_iter=2_000_000)
        info = s.info()
    assert st == P.OPTIMAL
    obj = float(0.5 * np.dot(qp.qdiag * x, x) + qp.c @ x)
    assert obj == pytest.approx(info["pobj"], rel=1e-12)
    assert abs(obj - qp.obj_star) <= 1e-6 * (1 + abs(qp.obj_star))
    # the oracle's own Sec. 4.1 test of the QP accepts the GPU's point
    assert oracle.passes(qp, x, y, 1e-8)
    r = oracle.solve(qp, tol=1e-8, max_iter=2_000_000)
    assert r.status == oracle.OPTIMAL
    assert abs(obj - r.pobj) <= 1e-6 * (1 + abs(r.pobj))


def test_clearing_the_hessian_restores_the_lp_bitwise():
    lp = lpgen.tiny_lp(6)
    with P.Solver(lp) as a:
        ref = a.solve(tol=1e-8)
    qp = lpgen.planted_qp(lp, seed=3)
    with P.Solver(lp) as b:
        b.set_quadratic(qp.qdiag)
        q = b.solve(tol=1e-8)
        b.set_quadratic(None)
        back = b.solve(tol=1e-8)
    assert not np.array_equal(q[0], ref[0])  # the Hessian did change the solve
    assert (back[2], back[3]) == (ref[2], ref[3])
    assert np.array_equal(back[0], ref[0]) and np.array_equal(back[1], ref[1])


def test_set_quadratic_rejects_negative_or_nonfinite_entries():
    lp = lpgen.tiny_lp(6)
    with P.Solver(lp) as s:
        for bad in (-1.0, np.nan, np.inf):
            d = np.ones(lp.n)
            d[7] = bad
            with pytest.raises(P.PdlpError) as e:
                s.set_quadratic(d)
            assert e.value.code == P.ERR_INVALID


@pytest.mark.parametrize("case,N", [("tiny", 60), ("powerlaw", 30)])
def test_qp_fp32_values_iterates_match_the_oracles_fp32_steps(case, N):
    """A QP with FP32 matrix values in the steps (value_bits = 32) against
    the oracle's FP32-values mode before the first check: the same trials
    and the same iterates elementwise; the FP64 method is elsewhere."""
    qp = _qp(case)
    with P.Solver(qp, check_period=64, value_bits=32) as s:
        x, y, st, it = s.solve(tol=1e-14, max_iter=N)
        info = s.info()
    r = oracle.solve(qp, tol=1e-14, max_iter=N, check_period=64, step_value_bits=32)
    r64 = oracle.solve(qp, tol=1e-14, max_iter=N, check_period=64)
    assert st == P.ITER_LIMIT == r.status and it == N == r.iters
    assert info["attempts"] == r.attempts
    np.testing.assert_allclose(x, r.x, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.x).max()))
    np.testing.assert_allclose(y, r.y, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.y).max()))
    assert np.abs(y - r64.y).max() > 1e-7 * max(1.0, np.abs(r64.y).max())
