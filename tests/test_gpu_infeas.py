"""GPU infeasibility detection (Sec. 2.2, last bullet) through the C ABI
against the FP64 oracle on the same LPs.

Both sides test the same two rays at every check with the same rule, but
the GPU forms K xr and K'yr from stored products (K x and K'y of the two
iterates) while the oracle multiplies the unscaled ray directly, so the
certificates' residuals differ by rounding: the check at which a
certificate first passes may differ, and the comparison is on the status,
on the returned ray passing the oracle's own test at eps, and on the
iteration count to within a factor of two."""

import numpy as np
import pytest

import lpgen
import oracle
from paper_2311_12180_gb300 import pdlp as P

pytestmark = pytest.mark.gpu

EPS = 1e-8


def _check_ray(lp, status, x, y):
    if status == P.PRIMAL_INFEASIBLE:
        t = oracle.infeas_terms(lp, np.zeros(lp.n), y)
        assert np.all(x >= lp.l) and np.all(x <= lp.u)
    else:
        t = oracle.infeas_terms(lp, x, np.zeros(lp.m))
    assert oracle.infeas_status(t, EPS) == status
    return t


@pytest.mark.parametrize("kind", ["primal", "primal_bounds", "dual"])
@pytest.mark.parametrize("size", ["tiny", "tiles"])
def test_detects_like_the_oracle(kind, size):
    kw = {} if size == "tiny" else dict(m_eq=1500, m_ineq=1500, n=5000, density=0.003)
    lp = lpgen.infeasible_lp(3, kind, **kw)
    r = oracle.solve(lp, tol=1e-8, max_iter=400000, eps_infeas=EPS)
    want = P.DUAL_INFEASIBLE if kind == "dual" else P.PRIMAL_INFEASIBLE
    assert r.status == want
    with P.Solver(lp, eps_infeas=EPS) as s:
        x, y, st, it = s.solve(tol=1e-8, max_iter=400000)
        info = s.info()
    assert st == want, P.STATUS_NAMES.get(st, st)
    assert info["which"] in (2, 3)
    assert it <= 2 * r.iters + 128 and r.iters <= 2 * it + 128
    t = _check_ray(lp, st, x, y)
    obj, res = (t[0], t[1]) if st == P.PRIMAL_INFEASIBLE else (t[2], t[3])
    assert info["ray_obj"] == pytest.approx(obj, rel=1e-6)
    assert info["ray_res"] <= EPS * info["ray_obj"]
    assert res <= EPS * obj


def test_detection_off_runs_to_the_limit():
    lp = lpgen.infeasible_lp(0, "primal")
    with P.Solver(lp, eps_infeas=0.0) as s:
        _, _, st, it = s.solve(tol=1e-8, max_iter=4096)
    r = oracle.solve(lp, tol=1e-8, max_iter=4096, eps_infeas=0.0)
    assert st == P.ITER_LIMIT == r.status and it == 4096 == r.iters


def test_detection_leaves_feasible_solves_unchanged():
    for seed in (0, 1):
        lp = lpgen.tiny_lp(seed)
        with P.Solver(lp, eps_infeas=EPS) as s:
            x1, y1, st1, it1 = s.solve(tol=1e-8, max_iter=200000)
        with P.Solver(lp, eps_infeas=0.0) as s:
            x0, y0, st0, it0 = s.solve(tol=1e-8, max_iter=200000)
        assert st1 == st0 == P.OPTIMAL and it1 == it0
        assert np.array_equal(x1, x0) and np.array_equal(y1, y0)



def test_batch_detects_like_the_oracle():
    """The batched solver runs the same tests per LP; two of the infeasible
    LPs are large enough for a team of CTAs (>= 32768 nonzeros)."""
    big = dict(m_eq=600, m_ineq=600, n=3000, density=0.02)
    lps = [lpgen.tiny_lp(50), lpgen.infeasible_lp(0, "primal"), lpgen.infeasible_lp(1, "primal_bounds"),
           lpgen.infeasible_lp(2, "dual"), lpgen.tiny_lp(51), lpgen.infeasible_lp(5, "primal", **big),
           lpgen.infeasible_lp(6, "dual", **big)]
    assert lps[5].nnz >= 32768 and lps[6].nnz >= 32768
    with P.BatchSolver(lps, eps_infeas=EPS) as b:
        xs, ys, st, it = b.solve(tol=1e-8, max_iter=400000)
    for i, lp in enumerate(lps):
        r = oracle.solve(lp, tol=1e-8, max_iter=400000, eps_infeas=EPS)
        assert st[i] == r.status, (i, st[i], r.status)
        assert it[i] <= 2 * r.iters + 128 and r.iters <= 2 * it[i] + 128
        if st[i] == P.OPTIMAL:
            assert oracle.passes(lp, xs[i], ys[i], 1e-8)
        else:
            _check_ray(lp, st[i], xs[i], ys[i])
    with P.BatchSolver(lps[1:4], eps_infeas=0.0) as b:
        _, _, st0, it0 = b.solve(tol=1e-8, max_iter=4096)
    assert list(st0) == [P.ITER_LIMIT] * 3 and list(it0) == [4096] * 3
