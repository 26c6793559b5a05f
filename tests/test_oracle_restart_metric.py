"""Restart-metric ablation in the oracle (not part of the GPU path): the
paper's KKT-error restarts (Sec. 3.4) against the normalized-duality-gap
restarts of CPU PDLP that they replace (Sec. 2.2 "Adaptive restarts",
Appendix A).  First the normalized gap itself is pinned (closed form without
bounds, an independent optimiser with bounds, zero at a planted saddle point,
its monotonicity in the radius); then both schemes solve the same families
and their iteration counts are compared."""

import math

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle


class _LP:
    def __init__(self, A, c, q, l, u, n_eq):
        S = sp.csr_matrix(A)
        self.m, self.n = A.shape
        self.n_eq = n_eq
        self.row_ptr, self.col_idx, self.val = S.indptr, S.indices, S.data
        self.c, self.q, self.l, self.u = c, q, l, u


def _random(seed, bounded):
    rng = np.random.default_rng(seed)
    m, n = 3, 5
    A = rng.standard_normal((m, n))
    c, q = rng.standard_normal(n), rng.standard_normal(m)
    if bounded:
        lp = _LP(A, c, q, np.zeros(n), np.full(n, 2.0), 1)
        x = rng.uniform(0, 2, n)
        y = np.abs(rng.standard_normal(m))
        y[0] = -0.3
    else:
        lp = _LP(A, c, q, np.full(n, -np.inf), np.full(n, np.inf), m)
        x, y = rng.standard_normal(n), rng.standard_normal(m)
    return lp, A, x, y


@pytest.mark.parametrize("omega", [0.4, 1.0, 2.5])
def test_gap_without_bounds_is_the_weighted_gradient_norm(omega):
    # no bounds: the maximiser is r h / ||h|| on the ball, so rho_r = ||h|| for every r
    lp, A, x, y = _random(0, bounded=False)
    h = np.concatenate([-(lp.c - A.T @ y) / math.sqrt(omega), math.sqrt(omega) * (lp.q - A @ x)])
    for r in (0.01, 1.0, 50.0):
        assert oracle.normalized_gap(lp, x, y, omega, r) == pytest.approx(np.linalg.norm(h), rel=1e-12)


def test_gap_with_bounds_matches_an_independent_optimiser():
    from scipy.optimize import minimize

    lp, A, x, y = _random(1, bounded=True)
    w = 2.5
    n, m = lp.n, lp.m
    gx, gy = -(lp.c - A.T @ y), lp.q - A @ x
    bnds = [(lp.l[j] - x[j], lp.u[j] - x[j]) for j in range(n)] + [(None, None)] + [(-y[i], None) for i in range(1, m)]
    for r in (0.05, 0.7, 3.0, 40.0):
        cons = [{"type": "ineq", "fun": lambda d: r * r - (w * d[:n] @ d[:n] + d[n:] @ d[n:] / w)}]
        best = min(minimize(lambda d: -(gx @ d[:n] + gy @ d[n:]), 1e-3 * np.random.default_rng(s).standard_normal(n + m),
                            method="SLSQP", bounds=bnds, constraints=cons, options={"ftol": 1e-14, "maxiter": 500}).fun
                   for s in range(8))
        assert oracle.normalized_gap(lp, x, y, w, r) == pytest.approx(-best / r, rel=1e-7, abs=1e-9)


def test_gap_is_zero_at_a_planted_saddle_point_and_monotone_in_r():
    lp = lpgen.tiny_lp(2)
    for r in (0.1, 1.0, 10.0):
        assert abs(oracle.normalized_gap(lp, lp.x_star, lp.y_star, 1.3, r)) < 1e-9
    rng = np.random.default_rng(3)
    x = np.clip(lp.x_star + rng.standard_normal(lp.n), lp.l, lp.u)
    y = lp.y_star + rng.standard_normal(lp.m)
    y[lp.n_eq:] = np.maximum(y[lp.n_eq:], 0)
    rs = np.geomspace(1e-3, 1e3, 13)
    g = np.array([oracle.normalized_gap(lp, x, y, 0.7, r) for r in rs])
    assert np.all(g > 0)
    assert np.all(np.diff(g) <= 1e-12 * g[:-1])          # rho_r does not increase with r
    assert np.all(np.diff(g * rs) >= -1e-12 * (g * rs)[1:])  # r rho_r (the maximum) does not decrease


def _families():
    return ([("tiny", s, lpgen.tiny_lp(s)) for s in range(6)] +
            [("boxed", s, lpgen.random_boxed_lp(s, 3, 3, 8)) for s in range(3)] +
            [("powerlaw", s, lpgen.large_lp(s, m=1000, n=2000, nnz=20000)) for s in range(3)])


def test_kkt_restarts_and_gap_restarts_take_comparable_iterations():
    """Appendix A argues that restarting on the KKT error behaves like the
    normalized-gap restarts of CPU PDLP.  Both schemes solve every LP of the
    tiny, boxed and power-law families to 1e-6 here, and the geometric mean
    of the iteration ratio stays within a factor of two."""
    ratios = []
    for name, s, lp in _families():
        r_kkt = oracle.solve(lp, tol=1e-6, max_iter=400000, restart_metric=0)
        r_gap = oracle.solve(lp, tol=1e-6, max_iter=400000, restart_metric=1)
        assert r_kkt.status == oracle.OPTIMAL and r_gap.status == oracle.OPTIMAL, (name, s)
        for r in (r_kkt, r_gap):
            assert abs(float(lp.c @ r.x) - lp.obj_star) <= 1e-5 * (1 + abs(lp.obj_star)), (name, s)
        ratios.append(r_kkt.iters / r_gap.iters)
    gm = math.exp(np.mean(np.log(ratios)))
    assert 0.5 <= gm <= 2.0, (gm, ratios)
