"""Pins for the oracle's infeasibility detection (Sec. 2.2, last bullet), no
GPU: hand-worked certificate measures (every cone case, a non-symmetric K,
both objective terms), the weak-duality bounds that any measure of a
feasible LP must obey, the exact certificates the generator builds in, and
HiGHS (scipy) as an independent judge of which LPs are infeasible."""

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle
from conftest import DictLP


# ---------------------------------------------------------------- hand examples


def test_infeas_terms_hand(golden):
    g = golden["infeas_terms"]
    lp = DictLP(g["lp"])
    for case in g["cases"]:
        out = oracle.infeas_terms(lp, np.array(case["xr"]), np.array(case["yr"]))
        np.testing.assert_allclose(out, case["out"], rtol=1e-15, atol=1e-15)
    ub = DictLP(g["unbounded_lp"])
    out = oracle.infeas_terms(ub, np.array(g["unbounded_ray"]["xr"]), np.zeros(1))
    np.testing.assert_allclose(out, g["unbounded_ray"]["out"], rtol=0, atol=0)


def test_infeas_status_rule():
    # positive objective and residual at most eps times it; dual ray first
    assert oracle.infeas_status([2.0, 0.0, 0.0, 0.0], 1e-8) == oracle.PRIMAL_INFEASIBLE
    assert oracle.infeas_status([2.0, 2e-8, 0.0, 0.0], 1e-8) == oracle.PRIMAL_INFEASIBLE
    assert oracle.infeas_status([2.0, 2.1e-8, 0.0, 0.0], 1e-8) == -1
    assert oracle.infeas_status([-2.0, 0.0, 0.0, 0.0], 1e-8) == -1
    assert oracle.infeas_status([0.0, 0.0, 1.0, 1e-9], 1e-8) == oracle.DUAL_INFEASIBLE
    assert oracle.infeas_status([0.0, 0.0, 0.0, 0.0], 1e-8) == -1
    assert oracle.infeas_status([1.0, 0.0, 1.0, 0.0], 1e-8) == oracle.PRIMAL_INFEASIBLE


# ---------------------------------------------------------------- weak duality


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_measures_obey_weak_duality_on_feasible_lps(seed):
    """For a feasible LP with point x* (slack s on the '>=' rows) any dual ray
    has objective <= residual * ||(x*, s)||; for a dual-feasible one with
    (y*, lam*) any primal ray has -c'xr <= residual * ||(y*, lam*)||.  A sign
    error in q'y, l'lam+ - u'lam-, c'x or the projection breaks one of them
    for some random ray."""
    lp = lpgen.large_lp(seed, m=60, n=90, nnz=500)  # free, [0, inf) and boxed variables
    rng = np.random.default_rng(seed)
    kx = np.array([lp.val[lp.row_ptr[i]:lp.row_ptr[i + 1]] @ lp.x_star[lp.col_idx[lp.row_ptr[i]:lp.row_ptr[i + 1]]]
                   for i in range(lp.m)])
    slack = np.concatenate([np.zeros(lp.n_eq), kx[lp.n_eq:] - lp.q[lp.n_eq:]])
    assert slack.min() >= -1e-9
    bx = np.sqrt(np.sum(lp.x_star ** 2) + np.sum(slack ** 2))
    by = np.sqrt(np.sum(lp.y_star ** 2) + np.sum(lp.lam_star ** 2))
    tight_d = tight_p = 0.0
    for _ in range(200):
        yr = rng.standard_normal(lp.m) * rng.uniform(0.1, 10)
        xr = rng.standard_normal(lp.n) * rng.uniform(0.1, 10)
        t = oracle.infeas_terms(lp, xr, yr)
        assert t[0] <= t[1] * bx * (1 + 1e-12) + 1e-9
        assert t[2] <= t[3] * by * (1 + 1e-12) + 1e-9
        if t[1] > 0:
            tight_d = max(tight_d, t[0] / (t[1] * bx))
        if t[3] > 0:
            tight_p = max(tight_p, t[2] / (t[3] * by))
    # the bounds are not vacuous: some random rays come within a factor of 50
    assert tight_d > 0.02 and tight_p > 0.02


def test_planted_pair_differences_certify_nothing():
    lp = lpgen.tiny_lp(7)
    for xr, yr in ((lp.x_star, lp.y_star), (lp.x_star - 1.0, lp.y_star + 1.0)):
        t = oracle.infeas_terms(lp, xr, yr)
        assert oracle.infeas_status(t, 1e-8) == -1


# ---------------------------------------------------------------- generator certificates


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_generator_rays_are_exact_certificates(seed):
    for kind in ("primal", "primal_bounds"):
        lp = lpgen.infeasible_lp(seed, kind)
        t = oracle.infeas_terms(lp, np.zeros(lp.n), lp.meta["ray_y"])
        assert t[1] == 0.0 and t[0] > 0.5
        assert oracle.infeas_status(t, 0.0) == oracle.PRIMAL_INFEASIBLE
        if kind == "primal":  # y = 1 on the two added rows: objective h1 - h2
            assert t[0] == pytest.approx(lp.q[-2] + lp.q[-1], rel=1e-15)
        else:  # the row's bound is above max over the box of a'x
            s, e = lp.row_ptr[-2], lp.row_ptr[-1]
            a, cols = lp.val[s:e], lp.col_idx[s:e]
            top = np.sum(np.maximum(a * lp.l[cols], a * lp.u[cols]))
            assert t[0] == pytest.approx(lp.q[-1] - top, rel=1e-12)
    lp = lpgen.infeasible_lp(seed, "dual")
    t = oracle.infeas_terms(lp, lp.meta["ray_x"], np.zeros(lp.m))
    assert t[2] == 0.5 and t[3] == 0.0
    assert oracle.infeas_status(t, 0.0) == oracle.DUAL_INFEASIBLE


@pytest.mark.parametrize("kind,seed", [("primal", 0), ("primal_bounds", 1), ("dual", 2)])
def test_highs_agrees_the_generated_lps_are_infeasible(kind, seed):
    linprog = pytest.importorskip("scipy.optimize").linprog
    sp = pytest.importorskip("scipy.sparse")
    lp = lpgen.infeasible_lp(seed, kind)
    K = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    r = linprog(lp.c, A_ub=-K[lp.n_eq:], b_ub=-lp.q[lp.n_eq:], A_eq=K[:lp.n_eq], b_eq=lp.q[:lp.n_eq],
                bounds=list(zip(lp.l, [None if np.isinf(v) else v for v in lp.u])), method="highs")
    assert r.status == (2 if kind != "dual" else 3)


# ---------------------------------------------------------------- solve


@pytest.mark.parametrize("kind", ["primal", "primal_bounds", "dual"])
@pytest.mark.parametrize("seed", [0, 1])
def test_solve_detects_and_returns_a_certificate(kind, seed):
    lp = lpgen.infeasible_lp(seed, kind)
    r = oracle.solve(lp, tol=1e-8, max_iter=200000, eps_infeas=1e-8)
    want = oracle.DUAL_INFEASIBLE if kind == "dual" else oracle.PRIMAL_INFEASIBLE
    assert r.status == want and r.which in (2, 3)
    if want == oracle.PRIMAL_INFEASIBLE:
        t = oracle.infeas_terms(lp, np.zeros(lp.n), r.y)
        assert np.all(r.x >= lp.l) and np.all(r.x <= lp.u)
    else:
        t = oracle.infeas_terms(lp, r.x, np.zeros(lp.m))
    assert oracle.infeas_status(t, 1e-8) == want
    assert (r.ray_obj, r.ray_res) == pytest.approx(tuple(t[:2] if want == oracle.PRIMAL_INFEASIBLE else t[2:]),
                                                   rel=1e-12, abs=1e-300)
    off = oracle.solve(lp, tol=1e-8, max_iter=r.iters + 256, eps_infeas=0.0)
    assert off.status == oracle.ITER_LIMIT


def test_detection_leaves_feasible_solves_unchanged():
    for seed in range(3):
        lp = lpgen.tiny_lp(seed)
        on = oracle.solve(lp, tol=1e-8, max_iter=200000, eps_infeas=1e-8)
        off = oracle.solve(lp, tol=1e-8, max_iter=200000, eps_infeas=0.0)
        assert on.status == off.status == oracle.OPTIMAL
        assert on.iters == off.iters and np.array_equal(on.x, off.x) and np.array_equal(on.y, off.y)


def _np_dual_ray_measures(lp, yr):
    """Primal-infeasibility certificate measures of a dual ray yr, written
    out in numpy: lambda = proj_Lambda(-K'yr) on the bounds' cone,
    objective q'yr + l'lambda+ - u'lambda-, residual
    ||(-K'yr - lambda, min(yr_G, 0))||."""
    K = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n)).toarray()
    g = -K.T @ yr
    lf, uf = np.isfinite(lp.l), np.isfinite(lp.u)
    lam = np.where(lf & uf, g, np.where(lf, np.maximum(g, 0), np.where(uf, np.minimum(g, 0), 0.0)))
    obj = lp.q @ yr + np.sum(np.where(lf, lp.l, 0.0) * np.maximum(lam, 0)) \
        - np.sum(np.where(uf, lp.u, 0.0) * np.maximum(-lam, 0))
    res = np.sqrt(np.sum((g - lam) ** 2) + np.sum(np.minimum(yr[lp.n_eq:], 0) ** 2))
    return obj, res


def _np_primal_ray_measures(lp, xr):
    """Dual-infeasibility certificate measures of a primal ray xr: objective
    -c'xr, residual ||(K_E xr, min(K_G xr, 0), xr's distance to the
    recession cone of the bounds)||."""
    K = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n)).toarray()
    kx = K @ xr
    lf, uf = np.isfinite(lp.l), np.isfinite(lp.u)
    cone = np.where(lf & uf, 0.0, np.where(lf, np.maximum(xr, 0), np.where(uf, np.minimum(xr, 0), xr)))
    res = np.sqrt(np.sum(kx[:lp.n_eq] ** 2) + np.sum(np.minimum(kx[lp.n_eq:], 0) ** 2) + np.sum((xr - cone) ** 2))
    return -lp.c @ xr, res


@pytest.mark.parametrize("kind,seed", [("primal", 0), ("primal_bounds", 1), ("dual", 0)])
def test_detection_fires_at_the_first_check_whose_difference_ray_certifies(kind, seed):
    """Without scaling the difference ray is the difference of the iterates
    that solves stopped at k and k - 1 return.  At the check where the
    solve declares infeasibility that ray, as the test computes it, is the
    returned ray and passes the certificate test written out in numpy; one
    check earlier it does not, and a solve stopped there has not fired."""
    eps = 1e-8
    lp = lpgen.infeasible_lp(seed, kind)
    kw = dict(tol=1e-8, ruiz_iters=0, pc_alpha=-1.0, check_period=64)
    r = oracle.solve(lp, max_iter=200000, eps_infeas=eps, **kw)
    primal = kind != "dual"
    assert r.status == (oracle.PRIMAL_INFEASIBLE if primal else oracle.DUAL_INFEASIBLE) and r.which == 2

    def ray(k):
        a = oracle.solve(lp, max_iter=k, eps_infeas=0.0, **kw)
        b = oracle.solve(lp, max_iter=k - 1, eps_infeas=0.0, **kw)
        assert a.iters == k and b.iters == k - 1
        return a.x - b.x, a.y - b.y

    def certifies(xr, yr):
        obj, res = _np_dual_ray_measures(lp, yr) if primal else _np_primal_ray_measures(lp, xr)
        return obj > 0 and res <= eps * obj

    xr, yr = ray(r.iters)
    np.testing.assert_allclose(r.y if primal else r.x, yr if primal else xr, rtol=1e-12, atol=1e-300)
    assert certifies(xr, yr)
    assert not certifies(*ray(r.iters - 64))
    earlier = oracle.solve(lp, max_iter=r.iters - 64, eps_infeas=eps, **kw)
    assert earlier.status == oracle.ITER_LIMIT
