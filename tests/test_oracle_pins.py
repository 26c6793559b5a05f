"""Pins for the FP64 CPU oracle (no GPU): every check here compares the oracle
with something other than itself -- hand-worked examples, closed forms,
brute-force vertex enumeration, an independent LP solver (HiGHS via scipy),
planted optima built by the generator, and invariants of the method."""

import math

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle
from brute import dense, vertex_enum
from conftest import DictLP


# ---------------------------------------------------------------- hand examples


def test_pdhg_step_hand(golden):
    g = golden["pdhg_step"]
    lp = DictLP(g["lp"])
    xn, yn = oracle.pdhg_step(lp, np.array(g["x"]), np.array(g["y"]), g["tau"], g["sigma"])
    np.testing.assert_allclose(xn, g["x_next"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(yn, g["y_next"], rtol=0, atol=1e-13)


def test_kkt_hand(golden):
    g = golden["kkt"]
    lp = DictLP(g["lp"])
    t = oracle.kkt_terms(lp, np.array(g["x"]), np.array(g["y"]))
    assert t["pobj"] == pytest.approx(g["pobj"], abs=1e-14)
    assert t["dobj"] == pytest.approx(g["dobj"], abs=1e-14)
    assert t["rp"] == pytest.approx(g["rp_norm"], abs=1e-14)
    assert t["rd"] == pytest.approx(g["rd_norm"], abs=1e-14)
    assert t["q_norm"] ** 2 == pytest.approx(g["q_norm_sq"], rel=1e-14)
    assert t["c_norm"] ** 2 == pytest.approx(g["c_norm_sq"], rel=1e-14)
    k = oracle.kkt_omega(lp, np.array(g["x"]), np.array(g["y"]), g["omega"])
    assert k * k == pytest.approx(g["kkt_omega_sq"], rel=1e-14)


def test_alg2_scalars(golden):
    g = golden["alg2_scalars"]
    for c in g["cases"]:
        want = math.inf if c["eta_bar"] == "inf" else c["eta_bar"]
        assert oracle.eta_bar(c["dx2"], c["dy2"], c["cross"], c["omega"]) == want
    for c in g["eta_next"]:
        assert oracle.eta_next(c["eta"], c["eta_bar"], c["k"]) == pytest.approx(c["expect"], rel=1e-15)
    # eta_bar = inf -> the growth branch: (1 + (k+2)^-0.6) eta
    assert oracle.eta_next(2.0, math.inf, 0) == pytest.approx(2.0 * (1 + 2 ** -0.6), rel=1e-15)


def test_primal_weight(golden):
    g = golden["primal_weight"]
    for c in g["init"]:
        assert oracle.primal_weight_init(c["c_norm"], c["q_norm"]) == pytest.approx(c["expect"], rel=1e-15)
    for c in g["update"]:
        got = oracle.primal_weight_update(c["dx"], c["dy"], c["omega"], c["theta"])
        assert got == pytest.approx(c["expect"], rel=1e-14)
    # theta = 1 keeps only the new ratio, theta = 0 keeps the old weight
    assert oracle.primal_weight_update(2.0, 6.0, 5.0, 1.0) == pytest.approx(3.0, rel=1e-14)
    assert oracle.primal_weight_update(2.0, 6.0, 5.0, 0.0) == pytest.approx(5.0, rel=1e-14)


def test_restart_mask_truth_table():
    # Sec. 3.4: (i) cand <= 0.2 start; (ii) cand <= 0.8 start and cand > prev; (iii) t >= 0.36 k
    assert oracle.restart_mask(0.19, 1.0, 0.3, 1, 100) == 1
    assert oracle.restart_mask(0.2, 1.0, 0.3, 1, 100) == 1  # boundary: <= ; not > prev
    assert oracle.restart_mask(0.5, 1.0, 0.4, 1, 100) == 2  # necessary decay + no local progress
    assert oracle.restart_mask(0.5, 1.0, 0.6, 1, 100) == 0  # still progressing
    assert oracle.restart_mask(0.81, 1.0, 0.1, 1, 100) == 0  # not enough decay
    assert oracle.restart_mask(0.9, 1.0, 0.1, 36, 100) == 4  # long inner loop, boundary t = 0.36 k
    assert oracle.restart_mask(0.9, 1.0, 0.1, 35, 100) == 0
    assert oracle.restart_mask(0.1, 1.0, 0.05, 50, 100) == 1 | 2 | 4


# ---------------------------------------------------------------- closed forms


def _lp_from_dense(K, c, q, l, u, n_eq):
    S = sp.csr_matrix(np.asarray(K, dtype=float).reshape(len(q), len(c)))
    return lpgen.LP(m=len(q), n=len(c), n_eq=n_eq, c=np.asarray(c, float), row_ptr=S.indptr.astype(np.int32),
                    col_idx=S.indices.astype(np.int32), val=S.data.astype(float), q=np.asarray(q, float),
                    l=np.asarray(l, float), u=np.asarray(u, float))


def test_closed_form_no_constraints():
    # m = 0: x_j = l_j if c_j > 0, u_j if c_j < 0
    rng = np.random.default_rng(3)
    n = 40
    c = rng.standard_normal(n)
    l = rng.uniform(-3, 0, n)
    u = rng.uniform(0, 3, n)
    lp = lpgen.LP(m=0, n=n, n_eq=0, c=c, row_ptr=np.zeros(1, np.int32), col_idx=np.zeros(0, np.int32),
                  val=np.zeros(0), q=np.zeros(0), l=l, u=u)
    r = oracle.solve(lp, tol=1e-10, max_iter=20000)
    assert r.status == oracle.OPTIMAL
    x_exp = np.where(c > 0, l, u)
    np.testing.assert_allclose(r.x, x_exp, atol=1e-9)
    assert r.pobj == pytest.approx(float(c @ x_exp), rel=1e-10)


def test_closed_form_fractional_knapsack():
    # max v'x s.t. w'x <= W, 0 <= x <= 1  ==  min -v'x s.t. -w'x >= -W
    rng = np.random.default_rng(5)
    n = 12
    v = rng.uniform(1, 5, n)
    w = rng.uniform(1, 3, n)
    W = 0.4 * w.sum()
    order = np.argsort(-v / w)
    x = np.zeros(n)
    cap = W
    for j in order:
        take = min(1.0, cap / w[j])
        x[j] = take
        cap -= take * w[j]
        if cap <= 0:
            break
    opt = -float(v @ x)
    lp = _lp_from_dense([-w], -v, [-W], np.zeros(n), np.ones(n), n_eq=0)
    r = oracle.solve(lp, tol=1e-10, max_iter=200000)
    assert r.status == oracle.OPTIMAL
    assert r.pobj == pytest.approx(opt, rel=1e-8)


# ---------------------------------------------------------------- brute force


@pytest.mark.parametrize("seed", range(12))
def test_vertex_enumeration(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 6))
    m_eq = int(rng.integers(0, 3))
    m_in = int(rng.integers(0, 3))
    lp = lpgen.random_boxed_lp(seed, m_eq, m_in, n, density=0.7, planted=bool(seed % 2))
    best, _ = vertex_enum(lp)
    assert np.isfinite(best)
    r = oracle.solve(lp, tol=1e-10, max_iter=500000)
    assert r.status == oracle.OPTIMAL
    assert r.pobj == pytest.approx(best, abs=1e-7 * (1 + abs(best)))
    if lp.obj_star is not None:
        assert best == pytest.approx(lp.obj_star, abs=1e-9 * (1 + abs(best)))


# ---------------------------------------------------------------- planted optima


def test_planted_pair_has_zero_kkt():
    for lp in (lpgen.tiny_lp(0), lpgen.large_lp(1, m=3000, n=6000, nnz=60000)):
        t = oracle.kkt_terms(lp, lp.x_star, lp.y_star)
        scale = 1 + abs(t["pobj"])
        assert abs(t["dobj"] - t["pobj"]) <= 1e-12 * scale
        assert t["rp"] <= 1e-11 * (1 + t["q_norm"])
        assert t["rd"] <= 1e-11 * (1 + t["c_norm"])
        assert t["pobj"] == pytest.approx(lp.obj_star, rel=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_planted_tiny_objective(seed):
    lp = lpgen.tiny_lp(seed)
    r = oracle.solve(lp, tol=1e-8)
    assert r.status == oracle.OPTIMAL
    assert abs(r.pobj - lp.obj_star) <= 1e-6 * abs(lp.obj_star)
    assert oracle.passes(lp, r.x, r.y, 1e-8)
    assert np.all(r.x >= lp.l) and np.all(r.x <= lp.u)
    assert np.all(r.y[lp.n_eq:] >= 0)


def test_warm_start_at_optimum_is_a_fixed_point():
    lp = lpgen.tiny_lp(4)
    r = oracle.solve(lp, tol=1e-12, x0=lp.x_star, y0=lp.y_star, check_period=8)
    assert r.status == oracle.OPTIMAL and r.iters == 8
    assert oracle.relative_kkt(lp, r.x, r.y) < 1e-12


# ---------------------------------------------------------------- independent solver


def _highs(lp):
    from scipy.optimize import linprog

    K = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    A_eq = K[: lp.n_eq] if lp.n_eq else None
    b_eq = lp.q[: lp.n_eq] if lp.n_eq else None
    A_ub = -K[lp.n_eq:] if lp.m > lp.n_eq else None
    b_ub = -lp.q[lp.n_eq:] if lp.m > lp.n_eq else None
    bounds = [(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b) for a, b in zip(lp.l, lp.u)]
    res = linprog(lp.c, A_ub=A_ub, b_ub=b_ub, A_eq=A_eq, b_eq=b_eq, bounds=bounds, method="highs")
    assert res.status == 0
    return res.fun


@pytest.mark.parametrize("case", ["tiny-mixed", "all-eq", "all-ineq", "power-law", "transport"])
def test_against_highs(case):
    if case == "transport":  # a 20 x 30 member of the warm-start family (incidence K, free-cost noise)
        fam = lpgen.transport_family(0, sources=20, sinks=30)
        lp = lpgen.transport_lp(fam, lpgen.transport_thetas(1, 0)[0], 0)
    elif case == "tiny-mixed":
        lp = lpgen.tiny_lp(7)
    elif case == "all-eq":
        lp = lpgen.tiny_lp(8, m_eq=120, m_ineq=0, n=300)
    elif case == "all-ineq":
        lp = lpgen.tiny_lp(9, m_eq=0, m_ineq=150, n=300)
    else:
        lp = lpgen.large_lp(2, m=600, n=1200, nnz=12000)
    ref = _highs(lp)
    r = oracle.solve(lp, tol=1e-8, max_iter=400000)
    assert r.status == oracle.OPTIMAL
    assert abs(r.pobj - ref) <= 1e-6 * (1 + abs(ref))


# ---------------------------------------------------------------- preconditioning


def test_ruiz_equilibrates_and_scaling_identity():
    lp = lpgen.large_lp(3, m=2000, n=4000, nnz=40000)
    K = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    sv, D1, D2 = oracle.precondition(lp, ruiz_iters=10, pc_alpha=-1.0)
    Kt = sp.csr_matrix((sv, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    # identity K~ = D1 K D2 (Sec. 2.2)
    ref = (sp.diags(D1) @ K @ sp.diags(D2)).tocsr()
    ref.sort_indices()
    np.testing.assert_allclose(sv, ref.data, rtol=1e-13)
    assert np.all(D1 > 0) and np.all(D2 > 0)

    # l_inf equilibration (Ruiz): every nonempty row / column max tends to 1,
    # the deviation shrinking geometrically with the number of passes
    def dev(passes):
        v, _, _ = oracle.precondition(lp, ruiz_iters=passes, pc_alpha=-1.0)
        A = abs(sp.csr_matrix((v, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n)))
        r = A.max(axis=1).toarray().ravel()
        c = A.max(axis=0).toarray().ravel()
        return max(np.abs(r[r > 0] - 1).max(), np.abs(c[c > 0] - 1).max())

    d = [dev(p) for p in (5, 10, 20, 40)]
    assert d[1] < 5e-2 and d[2] < 1e-4 and d[3] < 1e-9
    assert d[0] > d[1] > d[2] > d[3]


def test_pock_chambolle_single_pass_closed_form():
    lp = lpgen.tiny_lp(2)
    K = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    sv, D1, D2 = oracle.precondition(lp, ruiz_iters=0, pc_alpha=1.0)
    rs = np.asarray(abs(K).sum(axis=1)).ravel()
    cs = np.asarray(abs(K).sum(axis=0)).ravel()
    np.testing.assert_allclose(D1, 1 / np.sqrt(np.where(rs > 0, rs, 1)), rtol=1e-14)
    np.testing.assert_allclose(D2, 1 / np.sqrt(np.where(cs > 0, cs, 1)), rtol=1e-14)


def test_scaling_does_not_change_solution():
    lp = lpgen.tiny_lp(11)
    a = oracle.solve(lp, tol=1e-8)
    b = oracle.solve(lp, tol=1e-8, ruiz_iters=0, pc_alpha=-1.0, max_iter=400000)
    assert a.status == b.status == oracle.OPTIMAL
    assert a.pobj == pytest.approx(b.pobj, rel=1e-6)


# ---------------------------------------------------------------- Algorithm 3 (App. A)


def test_alg3_restart_decay_and_bounded_length():
    rng = np.random.default_rng(1)
    m, n = 6, 14
    A = rng.standard_normal((m, n))
    xs = np.abs(rng.standard_normal(n))
    xs[:6] = 0
    ys = rng.standard_normal(m)
    lam = np.zeros(n)
    lam[:6] = rng.uniform(0.1, 1, 6)
    c = A.T @ ys + lam
    b = A @ xs
    S = sp.csr_matrix(A)
    s = 1 / (2 * np.linalg.norm(A, 2))  # Theorem: s <= 1 / (2 ||A||_2)
    beta = 0.5
    x, y, kr, lr = oracle.alg3(S.indptr, S.indices, S.data, b, c, m, n, s, beta, 200000)
    assert len(lr) >= 20
    # restart rule: KKT(z^{n+1,0}) <= beta KKT(z^{n,0}), so KKT(z^{n,0}) <= beta^n KKT(z^{0,0})
    assert np.all(kr[1:] <= beta * kr[:-1] * (1 + 1e-12))
    assert np.all(kr <= beta ** np.arange(len(kr)) * kr[0] * (1 + 1e-9))
    # Theorem (ii): restart lengths stay bounded (no growth) while the KKT
    # error is above the rounding floor of FP64
    above = kr[: len(lr)] > 1e-10 * kr[0]
    assert above.sum() >= 20
    assert lr[above].max() <= 4 * np.median(lr[above])
    # the KKT error of Appendix A vanishes at the limit: optimal objective
    assert float(c @ x) == pytest.approx(float(c @ xs), abs=1e-9)
    # the Appendix A KKT function is zero at the planted optimum
    assert oracle.kkt_standard(S.indptr, S.indices, S.data, b, c, xs, ys, m, n) < 1e-12


def test_kkt_standard_hand(golden):
    """Appendix A's KKT error at two non-optimal points worked by hand: every
    term (primal residual, [-x]^+, [A'y - c]^+, [c'x - b'y]^+) is nonzero at
    the first, and the gap is negative at the second (its positive part is 0)."""
    g = golden["kkt_standard"]
    S = sp.csr_matrix(np.array(g["A"]))
    m, n = S.shape
    b, c = np.array(g["b"]), np.array(g["c"])
    for p in g["points"]:
        k = oracle.kkt_standard(S.indptr, S.indices, S.data, b, c, np.array(p["x"]), np.array(p["y"]), m, n)
        assert k * k == pytest.approx(p["kkt_sq"], rel=1e-14)


# ---------------------------------------------------------------- driver behaviour


def test_iteration_limit_and_trace():
    lp = lpgen.tiny_lp(1)
    r = oracle.solve(lp, tol=1e-12, max_iter=200, check_period=16)
    assert r.status == oracle.ITER_LIMIT and r.iters == 200
    ks = r.trace["k"]
    assert np.all(ks % 16 == 0) and np.all(np.diff(ks) == 16)
    assert np.all(r.trace["eta_hat"] > 0) and np.all(r.trace["omega"] > 0)
    # the first check of the run is in epoch 0 where t == k: criterion (iii) fires
    assert r.trace["restart"][0] & 4


def test_trace_metrics_match_a_solve_stopped_at_the_check():
    """Each check record's Sec. 4.1 measures are those of the current iterate
    on the original LP: a solve stopped by the iteration limit at that k
    returns that iterate, whose measures kkt_terms evaluates independently;
    its trial count is the record's, and the restart count is the running
    number of restart masks."""
    lp = lpgen.tiny_lp(1)
    r = oracle.solve(lp, tol=1e-12, max_iter=640, check_period=64)
    tr = r.trace
    assert len(tr) == 9
    assert np.array_equal(tr["restarts"], np.cumsum(tr["restart"] != 0))
    assert np.all(np.diff(tr["attempts"]) >= 64) and np.all(tr["attempts"] >= tr["k"])
    for rec in tr[[0, 3, 8]]:
        k = int(rec["k"])
        s = oracle.solve(lp, tol=1e-12, max_iter=k, check_period=64)
        assert s.status == oracle.ITER_LIMIT and s.iters == k and s.attempts == rec["attempts"]
        t = oracle.kkt_terms(lp, s.x, s.y)
        gap = abs(t["pobj"] - t["dobj"]) / (1.0 + abs(t["pobj"]) + abs(t["dobj"]))
        want = [gap, t["rp"] / (1.0 + t["q_norm"]), t["rd"] / (1.0 + t["c_norm"])]
        got = [rec["rel_gap"], rec["rel_primal"], rec["rel_dual"]]
        np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-15)
        assert max(got) > 1e-12  # the check did not end the solve


def test_invalid_inputs_rejected():
    lp = lpgen.tiny_lp(0)
    bad = lpgen.tiny_lp(0)
    bad.col_idx = bad.col_idx.copy()
    bad.col_idx[3] = lp.n  # out of range
    with pytest.raises(ValueError):
        oracle.solve(bad)
    bad = lpgen.tiny_lp(0)
    bad.l = bad.l.copy()
    bad.l[0] = 20.0  # l > u
    with pytest.raises(ValueError):
        oracle.solve(bad)
    bad = lpgen.tiny_lp(0)
    bad.c = bad.c.copy()
    bad.c[0] = np.nan
    with pytest.raises(ValueError):
        oracle.solve(bad)


def test_dense_helper_matches_csr():
    lp = lpgen.tiny_lp(0)
    K = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n)).toarray()
    np.testing.assert_array_equal(dense(lp), K)


def test_first_solve_step_is_eq_pdhg(golden):
    """The solver's inner step itself (not the separate helper): without
    scaling, one accepted step from (x0, y0) is eq. (pdhg) with
    tau = eta/omega, sigma = eta*omega, eta = 1/max|K_ij| (Alg. 1 init) and
    omega = ||c|| / ||q|| (InitializePrimalWeight), computed here in numpy."""
    g = golden["pdhg_step"]
    lp = DictLP(g["lp"])
    x0, y0 = np.array(g["x"]), np.array(g["y"])
    r = oracle.solve(lp, tol=0.0, max_iter=1, check_period=1, ruiz_iters=0, pc_alpha=-1.0, x0=x0, y0=y0)
    assert r.status == oracle.ITER_LIMIT and r.iters == 1 and r.attempts == 1
    K = dense(lp)
    eta = 1.0 / np.abs(lp.val).max()
    omega = np.linalg.norm(lp.c) / np.linalg.norm(lp.q)
    tau, sigma = eta / omega, eta * omega
    x1 = np.clip(x0 - tau * (lp.c - K.T @ y0), lp.l, lp.u)
    y1 = y0 + sigma * (lp.q - K @ (2 * x1 - x0))
    y1[lp.n_eq:] = np.maximum(y1[lp.n_eq:], 0)
    np.testing.assert_allclose(r.x, x1, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(r.y, y1, rtol=1e-14, atol=1e-15)


def test_iteration_limit_below_one_is_rejected():
    # the iteration limit counts accepted steps and must allow at least one
    with pytest.raises(ValueError):
        oracle.solve(lpgen.tiny_lp(0), tol=1e-6, max_iter=0)


def test_oracle_stalls_on_batch_lp_2581_by_primal_weight_runaway():
    """Member 2581 of the 4096-LP batch workload (147 x 120, planted, so
    feasible and bounded) ends at the iteration limit in the batched GPU
    solver; the oracle does the same.  After k ~ 1.5e3 every restart raises
    the primal weight (Sec. 2.2 PrimalWeightUpdate: the dual iterate moves
    far more than the primal one between restart points), omega passes 1e5,
    the primal step eta / omega all but vanishes, and from k ~ 1.6e4 only
    the artificial criterion (iii) restarts: a limit of the method as read
    (unbounded omega), not of the GPU path."""
    lp = lpgen.batch_lp(2581)
    assert (lp.m, lp.n, lp.nnz) == (147, 120, 399)
    r = oracle.solve(lp, tol=1e-6, max_iter=1_000_000, check_period=64)
    assert r.status == oracle.ITER_LIMIT and r.iters == 1_000_000
    restarts = r.trace[r.trace["restart"] != 0]
    assert restarts["omega"][-1] > 1e5
    late = restarts[restarts["k"] > 20000]
    assert len(late) >= 3 and np.all(late["restart"] == 4)  # only criterion (iii)
    assert np.all(np.diff(late["omega"]) > 0)
    # still near the optimum: the objective is off by a few 1e-6 relative
    assert abs(float(lp.c @ r.x) - lp.obj_star) < 1e-5 * abs(lp.obj_star)


def test_fp32_step_mode_first_step_uses_float_values(golden):
    """FP32-values mode of the steps: from a warm start, one accepted step is
    eq. (pdhg) with the dual step's product taken with K rounded to FP32 (the
    primal step's K'y0 is the start point's product, taken in FP64 like every
    check), eta = 1/max|K| from the FP64 values; and the rounding matters."""
    g = golden["pdhg_step"]
    lp = DictLP(g["lp"])
    lp.val = lp.val / 3.0  # not representable in FP32
    x0, y0 = np.array(g["x"]), np.array(g["y"])
    r = oracle.solve(lp, tol=0.0, max_iter=1, check_period=1, ruiz_iters=0, pc_alpha=-1.0, x0=x0, y0=y0,
                     step_value_bits=32)
    assert r.status == oracle.ITER_LIMIT and r.iters == 1 and r.attempts == 1
    K = dense(lp)
    K32 = K.astype(np.float32).astype(np.float64)
    eta = 1.0 / np.abs(lp.val).max()
    omega = np.linalg.norm(lp.c) / np.linalg.norm(lp.q)
    tau, sigma = eta / omega, eta * omega
    x1 = np.clip(x0 - tau * (lp.c - K.T @ y0), lp.l, lp.u)

    def dual(Km):
        y1 = y0 + sigma * (lp.q - Km @ (2 * x1 - x0))
        y1[lp.n_eq:] = np.maximum(y1[lp.n_eq:], 0)
        return y1

    np.testing.assert_allclose(r.x, x1, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(r.y, dual(K32), rtol=1e-14, atol=1e-15)
    assert np.abs(dual(K32) - dual(K)).max() > 1e-12 * np.abs(dual(K)).max()


def test_fp32_step_mode_equals_fp64_on_float_exact_values():
    """Without scaling and with every value exactly representable in FP32,
    the FP32-values mode of the steps is the FP64 method, bit for bit, over
    several restart periods."""
    lp = lpgen.tiny_lp(3)
    lp.val = np.round(lp.val * 8.0) / 8.0
    lp.val[lp.val == 0] = 0.125
    kw = dict(tol=0.0, max_iter=400, check_period=16, ruiz_iters=0, pc_alpha=-1.0)
    a = oracle.solve(lp, step_value_bits=64, **kw)
    b = oracle.solve(lp, step_value_bits=32, **kw)
    assert a.iters == b.iters == 400 and a.attempts == b.attempts and a.restarts == b.restarts > 0
    assert np.array_equal(a.x, b.x) and np.array_equal(a.y, b.y)
    assert a.trace.tobytes() == b.trace.tobytes()


def test_fp32_step_mode_rejects_other_widths():
    with pytest.raises(ValueError):
        oracle.solve(lpgen.tiny_lp(0), tol=1e-6, max_iter=10, step_value_bits=16)


def test_accepted_steps_satisfy_the_step_size_condition():
    """Algorithm 2's acceptance on a real trajectory: every step accepted at
    its first trial, from an iterate no restart moved, satisfies eq.
    (step-size), eta <= (omega ||dx||^2 + ||dy||^2 / omega) / (2 |dy' K dx|),
    with dx, dy the differences of the iterates the solve returns when it is
    stopped before and after the step (no scaling, so these are the LP's own
    iterates) and eta, omega from the check records in between."""
    lp = lpgen.tiny_lp(2)
    kw = dict(tol=0.0, check_period=1, ruiz_iters=0, pc_alpha=-1.0)
    N = 40
    runs = [oracle.solve(lp, max_iter=k, **kw) for k in range(1, N + 1)]
    tr = runs[-1].trace  # record i: the check after step i + 1
    assert np.array_equal(tr["k"], np.arange(1, N))
    K = dense(lp)
    checked = 0
    for k in range(1, N - 1):  # the step from k to k + 1 accepted steps
        before, after = tr[k - 1], tr[k]
        if after["attempts"] - before["attempts"] != 1 or before["restart"] != 0:
            continue
        dx = runs[k].x - runs[k - 1].x
        dy = runs[k].y - runs[k - 1].y
        eta, omega = before["eta_hat"], before["omega"]
        inter = abs(dy @ (K @ dx))
        eta_bar = (omega * (dx @ dx) + (dy @ dy) / omega) / (2.0 * inter) if inter > 0 else np.inf
        assert eta <= eta_bar * (1 + 1e-12), (k, eta, eta_bar)
        checked += 1
    assert checked >= 10


def test_restart_decisions_follow_the_recorded_kkt_values():
    """Sec. 3.4's bookkeeping on a real trajectory: at every check the
    recorded restart mask is the three criteria evaluated on the recorded
    values -- the candidate (the average unless the current KKT is strictly
    smaller), the epoch start's KKT as left by the previous check (recomputed
    with the new primal weight after a restart), the previous candidate's KKT
    (the restart point's right after a restart) and t = k minus the last
    restart's k (beta = 0.2, 0.8, 0.36)."""
    lp = lpgen.tiny_lp(1)
    r = oracle.solve(lp, tol=0.0, max_iter=64 * 60, check_period=64)
    tr = r.trace
    assert len(tr) == 59 and (tr["restart"] != 0).sum() >= 3
    last_restart = tr["k"][0] if tr["restart"][0] else 0
    bits = set()
    for i in range(1, len(tr)):
        prev, cur = tr[i - 1], tr[i]
        start = prev["kkt_start"]
        kprev = start if prev["restart"] else (prev["kkt_avg"] if prev["cand_avg"] else prev["kkt_cur"])
        cand_avg = not (cur["kkt_cur"] < cur["kkt_avg"])
        assert cur["cand_avg"] == cand_avg
        cand = cur["kkt_avg"] if cand_avg else cur["kkt_cur"]
        t = cur["k"] - last_restart
        mask = (cand <= 0.2 * start) | ((cand <= 0.8 * start and cand > kprev) << 1) | ((t >= 0.36 * cur["k"]) << 2)
        assert cur["restart"] == mask, (i, cur["restart"], mask)
        if mask:
            last_restart = cur["k"]
            bits |= {b for b in (1, 2, 4) if mask & b}
    assert len(bits) >= 2  # more than one criterion fired along the way


def test_primal_weight_updates_follow_the_restart_points():
    """PrimalWeightUpdate (Sec. 2.2, read in log space) on a real trajectory:
    between two restarts to the current iterate, omega moves to
    exp(theta log(||dy|| / ||dx||) + (1 - theta) log(omega)) with dx, dy the
    differences of the two restart points, which the test takes from solves
    stopped at those checks (no scaling, so these are the LP's own iterates);
    where either distance is below eps_zero omega stays."""
    lp = lpgen.large_lp(0, m=300, n=600, nnz=3000)
    kw = dict(tol=0.0, check_period=64, ruiz_iters=0, pc_alpha=-1.0)
    tr = oracle.solve(lp, max_iter=64 * 60, **kw).trace
    ks = {int(r["k"]): r for r in tr}
    restarts = [int(r["k"]) for r in tr if r["restart"]]
    pairs = [(a, b) for a, b in zip(restarts, restarts[1:]) if not ks[a]["cand_avg"] and not ks[b]["cand_avg"]]
    moved = 0
    for a, b in pairs:
        za, zb = oracle.solve(lp, max_iter=a, **kw), oracle.solve(lp, max_iter=b, **kw)
        dx, dy = np.linalg.norm(zb.x - za.x), np.linalg.norm(zb.y - za.y)
        before = ks[b - 64]["omega"]  # unchanged since the restart at a
        assert before == ks[a]["omega"]
        if dx > 1e-10 and dy > 1e-10:
            want = np.exp(0.5 * np.log(dy / dx) + 0.5 * np.log(before))
            assert ks[b]["omega"] == pytest.approx(want, rel=1e-12)
            assert abs(ks[b]["omega"] - before) > 1e-6 * before  # the update moved omega
            moved += 1
        else:
            assert ks[b]["omega"] == before
    assert moved >= 2


def test_average_iterate_is_weighted_by_the_accepted_steps():
    """Algorithm 1's average on a real trajectory: the KKT of the average
    recorded at the first check equals, to rounding, eq. (kkt) at the average
    of the first 64 iterates (taken from solves stopped after each step)
    weighted by their accepted step sizes (eta_1 = 1 / max|K|, then each
    solve's next trial step, every trial accepted here); the plain mean of the
    same iterates scores measurably differently."""
    lp = lpgen.tiny_lp(2)
    kw = dict(tol=0.0, check_period=64, ruiz_iters=0, pc_alpha=-1.0)
    runs = [oracle.solve(lp, max_iter=k, **kw) for k in range(1, 65)]
    assert runs[-1].attempts == 64  # no rejected trial: accepted eta = the trial eta
    rec = oracle.solve(lp, max_iter=128, **kw).trace[0]
    assert rec["k"] == 64
    eta = np.array([1.0 / np.abs(lp.val).max()] + [r.eta_hat for r in runs[:-1]])
    X, Y = np.array([r.x for r in runs]), np.array([r.y for r in runs])
    omega = np.linalg.norm(lp.c) / np.linalg.norm(lp.q)
    xb, yb = eta @ X / eta.sum(), eta @ Y / eta.sum()
    assert oracle.kkt_omega(lp, xb, yb, omega) == pytest.approx(rec["kkt_avg"], rel=1e-12)
    assert oracle.kkt_omega(lp, X[-1], Y[-1], omega) == pytest.approx(rec["kkt_cur"], rel=1e-12)
    plain = oracle.kkt_omega(lp, X.mean(0), Y.mean(0), omega)
    assert abs(plain - rec["kkt_avg"]) > 1e-6 * rec["kkt_avg"]
    # this first check restarts to the average (criteria (i) and (iii)): the
    # new primal weight comes from the distance of the average to the start
    # point z^{0,0} = 0, and the new epoch's KKT is the average's under it
    assert rec["restart"] == 5 and rec["cand_avg"] == 1
    omega1 = np.exp(0.5 * np.log(np.linalg.norm(yb) / np.linalg.norm(xb)) + 0.5 * np.log(omega))
    assert rec["omega"] == pytest.approx(omega1, rel=1e-12)
    assert rec["kkt_start"] == pytest.approx(oracle.kkt_omega(lp, xb, yb, omega1), rel=1e-12)


def test_solve_stops_at_the_first_check_that_passes():
    """Sec. 4.1 termination at the first opportunity: every check before the
    last recorded a current iterate whose relative measures exceed tol, the
    solve stopped at the next check, and its returned point meets tol on the
    original LP while the current iterate one check earlier does not."""
    lp = lpgen.tiny_lp(3)
    tol = 1e-6
    r = oracle.solve(lp, tol=tol, check_period=64)
    assert r.status == oracle.OPTIMAL and r.iters % 64 == 0
    tr = r.trace
    assert tr["k"][-1] == r.iters - 64 and len(tr) == r.iters // 64 - 1
    worst = np.maximum(np.maximum(tr["rel_gap"], tr["rel_primal"]), tr["rel_dual"])
    assert np.all(worst > tol)
    assert oracle.passes(lp, r.x, r.y, tol)
    earlier = oracle.solve(lp, tol=0.0, max_iter=r.iters - 64, check_period=64)
    assert not oracle.passes(lp, earlier.x, earlier.y, tol)
    assert oracle.relative_kkt(lp, earlier.x, earlier.y) == pytest.approx(worst[-1], rel=1e-9)


def test_algorithm_2_replayed_in_numpy_reproduces_every_step():
    """Algorithm 2 written out in numpy (trial step of eq. (pdhg), eta_bar
    of eq. (step-size) with |dy'K dx|, the next trial min((1 - (k+2)^-0.3)
    eta_bar, (1 + (k+2)^-0.6) eta) with k accepted steps so far, readings
    1-2) and replayed from the iterates of a solve stopped before each step:
    it takes as many trials as the solve recorded, lands on the iterates of
    the solve stopped after the step, and leaves the recorded next step
    size, rejected trials included.  A restart to the current iterate
    leaves the start point as the stopped solve returns it (with the new
    primal weight in the record); steps after a restart to the average
    are skipped."""
    lp = lpgen.tiny_lp(1)
    kw = dict(tol=0.0, check_period=1, ruiz_iters=0, pc_alpha=-1.0)
    N = 90
    runs = [oracle.solve(lp, max_iter=k, **kw) for k in range(1, N + 1)]
    tr = runs[-1].trace  # record i: the check after step i + 1
    K = dense(lp)
    replayed = rejections = restarted = 0
    for k in range(1, N - 1):  # the step from k to k + 1 accepted steps
        before, after = tr[k - 1], tr[k]
        if before["restart"] != 0 and before["cand_avg"] == 1:
            continue
        x, y = runs[k - 1].x, runs[k - 1].y
        eta, omega = before["eta_hat"], before["omega"]
        trials = 0
        while True:
            trials += 1
            x1 = np.clip(x - eta / omega * (lp.c - K.T @ y), lp.l, lp.u)
            y1 = y + eta * omega * (lp.q - K @ (2 * x1 - x))
            y1[lp.n_eq:] = np.maximum(y1[lp.n_eq:], 0.0)
            dx, dy = x1 - x, y1 - y
            inter = abs(dy @ (K @ dx))
            eta_bar = (omega * (dx @ dx) + (dy @ dy) / omega) / (2.0 * inter) if inter > 0 else np.inf
            kk = float(k + 2)
            eta_next = min((1 - kk ** -0.3) * eta_bar, (1 + kk ** -0.6) * eta)
            if eta <= eta_bar:
                break
            eta = eta_next
            assert trials < 50
        assert trials == after["attempts"] - before["attempts"], k
        np.testing.assert_allclose(runs[k].x, x1, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(runs[k].y, y1, rtol=1e-12, atol=1e-13)
        assert after["eta_hat"] == pytest.approx(eta_next, rel=1e-10)
        replayed += 1
        rejections += trials - 1
        restarted += before["restart"] != 0
    assert replayed >= 60 and rejections >= 4 and restarted >= 1


def test_termination_tests_the_current_iterate_before_the_average():
    """Reading 13's order: at the check where a solve ends on the average
    (which = 1), the current iterate there, from a solve stopped at the same
    step, fails the Sec. 4.1 test and the returned average passes it; at
    the check where a solve ends on the current iterate, that iterate
    is what a solve stopped there returns."""
    tol = 1e-4
    lp = lpgen.tiny_lp(3)
    r = oracle.solve(lp, tol=tol, check_period=64)
    assert r.status == oracle.OPTIMAL and r.which == 1
    cur = oracle.solve(lp, tol=0.0, max_iter=r.iters, check_period=64)
    assert cur.status == oracle.ITER_LIMIT and cur.iters == r.iters
    assert not oracle.passes(lp, cur.x, cur.y, tol) and oracle.passes(lp, r.x, r.y, tol)
    assert not np.array_equal(r.x, cur.x)
    lp = lpgen.tiny_lp(0)
    r = oracle.solve(lp, tol=1e-6, check_period=64)
    assert r.status == oracle.OPTIMAL and r.which == 0
    cur = oracle.solve(lp, tol=0.0, max_iter=r.iters, check_period=64)
    assert np.array_equal(r.x, cur.x) and np.array_equal(r.y, cur.y)
