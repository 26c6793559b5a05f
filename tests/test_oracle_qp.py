"""QP extension in the oracle (the introduction names the extension of the
method to quadratic programs; this is the diagonal-Hessian case): pinned by
closed forms, a KKT linear solve, planted optima and a hand-worked example."""

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle


class _QP:
    def __init__(self, A, c, q, l, u, n_eq, qd):
        S = sp.csr_matrix(A)
        self.m, self.n = A.shape
        self.n_eq = n_eq
        self.row_ptr, self.col_idx, self.val = S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data
        self.c, self.q, self.l, self.u, self.qdiag = c, q, l, u, qd

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


def test_qp_kkt_terms_hand():
    # min x1^2 + 0.5 x2^2 / 2 ... : Q = diag(2, 0.5), c = (1, -1), one equality x1 + x2 = 3, x >= 0
    qp = _QP(np.array([[1.0, 1.0]]), np.array([1.0, -1.0]), np.array([3.0]), np.zeros(2), np.full(2, np.inf), 1,
             np.array([2.0, 0.5]))
    x, y = np.array([1.0, 1.0]), np.array([0.5])
    # gradient c + Qx = (3, -0.5); minus K'y = (0.5, 0.5): d = (2.5, -1.0); only l finite: lambda = (2.5, 0)
    # r_d = (0, -1); primal residual 3 - 2 = 1; x'Qx = 2.5
    # pobj = c'x + 1.25 = 1.25; dobj = q'y + l'lambda+ - 1.25 = 1.5 + 0 - 1.25 = 0.25
    t = oracle.kkt_terms(qp, x, y)
    assert t["pobj"] == pytest.approx(1.25, abs=1e-15)
    assert t["dobj"] == pytest.approx(0.25, abs=1e-15)
    assert t["rp"] == pytest.approx(1.0, abs=1e-15)
    assert t["rd"] == pytest.approx(1.0, abs=1e-15)


def test_box_qp_without_rows_is_a_clamp():
    rng = np.random.default_rng(0)
    n = 40
    qd = rng.uniform(0.2, 3.0, n)
    c = rng.standard_normal(n) * 3
    l, u = np.full(n, -1.0), np.full(n, 1.5)
    qp = _QP(np.zeros((0, n)), c, np.zeros(0), l, u, 0, qd)
    r = oracle.solve(qp, tol=1e-10, max_iter=200000)
    assert r.status == oracle.OPTIMAL
    np.testing.assert_allclose(r.x, np.clip(-c / qd, l, u), atol=1e-8)


def test_equality_qp_matches_its_kkt_system():
    rng = np.random.default_rng(1)
    m, n = 4, 9
    A = rng.standard_normal((m, n))
    qd = rng.uniform(0.5, 2.0, n)
    c, b = rng.standard_normal(n), rng.standard_normal(m)
    # stationarity Q x + c - A'y = 0 and A x = b
    M = np.block([[np.diag(qd), -A.T], [A, np.zeros((m, m))]])
    sol = np.linalg.solve(M, np.concatenate([-c, b]))
    qp = _QP(A, c, b, np.full(n, -np.inf), np.full(n, np.inf), m, qd)
    r = oracle.solve(qp, tol=1e-10, max_iter=400000)
    assert r.status == oracle.OPTIMAL
    np.testing.assert_allclose(r.x, sol[:n], atol=1e-7)
    np.testing.assert_allclose(r.y, sol[n:], atol=1e-7)


@pytest.mark.parametrize("kind", ["tiny", "powerlaw"])
def test_planted_qp_optimum(kind):
    base = lpgen.tiny_lp(4) if kind == "tiny" else lpgen.large_lp(2, m=1000, n=2000, nnz=20000)
    qp = lpgen.planted_qp(base, seed=1)
    assert np.count_nonzero(qp.qdiag) > 0 and np.count_nonzero(qp.qdiag == 0) > 0
    t = oracle.kkt_terms(qp, qp.x_star, qp.y_star)  # the planted pair is a KKT point of the QP
    assert abs(t["pobj"] - t["dobj"]) <= 1e-9 * (1 + abs(t["pobj"]))
    assert t["rp"] <= 1e-9 * (1 + t["q_norm"]) and t["rd"] <= 1e-9 * (1 + t["c_norm"])
    assert t["pobj"] == pytest.approx(qp.obj_star, rel=1e-12)
    r = oracle.solve(qp, tol=1e-8, max_iter=400000)
    assert r.status == oracle.OPTIMAL
    obj = float(0.5 * np.dot(qp.qdiag * r.x, r.x) + qp.c @ r.x)
    assert abs(obj - qp.obj_star) <= 1e-6 * (1 + abs(qp.obj_star))
    assert oracle.passes(qp, r.x, r.y, 1e-8)


def test_qp_rejects_negative_curvature():
    base = lpgen.tiny_lp(4)
    qp = lpgen.planted_qp(base, seed=1)
    qp.qdiag = qp.qdiag.copy()
    qp.qdiag[3] = -1.0
    with pytest.raises(ValueError):
        oracle.solve(qp, tol=1e-6)


def test_first_qp_step_is_the_proximal_step():
    # no rows: eta-hat = 1 (K is empty), omega = 1 (q = 0), the first trial is
    # accepted (no interaction term), so tau = 1 and from x = 0:
    # x1 = proj_X((0 - (c - 0)) / (1 + Q)) -- an explicit gradient step on the
    # quadratic would give proj_X(-c) instead
    rng = np.random.default_rng(5)
    n = 12
    qd = rng.uniform(0.5, 4.0, n)
    c = rng.standard_normal(n)
    l, u = np.full(n, -0.3), np.full(n, 0.4)
    qp = _QP(np.zeros((0, n)), c, np.zeros(0), l, u, 0, qd)
    r = oracle.solve(qp, tol=1e-30, max_iter=1, check_period=1, ruiz_iters=0, pc_alpha=-1.0)
    assert r.iters == 1
    np.testing.assert_allclose(r.x, np.clip(-c / (1 + qd), l, u), rtol=1e-15, atol=0)


def test_every_accepted_qp_step_is_the_proximal_pdhg_step():
    """Along a QP trajectory (no scaling, check period 1), every step
    accepted at its first trial maps the iterates of the solve stopped
    before it to those of the solve stopped after it by the proximal primal
    step x' = proj_X((x - tau (c - K'y)) / (1 + tau Q_jj)) and the
    extrapolated dual step y' = proj_Y(y + sigma (q - K(2x' - x))), with
    tau = eta / omega, sigma = eta omega from the record in between: the
    Hessian enters every step, across restarts and primal-weight changes."""
    lp = lpgen.planted_qp(lpgen.tiny_lp(2), seed=3)
    kw = dict(tol=0.0, check_period=1, ruiz_iters=0, pc_alpha=-1.0)
    N = 40
    runs = [oracle.solve(lp, max_iter=k, **kw) for k in range(1, N + 1)]
    tr = runs[-1].trace  # record i: the check after step i + 1
    assert np.array_equal(tr["k"], np.arange(1, N))
    K = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n)).toarray()
    checked, omegas = 0, set()
    for k in range(1, N - 1):
        before, after = tr[k - 1], tr[k]
        if after["attempts"] - before["attempts"] != 1 or before["restart"] != 0:
            continue
        x, y = runs[k - 1].x, runs[k - 1].y
        eta, omega = before["eta_hat"], before["omega"]
        tau, sigma = eta / omega, eta * omega
        x1 = np.clip((x - tau * (lp.c - K.T @ y)) / (1.0 + tau * lp.qdiag), lp.l, lp.u)
        y1 = y + sigma * (lp.q - K @ (2 * x1 - x))
        y1[lp.n_eq:] = np.maximum(y1[lp.n_eq:], 0.0)
        np.testing.assert_allclose(runs[k].x, x1, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(runs[k].y, y1, rtol=1e-12, atol=1e-13)
        checked += 1
        omegas.add(float(omega))
    assert checked >= 10 and len(omegas) >= 2


def test_fp32_values_mode_of_a_qp_step():
    """The QP extension in the FP32-values mode of the steps: from a warm
    start, one accepted step is the proximal primal step (with the start
    point's K'y0 in FP64) and the extrapolated dual step whose product takes
    K rounded to FP32; the Hessian and the rounding both matter."""
    lp = lpgen.planted_qp(lpgen.tiny_lp(2), seed=1)
    rng = np.random.default_rng(5)
    x0 = np.clip(lp.x_star + rng.uniform(-0.5, 0.5, lp.n), lp.l + 0.1, lp.u - 0.1)
    y0 = lp.y_star + rng.uniform(-0.1, 0.1, lp.m)
    r = oracle.solve(lp, tol=0.0, max_iter=1, check_period=1, ruiz_iters=0, pc_alpha=-1.0, x0=x0, y0=y0,
                     step_value_bits=32)
    assert r.status == oracle.ITER_LIMIT and r.iters == 1 and r.attempts == 1
    K = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n)).toarray()
    K32 = K.astype(np.float32).astype(np.float64)
    eta = 1.0 / np.abs(lp.val).max()
    omega = np.linalg.norm(lp.c) / np.linalg.norm(lp.q)
    tau, sigma = eta / omega, eta * omega

    def primal(qd):
        return np.clip((x0 - tau * (lp.c - K.T @ y0)) / (1.0 + tau * qd), lp.l, lp.u)

    def dual(Km, x1):
        y1 = y0 + sigma * (lp.q - Km @ (2 * x1 - x0))
        y1[lp.n_eq:] = np.maximum(y1[lp.n_eq:], 0)
        return y1

    x1 = primal(lp.qdiag)
    np.testing.assert_allclose(r.x, x1, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(r.y, dual(K32, x1), rtol=1e-13, atol=1e-14)
    assert np.abs(x1 - primal(0.0)).max() > 1e-6 * np.abs(x1).max()
    assert np.abs(dual(K32, x1) - dual(K, x1)).max() > 1e-10 * np.abs(dual(K, x1)).max()
