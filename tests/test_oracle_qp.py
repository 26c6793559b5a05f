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
