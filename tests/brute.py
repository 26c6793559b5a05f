"""Brute-force LP optimum by vertex enumeration (test helper, numpy only).

For  min c'x  s.t.  A x = b (rows [0, n_eq)),  G x >= h (rows [n_eq, m)),
l <= x <= u  with every bound finite, an optimum is attained at a vertex: a
point where n linearly independent constraints are active.  Enumerate every
choice of active ">=" rows and every assignment of each variable to
{lower, upper, not fixed}, solve the square system, keep the feasible
solutions and return the smallest objective.  Exponential; only for n <= 6,
m <= 4.  Shares nothing with the oracle or the CUDA solver.
"""

from __future__ import annotations

import itertools

import numpy as np


def dense(lp):
    K = np.zeros((lp.m, lp.n))
    for i in range(lp.m):
        for e in range(int(lp.row_ptr[i]), int(lp.row_ptr[i + 1])):
            K[i, int(lp.col_idx[e])] += lp.val[e]
    return K


def vertex_enum(lp, feas_tol: float = 1e-9):
    assert np.all(np.isfinite(lp.l)) and np.all(np.isfinite(lp.u))
    n, m, n_eq = lp.n, lp.m, lp.n_eq
    K = dense(lp)
    best, best_x = np.inf, None
    ineq = list(range(n_eq, m))
    for r in range(len(ineq) + 1):
        for S in itertools.combinations(ineq, r):
            need = n - n_eq - r
            if need < 0:
                continue
            for fixed in itertools.combinations(range(n), need):
                for side in itertools.product((0, 1), repeat=need):
                    rows, rhs = [], []
                    for i in list(range(n_eq)) + list(S):
                        rows.append(K[i])
                        rhs.append(lp.q[i])
                    for j, sd in zip(fixed, side):
                        e = np.zeros(n)
                        e[j] = 1.0
                        rows.append(e)
                        rhs.append(lp.u[j] if sd else lp.l[j])
                    Mx = np.array(rows).reshape(len(rows), n)
                    if np.linalg.matrix_rank(Mx) < n:
                        continue
                    x = np.linalg.solve(Mx, np.array(rhs))
                    if np.any(x < lp.l - feas_tol) or np.any(x > lp.u + feas_tol):
                        continue
                    kx = K @ x
                    if n_eq and np.max(np.abs(kx[:n_eq] - lp.q[:n_eq])) > feas_tol * (1 + np.abs(lp.q[:n_eq]).max()):
                        continue
                    if m > n_eq and np.any(kx[n_eq:] < lp.q[n_eq:] - feas_tol):
                        continue
                    obj = float(lp.c @ x)
                    if obj < best:
                        best, best_x = obj, x
    return best, best_x
