"""Seeded synthetic linear programs with a planted optimal primal-dual pair.

This module only *builds instances*; it holds none of the solver's arithmetic
(no PDHG step, no scaling, no KKT evaluation).  Both the CUDA solver's tests
and the CPU oracle's tests draw their inputs from here.

Problem form (Sec. 2, eq. (lp) / (primal-dual) of the cuPDLP.jl paper):

    min c^T x   s.t.  A x = b,  G x >= h,  l <= x <= u,

stored with K = (A; G) in CSR and q = (b; h): rows [0, n_eq) are the
equalities, rows [n_eq, m) the ">=" rows (the paper lists G first; this is the
same problem with the rows permuted).

Planted optimum.  Draw x* inside the bounds with a fraction of the bounded
variables sitting on a bound, duals y* (free on equality rows, >= 0 and
complementary on ">=" rows) and reduced costs lam* (> 0 only where x* sits on
its lower bound, < 0 only on its upper bound), then set

    b = A x*,   h_i = (G x*)_i on active rows,  (G x*)_i - U(0.1, 1) otherwise,
    c = K^T y* + lam*.

(x*, y*, lam*) then satisfies the KKT system of the LP by construction, so
c^T x* is the exact optimal value and the dual objective
q^T y* + l^T lam*^+ - u^T lam*^- equals it.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "LP",
    "plant",
    "uniform_pattern",
    "zipf_pattern",
    "tiny_lp",
    "large_lp",
    "random_boxed_lp",
    "batch_lps",
    "batch_lp",
    "batch_subset",
    "batch_work",
    "planted_qp",
    "permuted",
    "infeasible_lp",
]


@dataclass
class LP:
    """One LP instance in the solver's C-ABI layout (int32 CSR, float64 values)."""

    m: int
    n: int
    n_eq: int
    c: np.ndarray
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray
    q: np.ndarray
    l: np.ndarray
    u: np.ndarray
    x_star: np.ndarray | None = None
    y_star: np.ndarray | None = None
    lam_star: np.ndarray | None = None
    obj_star: float | None = None
    meta: dict = field(default_factory=dict)
    qdiag: np.ndarray | None = None  # QP extension: objective x'Qx/2 + c'x with Q = diag(qdiag)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def arrays(self):
        """Contiguous arrays in C-ABI order: c, row_ptr, col_idx, val, q, l, u."""
        return (
            np.ascontiguousarray(self.c, dtype=np.float64),
            np.ascontiguousarray(self.row_ptr, dtype=np.int32),
            np.ascontiguousarray(self.col_idx, dtype=np.int32),
            np.ascontiguousarray(self.val, dtype=np.float64),
            np.ascontiguousarray(self.q, dtype=np.float64),
            np.ascontiguousarray(self.l, dtype=np.float64),
            np.ascontiguousarray(self.u, dtype=np.float64),
        )


# ----------------------------------------------------------------------------
# sparsity patterns
# ----------------------------------------------------------------------------


def _sample_rows(rng: np.random.Generator, lengths: np.ndarray, n: int):
    """Columns drawn uniformly without replacement inside each row, sorted.

    Returns (row_ptr int64, col int64).  Draws with replacement, then redraws
    the duplicates until every row holds distinct columns; rows that still
    hold duplicates after 200 rounds (nearly dense rows) take the rest of
    their columns from the ones they lack, without replacement."""
    lengths = np.minimum(np.asarray(lengths, dtype=np.int64), n)
    m = lengths.shape[0]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    rows = np.repeat(np.arange(m, dtype=np.int64), lengths)
    cols = rng.integers(0, n, size=nnz, dtype=np.int64)
    for _ in range(200):
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        key = key[order]
        cols = cols[order]  # rows stay sorted: key is row-major
        dup = np.zeros(nnz, dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum())
        if nd == 0:
            return row_ptr, cols
        cols[dup] = rng.integers(0, n, size=nd, dtype=np.int64)
    for r in np.unique(rows[dup]):
        a, b = int(row_ptr[r]), int(row_ptr[r + 1])
        have = np.unique(cols[a:b])
        missing = np.setdiff1d(np.arange(n, dtype=np.int64), have, assume_unique=True)
        extra = rng.choice(missing, size=(b - a) - have.size, replace=False)
        cols[a:b] = np.sort(np.concatenate([have, extra]))
    return row_ptr, cols


def _cover_columns(rng, row_ptr, cols, m, n):
    """Give every empty column one entry in a uniformly drawn row."""
    counts = np.bincount(cols, minlength=n)
    empty = np.flatnonzero(counts == 0)
    if empty.size == 0:
        return row_ptr, cols
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))
    add_rows = rng.integers(0, m, size=empty.size, dtype=np.int64)
    rows = np.concatenate([rows, add_rows])
    cols = np.concatenate([cols, empty.astype(np.int64)])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    return row_ptr, cols


def uniform_pattern(rng, m: int, n: int, density: float, cover: bool = True):
    """Each entry nonzero with probability `density`; every row (and, with
    `cover`, every column) gets at least one entry."""
    lengths = rng.binomial(n, density, size=m).astype(np.int64)
    lengths = np.maximum(lengths, 1)
    row_ptr, cols = _sample_rows(rng, lengths, n)
    if cover:
        row_ptr, cols = _cover_columns(rng, row_ptr, cols, m, n)
    return row_ptr, cols


def zipf_pattern(rng, m: int, n: int, nnz_target: int, alpha: float = 1.5, cap: int = 5000):
    """Power-law row lengths: Z ~ Zipf(alpha) clipped at `cap`, rescaled to
    d_i = max(1, round(s * Z_i)) with s found by bisection so that the total
    is within 0.1 % of `nnz_target`.  Columns uniform without replacement."""
    z = np.minimum(rng.zipf(alpha, size=m), cap).astype(np.float64)

    def total(s):
        return int(np.maximum(1, np.rint(s * z)).sum())

    lo, hi = 0.0, 1.0
    while total(hi) < nnz_target and hi < 1e9:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        t = total(mid)
        if abs(t - nnz_target) <= 1e-3 * nnz_target:
            lo = hi = mid
            break
        if t < nnz_target:
            lo = mid
        else:
            hi = mid
    s = 0.5 * (lo + hi)
    lengths = np.minimum(np.maximum(1, np.rint(s * z)), n).astype(np.int64)
    row_ptr, cols = _sample_rows(rng, lengths, n)
    return row_ptr, cols, s


# ----------------------------------------------------------------------------
# planted optimum
# ----------------------------------------------------------------------------


def _csr_matvec(row_ptr, cols, val, x, m):
    prod = val * x[cols]
    out = np.zeros(m, dtype=np.float64)
    nz = np.diff(row_ptr) > 0
    starts = row_ptr[:-1][nz]
    out[nz] = np.add.reduceat(prod, starts) if prod.size else 0.0
    return out


def _csr_rmatvec(cols, val, y_rep, n):
    return np.bincount(cols, weights=val * y_rep, minlength=n).astype(np.float64)


def plant(
    rng,
    m: int,
    n: int,
    n_eq: int,
    row_ptr,
    cols,
    val,
    l,
    u,
    at_bound_frac: float = 0.3,
    active_frac: float = 0.5,
    meta: dict | None = None,
) -> LP:
    """Build (q, c) from a planted optimal pair for the given K, l, u."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    l = np.asarray(l, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    lf, uf = np.isfinite(l), np.isfinite(u)

    x = np.empty(n)
    lam = np.zeros(n)
    box, low, upp, free = lf & uf, lf & ~uf, ~lf & uf, ~lf & ~uf
    at_bound = (rng.random(n) < at_bound_frac) & ~free
    pick_low = rng.random(n) < 0.5
    at_l = at_bound & (low | (box & pick_low))
    at_u = at_bound & (upp | (box & ~pick_low))
    inner = ~(at_l | at_u)
    x[box & inner] = rng.uniform(l[box & inner], u[box & inner])
    x[low & inner] = l[low & inner] + rng.uniform(0.0, 5.0, size=int((low & inner).sum()))
    x[upp & inner] = u[upp & inner] - rng.uniform(0.0, 5.0, size=int((upp & inner).sum()))
    x[free] = rng.standard_normal(int(free.sum()))
    x[at_l] = l[at_l]
    x[at_u] = u[at_u]
    lam[at_l] = rng.uniform(0.1, 1.0, size=int(at_l.sum()))
    lam[at_u] = -rng.uniform(0.1, 1.0, size=int(at_u.sum()))

    y = np.zeros(m)
    y[:n_eq] = rng.standard_normal(n_eq)
    n_in = m - n_eq
    active = rng.random(n_in) < active_frac
    y[n_eq:][active] = rng.uniform(0.1, 1.0, size=int(active.sum()))

    kx = _csr_matvec(row_ptr, cols, val, x, m)
    q = kx.copy()
    slack = rng.uniform(0.1, 1.0, size=n_in)
    q[n_eq:][~active] = kx[n_eq:][~active] - slack[~active]

    y_rep = np.repeat(y, np.diff(row_ptr))
    c = _csr_rmatvec(cols, val, y_rep, n) + lam
    obj = math.fsum((c * x).tolist())
    return LP(
        m=m,
        n=n,
        n_eq=n_eq,
        c=c,
        row_ptr=row_ptr.astype(np.int32),
        col_idx=cols.astype(np.int32),
        val=val,
        q=q,
        l=l,
        u=u,
        x_star=x,
        y_star=y,
        lam_star=lam,
        obj_star=obj,
        meta=dict(meta or {}),
    )


# ----------------------------------------------------------------------------
# workload recipes
# ----------------------------------------------------------------------------


def tiny_lp(seed: int = 0, m_eq: int = 100, m_ineq: int = 100, n: int = 500, density: float = 0.02) -> LP:
    """Small LP: 0 <= x <= 10, N(0,1) values, uniform sparsity (default 2 %),
    equality rows first, 30 % of x* on a bound."""
    rng = np.random.default_rng([0x7A11, seed])
    m = m_eq + m_ineq
    row_ptr, cols = uniform_pattern(rng, m, n, density, cover=True)
    val = rng.standard_normal(cols.size)
    l = np.zeros(n)
    u = np.full(n, 10.0)
    return plant(rng, m, n, m_eq, row_ptr, cols, val, l, u,
                 meta=dict(kind="tiny", seed=seed, density=density))


def large_lp(seed: int = 0, m: int = 1_000_000, n: int = 2_000_000, nnz: int = 20_000_000,
             eq_frac: float = 0.4, alpha: float = 1.5, cap: int = 5000) -> LP:
    """Power-law planted LP: Zipf(alpha) row lengths (clipped at `cap`,
    rescaled to `nnz` total), lognormal(0, 2) magnitudes with random signs,
    bounds 50 % [0, inf), 30 % [l, u] (l ~ U(-5,0), u ~ U(0,5)), 20 % free."""
    rng = np.random.default_rng([0x1A26E, seed])
    n_eq = int(round(eq_frac * m))
    row_ptr, cols, s = zipf_pattern(rng, m, n, nnz, alpha=alpha, cap=cap)
    k = cols.size
    val = rng.lognormal(0.0, 2.0, size=k) * np.where(rng.random(k) < 0.5, -1.0, 1.0)
    kind = rng.random(n)
    l = np.zeros(n)
    u = np.full(n, np.inf)
    boxed = (kind >= 0.5) & (kind < 0.8)
    free = kind >= 0.8
    l[boxed] = rng.uniform(-5.0, 0.0, size=int(boxed.sum()))
    u[boxed] = rng.uniform(0.0, 5.0, size=int(boxed.sum()))
    l[free] = -np.inf
    u[free] = np.inf
    lengths = np.diff(row_ptr)
    return plant(rng, m, n, n_eq, row_ptr, cols, val, l, u,
                 meta=dict(kind="large", seed=seed, zipf_scale=s,
                           max_row=int(lengths.max()) if m else 0,
                           mean_row=float(lengths.mean()) if m else 0.0))


def random_boxed_lp(seed: int, m_eq: int, m_ineq: int, n: int, density: float = 0.5,
                    lo: float = -1.0, hi: float = 2.0, planted: bool = True) -> LP:
    """Tiny dense-ish boxed LP (all bounds finite) for brute-force checks.
    With planted=False, c and q are drawn at random (the LP is still feasible
    because q is taken from a random point inside the box)."""
    rng = np.random.default_rng([0xB0C5, seed])
    m = m_eq + m_ineq
    if m:
        row_ptr, cols = uniform_pattern(rng, m, n, density, cover=False)
    else:
        row_ptr, cols = np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int64)
    val = rng.standard_normal(cols.size)
    l = np.full(n, lo)
    u = np.full(n, hi)
    if planted:
        return plant(rng, m, n, m_eq, row_ptr, cols, val, l, u, meta=dict(kind="boxed", seed=seed))
    x0 = rng.uniform(lo, hi, size=n)
    kx = _csr_matvec(row_ptr, cols, val, x0, m)
    q = kx.copy()
    q[m_eq:] -= rng.uniform(0.0, 1.0, size=m_ineq)
    c = rng.standard_normal(n)
    return LP(m=m, n=n, n_eq=m_eq, c=c, row_ptr=row_ptr.astype(np.int32),
              col_idx=cols.astype(np.int32), val=val, q=q, l=l, u=u,
              meta=dict(kind="boxed-random", seed=seed))


def _from_coo(m, rows, cols, vals):
    """CSR (row_ptr, cols, vals) of COO entries, sorted by (row, column)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    return row_ptr, cols[order], vals[order]


def infeasible_lp(seed: int, kind: str, m_eq: int = 30, m_ineq: int = 30, n: int = 120,
                  density: float = 0.05) -> LP:
    """A small LP with a known infeasibility, built around a planted feasible
    one (0 <= x <= 10, N(0,1) values); meta["ray"] holds an exact certificate.

      "primal":        two ">=" rows a'x >= h1 and -a'x >= -h2 with h2 < h1
                       (dual ray: 1 on both rows);
      "primal_bounds": one ">=" row a'x >= h with h above the largest value
                       of a'x over the box (dual ray: 1 on that row);
      "dual":          two extra columns v and -v with bounds [0, inf) and
                       costs -1 and 0.5, so x = t (e_n + e_{n+1}) is feasible
                       for all t >= 0 and lowers c'x without bound (primal
                       ray e_n + e_{n+1}).
    """
    rng = np.random.default_rng([0x1F3A, seed, ["primal", "primal_bounds", "dual"].index(kind)])
    base = tiny_lp(1000 + seed, m_eq=m_eq, m_ineq=m_ineq, n=n, density=density)
    rows = np.repeat(np.arange(base.m, dtype=np.int64), np.diff(base.row_ptr))
    cols = base.col_idx.astype(np.int64)
    vals = base.val.copy()
    m, nn = base.m, base.n
    q, c, l, u = base.q.copy(), base.c.copy(), base.l.copy(), base.u.copy()
    if kind in ("primal", "primal_bounds"):
        k = max(3, n // 10)
        a_cols = np.sort(rng.choice(n, size=k, replace=False))
        a_val = rng.standard_normal(k)
        if kind == "primal":
            h1 = float(a_val @ base.x_star[a_cols]) + rng.uniform(0.5, 1.0)
            h2 = h1 - rng.uniform(0.5, 1.0)
            new_rows = [(a_cols, a_val, h1), (a_cols, -a_val, -h2)]
            ray_y = np.zeros(m + 2)
            ray_y[m:] = 1.0
        else:
            top = float(np.sum(np.maximum(a_val * l[a_cols], a_val * u[a_cols])))
            new_rows = [(a_cols, a_val, top + rng.uniform(0.5, 1.0))]
            ray_y = np.zeros(m + 1)
            ray_y[m] = 1.0
        for cc_, vv_, hh_ in new_rows:
            rows = np.concatenate([rows, np.full(cc_.size, m, dtype=np.int64)])
            cols = np.concatenate([cols, cc_])
            vals = np.concatenate([vals, vv_])
            q = np.concatenate([q, [hh_]])
            m += 1
        row_ptr, cols, vals = _from_coo(m, rows, cols, vals)
        return LP(m=m, n=nn, n_eq=base.n_eq, c=c, row_ptr=row_ptr.astype(np.int32),
                  col_idx=cols.astype(np.int32), val=vals, q=q, l=l, u=u,
                  meta=dict(kind="infeasible-" + kind, seed=seed, ray_y=ray_y, ray_x=None))
    if kind != "dual":
        raise ValueError("kind must be 'primal', 'primal_bounds' or 'dual'")
    k = max(3, m // 10)
    v_rows = np.sort(rng.choice(m, size=k, replace=False))
    v_val = rng.standard_normal(k)
    rows = np.concatenate([rows, v_rows, v_rows])
    cols = np.concatenate([cols, np.full(k, nn, dtype=np.int64), np.full(k, nn + 1, dtype=np.int64)])
    vals = np.concatenate([vals, v_val, -v_val])
    row_ptr, cols, vals = _from_coo(m, rows, cols, vals)
    c = np.concatenate([c, [-1.0, 0.5]])
    l = np.concatenate([l, [0.0, 0.0]])
    u = np.concatenate([u, [np.inf, np.inf]])
    ray_x = np.zeros(nn + 2)
    ray_x[nn:] = 1.0
    return LP(m=m, n=nn + 2, n_eq=base.n_eq, c=c, row_ptr=row_ptr.astype(np.int32),
              col_idx=cols.astype(np.int32), val=vals, q=q, l=l, u=u,
              meta=dict(kind="infeasible-dual", seed=seed, ray_x=ray_x, ray_y=None))


def _batch_shapes(count: int, seed: int, m_lo: int, m_hi: int, dens_lo: float, dens_hi: float):
    rng = np.random.default_rng([0xBA7C, seed])
    for _ in range(count):
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        n = int(round(math.exp(rng.uniform(math.log(2 * m / 3), math.log(2.5 * m)))))
        d = float(rng.uniform(dens_lo, dens_hi))
        yield m, n, d


def _batch_member(i: int, seed: int, m: int, n: int, d: float) -> LP:
    n_eq = m // 2
    sub = np.random.default_rng([0xBA7C, seed, i])
    row_ptr, cols = uniform_pattern(sub, m, n, d, cover=True)
    val = sub.standard_normal(cols.size)
    return plant(sub, m, n, n_eq, row_ptr, cols, val, np.zeros(n), np.full(n, 10.0),
                 meta=dict(kind="batch", seed=seed, index=i, density=d))


def batch_lps(count: int, seed: int = 0, m_lo: int = 50, m_hi: int = 4000,
              dens_lo: float = 0.005, dens_hi: float = 0.05) -> list[LP]:
    """Uneven batch: m ~ logU[m_lo, m_hi], n ~ logU[2m/3, 2.5m], density ~
    U[dens_lo, dens_hi], N(0,1) values, half equality rows, 0 <= x <= 10."""
    return [_batch_member(i, seed, m, n, d)
            for i, (m, n, d) in enumerate(_batch_shapes(count, seed, m_lo, m_hi, dens_lo, dens_hi))]


def batch_lp(index: int, seed: int = 0, m_lo: int = 50, m_hi: int = 4000,
             dens_lo: float = 0.005, dens_hi: float = 0.05) -> LP:
    """Member `index` of batch_lps(count > index, seed, ...), built alone."""
    for i, (m, n, d) in enumerate(_batch_shapes(index + 1, seed, m_lo, m_hi, dens_lo, dens_hi)):
        if i == index:
            return _batch_member(i, seed, m, n, d)
    raise IndexError(index)


def batch_subset(indices, count: int, seed: int = 0, m_lo: int = 50, m_hi: int = 4000,
                 dens_lo: float = 0.005, dens_hi: float = 0.05) -> list[LP]:
    """Members `indices` of batch_lps(count, seed, ...), each built alone (a
    rank of a sharded run builds only its own)."""
    shapes = list(_batch_shapes(count, seed, m_lo, m_hi, dens_lo, dens_hi))
    return [_batch_member(int(i), seed, *shapes[int(i)]) for i in indices]


def batch_work(count: int, seed: int = 0, m_lo: int = 50, m_hi: int = 4000,
               dens_lo: float = 0.005, dens_hi: float = 0.05) -> np.ndarray:
    """Expected nonzeros m n density of each member of batch_lps(count, seed),
    from the shapes alone (no member is built)."""
    return np.array([m * n * d for m, n, d in _batch_shapes(count, seed, m_lo, m_hi, dens_lo, dens_hi)])


def planted_qp(lp: LP, seed: int = 0, frac: float = 0.6, lo: float = 0.0, hi: float = 2.0) -> LP:
    """The QP min x'Qx/2 + c'x over the planted LP's feasible set, Q =
    diag(qdiag) with a fraction `frac` of its entries ~ U(lo, hi), the rest 0,
    and c shifted by -Q x* so that the LP's planted pair (x*, y*, lambda*)
    satisfies the QP's KKT system (stationarity c + Q x* - K'y* - lambda* = 0,
    the same complementarity): x* is optimal with value x*'Qx*/2 + c'x*."""
    rng = np.random.default_rng([0x0D1A, seed])
    qd = np.where(rng.random(lp.n) < frac, rng.uniform(lo, hi, lp.n), 0.0)
    c = lp.c - qd * lp.x_star
    obj = float(0.5 * np.dot(qd * lp.x_star, lp.x_star) + np.dot(c, lp.x_star))
    out = LP(m=lp.m, n=lp.n, n_eq=lp.n_eq, c=c, row_ptr=lp.row_ptr, col_idx=lp.col_idx, val=lp.val, q=lp.q,
             l=lp.l, u=lp.u, x_star=lp.x_star, y_star=lp.y_star, lam_star=lp.lam_star, obj_star=obj,
             meta=dict(lp.meta, qp=True, qp_seed=seed), qdiag=qd)
    return out


def permuted(lp: LP, seed: int) -> LP:
    """The same LP with its columns permuted and its rows permuted within the
    equality and the ">=" groups (and the planted pair with them): another
    summation order for every solver, nothing else changed."""
    rng = np.random.default_rng([0x9E57, seed])
    pc = rng.permutation(lp.n)
    pr = np.concatenate([rng.permutation(lp.n_eq), lp.n_eq + rng.permutation(lp.m - lp.n_eq)])
    inv_c = np.empty(lp.n, dtype=np.int64)
    inv_c[pc] = np.arange(lp.n)
    lens = np.diff(lp.row_ptr)[pr]
    row_ptr = np.zeros(lp.m + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    starts = np.asarray(lp.row_ptr)[pr]
    src = np.repeat(starts - row_ptr[:-1], lens) + np.arange(int(row_ptr[-1]))
    cols = inv_c[np.asarray(lp.col_idx)[src]]
    vals = np.asarray(lp.val)[src]
    rows = np.repeat(np.arange(lp.m), lens)
    order = np.lexsort((cols, rows))  # columns increasing inside each row
    return LP(m=lp.m, n=lp.n, n_eq=lp.n_eq, c=lp.c[pc], row_ptr=row_ptr.astype(np.int32),
              col_idx=cols[order].astype(np.int32), val=vals[order], q=lp.q[pr], l=lp.l[pc], u=lp.u[pc],
              x_star=None if lp.x_star is None else lp.x_star[pc],
              y_star=None if lp.y_star is None else lp.y_star[pr],
              lam_star=None if lp.lam_star is None else lp.lam_star[pc], obj_star=lp.obj_star,
              meta=dict(lp.meta, permuted=seed), qdiag=None if lp.qdiag is None else lp.qdiag[pc])


# ----------------------------------------------------------------------------
# parametric transportation family
# ----------------------------------------------------------------------------


@dataclass
class TransportFamily:
    """min sum c_ij x_ij  s.t.  sum_i x_ij = d_j (sinks, equality rows first),
    -sum_j x_ij >= -s_i (sources), x >= 0, with x_ij at column i * sinks + j.
    Costs, supplies and demands are affine in a latent theta ~ N(0, I_dim)
    through fixed seeded matrices, plus N(0, noise) noise; supplies and
    demands are clipped at `floor` (keeps every instance feasible) and the
    supplies rescaled so that sum s = slack * sum d."""

    sources: int
    sinks: int
    dim: int
    c0: np.ndarray
    Cc: np.ndarray
    s0: np.ndarray
    Cs: np.ndarray
    d0: np.ndarray
    Cd: np.ndarray
    noise: float
    floor: float
    slack: float
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def n(self):
        return self.sources * self.sinks

    @property
    def m(self):
        return self.sources + self.sinks


def transport_family(seed: int = 0, sources: int = 200, sinks: int = 300, dim: int = 16, noise: float = 0.1,
                     floor: float = 0.05, slack: float = 1.05, cost_scale: float = 1.0) -> TransportFamily:
    """cost_scale multiplies the latent cost directions (0: fixed costs, only
    supplies and demands move with theta)."""
    rng = np.random.default_rng([0x7A45, seed])
    n = sources * sinks
    # costs: a base geometry (sources and sinks on the unit square) plus latent directions
    ps, pk = rng.random((sources, 2)), rng.random((sinks, 2))
    c0 = np.sqrt(((ps[:, None, :] - pk[None, :, :]) ** 2).sum(-1)).ravel() * 10.0 + 1.0
    Cc = rng.standard_normal((n, dim)) * 0.5 * cost_scale
    s0 = rng.uniform(1.0, 3.0, sources)
    Cs = rng.standard_normal((sources, dim)) * 0.3
    d0 = rng.uniform(1.0, 2.0, sinks)
    Cd = rng.standard_normal((sinks, dim)) * 0.2
    # K: sink rows (+1) first, then source rows (-1)
    rows_sink = [np.arange(sources) * sinks + j for j in range(sinks)]
    rows_src = [np.arange(sinks) + i * sinks for i in range(sources)]
    cols = np.concatenate(rows_sink + rows_src)
    val = np.concatenate([np.ones(n), -np.ones(n)])
    row_ptr = np.concatenate([[0], np.cumsum([sources] * sinks + [sinks] * sources)])
    return TransportFamily(sources, sinks, dim, c0, Cc, s0, Cs, d0, Cd, noise, floor, slack,
                           row_ptr.astype(np.int32), cols.astype(np.int32), val)


def transport_thetas(count: int, seed: int, dim: int = 16) -> np.ndarray:
    return np.random.default_rng([0x7E7A, seed]).standard_normal((count, dim))


def transport_lp(fam: TransportFamily, theta: np.ndarray, noise_seed: int) -> LP:
    """The family member at latent `theta` (noise drawn from `noise_seed`)."""
    rng = np.random.default_rng([0x7A46, noise_seed])
    c = fam.c0 + fam.Cc @ theta + rng.normal(0.0, fam.noise, fam.n)
    s = np.maximum(fam.s0 + fam.Cs @ theta + rng.normal(0.0, fam.noise, fam.sources), fam.floor)
    d = np.maximum(fam.d0 + fam.Cd @ theta + rng.normal(0.0, fam.noise, fam.sinks), fam.floor)
    s = s * (fam.slack * d.sum() / s.sum())
    q = np.concatenate([d, -s])
    return LP(m=fam.m, n=fam.n, n_eq=fam.sinks, c=c, row_ptr=fam.row_ptr, col_idx=fam.col_idx, val=fam.val, q=q,
              l=np.zeros(fam.n), u=np.full(fam.n, np.inf), meta=dict(kind="transport", noise_seed=noise_seed))
