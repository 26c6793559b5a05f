"""Input generators (no solver arithmetic): the benchmark LP, the uneven
batch and the transportation family follow their stated recipes, and single
members of a batch are rebuilt exactly, so a member can be studied without
its batch."""

import numpy as np
import pytest

import lpgen


def test_batch_lp_equals_the_member_of_its_batch():
    batch = lpgen.batch_lps(12, seed=3, m_lo=20, m_hi=400)
    for i in (0, 5, 11):
        one = lpgen.batch_lp(i, seed=3, m_lo=20, m_hi=400)
        ref = batch[i]
        assert (one.m, one.n, one.n_eq) == (ref.m, ref.n, ref.n_eq)
        for f in ("row_ptr", "col_idx", "val", "c", "q", "l", "u", "x_star", "y_star"):
            assert np.array_equal(getattr(one, f), getattr(ref, f)), f


def test_permuted_lp_is_the_same_lp():
    import oracle

    lp = lpgen.tiny_lp(3)
    p = lpgen.permuted(lp, 1)
    assert p.nnz == lp.nnz and np.all(np.diff(p.row_ptr) >= 0)
    assert sorted(p.val.tolist()) == sorted(lp.val.tolist())
    t = oracle.kkt_terms(p, p.x_star, p.y_star)  # the planted pair, permuted, is still optimal
    assert t["rp"] < 1e-12 and t["rd"] < 1e-12 and abs(t["pobj"] - lp.obj_star) < 1e-10 * (1 + abs(lp.obj_star))
    # equality rows stay first
    assert p.n_eq == lp.n_eq and np.array_equal(np.sort(p.q[: p.n_eq]), np.sort(lp.q[: lp.n_eq]))


def test_batch_subset_builds_the_same_members():
    """A rank of a sharded batch builds only its LPs: each equals the member of
    the whole batch, and the expected work follows the realised nonzeros."""
    full = lpgen.batch_lps(10, seed=3)
    sub = lpgen.batch_subset([2, 5, 9], 10, seed=3)
    for i, lp in zip([2, 5, 9], sub):
        assert np.array_equal(lp.row_ptr, full[i].row_ptr) and np.array_equal(lp.col_idx, full[i].col_idx)
        assert np.array_equal(lp.val, full[i].val) and np.array_equal(lp.c, full[i].c)
    w = lpgen.batch_work(10, seed=3)
    assert np.corrcoef(w, [lp.nnz for lp in full])[0, 1] > 0.99


def test_large_lp_follows_its_recipe():
    """The 1e6 x 2e6 benchmark LP has the stated shape: 2e7 nonzeros within
    0.1 %, 40 % equality rows, Zipf(1.5) row lengths (the tail P(L >= 2d) /
    P(L >= d) of a Zipf(1.5) law is 2^-0.5; realised maximum ~910, mean 20),
    lognormal(0, 2) magnitudes with random signs, bounds 50 % [0, inf),
    30 % [l, u] with l in [-5, 0] and u in [0, 5], 20 % free; a valid CSR
    matrix (sorted, distinct columns per row) whose planted pair is a KKT
    point (b = A x*, c = K'y* + lambda*, complementary slackness)."""
    lp = lpgen.large_lp(0)
    m, n = lp.m, lp.n
    L = np.diff(lp.row_ptr)
    assert (m, n, lp.n_eq) == (1_000_000, 2_000_000, 400_000)
    assert abs(lp.nnz - 20_000_000) <= 20_000 and L.min() >= 1 and 800 <= L.max() <= 1000
    for d in (8, 16, 32, 64):
        assert abs((L >= 2 * d).sum() / (L >= d).sum() - 2 ** -0.5) < 0.02, d
    lv = np.log(np.abs(lp.val))
    assert abs(lv.mean()) < 0.01 and abs(lv.std() - 2.0) < 0.01 and abs((lp.val < 0).mean() - 0.5) < 0.002
    fl, fu = np.isfinite(lp.l), np.isfinite(lp.u)
    assert abs((fl & ~fu).mean() - 0.5) < 0.002 and np.all(lp.l[fl & ~fu] == 0)
    assert abs((fl & fu).mean() - 0.3) < 0.002 and abs((~fl & ~fu).mean() - 0.2) < 0.002
    assert not np.any(~fl & fu)
    box = fl & fu
    assert lp.l[box].min() >= -5 and lp.l[box].max() <= 0 and lp.u[box].min() >= 0 and lp.u[box].max() <= 5
    rows = np.repeat(np.arange(m), L)
    key = rows.astype(np.int64) * n + lp.col_idx
    assert np.all(np.diff(key) > 0) and lp.col_idx.min() >= 0 and lp.col_idx.max() < n
    # the planted pair, in plain numpy over the CSR arrays
    kx = np.bincount(rows, weights=lp.val * lp.x_star[lp.col_idx], minlength=m)
    kty = np.bincount(lp.col_idx, weights=lp.val * lp.y_star[rows], minlength=n)
    scale = 1.0 + np.abs(lp.q)
    assert np.all(np.abs(kx[:lp.n_eq] - lp.q[:lp.n_eq]) <= 1e-9 * scale[:lp.n_eq])
    assert np.all(kx[lp.n_eq:] - lp.q[lp.n_eq:] >= -1e-9 * scale[lp.n_eq:])
    assert np.all(lp.y_star[lp.n_eq:] >= 0)
    act = np.abs(kx[lp.n_eq:] - lp.q[lp.n_eq:]) * lp.y_star[lp.n_eq:]
    assert np.all(act <= 1e-9 * (1 + np.abs(lp.q[lp.n_eq:])))
    assert np.allclose(lp.c, kty + lp.lam_star, rtol=1e-12, atol=1e-9)
    assert np.all((lp.x_star >= lp.l) & (lp.x_star <= lp.u))
    assert np.all(lp.x_star[lp.lam_star > 0] == lp.l[lp.lam_star > 0])
    assert np.all(lp.x_star[lp.lam_star < 0] == lp.u[lp.lam_star < 0])


def test_batch_shapes_and_members_follow_their_recipe():
    """The 4096-LP batch: m log-uniform on [50, 4000], n / m log-uniform on
    [2/3, 2.5], density uniform on [0.5 %, 5 %] (about 2.8e8 expected
    nonzeros in all); sampled members have half equality rows, 0 <= x <= 10,
    N(0, 1) values, every row and column covered, and the density drawn."""
    import math

    count = 4096
    shapes = np.array(list(lpgen._batch_shapes(count, 0, 50, 4000, 0.005, 0.05)))
    m, n, d = shapes[:, 0], shapes[:, 1], shapes[:, 2]
    assert m.min() >= 50 and m.max() <= 4000
    u = (np.log(m) - math.log(50)) / (math.log(4000) - math.log(50))
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.std() - (1 / 12) ** 0.5) < 0.02
    r = np.log(n / m)
    assert r.min() >= math.log(2 / 3) - 0.02 and r.max() <= math.log(2.5) + 0.01
    assert abs(r.mean() - 0.5 * (math.log(2 / 3) + math.log(2.5))) < 0.02
    assert d.min() >= 0.005 and d.max() <= 0.05 and abs(d.mean() - 0.0275) < 0.001
    assert abs(lpgen.batch_work(count, 0).sum() / 2.8e8 - 1) < 0.02
    for i, lp in zip((0, 7, 2581), lpgen.batch_subset([0, 7, 2581], count, seed=0)):
        assert (lp.m, lp.n) == (m[i], n[i]) and lp.n_eq == lp.m // 2
        assert np.all(lp.l == 0) and np.all(lp.u == 10)
        assert np.all(np.diff(lp.row_ptr) >= 1) and np.unique(lp.col_idx).size == lp.n
        assert abs(lp.nnz / (lp.m * lp.n) - d[i]) < 0.3 * d[i] + 2.0 / lp.n
        assert abs(lp.val.mean()) < 0.2 and abs(lp.val.std() - 1) < 0.2


def test_transport_family_members_are_feasible_transportation_lps():
    """A member of the warm-start family is a transportation LP: each column
    x_ij appears once with +1 in sink j's equality row and once with -1 in
    source i's ">=" row; supplies and demands are at least the floor and
    total supply is 1.05 x total demand, so the proportional plan
    x_ij = s_i d_j / S meets every demand and uses 1 / 1.05 of each supply."""
    fam = lpgen.transport_family(0, sources=20, sinks=30)
    lp = lpgen.transport_lp(fam, lpgen.transport_thetas(1, 0)[0], 0)
    S, T = 20, 30
    assert (lp.m, lp.n, lp.n_eq) == (S + T, S * T, T)
    L = np.diff(lp.row_ptr)
    assert np.all(L[:T] == S) and np.all(L[T:] == T)
    rows = np.repeat(np.arange(lp.m), L)
    j, i = lp.col_idx % T, lp.col_idx // T  # column i * T + j: source i, sink j
    sink_part = rows < T
    assert np.all(j[sink_part] == rows[sink_part]) and np.all(lp.val[sink_part] == 1)
    assert np.all(i[~sink_part] == rows[~sink_part] - T) and np.all(lp.val[~sink_part] == -1)
    assert np.array_equal(np.sort(lp.col_idx[sink_part]), np.arange(S * T))
    d, s = lp.q[:T], -lp.q[T:]
    assert d.min() >= 0.05 and s.sum() == pytest.approx(1.05 * d.sum(), rel=1e-12)
    x = np.outer(s, d).ravel() / s.sum()
    kx = np.bincount(rows, weights=lp.val * x[lp.col_idx], minlength=lp.m)
    np.testing.assert_allclose(kx[:T], d, rtol=1e-12)
    assert np.all(kx[T:] >= lp.q[T:]) and np.all(lp.l == 0) and np.all(np.isinf(lp.u))


def test_nearly_dense_rows_still_get_distinct_columns():
    """A small power-law LP can draw a row as long as n (seed 4 below): its
    columns are still distinct and sorted, every row of the matrix too."""
    lp = lpgen.large_lp(4, m=300, n=600, nnz=3000)
    L = np.diff(lp.row_ptr)
    assert L.max() == lp.n
    rows = np.repeat(np.arange(lp.m), L)
    assert np.all(np.diff(rows.astype(np.int64) * lp.n + lp.col_idx) > 0)
    dense = int(np.argmax(L))
    assert np.array_equal(lp.col_idx[lp.row_ptr[dense]:lp.row_ptr[dense + 1]], np.arange(lp.n))
