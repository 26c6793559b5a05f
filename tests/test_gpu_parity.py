"""GPU parity: the CUDA solver (through the C ABI) against the FP64 CPU
oracle on the same seeded inputs.

Tolerances (derived from the arithmetic, not tuned):
  * Scaling: the Ruiz passes are max / sqrt / divide -- exact and correctly
    rounded on both sides -- so only the Pock-Chambolle row / column sums differ
    in summation order: |D1, D2, K~| agree to a few ulps (rtol 1e-13).
  * Iterates after N steps with identical accept / restart decisions: both
    sides compute the same formulas in FP64; summation order and FMA
    contraction differ, so every step adds O(1e-16) relative noise and PDHG
    is non-expansive: rtol 1e-9 with an absolute floor of 1e-9 * max|x|.
  * Solutions: the optimum need not be unique, so vectors are never compared
    after convergence; the objective must match the oracle's to 1e-6 relative
    at tol = 1e-8 (a tol-eps solution's objective is only fixed to
    eps * (1 + |obj|)), and the oracle's own Sec. 4.1 evaluation of the GPU's
    (x, y) must pass the requested tolerance.
"""

import numpy as np
import pytest

import lpgen
import oracle
from paper_2311_12180_gb300 import pdlp as P

pytestmark = pytest.mark.gpu


def _solver(lp, **kw):
    return P.Solver(lp, **kw)


def _oracle(lp, **kw):
    return oracle.solve(lp, **kw)


def _assert_feasible_signs(lp, x, y):
    assert np.all(x >= lp.l) and np.all(x <= lp.u)
    assert np.all(y[lp.n_eq:] >= 0)


# ---------------------------------------------------------------- scaling


@pytest.mark.parametrize("seed", [0, 1])
def test_scaling_matches_oracle(seed):
    lp = lpgen.large_lp(seed, m=3000, n=6000, nnz=60000)
    with _solver(lp) as s:
        D1, D2, v = s.scaling()
    sv, oD1, oD2 = oracle.precondition(lp, ruiz_iters=10, pc_alpha=1.0)
    np.testing.assert_allclose(D1, oD1, rtol=1e-13)
    np.testing.assert_allclose(D2, oD2, rtol=1e-13)
    np.testing.assert_allclose(v, sv, rtol=1e-13)


@pytest.mark.parametrize("case", ["tiny", "powerlaw"])
def test_ruiz_only_scaling_is_bitwise(case):
    """Ten Ruiz passes: every entry divided twice per pass, on the GPU by a
    reciprocal and one correction step (correctly rounded) and in the oracle by
    plain division: bitwise equal on 2e3 and on 4e5 lognormal entries."""
    lp = lpgen.tiny_lp(3) if case == "tiny" else lpgen.large_lp(4, m=20000, n=40000, nnz=400000)
    with _solver(lp, pc_alpha=-1.0) as s:
        D1, D2, v = s.scaling()
    sv, oD1, oD2 = oracle.precondition(lp, ruiz_iters=10, pc_alpha=-1.0)
    assert np.array_equal(D1, oD1) and np.array_equal(D2, oD2) and np.array_equal(v, sv)


# ---------------------------------------------------------------- iterates


@pytest.mark.parametrize("case,P_,N", [("tiny", 64, 40), ("tiny", 1, 12), ("tiny", 8, 130), ("powerlaw", 64, 30)])
def test_iterates_match_oracle(case, P_, N):
    lp = lpgen.tiny_lp(5) if case == "tiny" else lpgen.large_lp(4, m=20000, n=40000, nnz=400000)
    with _solver(lp, check_period=P_) as s:
        x, y, st, it = s.solve(tol=1e-14, max_iter=N)
        tr = s.trace()
        info = s.info()
    r = _oracle(lp, tol=1e-14, max_iter=N, check_period=P_)
    assert st == P.ITER_LIMIT == r.status and it == N == r.iters
    assert info["attempts"] == r.attempts and info["restarts"] == r.restarts
    assert len(tr) == len(r.trace)
    np.testing.assert_array_equal(tr["k"], r.trace["k"])
    np.testing.assert_array_equal(tr["restart"], r.trace["restart"])
    np.testing.assert_array_equal(tr["attempts"], r.trace["attempts"])
    np.testing.assert_array_equal(tr["restarts"], r.trace["restarts"])
    # GetRestartCandidate is decided by KKT(current) < KKT(average); where the
    # two agree to rounding (e.g. t = 1, when the average is the current
    # iterate up to (1/eta)(eta x)), both candidates are the same point and
    # either choice is correct, so only distinguishable cases are compared
    tie = np.abs(r.trace["kkt_cur"] - r.trace["kkt_avg"]) <= 1e-12 * np.maximum(r.trace["kkt_cur"], r.trace["kkt_avg"])
    np.testing.assert_array_equal(tr["cand_avg"][~tie], r.trace["cand_avg"][~tie])
    for f in ("kkt_cur", "kkt_avg", "kkt_start", "omega", "eta_hat", "rel_gap", "rel_primal", "rel_dual"):
        np.testing.assert_allclose(tr[f], r.trace[f], rtol=1e-9, err_msg=f)
    np.testing.assert_allclose(x, r.x, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.x).max()))
    np.testing.assert_allclose(y, r.y, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.y).max()))


def _long_column_lp(seed, longest):
    """K whose columns run from 1 entry to `longest`: columns of at most 32
    entries, of 33..4096 entries and (longest > 4096) longer ones, with K's
    rows drawn per column, so that the stable transpose sorts every kind."""
    rng = np.random.default_rng(seed)
    m, n = longest + 300, 260
    lens = np.concatenate([rng.integers(1, 33, 200), rng.integers(33, 600, 50), [1000, 2048, 3000, 4095, 4096],
                           rng.integers(100, 300, 4), [longest]])
    cp, rows = lpgen._sample_rows(rng, lens, m)  # K' pattern: row j holds column j's rows
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(cp))
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    row_ptr, cols = lpgen._cover_columns(rng, row_ptr, cols, m, n)
    assert np.all(np.diff(row_ptr) > 0), "every row needs an entry"
    val = rng.standard_normal(cols.size)
    return lpgen.plant(rng, m, n, m // 3, row_ptr, cols, val, np.zeros(n), np.full(n, 10.0))


@pytest.mark.parametrize("longest", [4096, 5000])
def test_long_columns_match_oracle(longest):
    # 4096: K' built on the device (every column sorted there); 5000: one
    # column too long for the per-column device sort, K' built on the host
    lp = _long_column_lp(31, longest)
    assert np.bincount(lp.col_idx, minlength=lp.n).max() == longest
    with _solver(lp) as s:
        D1, D2, v = s.scaling()
    sv, oD1, oD2 = oracle.precondition(lp, ruiz_iters=10, pc_alpha=1.0)
    np.testing.assert_allclose(D1, oD1, rtol=1e-13)
    np.testing.assert_allclose(D2, oD2, rtol=1e-13)
    np.testing.assert_allclose(v, sv, rtol=1e-13)
    N = 40
    with _solver(lp, check_period=8) as s:
        x, y, st, it = s.solve(tol=1e-14, max_iter=N)
    r = _oracle(lp, tol=1e-14, max_iter=N, check_period=8)
    assert it == N == r.iters
    np.testing.assert_allclose(x, r.x, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.x).max()))
    np.testing.assert_allclose(y, r.y, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.y).max()))


def test_deterministic():
    lp = lpgen.large_lp(6, m=20000, n=40000, nnz=400000)
    with _solver(lp) as s:
        a = s.solve(tol=1e-12, max_iter=300)
        b = s.solve(tol=1e-12, max_iter=300)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[3] == b[3]


# ---------------------------------------------------------------- solutions


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_solution_parity(seed):
    lp = lpgen.tiny_lp(seed)
    r4 = _oracle(lp, tol=1e-4)
    r8 = _oracle(lp, tol=1e-8)
    with _solver(lp) as s:
        x4, y4, st4, it4 = s.solve(tol=1e-4)
        x8, y8, st8, it8 = s.solve(tol=1e-8)
        info8 = s.info()
    assert st4 == st8 == P.OPTIMAL
    assert oracle.passes(lp, x4, y4, 1e-4) and oracle.passes(lp, x8, y8, 1e-8)
    _assert_feasible_signs(lp, x8, y8)
    obj8 = float(lp.c @ x8)
    assert abs(obj8 - r8.pobj) <= 1e-6 * abs(r8.pobj)
    assert abs(obj8 - lp.obj_star) <= 1e-6 * abs(lp.obj_star)
    assert abs(float(lp.c @ x4) - r4.pobj) <= 2e-4 * (1 + abs(r4.pobj))
    # Restart / termination decisions compare FP64 values that can tie to
    # rounding (candidate choice at t = 1, a relative KKT error at tol), so
    # long runs may take different decision paths on the two sides; the
    # iteration counts must still agree to within a factor of two (a broken
    # restart or step rule shows up as a much larger gap).
    for a, b in ((it4, r4.iters), (it8, r8.iters)):
        assert a <= 2 * b + 128 and b <= 2 * a + 128
    assert info8["pobj"] == pytest.approx(obj8, rel=1e-9)


@pytest.mark.parametrize("case", ["all_eq", "all_ineq", "no_rows", "free_vars", "long_rows", "empty_lines",
                                  "ragged_tiles"])
def test_edge_cases(case):
    rng = np.random.default_rng(17)
    if case == "all_eq":
        lp = lpgen.tiny_lp(21, m_eq=150, m_ineq=0, n=400)
    elif case == "all_ineq":
        lp = lpgen.tiny_lp(22, m_eq=0, m_ineq=150, n=400)
    elif case == "no_rows":
        n = 300
        c = rng.standard_normal(n)
        lp = lpgen.LP(m=0, n=n, n_eq=0, c=c, row_ptr=np.zeros(1, np.int32), col_idx=np.zeros(0, np.int32),
                      val=np.zeros(0), q=np.zeros(0), l=rng.uniform(-2, 0, n), u=rng.uniform(0, 2, n))
    elif case == "free_vars":
        lp = lpgen.large_lp(23, m=400, n=800, nnz=6000)  # 20 % free, 50 % [0, inf)
    elif case == "long_rows":
        # rows far beyond the 48-entry slice limit (one warp each, up to 157
        # strides of 32 entries) next to short ones
        m, n = 40, 12000
        lens = np.array([1, 2, 5000, 3, 2500, 1] + [40] * (m - 6))
        row_ptr, cols = lpgen._sample_rows(rng, lens, n)
        row_ptr, cols = lpgen._cover_columns(rng, row_ptr, cols, m, n)
        val = rng.standard_normal(cols.size)
        lp = lpgen.plant(rng, m, n, 20, row_ptr, cols, val, np.zeros(n), np.full(n, 10.0))
    elif case == "empty_lines":
        # an empty ">=" row with q <= 0 and empty columns (variables only in c)
        base = lpgen.tiny_lp(24, m_eq=60, m_ineq=60, n=300)
        m, n = base.m + 1, base.n + 7
        row_ptr = np.concatenate([base.row_ptr, [base.row_ptr[-1]]]).astype(np.int32)
        c = np.concatenate([base.c, rng.uniform(0.5, 1.0, 7)])
        q = np.concatenate([base.q, [-1.0]])
        lp = lpgen.LP(m=m, n=n, n_eq=base.n_eq, c=c, row_ptr=row_ptr, col_idx=base.col_idx, val=base.val, q=q,
                      l=np.concatenate([base.l, np.zeros(7)]), u=np.concatenate([base.u, np.full(7, 3.0)]))
    else:  # sizes that leave a ragged last slice of 32 rows on both sides
        lp = lpgen.tiny_lp(25, m_eq=257, m_ineq=300, n=2049, density=0.004)
    r = _oracle(lp, tol=1e-8, max_iter=200000)
    assert r.status == oracle.OPTIMAL
    with _solver(lp) as s:
        x, y, st, it = s.solve(tol=1e-8, max_iter=200000)
    assert st == P.OPTIMAL
    assert oracle.passes(lp, x, y, 1e-8)
    _assert_feasible_signs(lp, x, y)
    assert abs(float(lp.c @ x) - r.pobj) <= 1e-6 * (1 + abs(r.pobj))


def test_warm_start_at_planted_optimum():
    lp = lpgen.tiny_lp(4)
    with _solver(lp, check_period=8) as s:
        x, y, st, it = s.solve(tol=1e-12, x0=lp.x_star, y0=lp.y_star)
    assert st == P.OPTIMAL and it == 8
    assert oracle.relative_kkt(lp, x, y) < 1e-12


def test_limits_and_info():
    lp = lpgen.tiny_lp(6)
    with _solver(lp, check_period=16) as s:
        x, y, st, it = s.solve(tol=1e-14, max_iter=100)
        inf = s.info()
        assert st == P.ITER_LIMIT and it == 100
        assert inf["status"] == P.ITER_LIMIT and inf["iters"] == 100
        assert inf["attempts"] >= 100 and inf["checks"] >= 6
        assert inf["graph_launches"] >= 7
        assert s.device_bytes() > 0 and s.stream != 0
    big = lpgen.large_lp(7, m=20000, n=40000, nnz=400000)
    with _solver(big, time_limit_s=0.05) as s:
        x, y, st, it = s.solve(tol=1e-14, max_iter=10**9)
    assert st == P.TIME_LIMIT and it > 0


def test_async_pieces_match_blocking_solve():
    lp = lpgen.tiny_lp(8)
    with _solver(lp) as s:
        xa, ya, sa, ia = s.solve(tol=1e-6)
        s.begin(tol=1e-6)
        for _ in range(10000):
            s.run_periods(4)
            st, k = s.poll()
            if st != -1:
                break
        xb, yb, sb, ib = s.finish()
    assert sa == sb == P.OPTIMAL and ia == ib
    assert np.array_equal(xa, xb) and np.array_equal(ya, yb)


def test_kernel_timing_mode_runs_same_arithmetic():
    lp = lpgen.tiny_lp(9)
    with _solver(lp) as s:
        x1, y1, s1, i1 = s.solve(tol=1e-12, max_iter=256)
        s.begin(tol=1e-12, max_iter=256)
        t = s.time_kernels(4)
        x2, y2, s2, i2 = s.finish()
    assert i1 == i2 == 256 and np.array_equal(x1, x2) and np.array_equal(y1, y2)
    assert t["k_primal"][1] + t["k_primal_reuse_g"][1] >= 256 and t["k_dual"][1] >= 256
    assert t["k_check_dual"][1] == 4
    assert all(v[0] >= 0 for v in t.values())


# ---------------------------------------------------------------- full-size workload


@pytest.mark.slow
def test_full_size_iterates_match_oracle():
    """The 1e6 x 2e6, nnz 2e7 power-law LP in the benchmark's launch
    configuration: 20 PDHG steps on the GPU against the oracle, elementwise."""
    lp = lpgen.large_lp(0)
    N = 20
    with _solver(lp) as s:
        x, y, st, it = s.solve(tol=1e-14, max_iter=N)
        tr = s.trace()
    r = _oracle(lp, tol=1e-14, max_iter=N)
    assert st == r.status == P.ITER_LIMIT and it == r.iters == N
    np.testing.assert_allclose(x, r.x, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.x).max()))
    np.testing.assert_allclose(y, r.y, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.y).max()))
    assert len(tr) == len(r.trace)


# ---------------------------------------------------------------- FP32-values mode


@pytest.mark.parametrize("seed", [0, 1])
def test_fp32_values_solution_parity(seed):
    """K values stored FP32 for the step kernels (gathers, accumulation and
    iterates FP64); termination is evaluated with the FP64 K, so the returned
    point must pass the oracle's FP64 Sec. 4.1 test at the requested tol."""
    lp = lpgen.tiny_lp(seed)
    r8 = _oracle(lp, tol=1e-8)
    with _solver(lp, value_bits=32) as s:
        x6, y6, st6, it6 = s.solve(tol=1e-6)
        x8, y8, st8, it8 = s.solve(tol=1e-8)
        info = s.info()
    assert st6 == st8 == P.OPTIMAL
    assert oracle.passes(lp, x6, y6, 1e-6) and oracle.passes(lp, x8, y8, 1e-8)
    _assert_feasible_signs(lp, x8, y8)
    assert abs(float(lp.c @ x8) - r8.pobj) <= 1e-6 * abs(r8.pobj)
    assert abs(float(lp.c @ x6) - lp.obj_star) <= 2e-6 * (1 + abs(lp.obj_star))
    assert info["f64_switch_iter"] == -1 or 0 < info["f64_switch_iter"] <= it8


def test_fp32_values_with_entries_below_the_float_range():
    """Entries far below the smallest normal float (1e-42 and -3e-45 next to
    O(1) ones) become signed zeros in the FP32 copy the step kernels read; the
    solve still meets tol on the FP64 LP (termination uses the FP64 K) and
    matches the oracle's objective on the same LP."""
    lp = lpgen.tiny_lp(6)
    lp.val = lp.val.copy()
    lp.val[[5, 17]] = [1e-42, -3e-45]
    r8 = _oracle(lp, tol=1e-8)
    with _solver(lp, value_bits=32) as s:
        x8, y8, st8, _ = s.solve(tol=1e-8)
    assert st8 == P.OPTIMAL and r8.status == P.OPTIMAL
    assert oracle.passes(lp, x8, y8, 1e-8)
    assert abs(float(lp.c @ x8) - r8.pobj) <= 1e-6 * (1 + abs(r8.pobj))


@pytest.mark.parametrize("case,N", [("tiny", 60), ("powerlaw", 60)])
def test_fp32_values_iterates_match_the_oracles_fp32_steps(case, N):
    """X1 against the oracle's FP32-values mode of the steps (K~ rounded to
    FP32 in Algorithm 2's products, FP64 everywhere else) before the first
    restart / termination check: the same trials and the same iterates
    elementwise, as in the FP64 parity test."""
    lp = lpgen.tiny_lp(5) if case == "tiny" else lpgen.large_lp(4, m=20000, n=40000, nnz=400000)
    with _solver(lp, check_period=64, value_bits=32) as s:
        x, y, st, it = s.solve(tol=1e-14, max_iter=N)
        info = s.info()
    r = _oracle(lp, tol=1e-14, max_iter=N, check_period=64, step_value_bits=32)
    r64 = _oracle(lp, tol=1e-14, max_iter=N, check_period=64)
    assert st == P.ITER_LIMIT == r.status and it == N == r.iters
    assert info["attempts"] == r.attempts
    np.testing.assert_allclose(x, r.x, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.x).max()))
    np.testing.assert_allclose(y, r.y, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.y).max()))
    # the FP32 rounding of the matrix is visible at this tolerance: the FP64
    # method's iterates are elsewhere
    assert np.abs(y - r64.y).max() > 1e-7 * max(1.0, np.abs(r64.y).max())


def test_fp32_values_first_steps_track_fp64():
    """Before any restart decision can differ, the FP32-valued steps follow
    the FP64 trajectory to within the FP32 rounding of the matrix (2^-24
    relative per value)."""
    lp = lpgen.large_lp(4, m=20000, n=40000, nnz=400000)
    with _solver(lp) as a, _solver(lp, value_bits=32) as b:
        xa, ya, _, _ = a.solve(tol=1e-14, max_iter=10)
        xb, yb, _, _ = b.solve(tol=1e-14, max_iter=10)
    sx = max(1.0, np.abs(xa).max())
    sy = max(1.0, np.abs(ya).max())
    assert np.abs(xa - xb).max() <= 1e-5 * sx and np.abs(ya - yb).max() <= 1e-5 * sy
    assert np.abs(xa - xb).max() > 0  # the FP32 copy is really in use
