"""Batched solver (one persistent launch, one CTA per LP) against the FP64
oracle, LP by LP, on the same seeded inputs."""

import numpy as np
import pytest

import lpgen
import oracle
from paper_2311_12180_gb300 import pdlp as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    lps = lpgen.batch_lps(24, seed=3, m_lo=20, m_hi=400)
    # edge cases: all equalities, all inequalities, no constraint rows
    lps.append(lpgen.tiny_lp(31, m_eq=60, m_ineq=0, n=150))
    lps.append(lpgen.tiny_lp(32, m_eq=0, m_ineq=60, n=150))
    # large enough (72k nonzeros) to be solved by a team of CTAs (threshold 32768)
    lps.append(lpgen.tiny_lp(41, m_eq=600, m_ineq=600, n=3000, density=0.02))
    rng = np.random.default_rng(9)
    n = 40
    lps.append(lpgen.LP(m=0, n=n, n_eq=0, c=rng.standard_normal(n), row_ptr=np.zeros(1, np.int32),
                        col_idx=np.zeros(0, np.int32), val=np.zeros(0), q=np.zeros(0), l=np.full(n, -1.0),
                        u=np.full(n, 2.0)))
    return lps


def test_batch_solutions_match_oracle(batch):
    with P.BatchSolver(batch) as b:
        xs, ys, st, it = b.solve(tol=1e-6)
        # both schedules run: LPs solved from shared memory and from global memory
        assert 0 < b.stats()["resident"] < len(batch)
        assert b.stats()["team_lps"] == 1
        stats = b.stats()
        lk, lt = b.lanes()
    assert stats["count"] == len(batch) and stats["entries_per_lane"] in (4.0, 8.0, 16.0)
    assert set(np.unique(np.concatenate([lk, lt]))) <= {1, 2, 4, 8, 16, 32}
    for i, lp in enumerate(batch):
        assert st[i] == P.OPTIMAL, i
        assert oracle.passes(lp, xs[i], ys[i], 1e-6), i
        assert np.all(xs[i] >= lp.l) and np.all(xs[i] <= lp.u)
        assert np.all(ys[i][lp.n_eq:] >= 0)
        r = oracle.solve(lp, tol=1e-6)
        obj = float(lp.c @ xs[i])
        assert abs(obj - r.pobj) <= 4e-6 * (1 + abs(r.pobj)), i
        if lp.obj_star is not None:
            assert abs(obj - lp.obj_star) <= 4e-6 * (1 + abs(lp.obj_star)), i


def test_batch_iterates_match_oracle(batch):
    """Short horizon (identical accept / restart decisions): every LP's
    iterate after 40 accepted steps equals the oracle's to rounding."""
    N = 40
    with P.BatchSolver(batch) as b:
        xs, ys, st, it = b.solve(tol=1e-14, max_iter=N)
    for i, lp in enumerate(batch):
        r = oracle.solve(lp, tol=1e-14, max_iter=N)
        assert st[i] == r.status and it[i] == r.iters <= N, i
        np.testing.assert_allclose(xs[i], r.x, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.x).max()), err_msg=str(i))
        if lp.m:
            np.testing.assert_allclose(ys[i], r.y, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(r.y).max()),
                                       err_msg=str(i))


def test_batch_deterministic_and_warm_start(batch):
    with P.BatchSolver(batch[:8]) as b:
        a = b.solve(tol=1e-6)
        c = b.solve(tol=1e-6)
        assert all(np.array_equal(u, v) for u, v in zip(a[0], c[0])) and np.array_equal(a[3], c[3])
        lps = batch[:8]
        w = b.solve(tol=1e-10, x0=[lp.x_star for lp in lps], y0=[lp.y_star for lp in lps])
    assert np.all(w[2] == P.OPTIMAL) and np.all(w[3] == 64)
    for i, lp in enumerate(lps):
        assert oracle.relative_kkt(lp, w[0][i], w[1][i]) < 1e-10


def test_batch_matches_single_instance_solver(batch):
    lps = batch[:4]
    with P.BatchSolver(lps) as b:
        xs, ys, st, it = b.solve(tol=1e-8)
    for i, lp in enumerate(lps):
        with P.Solver(lp) as s:
            x, y, s1, i1 = s.solve(tol=1e-8)
        assert st[i] == s1 == P.OPTIMAL
        assert float(lp.c @ xs[i]) == pytest.approx(float(lp.c @ x), rel=1e-6)


def test_batch_times_describe_the_schedule(batch):
    import time

    with P.BatchSolver(batch) as b:
        b.solve(tol=1e-6, max_iter=2)
        t = time.perf_counter()
        b.solve(tol=1e-6)
        wall = time.perf_counter() - t
        t0, t1 = b.times()
    assert t0.min() == 0.0
    assert np.all(t1 >= t0) and t1.max() <= wall


def test_team_barrier_timeout_is_reported_and_context_survives(batch, monkeypatch):
    # a team member that never arrives: its teammates give up after 2 s, the
    # call fails with an error, and the next solve on the same batch is normal
    with P.BatchSolver(batch) as b:
        ok = b.solve(tol=1e-6)
        monkeypatch.setenv("PDLP_TEST_TEAM_STALL", "1")
        with pytest.raises(P.PdlpError) as e:
            b.solve(tol=1e-6)
        assert "timed out" in str(e.value)
        monkeypatch.delenv("PDLP_TEST_TEAM_STALL")
        again = b.solve(tol=1e-6)
    assert np.array_equal(ok[2], again[2]) and np.array_equal(ok[3], again[3])
    assert all(np.array_equal(a, c) for a, c in zip(ok[0], again[0]))


_SUBPROCESS_SOLVE = """
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import lpgen
from paper_2311_12180_gb300 import pdlp as P
lps = lpgen.batch_lps(24, seed=3, m_lo=20, m_hi=400)
lps.append(lpgen.tiny_lp(41, m_eq=600, m_ineq=600, n=3000, density=0.02))
with P.BatchSolver(lps) as b:
    xs, ys, st, it = b.solve(tol=1e-6)
np.savez(sys.argv[2], x=np.concatenate(xs), y=np.concatenate(ys), st=st, it=it)
"""


def test_batch_results_do_not_depend_on_schedule_create_or_process(batch, monkeypatch, tmp_path):
    """Row sums have one order for every lanes-per-row choice, so the
    autotuned schedule (timing-dependent, redone at every create) changes
    speed only: every forced schedule, a second create and a second process
    give bitwise the same iterates and iteration counts."""
    import os
    import subprocess
    import sys

    lps = batch[:24] + [batch[26]]  # the subprocess builds the same list
    runs = []
    for target in (None, "4", "8", "16"):
        if target:
            monkeypatch.setenv("PDLP_TEST_BATCH_TARGET", target)
        else:
            monkeypatch.delenv("PDLP_TEST_BATCH_TARGET", raising=False)
        with P.BatchSolver(lps) as b:
            runs.append((b.solve(tol=1e-6), b.lanes()))
    monkeypatch.delenv("PDLP_TEST_BATCH_TARGET", raising=False)
    ref = runs[0][0]
    lanes = {tuple(np.concatenate(r[1])) for r in runs}
    assert len(lanes) >= 3  # the forced schedules really differ
    for (xs, ys, st, it), _ in runs[1:]:
        assert np.array_equal(st, ref[2]) and np.array_equal(it, ref[3])
        assert all(np.array_equal(u, v) for u, v in zip(xs, ref[0]))
        assert all(np.array_equal(u, v) for u, v in zip(ys, ref[1]))
    out = tmp_path / "batch.npz"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([sys.executable, "-c", _SUBPROCESS_SOLVE, root, str(out)], check=True, timeout=600)
    other = np.load(out)
    assert np.array_equal(other["st"], ref[2]) and np.array_equal(other["it"], ref[3])
    assert np.array_equal(other["x"], np.concatenate(ref[0])) and np.array_equal(other["y"], np.concatenate(ref[1]))
