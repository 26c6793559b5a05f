"""The per-check metrics ring (pdlp_get_trace) and host-side fault injection,
through the C ABI on the GPU.  Faults are made on the host only: a NaN
written into a saved solver state, or an input the create call rejects; no
test faults, traps or hangs the GPU."""

import numpy as np
import pytest

import lpgen
from paper_2311_12180_gb300 import pdlp as P

pytestmark = pytest.mark.gpu


def test_trace_ring_keeps_the_last_checks_in_order():
    """One check per accepted step (P = 1) for more steps than the ring holds:
    the records of the last TRACE_RETAINED checks come back oldest first,
    equal bit for bit to those of a shorter solve where they overlap."""
    lp = lpgen.tiny_lp(3)
    total = P.TRACE_RETAINED + 4000
    with P.Solver(lp, check_period=1) as a:
        _, _, st, it = a.solve(tol=0.0, max_iter=total)
        tr = a.trace()
        n_rec = a.checks_recorded()
    assert st == P.ITER_LIMIT and it == total
    assert n_rec == total - 1  # every check but the one that ends the solve
    assert len(tr) == P.TRACE_RETAINED
    np.testing.assert_array_equal(tr["k"], np.arange(total - P.TRACE_RETAINED, total))
    assert np.all(np.diff(tr["restarts"]) == (tr["restart"][1:] != 0))
    with P.Solver(lp, check_period=1) as b:
        _, _, st_b, _ = b.solve(tol=0.0, max_iter=5000)
        tb = b.trace()
    assert st_b == P.ITER_LIMIT and len(tb) == 4999
    k0 = int(tr["k"][0])
    assert tr[: 5000 - k0].tobytes() == tb[k0 - 1 :].tobytes()


def test_trace_metrics_are_those_of_the_returned_iterate():
    """A solve stopped by the iteration limit returns the current iterate of
    its last check: the longer solve's record at that k carries the same
    Sec. 4.1 measures as the oracle's evaluation of that iterate."""
    import oracle

    lp = lpgen.tiny_lp(4)
    with P.Solver(lp) as a:
        a.solve(tol=0.0, max_iter=640)
        tr = a.trace()
    rec = tr[tr["k"] == 384][0]
    with P.Solver(lp) as b:
        x, y, st, it = b.solve(tol=0.0, max_iter=384)
        info = b.info()
    assert st == P.ITER_LIMIT and it == 384 and info["attempts"] == rec["attempts"]
    t = oracle.kkt_terms(lp, x, y)
    gap = abs(t["pobj"] - t["dobj"]) / (1.0 + abs(t["pobj"]) + abs(t["dobj"]))
    want = [gap, t["rp"] / (1.0 + t["q_norm"]), t["rd"] / (1.0 + t["c_norm"])]
    np.testing.assert_allclose([rec["rel_gap"], rec["rel_primal"], rec["rel_dual"]], want, rtol=1e-8, atol=1e-14)


def _vector_offset(blob, lp, which, j):
    """Byte offset of entry j of one exported state vector: the state ends
    with six n-vectors (x first) and five m-vectors (y first), in the
    original order."""
    start = len(blob) - 8 * (6 * lp.n + 5 * lp.m)
    return start + (0 if which == "x" else 8 * 6 * lp.n) + 8 * j


@pytest.mark.parametrize("where", ["x", "y"])
def test_nan_injected_into_the_state_ends_with_numerical_error(where):
    """A NaN written into the saved iterate on the host: the next step test
    sees a non-finite ||dx||^2 or ||dy||^2 and the solve ends with
    PDLP_NUMERICAL; the same state without the NaN resumes normally."""
    lp = lpgen.tiny_lp(2)
    with P.Solver(lp, check_period=8) as s:
        s.begin(tol=1e-6)
        s.run_periods(2)
        s.poll()
        blob = s.get_state()
        bad = bytearray(blob)
        off = _vector_offset(blob, lp, where, 3)
        bad[off:off + 8] = np.array([np.nan]).tobytes()
        s.set_state(bytes(bad))
        _, _, st, _ = s.resume()
        assert st == P.NUMERICAL
        s.set_state(blob)
        _, _, st2, _ = s.resume()
        assert st2 == P.OPTIMAL
