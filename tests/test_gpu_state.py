"""Checkpoint / resume of Algorithm 1's state (pdlp_get_state, pdlp_set_state,
pdlp_resume) and the device-pointer create (pdlp_create_device), through the
C ABI on the GPU: both must reproduce the plain host path bit for bit."""

import numpy as np
import pytest

import lpgen
from paper_2311_12180_gb300 import pdlp as P

pytestmark = pytest.mark.gpu


def _powerlaw():
    return lpgen.large_lp(4, m=20000, n=40000, nnz=400000)


def test_resume_after_moving_the_state_is_bitwise():
    lp = _powerlaw()
    total, first = 64 * 14, 6  # iterations of the whole solve; graph periods before the checkpoint
    with P.Solver(lp) as a:
        x_ref, y_ref, st_ref, it_ref = a.solve(tol=1e-14, max_iter=total)
        info_ref = a.info()
        trace_ref = a.trace()
    assert st_ref == P.ITER_LIMIT and it_ref == total
    with P.Solver(lp) as b:
        b.begin(tol=1e-14, max_iter=total)
        b.run_periods(first)
        st, k = b.poll()
        assert st == -1 and 0 < k < total
        blob = b.get_state()
    # restarts happened both before and after the checkpoint
    ks = trace_ref["k"][trace_ref["restart"] != 0]
    assert (ks <= k).any() and (ks > k).any()
    with P.Solver(lp) as c:  # a fresh solver of the same LP
        c.set_state(blob)
        x, y, st2, it2 = c.resume()
        info = c.info()
    assert st2 == st_ref and it2 == it_ref
    assert np.array_equal(x, x_ref) and np.array_equal(y, y_ref)
    assert info["restarts"] == info_ref["restarts"] and info["attempts"] == info_ref["attempts"]
    assert info["omega"] == info_ref["omega"] and info["eta_hat"] == info_ref["eta_hat"]


def test_state_round_trip_in_place_and_to_optimality():
    lp = lpgen.tiny_lp(2)
    with P.Solver(lp, check_period=8) as a:
        x_ref, y_ref, st_ref, it_ref = a.solve(tol=1e-6)
    assert st_ref == P.OPTIMAL
    with P.Solver(lp, check_period=8) as b:
        b.begin(tol=1e-6)
        b.run_periods(3)
        b.poll()
        blob = b.get_state()
        b.run_periods(5)  # move on, then go back to the checkpoint on the same solver
        b.poll()
        b.set_state(blob)
        assert b.get_state() == blob
        x, y, st, it = b.resume()
    assert (st, it) == (st_ref, it_ref)
    assert np.array_equal(x, x_ref) and np.array_equal(y, y_ref)


def test_state_rejects_other_lp_and_sizes():
    a_lp, b_lp = lpgen.tiny_lp(1), lpgen.tiny_lp(2)
    with P.Solver(a_lp) as a, P.Solver(b_lp) as b, P.Solver(a_lp, check_period=16) as c:
        a.begin(tol=1e-6)
        blob = a.get_state()
        for target, data in ((b, blob), (c, blob), (a, blob[:-8]), (a, b"\0" * len(blob))):
            with pytest.raises(P.PdlpError) as e:
                target.set_state(data)
            assert e.value.code == P.ERR_INVALID


def _device_arrays(lp, torch):
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    keep = dict(c=t(lp.c, torch.float64), row_ptr=t(lp.row_ptr, torch.int32), col_idx=t(lp.col_idx, torch.int32),
                val=t(lp.val, torch.float64), q=t(lp.q if lp.m else np.zeros(1), torch.float64),
                l=t(lp.l, torch.float64), u=t(lp.u, torch.float64))
    return keep, {k: v.data_ptr() for k, v in keep.items()}


class _Dims:
    def __init__(self, lp):
        self.m, self.n, self.n_eq, self.nnz = lp.m, lp.n, lp.n_eq, int(lp.row_ptr[-1])
        self.row_ptr = None


@pytest.mark.parametrize("case", ["tiny", "powerlaw", "fp32"])
def test_device_create_matches_host_create_bitwise(case):
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    lp = lpgen.tiny_lp(3) if case == "tiny" else _powerlaw()
    kw = dict(value_bits=32) if case == "fp32" else {}
    tol, max_iter = (1e-6, 100000) if case == "tiny" else (1e-14, 640)
    with P.Solver(lp, **kw) as a:
        xa, ya, sa, ia = a.solve(tol=tol, max_iter=max_iter)
        scal_a = a.scaling()
    keep, ptrs = _device_arrays(lp, torch)
    torch.cuda.synchronize()
    with P.Solver(_Dims(lp), device=ptrs, **kw) as b:
        del keep  # the solver holds its own copies
        xb, yb, sb, ib = b.solve(tol=tol, max_iter=max_iter)
        scal_b = b.scaling()
    assert (sa, ia) == (sb, ib)
    assert np.array_equal(xa, xb) and np.array_equal(ya, yb)
    assert all(np.array_equal(u, v) for u, v in zip(scal_a, scal_b))


@pytest.mark.parametrize("defect", ["col_range", "nan_val", "row_ptr_order", "bad_bound"])
def test_device_create_rejects_bad_input(defect):
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    lp = lpgen.tiny_lp(0)
    lp.col_idx, lp.val, lp.row_ptr, lp.l = lp.col_idx.copy(), lp.val.copy(), lp.row_ptr.copy(), lp.l.copy()
    if defect == "col_range":
        lp.col_idx[17] = lp.n
    elif defect == "nan_val":
        lp.val[5] = np.nan
    elif defect == "row_ptr_order":
        lp.row_ptr[3] = lp.row_ptr[4] + 1
    else:
        lp.l[4] = np.inf
    keep, ptrs = _device_arrays(lp, torch)
    torch.cuda.synchronize()
    with pytest.raises(P.PdlpError) as e:
        P.Solver(_Dims(lp), device=ptrs)
    assert e.value.code == P.ERR_INVALID
    if defect in ("col_range", "nan_val"):
        assert str(17 if defect == "col_range" else 5) in str(e.value)
    del keep


def test_probe_rates_are_ordered():
    """The roofline probes: random gathers alone, and with an SpMV's index and
    value stream beside them (more bytes per gather, so no faster), and the
    FP64 FMA rate, all positive and finite on this GPU."""
    g, f = P.probe_rates()
    gs = P.probe_stream_gathers()
    assert np.isfinite(g) and np.isfinite(gs) and np.isfinite(f)
    assert g > 0 and gs > 0 and f > 0
    assert gs <= 1.05 * g
