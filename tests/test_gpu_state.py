"""Checkpoint / resume of Algorithm 1's state (pdlp_get_state, pdlp_set_state,
pdlp_resume) and the device-pointer create (pdlp_create_device), through the
C ABI on the GPU: both must reproduce the plain host path bit for bit."""

import ctypes as C

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
        c_trace = c.trace()
    assert st2 == st_ref and it2 == it_ref
    assert np.array_equal(x, x_ref) and np.array_equal(y, y_ref)
    assert info["restarts"] == info_ref["restarts"] and info["attempts"] == info_ref["attempts"]
    assert info["omega"] == info_ref["omega"] and info["eta_hat"] == info_ref["eta_hat"]
    # the trace is not part of the state: the new solver holds the checks
    # made after the load, equal to the uninterrupted solve's
    tr = trace_ref[trace_ref["k"] > k]
    assert len(tr) > 0 and c_trace.tobytes() == tr.tobytes()


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


class _Header(C.Structure):
    """The blob's header as pdlp_get_state writes it (host layout)."""

    _fields_ = [("magic", C.c_uint64), ("version", C.c_uint32), ("m", C.c_int32), ("n", C.c_int32),
                ("check_period", C.c_int32), ("value_bits", C.c_int32), ("pad", C.c_int32), ("nnz", C.c_int64),
                ("devstate_bytes", C.c_uint64), ("fingerprint", C.c_uint64)]


class _State(C.Structure):
    """The solver's scalar state that follows the header: 25 doubles
    (step size, primal weight, epoch sums, KKT references, parameters,
    candidate and term pieces, certificate), 7 counters, 13 ints of flags
    and positions, 8 block counters."""

    _fields_ = [("d", C.c_double * 25), ("k", C.c_int64), ("t", C.c_int64), ("attempts", C.c_int64),
                ("restarts", C.c_int64), ("checks", C.c_int64), ("max_iter", C.c_int64),
                ("f64_switch_k", C.c_int64), ("cur", C.c_int32), ("need_g", C.c_int32),
                ("check_pending", C.c_int32), ("status", C.c_int32), ("which", C.c_int32),
                ("restart_to", C.c_int32), ("mode", C.c_int32), ("P", C.c_int32), ("ntrace", C.c_int32),
                ("trace_cap", C.c_int32), ("use_f32", C.c_int32), ("polish", C.c_int32), ("stall", C.c_int32),
                ("cnt", C.c_uint32 * 8)]


def test_state_with_out_of_range_counters_is_rejected_on_the_host():
    """Fields the kernels index or divide with (check period, trace ring
    size and position, step counts, the FP32 switch) are checked before
    any device work; the unmodified blob still loads and resumes."""
    lp = lpgen.tiny_lp(2)
    with P.Solver(lp, check_period=8) as a:
        a.begin(tol=1e-6)
        a.run_periods(3)
        _, k = a.poll()
        blob = a.get_state()
        hdr = _Header.from_buffer_copy(blob)
        off = C.sizeof(_Header)
        d = _State.from_buffer_copy(blob, off)
        # the mirror matches this build's layout
        assert hdr.devstate_bytes == C.sizeof(_State) and (hdr.m, hdr.n) == (lp.m, lp.n)
        assert (d.k, d.P, d.trace_cap, d.ntrace, d.check_pending) == (k, 8, P.TRACE_RETAINED, 0, 0)
        assert d.cur in (0, 1) and d.use_f32 == 0 and d.attempts >= d.k > 0 and d.max_iter >= 1
        bad_values = dict(P=[0, 9, -8], trace_cap=[0, 1 << 20], ntrace=[5, -1], k=[-1], t=[-1],
                          attempts=[k - 1], max_iter=[0], use_f32=[1, 2], need_g=[2])
        for field, values in bad_values.items():
            for v in values:
                e = _State.from_buffer_copy(blob, off)
                setattr(e, field, v)
                data = blob[:off] + bytes(e) + blob[off + C.sizeof(_State):]
                with pytest.raises(P.PdlpError) as err:
                    a.set_state(data)
                assert err.value.code == P.ERR_INVALID, (field, v)
        a.set_state(blob)
        _, _, st, _ = a.resume()
    assert st == P.OPTIMAL


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
