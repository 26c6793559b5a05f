"""C-ABI checks that need no GPU: the library loads, exports every function
include/pdlp.h declares, and rejects malformed input on the host before any
CUDA call."""

import ctypes as C
import os
import re

import numpy as np
import pytest

import lpgen
from paper_2311_12180_gb300 import _build
from paper_2311_12180_gb300 import pdlp as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    _build.build()
    return P.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "pdlp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pdlp_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(P.EXPORTS) == names


def test_default_params(L):
    p = P.pdlp_default_params()
    assert p.check_period == 64 and p.ruiz_iters == 10 and p.pc_alpha == 1.0
    assert (p.beta_suff, p.beta_nec, p.beta_art) == (0.2, 0.8, 0.36)
    assert p.theta == 0.5 and p.eps_zero == 1e-10 and p.value_bits == 64
    assert p.eps_infeas == 1e-8


def test_kernel_names(L):
    names = P.kernel_names()
    assert names[:2] == ["k_primal", "k_dual"]
    assert "k_infeas" in names


def _create(lp, **kw):
    return P.pdlp_create(lp.m, lp.n, lp.n_eq, lp.c, lp.row_ptr, lp.col_idx, lp.val, lp.q, lp.l, lp.u, **kw)


@pytest.mark.parametrize("defect", ["col_range", "row_ptr_order", "row_ptr_start", "nan_val", "l_gt_u",
                                    "nan_c", "inf_q", "l_plus_inf", "n_eq_too_big", "n_zero"])
def test_invalid_input_rejected_on_host(L, defect):
    lp = lpgen.tiny_lp(0)
    lp.col_idx = lp.col_idx.copy()
    lp.row_ptr = lp.row_ptr.copy()
    lp.val, lp.c, lp.q, lp.l, lp.u = lp.val.copy(), lp.c.copy(), lp.q.copy(), lp.l.copy(), lp.u.copy()
    if defect == "col_range":
        lp.col_idx[5] = lp.n
    elif defect == "row_ptr_order":
        lp.row_ptr[3] = lp.row_ptr[4] + 1
    elif defect == "row_ptr_start":  # lengths consistent, so the C side sees row_ptr[0] = 1
        lp.row_ptr = lp.row_ptr + 1
        lp.col_idx = np.append(lp.col_idx, 0)
        lp.val = np.append(lp.val, 1.0)
    elif defect == "nan_val":
        lp.val[0] = np.nan
    elif defect == "l_gt_u":
        lp.l[2] = 11.0
    elif defect == "nan_c":
        lp.c[1] = np.nan
    elif defect == "inf_q":
        lp.q[0] = np.inf
    elif defect == "l_plus_inf":
        lp.l[0] = np.inf
        lp.u[0] = np.inf
    elif defect == "n_eq_too_big":
        lp.n_eq = lp.m + 1
    elif defect == "n_zero":
        lp.n = 0
        lp.c = lp.c[:0]
        lp.l = lp.l[:0]
        lp.u = lp.u[:0]
    with pytest.raises(P.PdlpError) as e:
        _create(lp)
    assert e.value.code == P.ERR_INVALID
    assert L.pdlp_last_error().decode() != ""


def test_invalid_params_rejected(L):
    lp = lpgen.tiny_lp(0)
    p = P.pdlp_default_params()
    p.check_period = 0
    with pytest.raises(P.PdlpError) as e:
        _create(lp, params=p)
    assert e.value.code == P.ERR_INVALID
    p = P.pdlp_default_params()
    p.value_bits = 16
    with pytest.raises(P.PdlpError):
        _create(lp, params=p)
    for bad in (-1e-8, float("nan")):
        p = P.pdlp_default_params()
        p.eps_infeas = bad
        with pytest.raises(P.PdlpError) as e:
            _create(lp, params=p)
        assert e.value.code == P.ERR_INVALID


def test_null_handles_are_safe(L):
    L.pdlp_destroy(None)
    assert L.pdlp_device_bytes(None) == 0
    assert L.pdlp_get_stream(None) is None
    assert L.pdlp_run_periods(None, 1) == P.ERR_INVALID
    assert L.pdlp_begin(None, None, None, 1e-4, 10) == P.ERR_INVALID


def test_batch_rejects_bad_lp_on_host(L):
    good = lpgen.tiny_lp(0)
    bad = lpgen.tiny_lp(1)
    bad.col_idx = bad.col_idx.copy()
    bad.col_idx[7] = bad.n + 3
    with pytest.raises(P.PdlpError) as e:
        P.BatchSolver([good, bad])
    assert e.value.code == P.ERR_INVALID and "LP 1" in str(e.value)


@pytest.mark.parametrize("dims", [(0, 8, 8, 8), (4, 0, 8, 8), (4, 8, 0, 8), (4, 8, 8, 0), (4, 8, 8, 70000),
                                  (4, 65536, 65536, 8)])
def test_mlp_create_rejects_bad_dims_on_host(L, dims):
    h = C.c_void_p()
    assert L.pdlp_mlp_create(C.byref(h), *dims, None) == P.ERR_INVALID
    assert not h.value


def test_batch_times_rejects_null(L):
    assert L.pdlp_batch_times(None, None, None) == P.ERR_INVALID


@pytest.mark.parametrize("null", ["K_ptr", "K_idx", "K_val", "KT_ptr", "KT_idx", "KT_val", "D1", "D2"])
def test_noalloc_scaling_rejects_null_pointers_on_host(L, null):
    # non-null dummies that are never dereferenced: the checks run before any
    # CUDA call, so a null argument must be rejected without touching the GPU
    args = dict(K_ptr=8, K_idx=8, K_val=8, KT_ptr=8, KT_idx=8, KT_val=8, D1=8, D2=8)
    args[null] = None
    rc = L.pdlp_scale_device_noalloc(4, 6, args["K_ptr"], args["K_idx"], args["K_val"], args["KT_ptr"],
                                     args["KT_idx"], args["KT_val"], 10, 1.0, args["D1"], args["D2"], None)
    assert rc == P.ERR_INVALID
    assert "null" in L.pdlp_last_error().decode()


def test_error_message_is_per_thread(L):
    """pdlp_last_error is thread-local: a rejected call on one thread sets
    that thread's message and leaves another thread's untouched."""
    import threading

    L.pdlp_last_error.restype = C.c_char_p
    lp = lpgen.tiny_lp(0)
    bad = lpgen.tiny_lp(0)
    bad.col_idx = bad.col_idx.copy()
    bad.col_idx[3] = bad.n
    seen = {}

    def worker():
        with pytest.raises(P.PdlpError):
            _create(bad)
        seen["worker"] = L.pdlp_last_error().decode()

    assert L.pdlp_get_info(None, None) == P.ERR_INVALID
    main_msg = L.pdlp_last_error().decode()
    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert "col_idx" in seen["worker"] and "3" in seen["worker"]
    assert main_msg and L.pdlp_last_error().decode() == main_msg != seen["worker"]


@pytest.mark.parametrize("defect", ["short_row_ptr", "short_col_idx", "short_val", "int32_overflow", "short_c",
                                    "short_q"])
def test_binding_checks_array_lengths_before_the_call(L, defect):
    """The Python binding hands the C call only arrays of the lengths it
    reads (m + 1 row starts, row_ptr[m] indices and values, n- and
    m-vectors) and indices that fit in int32; anything else is a ValueError
    before any C call."""
    lp = lpgen.tiny_lp(0)
    rp, ci, v, c, q = lp.row_ptr, lp.col_idx, lp.val, lp.c, lp.q
    if defect == "short_row_ptr":
        rp = rp[:-1]
    elif defect == "short_col_idx":
        ci = ci[:-1]
    elif defect == "short_val":
        v = v[:-1]
    elif defect == "int32_overflow":
        ci = ci.astype(np.int64)
        ci[0] = 2**32
    elif defect == "short_c":
        c = c[:-1]
    elif defect == "short_q":
        q = q[:-1]
    with pytest.raises(ValueError):
        P.pdlp_create(lp.m, lp.n, lp.n_eq, c, rp, ci, v, q, lp.l, lp.u)
    bad = lpgen.tiny_lp(1)
    bad.row_ptr, bad.col_idx, bad.val, bad.c, bad.q = rp, ci, v, c, q
    with pytest.raises(ValueError):
        P.BatchSolver([lpgen.tiny_lp(2), bad])


def test_mlp_binding_rejects_bad_shapes_before_the_call(L):
    """The MLP binding checks array shapes before any C call (a handle that
    was never created is enough to reach the checks)."""
    net = object.__new__(P.Mlp)
    net.in_dim, net.hidden, net.out_dim, net.max_batch, net.h = 4, 8, 3, 16, None
    with pytest.raises(ValueError):
        net.set_data(np.zeros((5, 3)), np.zeros((5, 3)))  # X has the wrong width
    with pytest.raises(ValueError):
        net.set_data(np.zeros((5, 4)), np.zeros((6, 3)))  # row counts differ
    with pytest.raises(ValueError):
        net.train(np.zeros(7, dtype=np.int32))  # not (steps, batch)
    with pytest.raises(ValueError):
        net.predict(np.zeros((2, 5)))
    with pytest.raises(ValueError):
        net.set_params(np.zeros(3))  # param_count of a NULL handle is 0, 3 != 0
