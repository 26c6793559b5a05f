"""ctypes binding of the C ABI in include/pdlp.h (argument marshalling only).

Every step of the solve runs in the CUDA kernels of libpdlp_gb300.so; this
module only converts numpy arrays to pointers.  There is no CPU fallback: if
the library is missing or no GB300 is visible, the calls raise.

Module-level functions carry the C names (pdlp_create, pdlp_solve, ...);
``Solver`` wraps them for convenience.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

OK, ERR_INVALID, ERR_CUDA, ERR_OOM = 0, -1, -2, -3
OPTIMAL, ITER_LIMIT, TIME_LIMIT, NUMERICAL, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE = 0, 1, 2, 3, 4, 5
STATUS_NAMES = {OPTIMAL: "optimal", ITER_LIMIT: "iteration_limit", TIME_LIMIT: "time_limit",
                NUMERICAL: "numerical_error", PRIMAL_INFEASIBLE: "primal_infeasible",
                DUAL_INFEASIBLE: "dual_infeasible", -1: "running"}


class PdlpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("pdlp error %d: %s" % (code, msg))
        self.code = code


class pdlp_params(C.Structure):
    _fields_ = [
        ("check_period", C.c_int32),
        ("ruiz_iters", C.c_int32),
        ("pc_alpha", C.c_double),
        ("theta", C.c_double),
        ("eps_zero", C.c_double),
        ("beta_suff", C.c_double),
        ("beta_nec", C.c_double),
        ("beta_art", C.c_double),
        ("time_limit_s", C.c_double),
        ("value_bits", C.c_int32),
        ("f32_polish", C.c_int32),
        ("eps_infeas", C.c_double),
    ]


class pdlp_info(C.Structure):
    _fields_ = [
        ("status", C.c_int32),
        ("which", C.c_int32),
        ("iters", C.c_int64),
        ("attempts", C.c_int64),
        ("restarts", C.c_int64),
        ("checks", C.c_int64),
        ("pobj", C.c_double),
        ("dobj", C.c_double),
        ("rp_norm", C.c_double),
        ("rd_norm", C.c_double),
        ("q_norm", C.c_double),
        ("c_norm", C.c_double),
        ("omega", C.c_double),
        ("eta_hat", C.c_double),
        ("setup_ms", C.c_double),
        ("solve_ms", C.c_double),
        ("graph_launches", C.c_int64),
        ("f64_switch_iter", C.c_int64),
        ("ray_obj", C.c_double),
        ("ray_res", C.c_double),
    ]


# check records the device ring keeps (pdlp_get_trace)
TRACE_RETAINED = 1 << 16

CHECK_DTYPE = np.dtype(
    [
        ("k", np.int64),
        ("attempts", np.int64),
        ("restarts", np.int64),
        ("restart", np.int32),
        ("cand_avg", np.int32),
        ("kkt_cur", np.float64),
        ("kkt_avg", np.float64),
        ("kkt_start", np.float64),
        ("omega", np.float64),
        ("eta_hat", np.float64),
        ("rel_gap", np.float64),
        ("rel_primal", np.float64),
        ("rel_dual", np.float64),
    ]
)

# every symbol include/pdlp.h declares
EXPORTS = (
    "pdlp_default_params", "pdlp_create", "pdlp_create_ex", "pdlp_solve", "pdlp_solve_warm", "pdlp_begin",
    "pdlp_run_periods", "pdlp_poll", "pdlp_finish", "pdlp_time_kernels", "pdlp_kernel_count",
    "pdlp_kernel_name", "pdlp_get_info", "pdlp_get_trace", "pdlp_get_scaling", "pdlp_get_stream",
    "pdlp_device_bytes", "pdlp_destroy", "pdlp_last_error", "pdlp_scale_device_noalloc",
    "pdlp_create_device", "pdlp_get_state", "pdlp_set_state", "pdlp_resume", "pdlp_get_layout",
    "pdlp_probe_rates", "pdlp_probe_stream_gathers", "pdlp_set_quadratic",
    "pdlp_batch_create", "pdlp_batch_solve", "pdlp_batch_info", "pdlp_batch_lanes", "pdlp_batch_times", "pdlp_batch_destroy",
    "pdlp_mlp_create", "pdlp_mlp_param_count", "pdlp_mlp_set_params", "pdlp_mlp_get_params", "pdlp_mlp_set_data",
    "pdlp_mlp_train", "pdlp_mlp_predict", "pdlp_mlp_gradients", "pdlp_mlp_stats", "pdlp_mlp_destroy",
)


class pdlp_layout_info(C.Structure):
    _fields_ = [(f, C.c_int64) for f in ("K_stored", "K_slices", "K_long_rows", "KT_stored", "KT_slices",
                                          "KT_long_rows")] + [("long_threshold", C.c_int32), ("pad_", C.c_int32)]


class pdlp_lp(C.Structure):
    _fields_ = [
        ("m", C.c_int32),
        ("n", C.c_int32),
        ("n_eq", C.c_int32),
        ("pad_", C.c_int32),
        ("c", C.c_void_p),
        ("row_ptr", C.c_void_p),
        ("col_idx", C.c_void_p),
        ("val", C.c_void_p),
        ("q", C.c_void_p),
        ("l", C.c_void_p),
        ("u", C.c_void_p),
    ]


class pdlp_batch_stats(C.Structure):
    _fields_ = [
        ("count", C.c_int32),
        ("grid", C.c_int32),
        ("sum_m", C.c_int64),
        ("sum_n", C.c_int64),
        ("sum_nnz", C.c_int64),
        ("setup_ms", C.c_double),
        ("tune_ms", C.c_double),
        ("solve_ms", C.c_double),
        ("entries_per_lane", C.c_double),
        ("device_bytes", C.c_size_t),
        ("resident", C.c_int32),
        ("resident_max_bytes", C.c_int32),
        ("team_lps", C.c_int32),
        ("team_size", C.c_int32),
        ("team_min_nnz", C.c_int32),
    ]

_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libpdlp_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("libpdlp_gb300.so is not built; run __graft_entry__.build() or "
                           "python -m paper_2311_12180_gb300._build")
    L = C.CDLL(path)
    vp, i32, i64, d, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    P = C.POINTER
    L.pdlp_default_params.argtypes = [P(pdlp_params)]
    L.pdlp_default_params.restype = None
    L.pdlp_create.argtypes = [P(vp), i32, i32, i32, vp, vp, vp, vp, vp, vp, vp]
    L.pdlp_create.restype = C.c_int
    L.pdlp_create_ex.argtypes = [P(vp), i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, P(pdlp_params), vp]
    L.pdlp_create_ex.restype = C.c_int
    L.pdlp_create_device.argtypes = [P(vp), i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, P(pdlp_params), vp]
    L.pdlp_create_device.restype = C.c_int
    L.pdlp_get_state.argtypes = [vp, vp, sz, P(sz)]
    L.pdlp_get_state.restype = C.c_int
    L.pdlp_set_state.argtypes = [vp, vp, sz]
    L.pdlp_set_state.restype = C.c_int
    L.pdlp_resume.argtypes = [vp, vp, vp, P(C.c_int), P(i64)]
    L.pdlp_resume.restype = C.c_int
    L.pdlp_set_quadratic.argtypes = [vp, vp]
    L.pdlp_set_quadratic.restype = C.c_int
    L.pdlp_get_layout.argtypes = [vp, P(pdlp_layout_info)]
    L.pdlp_get_layout.restype = C.c_int
    L.pdlp_probe_rates.argtypes = [P(d), P(d)]
    L.pdlp_probe_rates.restype = C.c_int
    L.pdlp_probe_stream_gathers.argtypes = [P(d)]
    L.pdlp_probe_stream_gathers.restype = C.c_int
    L.pdlp_solve.argtypes = [vp, d, i64, vp, vp, P(C.c_int), P(i64)]
    L.pdlp_solve.restype = C.c_int
    L.pdlp_solve_warm.argtypes = [vp, vp, vp, d, i64, vp, vp, P(C.c_int), P(i64)]
    L.pdlp_solve_warm.restype = C.c_int
    L.pdlp_begin.argtypes = [vp, vp, vp, d, i64]
    L.pdlp_begin.restype = C.c_int
    L.pdlp_run_periods.argtypes = [vp, i32]
    L.pdlp_run_periods.restype = C.c_int
    L.pdlp_poll.argtypes = [vp, P(C.c_int), P(i64)]
    L.pdlp_poll.restype = C.c_int
    L.pdlp_finish.argtypes = [vp, vp, vp, P(C.c_int), P(i64)]
    L.pdlp_finish.restype = C.c_int
    L.pdlp_time_kernels.argtypes = [vp, i32, vp, vp]
    L.pdlp_time_kernels.restype = C.c_int
    L.pdlp_kernel_count.argtypes = []
    L.pdlp_kernel_count.restype = i32
    L.pdlp_kernel_name.argtypes = [i32]
    L.pdlp_kernel_name.restype = C.c_char_p
    L.pdlp_get_info.argtypes = [vp, P(pdlp_info)]
    L.pdlp_get_info.restype = C.c_int
    L.pdlp_get_trace.argtypes = [vp, vp, i32, P(i32)]
    L.pdlp_get_trace.restype = C.c_int
    L.pdlp_get_scaling.argtypes = [vp, vp, vp, vp]
    L.pdlp_get_scaling.restype = C.c_int
    L.pdlp_get_stream.argtypes = [vp]
    L.pdlp_get_stream.restype = vp
    L.pdlp_device_bytes.argtypes = [vp]
    L.pdlp_device_bytes.restype = sz
    L.pdlp_destroy.argtypes = [vp]
    L.pdlp_destroy.restype = None
    L.pdlp_last_error.argtypes = []
    L.pdlp_last_error.restype = C.c_char_p
    L.pdlp_scale_device_noalloc.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, i32, d, vp, vp, vp]
    L.pdlp_scale_device_noalloc.restype = C.c_int
    L.pdlp_batch_create.argtypes = [P(vp), i32, P(pdlp_lp), P(pdlp_params), vp]
    L.pdlp_batch_create.restype = C.c_int
    L.pdlp_batch_solve.argtypes = [vp, vp, vp, d, i64, vp, vp, vp, vp]
    L.pdlp_batch_solve.restype = C.c_int
    L.pdlp_batch_info.argtypes = [vp, P(pdlp_batch_stats)]
    L.pdlp_batch_info.restype = C.c_int
    L.pdlp_batch_lanes.argtypes = [vp, vp, vp]
    L.pdlp_batch_lanes.restype = C.c_int
    L.pdlp_batch_times.argtypes = [vp, vp, vp]
    L.pdlp_batch_times.restype = C.c_int
    L.pdlp_batch_destroy.argtypes = [vp]
    L.pdlp_batch_destroy.restype = None
    L.pdlp_mlp_create.argtypes = [P(vp), i32, i32, i32, i32, vp]
    L.pdlp_mlp_create.restype = C.c_int
    L.pdlp_mlp_param_count.argtypes = [vp]
    L.pdlp_mlp_param_count.restype = i64
    L.pdlp_mlp_set_params.argtypes = [vp, vp]
    L.pdlp_mlp_set_params.restype = C.c_int
    L.pdlp_mlp_get_params.argtypes = [vp, vp]
    L.pdlp_mlp_get_params.restype = C.c_int
    L.pdlp_mlp_set_data.argtypes = [vp, i32, vp, vp]
    L.pdlp_mlp_set_data.restype = C.c_int
    L.pdlp_mlp_train.argtypes = [vp, i32, i32, vp, C.c_float, C.c_float, C.c_float, C.c_float, vp]
    L.pdlp_mlp_train.restype = C.c_int
    L.pdlp_mlp_predict.argtypes = [vp, i32, vp, vp]
    L.pdlp_mlp_predict.restype = C.c_int
    L.pdlp_mlp_gradients.argtypes = [vp, i32, vp, vp, vp]
    L.pdlp_mlp_gradients.restype = C.c_int
    L.pdlp_mlp_stats.argtypes = [vp, vp, vp]
    L.pdlp_mlp_stats.restype = C.c_int
    L.pdlp_mlp_destroy.argtypes = [vp]
    L.pdlp_mlp_destroy.restype = None
    _lib = L
    return L


def _check(rc):
    if rc != OK:
        raise PdlpError(rc, lib().pdlp_last_error().decode())
    return rc


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.shape[0] != n:
        raise ValueError("expected length %d, got %d" % (n, a.shape[0]))
    return a


def _i32(a, n=None):
    a = np.asarray(a)
    if a.dtype != np.int32 and a.size and (a.min() < -2**31 or a.max() >= 2**31):
        raise ValueError("index array does not fit in int32")
    a = np.ascontiguousarray(a, dtype=np.int32)
    if n is not None and a.shape[0] != n:
        raise ValueError("expected length %d, got %d" % (n, a.shape[0]))
    return a


def _csr(m, row_ptr, col_idx, val):
    """K's CSR arrays as int32 / float64, with the lengths the C call reads:
    m + 1 row starts and at least row_ptr[m] indices and values."""
    row_ptr = _i32(row_ptr, m + 1)
    nnz = int(row_ptr[m])
    col_idx, val = _i32(col_idx), _f64(val)
    if col_idx.shape[0] < nnz or val.shape[0] < nnz:
        raise ValueError("row_ptr[m] = %d but col_idx has %d and val %d entries" % (nnz, col_idx.shape[0], val.shape[0]))
    return row_ptr, col_idx, val


# ---------------------------------------------------------------- C-named functions


def pdlp_default_params() -> pdlp_params:
    p = pdlp_params()
    lib().pdlp_default_params(C.byref(p))
    return p


def pdlp_create(m, n, n_eq, c, row_ptr, col_idx, val, q, l, u, params=None, stream=None):
    """pdlp_create / pdlp_create_ex; returns the opaque handle (c_void_p)."""
    h = C.c_void_p()
    c, q, l, u = _f64(c, n), _f64(q, m), _f64(l, n), _f64(u, n)
    row_ptr, col_idx, val = _csr(m, row_ptr, col_idx, val)
    if params is None and stream is None:
        rc = lib().pdlp_create(C.byref(h), m, n, n_eq, _ptr(c), _ptr(row_ptr), _ptr(col_idx), _ptr(val), _ptr(q),
                               _ptr(l), _ptr(u))
    else:
        rc = lib().pdlp_create_ex(C.byref(h), m, n, n_eq, _ptr(c), _ptr(row_ptr), _ptr(col_idx), _ptr(val),
                                  _ptr(q), _ptr(l), _ptr(u), C.byref(params) if params is not None else None,
                                  C.c_void_p(stream) if stream else None)
    _check(rc)
    return h


def pdlp_create_device(m, n, n_eq, c, row_ptr, col_idx, val, q, l, u, params=None, stream=None):
    """pdlp_create_device: every array argument is a DEVICE address (int,
    e.g. a torch tensor's data_ptr()); returns the opaque handle."""
    h = C.c_void_p()
    _check(lib().pdlp_create_device(C.byref(h), m, n, n_eq, c, row_ptr, col_idx, val, q, l, u,
                                    C.byref(params) if params is not None else None,
                                    C.c_void_p(stream) if stream else None))
    return h


def pdlp_solve_warm(h, x0, y0, tol, max_iter, n, m):
    x = np.empty(n)
    y = np.empty(max(m, 1))
    st = C.c_int(-9)
    it = C.c_int64(0)
    _check(lib().pdlp_solve_warm(h, _ptr(_f64(x0, n)), _ptr(_f64(y0, m)), tol, int(max_iter), _ptr(x), _ptr(y),
                                 C.byref(st), C.byref(it)))
    return x, y[:m], st.value, it.value


def pdlp_solve(h, tol, max_iter, n, m):
    return pdlp_solve_warm(h, None, None, tol, max_iter, n, m)


def pdlp_destroy(h):
    if h:
        lib().pdlp_destroy(h)


def pdlp_scale_device_noalloc(m, n, K_ptr, K_idx, K_val, KT_ptr, KT_idx, KT_val, ruiz_iters, pc_alpha, D1, D2,
                              stream=None):
    """Allocation-free scaling of a device-resident K and K' (all arguments
    are device addresses as ints, e.g. torch tensors' data_ptr())."""
    _check(lib().pdlp_scale_device_noalloc(m, n, K_ptr, K_idx, K_val, KT_ptr, KT_idx, KT_val, int(ruiz_iters),
                                           float(pc_alpha), D1, D2, stream))


def probe_rates():
    """(random 8-byte gathers per second, FP64 FMA lane operations per second)
    measured on the current GPU (pdlp_probe_rates)."""
    g, f = C.c_double(0), C.c_double(0)
    _check(lib().pdlp_probe_rates(C.byref(g), C.byref(f)))
    return g.value, f.value


def probe_stream_gathers():
    """Random 8-byte gathers per second with an SpMV's index and value stream
    beside them (pdlp_probe_stream_gathers)."""
    g = C.c_double(0)
    _check(lib().pdlp_probe_stream_gathers(C.byref(g)))
    return g.value


def kernel_names():
    L = lib()
    return [L.pdlp_kernel_name(i).decode() for i in range(L.pdlp_kernel_count())]


# ---------------------------------------------------------------- convenience wrapper


class Solver:
    """One LP on the GPU.  `lp` is anything with fields m, n, n_eq, c,
    row_ptr, col_idx, val, q, l, u (e.g. lpgen.LP)."""

    def __init__(self, lp, params: pdlp_params | None = None, stream: int | None = None, device=None, **kw):
        """device: None for host arrays in `lp`; otherwise a dict of DEVICE
        addresses with keys c, row_ptr, col_idx, val, q, l, u (and `lp` only
        supplies m, n, n_eq, nnz): pdlp_create_device."""
        if kw:
            params = params or pdlp_default_params()
            for k, v in kw.items():
                setattr(params, k, v)
        self.m, self.n, self.n_eq = int(lp.m), int(lp.n), int(lp.n_eq)
        self.nnz = int(lp.row_ptr[-1]) if device is None else int(lp.nnz)
        if device is None:
            self.h = pdlp_create(self.m, self.n, self.n_eq, lp.c, lp.row_ptr, lp.col_idx, lp.val, lp.q, lp.l,
                                 lp.u, params=params, stream=stream)
        else:
            d = device
            self.h = pdlp_create_device(self.m, self.n, self.n_eq, d["c"], d["row_ptr"], d["col_idx"], d["val"],
                                        d["q"], d["l"], d["u"], params=params, stream=stream)
        qd = getattr(lp, "qdiag", None)
        if qd is not None:  # a QP (objective x'Qx/2 + c'x, Q = diag(qdiag))
            self.set_quadratic(qd)

    def set_quadratic(self, qdiag):
        """pdlp_set_quadratic: Q = diag(qdiag) from the next solve on (None: LP)."""
        arr = None if qdiag is None else _f64(qdiag, self.n)
        _check(lib().pdlp_set_quadratic(self.h, _ptr(arr)))

    def close(self):
        if getattr(self, "h", None):
            pdlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, tol=1e-4, max_iter=1_000_000, x0=None, y0=None):
        """Returns (x, y, status, iters) in the original space."""
        return pdlp_solve_warm(self.h, x0, y0, tol, max_iter, self.n, self.m)

    # non-blocking pieces
    def begin(self, tol=1e-4, max_iter=1_000_000, x0=None, y0=None):
        _check(lib().pdlp_begin(self.h, _ptr(_f64(x0, self.n)), _ptr(_f64(y0, self.m)), tol, int(max_iter)))

    def run_periods(self, n):
        _check(lib().pdlp_run_periods(self.h, int(n)))

    def poll(self):
        st = C.c_int(-9)
        it = C.c_int64(0)
        _check(lib().pdlp_poll(self.h, C.byref(st), C.byref(it)))
        return st.value, it.value

    def finish(self):
        x = np.empty(self.n)
        y = np.empty(max(self.m, 1))
        st = C.c_int(-9)
        it = C.c_int64(0)
        _check(lib().pdlp_finish(self.h, _ptr(x), _ptr(y), C.byref(st), C.byref(it)))
        return x, y[: self.m], st.value, it.value

    # checkpoint / resume
    def get_state(self) -> bytes:
        need = C.c_size_t(0)
        _check(lib().pdlp_get_state(self.h, None, 0, C.byref(need)))
        buf = (C.c_char * need.value)()
        _check(lib().pdlp_get_state(self.h, buf, need.value, C.byref(need)))
        return bytes(buf)

    def set_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib().pdlp_set_state(self.h, buf, len(blob)))

    def resume(self):
        """Continues a begun or loaded solve to its end: (x, y, status, iters)."""
        x = np.empty(self.n)
        y = np.empty(max(self.m, 1))
        st = C.c_int(-9)
        it = C.c_int64(0)
        _check(lib().pdlp_resume(self.h, _ptr(x), _ptr(y), C.byref(st), C.byref(it)))
        return x, y[: self.m], st.value, it.value

    def time_kernels(self, n_periods):
        k = lib().pdlp_kernel_count()
        ms = np.zeros(k)
        ln = np.zeros(k, dtype=np.int64)
        _check(lib().pdlp_time_kernels(self.h, int(n_periods), _ptr(ms), _ptr(ln)))
        return {name: (float(ms[i]), int(ln[i])) for i, name in enumerate(kernel_names())}

    def info(self) -> dict:
        inf = pdlp_info()
        _check(lib().pdlp_get_info(self.h, C.byref(inf)))
        return {f: getattr(inf, f) for f, _ in pdlp_info._fields_}

    def trace(self, cap=TRACE_RETAINED):
        """Check records of the last solve, oldest retained first (the device
        ring keeps the last TRACE_RETAINED); checks_recorded() gives the total."""
        out = np.zeros(cap, dtype=CHECK_DTYPE)
        cnt = C.c_int32(0)
        _check(lib().pdlp_get_trace(self.h, _ptr(out), cap, C.byref(cnt)))
        self._checks_recorded = cnt.value
        return out[: min(cnt.value, cap, TRACE_RETAINED)].copy()

    def checks_recorded(self) -> int:
        cnt = C.c_int32(0)
        _check(lib().pdlp_get_trace(self.h, None, 0, C.byref(cnt)))
        return cnt.value

    def scaling(self):
        D1 = np.zeros(max(self.m, 1))
        D2 = np.zeros(self.n)
        v = np.zeros(max(self.nnz, 1))
        _check(lib().pdlp_get_scaling(self.h, _ptr(D1), _ptr(D2), _ptr(v)))
        return D1[: self.m], D2, v[: self.nnz]

    def layout(self) -> dict:
        info = pdlp_layout_info()
        _check(lib().pdlp_get_layout(self.h, C.byref(info)))
        return {f: int(getattr(info, f)) for f, _ in pdlp_layout_info._fields_ if f != "pad_"}

    @property
    def stream(self) -> int:
        return lib().pdlp_get_stream(self.h) or 0

    def device_bytes(self) -> int:
        return int(lib().pdlp_device_bytes(self.h))


class BatchSolver:
    """Many LPs solved together in one persistent launch (pdlp_batch_*).
    `lps` is a sequence of objects with the fields of lpgen.LP."""

    def __init__(self, lps, params: pdlp_params | None = None, stream: int | None = None, **kw):
        if kw:
            params = params or pdlp_default_params()
            for k, v in kw.items():
                setattr(params, k, v)
        self._keep = []
        arr = (pdlp_lp * len(lps))()
        self.ms, self.ns = [], []
        for i, lp in enumerate(lps):
            m, n = int(lp.m), int(lp.n)
            c, q, l, u = _f64(lp.c, n), _f64(lp.q, m), _f64(lp.l, n), _f64(lp.u, n)
            rp, ci, v = _csr(m, lp.row_ptr, lp.col_idx, lp.val)
            q = q if q.size else np.zeros(1)
            ci = ci if ci.size else np.zeros(1, np.int32)
            v = v if v.size else np.zeros(1)
            self._keep += [c, q, l, u, rp, ci, v]
            arr[i] = pdlp_lp(int(lp.m), int(lp.n), int(lp.n_eq), 0, _ptr(c), _ptr(rp), _ptr(ci), _ptr(v), _ptr(q),
                             _ptr(l), _ptr(u))
            self.ms.append(int(lp.m))
            self.ns.append(int(lp.n))
        self.count = len(lps)
        self.xo = np.concatenate([[0], np.cumsum(self.ns)]).astype(np.int64)
        self.yo = np.concatenate([[0], np.cumsum(self.ms)]).astype(np.int64)
        self.h = C.c_void_p()
        _check(lib().pdlp_batch_create(C.byref(self.h), self.count, arr, C.byref(params) if params else None,
                                       C.c_void_p(stream) if stream else None))
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            lib().pdlp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, tol=1e-6, max_iter=1_000_000, x0=None, y0=None):
        """Returns (list of x, list of y, status array, iters array)."""
        X = np.empty(int(self.xo[-1]))
        Y = np.empty(max(int(self.yo[-1]), 1))
        st = np.empty(self.count, dtype=np.int32)
        it = np.empty(self.count, dtype=np.int64)
        # the start points of all LPs back to back: sum n and sum m entries
        x0p = None if x0 is None else _f64(np.concatenate(x0) if isinstance(x0, (list, tuple)) else x0,
                                           int(self.xo[-1]))
        y0p = None if y0 is None else _f64(np.concatenate(y0) if isinstance(y0, (list, tuple)) else y0,
                                           int(self.yo[-1]))
        _check(lib().pdlp_batch_solve(self.h, _ptr(x0p), _ptr(y0p), tol, int(max_iter), _ptr(X), _ptr(Y), _ptr(st),
                                      _ptr(it)))
        xs = [X[self.xo[i]:self.xo[i + 1]] for i in range(self.count)]
        ys = [Y[self.yo[i]:self.yo[i + 1]] for i in range(self.count)]
        return xs, ys, st, it

    def stats(self) -> dict:
        s = pdlp_batch_stats()
        _check(lib().pdlp_batch_info(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in pdlp_batch_stats._fields_}

    def times(self):
        """(start, end) seconds of each LP in the last solve, after the earliest start."""
        a = np.zeros(self.count)
        b = np.zeros(self.count)
        _check(lib().pdlp_batch_times(self.h, _ptr(a), _ptr(b)))
        return a, b

    def lanes(self):
        a = np.zeros(self.count, dtype=np.int32)
        b = np.zeros(self.count, dtype=np.int32)
        _check(lib().pdlp_batch_lanes(self.h, _ptr(a), _ptr(b)))
        return a, b


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class Mlp:
    """The warm-start MLP (pdlp_mlp_*): in -> hidden -> hidden -> out."""

    def __init__(self, in_dim, hidden, out_dim, max_batch=256, stream=None):
        self.in_dim, self.hidden, self.out_dim, self.max_batch = int(in_dim), int(hidden), int(out_dim), int(max_batch)
        self.h = C.c_void_p()
        _check(lib().pdlp_mlp_create(C.byref(self.h), self.in_dim, self.hidden, self.out_dim, self.max_batch,
                                     C.c_void_p(stream) if stream else None))

    def close(self):
        if getattr(self, "h", None):
            lib().pdlp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def param_count(self) -> int:
        return int(lib().pdlp_mlp_param_count(self.h))

    def set_params(self, p):
        p = _f32(p).ravel()
        if p.size != self.param_count:
            raise ValueError("expected %d parameters, got %d" % (self.param_count, p.size))
        _check(lib().pdlp_mlp_set_params(self.h, _ptr(p)))

    def get_params(self):
        p = np.empty(self.param_count, dtype=np.float32)
        _check(lib().pdlp_mlp_get_params(self.h, _ptr(p)))
        return p

    def set_data(self, X, T):
        X, T = _f32(X), _f32(T)
        if X.ndim != 2 or T.ndim != 2 or X.shape[1] != self.in_dim or T.shape[1] != self.out_dim \
                or X.shape[0] != T.shape[0]:
            raise ValueError("need X (samples, %d) and T (samples, %d)" % (self.in_dim, self.out_dim))
        _check(lib().pdlp_mlp_set_data(self.h, X.shape[0], _ptr(X), _ptr(T)))

    def train(self, idx, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        """idx: (steps, batch) int array of data-set rows; returns per-step losses."""
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        if idx.ndim != 2:
            raise ValueError("idx must be (steps, batch)")
        steps, batch = idx.shape
        losses = np.empty(steps, dtype=np.float32)
        _check(lib().pdlp_mlp_train(self.h, steps, batch, _ptr(idx), lr, beta1, beta2, eps, _ptr(losses)))
        return losses

    def predict(self, X):
        X = _f32(X)
        if X.ndim != 2 or X.shape[1] != self.in_dim:
            raise ValueError("need X (count, %d)" % self.in_dim)
        Y = np.empty((X.shape[0], self.out_dim), dtype=np.float32)
        _check(lib().pdlp_mlp_predict(self.h, X.shape[0], _ptr(X), _ptr(Y)))
        return Y

    def gradients(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        loss = np.zeros(1, dtype=np.float32)
        g = np.empty(self.param_count, dtype=np.float32)
        _check(lib().pdlp_mlp_gradients(self.h, idx.size, _ptr(idx), _ptr(loss), _ptr(g)))
        return float(loss[0]), g

    def stats(self):
        mu = np.empty(self.out_dim, dtype=np.float32)
        sd = np.empty(self.out_dim, dtype=np.float32)
        _check(lib().pdlp_mlp_stats(self.h, _ptr(mu), _ptr(sd)))
        return mu, sd
