"""FP64 CPU oracle for the restarted-PDHG LP solver (test infrastructure).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
import this module; the solver itself never does.  The arithmetic lives in
``pdlp_oracle.c`` (plain C, compiled here with gcc); this file only builds it
and marshals numpy arrays through ctypes.

Parity pins: see tests/test_oracle_*.py (brute-force vertex enumeration,
closed forms, planted optima, an independent LP solver, hand-computed KKT and
PDHG-step examples, Algorithm 3 restart behaviour, and trajectories replayed
in numpy from solves stopped before and after each step or check: Algorithm
2's trials, the weighted average, the restart decisions, the primal-weight
updates, termination and infeasibility detection).  The restart heuristics'
constants (beta = 0.2 / 0.8 / 0.36, theta, check period) are "parity unpinned"
beyond the oracle implementing the printed rules.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdlp_oracle.c")
_LIB = os.path.join(_HERE, "libpdlp_oracle.so")

OPTIMAL, ITER_LIMIT, NUMERICAL, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE = 0, 1, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/libpdlp_oracle.so (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _LPStruct(C.Structure):
    _fields_ = [
        ("m", C.c_int32),
        ("n", C.c_int32),
        ("n_eq", C.c_int32),
        ("pad_", C.c_int32),
        ("row_ptr", C.c_void_p),
        ("col_idx", C.c_void_p),
        ("val", C.c_void_p),
        ("c", C.c_void_p),
        ("q", C.c_void_p),
        ("l", C.c_void_p),
        ("u", C.c_void_p),
        ("qd", C.c_void_p),
    ]


class _Params(C.Structure):
    _fields_ = [
        ("tol", C.c_double),
        ("max_iter", C.c_int64),
        ("check_period", C.c_int32),
        ("ruiz_iters", C.c_int32),
        ("pc_alpha", C.c_double),
        ("theta", C.c_double),
        ("eps_zero", C.c_double),
        ("beta_suff", C.c_double),
        ("beta_nec", C.c_double),
        ("beta_art", C.c_double),
        ("eps_infeas", C.c_double),
        ("restart_metric", C.c_int32),
        ("step_value_bits", C.c_int32),
    ]


class _Info(C.Structure):
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
        ("ray_obj", C.c_double),
        ("ray_res", C.c_double),
    ]


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

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, d, i32, i64 = C.c_void_p, C.c_double, C.c_int32, C.c_int64
        L.orc_solve.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, i32]
        L.orc_solve.restype = C.c_int
        L.orc_precondition.argtypes = [i32, i32, vp, vp, vp, i32, d, vp, vp]
        L.orc_precondition.restype = C.c_int
        L.orc_kkt_terms.argtypes = [vp, vp, vp, vp]
        L.orc_kkt_terms.restype = C.c_int
        L.orc_kkt_omega.argtypes = [vp, vp, vp, d]
        L.orc_kkt_omega.restype = d
        L.orc_terms_pass.argtypes = [vp, d]
        L.orc_terms_pass.restype = C.c_int
        L.orc_infeas_terms.argtypes = [vp, vp, vp, vp]
        L.orc_infeas_terms.restype = C.c_int
        L.orc_infeas_status.argtypes = [vp, d]
        L.orc_infeas_status.restype = C.c_int
        L.orc_primal_weight_init.argtypes = [d, d, d]
        L.orc_primal_weight_init.restype = d
        L.orc_primal_weight_update.argtypes = [d, d, d, d, d]
        L.orc_primal_weight_update.restype = d
        L.orc_eta_bar.argtypes = [d, d, d, d]
        L.orc_eta_bar.restype = d
        L.orc_eta_next.argtypes = [d, d, i64]
        L.orc_eta_next.restype = d
        L.orc_restart_mask.argtypes = [d, d, d, i64, i64, d, d, d]
        L.orc_restart_mask.restype = i32
        L.orc_pdhg_step.argtypes = [vp, vp, vp, d, d, vp, vp]
        L.orc_pdhg_step.restype = C.c_int
        L.orc_normalized_gap.argtypes = [vp, vp, vp, d, d]
        L.orc_normalized_gap.restype = d
        L.orc_kkt_standard.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp]
        L.orc_kkt_standard.restype = d
        L.orc_alg3.argtypes = [i32, i32, vp, vp, vp, vp, vp, d, d, i64, vp, vp, vp, vp, i32]
        L.orc_alg3.restype = i32
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class _Holder:
    """Keeps the arrays behind an _LPStruct alive."""

    def __init__(self, m, n, n_eq, c, row_ptr, col_idx, val, q, l, u, qd=None):
        self.arrs = [
            np.ascontiguousarray(row_ptr, dtype=np.int32),
            np.ascontiguousarray(col_idx, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64),
            np.ascontiguousarray(c, dtype=np.float64),
            np.ascontiguousarray(q, dtype=np.float64),
            np.ascontiguousarray(l, dtype=np.float64),
            np.ascontiguousarray(u, dtype=np.float64),
        ]
        # keep zero-length arrays addressable
        self.arrs = [a if a.size else np.zeros(1, dtype=a.dtype) for a in self.arrs]
        rp, ci, v, cc, qq, ll, uu = self.arrs
        self.qd = None if qd is None else np.ascontiguousarray(qd, dtype=np.float64)
        if self.qd is not None and self.qd.size == 0:
            self.qd = np.zeros(1)
        self.s = _LPStruct(m, n, n_eq, 0, _p(rp), _p(ci), _p(v), _p(cc), _p(qq), _p(ll), _p(uu), _p(self.qd))

    @property
    def ref(self):
        return C.byref(self.s)


def _holder(lp):
    """The LP (or, with a `qdiag` field that is not None, the QP with
    objective x'Qx/2 + c'x, Q = diag(qdiag)) as the C structure."""
    return _Holder(lp.m, lp.n, lp.n_eq, lp.c, lp.row_ptr, lp.col_idx, lp.val, lp.q, lp.l, lp.u,
                   getattr(lp, "qdiag", None))


@dataclass
class Params:
    tol: float = 1e-4
    max_iter: int = 100000
    check_period: int = 64
    ruiz_iters: int = 10
    pc_alpha: float = 1.0
    theta: float = 0.5
    eps_zero: float = 1e-10
    beta_suff: float = 0.2
    beta_nec: float = 0.8
    beta_art: float = 0.36
    eps_infeas: float = 1e-8
    restart_metric: int = 0  # 0: KKT error (Sec. 3.4); 1: normalized duality gap (ablation only)
    # 64: FP64 K~; 32: Algorithm 2's products with K~ rounded to FP32 (the
    # FP32-values mode of the steps, up to the first check)
    step_value_bits: int = 64

    def struct(self):
        return _Params(self.tol, self.max_iter, self.check_period, self.ruiz_iters, self.pc_alpha,
                       self.theta, self.eps_zero, self.beta_suff, self.beta_nec, self.beta_art,
                       self.eps_infeas, self.restart_metric, self.step_value_bits)


@dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    status: int
    which: int
    iters: int
    attempts: int
    restarts: int
    checks: int
    pobj: float
    dobj: float
    rp_norm: float
    rd_norm: float
    q_norm: float
    c_norm: float
    omega: float
    eta_hat: float
    trace: np.ndarray
    ray_obj: float = 0.0
    ray_res: float = 0.0


def solve(lp, params: Params | None = None, x0=None, y0=None, trace_cap: int = 4096, **kw) -> Result:
    """Algorithm 1 + 2 on `lp` (an lpgen.LP or anything with the same fields)."""
    params = params or Params(**kw)
    h = _holder(lp)
    x = np.zeros(max(lp.n, 1))
    y = np.zeros(max(lp.m, 1))
    info = _Info()
    trace = np.zeros(max(trace_cap, 1), dtype=CHECK_DTYPE)
    x0a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    y0a = None if y0 is None else np.ascontiguousarray(y0, dtype=np.float64)
    ps = params.struct()
    nt = lib().orc_solve(h.ref, C.byref(ps), _p(x0a), _p(y0a), _p(x), _p(y), C.byref(info),
                         _p(trace), trace_cap)
    if nt < 0:
        raise ValueError("oracle rejected the LP (code %d)" % nt)
    return Result(x=x[: lp.n], y=y[: lp.m], status=info.status, which=info.which, iters=info.iters,
                  attempts=info.attempts, restarts=info.restarts, checks=info.checks, pobj=info.pobj,
                  dobj=info.dobj, rp_norm=info.rp_norm, rd_norm=info.rd_norm, q_norm=info.q_norm,
                  c_norm=info.c_norm, omega=info.omega, eta_hat=info.eta_hat, trace=trace[:nt].copy(),
                  ray_obj=info.ray_obj, ray_res=info.ray_res)


def precondition(lp, ruiz_iters: int = 10, pc_alpha: float = 1.0):
    """Sec. 2.2 scaling: returns (scaled values, D1, D2)."""
    sv = np.array(lp.val, dtype=np.float64, copy=True)
    if sv.size == 0:
        sv = np.zeros(1)
    D1 = np.zeros(max(lp.m, 1))
    D2 = np.zeros(max(lp.n, 1))
    rp = np.ascontiguousarray(lp.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(lp.col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)
    lib().orc_precondition(lp.m, lp.n, _p(rp), _p(ci), _p(sv), ruiz_iters, pc_alpha, _p(D1), _p(D2))
    return sv[: lp.nnz], D1[: lp.m], D2[: lp.n]


def normalized_gap(lp, x, y, omega, r):
    """rho_r(z): the normalized duality gap of (x, y) on `lp` as given (no
    scaling) over the omega-norm ball of radius r cut by X x Y (restart-metric
    ablation; see normalized_gap in pdlp_oracle.c)."""
    h = _holder(lp)
    xa = np.ascontiguousarray(x, dtype=np.float64)
    ya = np.ascontiguousarray(y, dtype=np.float64)
    xa = xa if xa.size else np.zeros(1)
    ya = ya if ya.size else np.zeros(1)
    return lib().orc_normalized_gap(h.ref, _p(xa), _p(ya), float(omega), float(r))


def kkt_terms(lp, x, y):
    """Sec. 4.1 quantities {pobj, dobj, ||r_p||, ||r_d||, ||q||, ||c||} at (x, y)."""
    h = _holder(lp)
    xa = np.ascontiguousarray(x, dtype=np.float64)
    ya = np.ascontiguousarray(y, dtype=np.float64)
    xa = xa if xa.size else np.zeros(1)
    ya = ya if ya.size else np.zeros(1)
    out = np.zeros(6)
    lib().orc_kkt_terms(h.ref, _p(xa), _p(ya), _p(out))
    return dict(pobj=out[0], dobj=out[1], rp=out[2], rd=out[3], q_norm=out[4], c_norm=out[5], raw=out)


def relative_kkt(lp, x, y):
    """The three left-hand sides of Sec. 4.1 divided by their right-hand
    factors: the smallest epsilon for which (x, y) passes."""
    t = kkt_terms(lp, x, y)
    gap = abs(t["dobj"] - t["pobj"]) / (1.0 + abs(t["dobj"]) + abs(t["pobj"]))
    return max(gap, t["rp"] / (1.0 + t["q_norm"]), t["rd"] / (1.0 + t["c_norm"]))


def passes(lp, x, y, tol: float) -> bool:
    t = kkt_terms(lp, x, y)
    return bool(lib().orc_terms_pass(_p(t["raw"]), tol))


def infeas_terms(lp, xr, yr):
    """Certificate measures of a primal ray xr and a dual ray yr on the LP as
    given: {dual-ray objective, dual-ray residual, primal-ray objective
    (-c'xr), primal-ray residual}."""
    h = _holder(lp)
    xa = np.ascontiguousarray(xr, dtype=np.float64)
    ya = np.ascontiguousarray(yr, dtype=np.float64)
    xa = xa if xa.size else np.zeros(1)
    ya = ya if ya.size else np.zeros(1)
    out = np.zeros(4)
    lib().orc_infeas_terms(h.ref, _p(xa), _p(ya), _p(out))
    return out


def infeas_status(terms, eps: float) -> int:
    """PRIMAL_INFEASIBLE / DUAL_INFEASIBLE certified by infeas_terms' output at
    relative tolerance eps, else -1."""
    t = np.ascontiguousarray(terms, dtype=np.float64)
    return int(lib().orc_infeas_status(_p(t), eps))


def kkt_omega(lp, x, y, omega: float) -> float:
    h = _holder(lp)
    xa = np.ascontiguousarray(x, dtype=np.float64)
    ya = np.ascontiguousarray(y, dtype=np.float64)
    xa = xa if xa.size else np.zeros(1)
    ya = ya if ya.size else np.zeros(1)
    return lib().orc_kkt_omega(h.ref, _p(xa), _p(ya), omega)


def pdhg_step(lp, x, y, tau: float, sigma: float):
    """eq. (pdhg): one vanilla step with explicit tau, sigma (no scaling)."""
    h = _holder(lp)
    xa = np.ascontiguousarray(x, dtype=np.float64)
    ya = np.ascontiguousarray(y, dtype=np.float64)
    xo = np.zeros(max(lp.n, 1))
    yo = np.zeros(max(lp.m, 1))
    lib().orc_pdhg_step(h.ref, _p(xa), _p(ya), tau, sigma, _p(xo), _p(yo))
    return xo[: lp.n], yo[: lp.m]


def primal_weight_init(c_norm, q_norm, eps_zero=1e-10):
    return lib().orc_primal_weight_init(c_norm, q_norm, eps_zero)


def primal_weight_update(dx, dy, omega, theta=0.5, eps_zero=1e-10):
    return lib().orc_primal_weight_update(dx, dy, omega, theta, eps_zero)


def eta_bar(dx2, dy2, cross, omega):
    return lib().orc_eta_bar(dx2, dy2, cross, omega)


def eta_next(eta, eta_b, k):
    return lib().orc_eta_next(eta, eta_b, k)


def restart_mask(kkt_cand, kkt_start, kkt_prev, t, k, beta_suff=0.2, beta_nec=0.8, beta_art=0.36):
    return lib().orc_restart_mask(kkt_cand, kkt_start, kkt_prev, t, k, beta_suff, beta_nec, beta_art)


def kkt_standard(A_rp, A_ci, A_v, b, c, x, y, m, n):
    rp = np.ascontiguousarray(A_rp, dtype=np.int32)
    ci = np.ascontiguousarray(A_ci, dtype=np.int32)
    v = np.ascontiguousarray(A_v, dtype=np.float64)
    return lib().orc_kkt_standard(m, n, _p(rp), _p(ci), _p(v), _p(np.ascontiguousarray(b, dtype=np.float64)),
                                  _p(np.ascontiguousarray(c, dtype=np.float64)),
                                  _p(np.ascontiguousarray(x, dtype=np.float64)),
                                  _p(np.ascontiguousarray(y, dtype=np.float64)))


def alg3(A_rp, A_ci, A_v, b, c, m, n, s, beta, max_iter, cap=1000):
    """Algorithm 3 (Appendix A) from zero: returns (x, y, kkt at restart
    points [kkt(z^{0,0}), kkt(z^{1,0}), ...], inner-loop lengths)."""
    rp = np.ascontiguousarray(A_rp, dtype=np.int32)
    ci = np.ascontiguousarray(A_ci, dtype=np.int32)
    v = np.ascontiguousarray(A_v, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    cc = np.ascontiguousarray(c, dtype=np.float64)
    x = np.zeros(n)
    y = np.zeros(m)
    kr = np.zeros(cap)
    lr = np.zeros(cap, dtype=np.int64)
    nr = lib().orc_alg3(m, n, _p(rp), _p(ci), _p(v), _p(bb), _p(cc), s, beta, max_iter, _p(x), _p(y),
                        _p(kr), _p(lr), cap)
    if nr < 0:
        raise MemoryError("alg3 allocation failed")
    return x, y, kr[: min(nr + 1, cap)], lr[: min(nr, cap)]
