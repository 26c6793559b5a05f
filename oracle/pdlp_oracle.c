/*
 * pdlp_oracle.c -- plain, slow, single-threaded FP64 restarted PDHG for LP.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the CUDA
 * solver: it shares no code, header, table or helper with the CUDA path, and
 * only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg load it.  It is written for a reader checking it against the cuPDLP.jl
 * paper (Lu & Yang, arXiv 2311.12180) line by line: straightforward loops over
 * CSR, naive left-to-right sums, no blocking, fusion or reordering.
 *
 * What it computes, in the paper's notation:
 *   LP (Sec. 2, eq. lp):  min c'x  s.t.  Gx >= h, Ax = b, l <= x <= u,
 *     with K = (A; G) (equality rows first), q = (b; h).
 *   Saddle problem (eq. primal-dual): L(x,y) = c'x - y'Kx + q'y over
 *     X = {l <= x <= u}, Y = {y_i >= 0 on ">=" rows}.
 *   Preconditioning (Sec. 2.2, first bullet): Ruiz (l_inf) passes, then
 *     Pock-Chambolle with exponent alpha; K~ = D1 K D2, c~ = D2 c,
 *     q~ = D1 q, l~ = l / D2, u~ = u / D2.
 *   Restarted PDHG (Algorithm 1) with the adaptive step of Algorithm 2 and
 *     step-size condition eq. (step-size), running average weighted by the
 *     accepted step sizes, restart candidate / criteria of Sec. 3.4 on the
 *     KKT error eq. (kkt), primal-weight initialisation and update of
 *     Sec. 2.2, relative-KKT termination on the ORIGINAL LP (Sec. 4.1).
 *   Restarted PDHG for standard-form LP with fixed step and uniform average
 *     (Algorithm 3, Appendix A) as a separate test-only routine.
 *   QP extension (orc_lp.qd != NULL; the introduction names the extension
 *     to quadratic programs): objective x'Qx/2 + c'x with Q diagonal; the
 *     primal step is the exact proximal step x' = proj_X((x - tau(c - K'y)) /
 *     (1 + tau Q)) (per coordinate), the KKT pieces use the objective's
 *     gradient c + Qx and the QP's objectives (kkt_pieces), Q is scaled as
 *     D2 Q D2, and infeasibility detection is off.
 *   Restart-metric ablation (orc_params.restart_metric = 1, not the paper's
 *     method): the same restart scheme driven by the normalized duality gap
 *     of the CPU PDLP restart scheme the paper replaces (normalized_gap),
 *     with the readings listed there.
 *
 * Readings where the paper is silent or garbled (each also used by the CUDA
 * path, which implements them independently):
 *   - PrimalWeightUpdate: omega = exp(theta*log(dy/dx) + (1-theta)*log(omega))
 *     (the printed formula mixes log and linear terms); theta = 0.5.
 *   - The running average restarts with each epoch; its weights are the
 *     accepted step sizes eta returned by Algorithm 2.
 *   - lambda = proj_Lambda(c - K'y) with Lambda_j = R (both bounds finite),
 *     R+ (only l finite), R- (only u finite), {0} (free); 0*inf = 0.
 *   - ||K||_inf in the initial step size = max |K~_ij| of the scaled matrix
 *     (1 if K is empty).
 *   - eps_zero = 1e-10.
 *   - The restart / termination check runs after every accepted iteration k
 *     with k % P == 0 (and at k == max_iter); P = 64 by default.
 *   - k in the exponents of Algorithm 2 counts accepted steps over the whole
 *     run (never reset), from 1: the base is k + 2 for k accepted steps so
 *     far (the literal (0+1)^-0.3 = 1 would zero the first step size).
 *   - eq. (step-size) uses |(y'-y)'K(x'-x)| in the denominator (see
 *     orc_eta_bar); eta_bar = +inf when it is exactly zero.
 *   - KKT_omega weights the primal residual by omega^2 and the dual one by
 *     omega^-2, as printed in eq. (kkt); it is evaluated on the scaled LP.
 *   - After a restart with a new omega, KKT(z^{n,0}) is re-evaluated with the
 *     new omega; the "previous candidate" at the first check of an epoch is
 *     z^{n,0} itself.
 *   - Candidate tie -> average.  Termination tests the current iterate first,
 *     then the average.
 *   - The returned x = D2 x^ is projected onto X (removes unscaling rounding).
 *   - Ruiz: 10 passes, row/col factor sqrt(max|K~|) (1 for an empty line);
 *     Pock-Chambolle alpha = 1: row factor sqrt(sum_j |K~_ij|^(2-alpha)),
 *     column factor sqrt(sum_i |K~_ij|^alpha).
 *   - Infeasibility detection (Sec. 2.2, last bullet, which names the two
 *     sequences but not the certificate tests): at every check, after the
 *     Sec. 4.1 test fails, the ray z^{n,t} - z^{n,t-1} (difference of the
 *     last two accepted iterates) and then z^{n,t} - z^{n,0} (the normalised
 *     iterate times t; the tests are invariant to positive scaling) are
 *     unscaled to the original LP and tested by orc_infeas_terms /
 *     infeas_status, dual ray (primal infeasibility) before primal ray (dual
 *     infeasibility); both tests use relative tolerance eps_infeas (0 turns
 *     detection off).  Then the iteration limit, then the restart.
 *
 * Pins (tests/test_oracle_pins.py) tie every routine to hand-worked
 * examples, closed forms, brute force or an independent solver, except the
 * restart constants themselves (beta = 0.2 / 0.8 / 0.36, theta = 0.5, the
 * check period): those are "parity unpinned" beyond implementing the printed
 * rules.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fused multiply-add, so
 * the results are the same on x86-64 and aarch64).
 */

#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_NOMEM (-3)

#define ORC_OPTIMAL 0
#define ORC_ITER_LIMIT 1
#define ORC_NUMERICAL 3
#define ORC_PRIMAL_INFEASIBLE 4
#define ORC_DUAL_INFEASIBLE 5

typedef struct {
  int32_t m, n, n_eq, pad_;
  const int32_t *row_ptr;
  const int32_t *col_idx;
  const double *val;
  const double *c, *q, *l, *u;
  const double *qd; /* diagonal of Q for the QP extension (objective 1/2 x'Qx + c'x), NULL for an LP */
} orc_lp;

typedef struct {
  double tol;
  int64_t max_iter;
  int32_t check_period;
  int32_t ruiz_iters;
  double pc_alpha; /* < 0 disables Pock-Chambolle */
  double theta;
  double eps_zero;
  double beta_suff, beta_nec, beta_art;
  double eps_infeas; /* relative tolerance of the infeasibility certificates; 0 = off */
  int32_t restart_metric; /* 0: KKT error, eq. (kkt) (Sec. 3.4); 1: normalized duality gap
                             (the restart metric of CPU PDLP the paper compares against) */
  int32_t step_value_bits; /* 64 (or 0): FP64 K~ throughout; 32: the products of Algorithm 2's
                              trials and of the accepted iterate use K~ rounded to FP32 (values
                              below the smallest normal float become signed zeros), everything
                              else stays FP64 -- the FP32-values mode of the steps, followed up to
                              the first restart / termination check (the GPU's checks then
                              recompute their products with the FP64 K~) */
} orc_params;

typedef struct {
  int32_t status;
  int32_t which; /* 0 = current iterate returned, 1 = average; infeasible:
                    2 = difference ray, 3 = normalised-iterate ray */
  int64_t iters;
  int64_t attempts;
  int64_t restarts;
  int64_t checks;
  double pobj, dobj, rp_norm, rd_norm, q_norm, c_norm;
  double omega, eta_hat;
  double ray_obj, ray_res; /* infeasible: the certificate's objective and residual norm */
} orc_info;

typedef struct {
  int64_t k;
  int64_t attempts; /* Algorithm 2 trials so far */
  int64_t restarts; /* restarts so far, this check's included */
  int32_t restart;  /* bit0 (i) sufficient, bit1 (ii) necessary, bit2 (iii) artificial */
  int32_t cand_avg; /* 1 if the restart candidate is the average */
  double kkt_cur, kkt_avg, kkt_start;
  double omega, eta_hat;
  /* Sec. 4.1 relative measures of the current iterate on the original LP:
   * |pobj - dobj| / (1 + |pobj| + |dobj|), ||rp|| / (1 + ||q||), ||rd|| / (1 + ||c||) */
  double rel_gap, rel_primal, rel_dual;
} orc_check;

/* ------------------------------------------------------------------------ */
/* basic sparse / dense pieces                                               */
/* ------------------------------------------------------------------------ */

/* y = K x (row-major CSR). */
static void spmv(int32_t m, const int32_t *rp, const int32_t *ci, const double *v, const double *x,
                 double *y) {
  for (int32_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) s += v[e] * x[ci[e]];
    y[i] = s;
  }
}

/* Transpose pattern: CSR of K' (n rows) with perm[e'] = index into K's arrays. */
static int transpose_pattern(int32_t m, int32_t n, const int32_t *rp, const int32_t *ci, int32_t *tp,
                             int32_t *ti, int64_t *perm) {
  memset(tp, 0, sizeof(int32_t) * ((size_t)n + 1));
  for (int32_t i = 0; i < m; ++i)
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) tp[ci[e] + 1]++;
  for (int32_t j = 0; j < n; ++j) tp[j + 1] += tp[j];
  int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  if (!fill) return ORC_ERR_NOMEM;
  memcpy(fill, tp, sizeof(int32_t) * ((size_t)n + 1));
  for (int32_t i = 0; i < m; ++i)
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
      int32_t pos = fill[ci[e]]++;
      ti[pos] = i;
      perm[pos] = e;
    }
  free(fill);
  return ORC_OK;
}

static double dot(int32_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double norm2(int32_t n, const double *a) { return sqrt(dot(n, a, a)); }

static double clamp(double v, double lo, double hi) {
  if (v < lo) v = lo;
  if (v > hi) v = hi;
  return v;
}

/* lambda_j = proj onto Lambda_j of d = (c - K'y)_j (reading in the header). */
static double proj_lambda(double d, double lj, double uj) {
  int lf = isfinite(lj), uf = isfinite(uj);
  if (lf && uf) return d;
  if (lf) return d > 0.0 ? d : 0.0;
  if (uf) return d < 0.0 ? d : 0.0;
  return 0.0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2: diagonal preconditioning                                        */
/* ------------------------------------------------------------------------ */

/* Scales sv (a copy of K's values) in place to K~ = D1 K D2 and returns D1,
 * D2.  Ruiz: `ruiz_iters` l_inf passes; then Pock-Chambolle with exponent
 * alpha (skipped when alpha < 0). */
int orc_precondition(int32_t m, int32_t n, const int32_t *rp, const int32_t *ci, double *sv,
                     int32_t ruiz_iters, double alpha, double *D1, double *D2) {
  double *r = (double *)malloc(sizeof(double) * ((size_t)m + 1));
  double *s = (double *)malloc(sizeof(double) * ((size_t)n + 1));
  if (!r || !s) {
    free(r);
    free(s);
    return ORC_ERR_NOMEM;
  }
  for (int32_t i = 0; i < m; ++i) D1[i] = 1.0;
  for (int32_t j = 0; j < n; ++j) D2[j] = 1.0;
  int passes = ruiz_iters + (alpha >= 0.0 ? 1 : 0);
  for (int it = 0; it < passes; ++it) {
    int ruiz = it < ruiz_iters;
    for (int32_t i = 0; i < m; ++i) r[i] = 0.0;
    for (int32_t j = 0; j < n; ++j) s[j] = 0.0;
    for (int32_t i = 0; i < m; ++i)
      for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
        double a = fabs(sv[e]);
        int32_t j = ci[e];
        if (ruiz) {
          if (a > r[i]) r[i] = a;
          if (a > s[j]) s[j] = a;
        } else {
          r[i] += (alpha == 1.0) ? a : pow(a, 2.0 - alpha);
          s[j] += (alpha == 1.0) ? a : pow(a, alpha);
        }
      }
    for (int32_t i = 0; i < m; ++i) r[i] = r[i] > 0.0 ? sqrt(r[i]) : 1.0;
    for (int32_t j = 0; j < n; ++j) s[j] = s[j] > 0.0 ? sqrt(s[j]) : 1.0;
    for (int32_t i = 0; i < m; ++i)
      for (int32_t e = rp[i]; e < rp[i + 1]; ++e) sv[e] = sv[e] / r[i] / s[ci[e]];
    for (int32_t i = 0; i < m; ++i) D1[i] = D1[i] / r[i];
    for (int32_t j = 0; j < n; ++j) D2[j] = D2[j] / s[j];
  }
  free(r);
  free(s);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* KKT quantities                                                            */
/* ------------------------------------------------------------------------ */

/* The three pieces of eq. (kkt) / Sec. 4.1 for the LP (c, K, q, l, u) at
 * (x, y), given Kx = K x and KTy = K' y:
 *   rp2 = ||(Ax - b, [h - Gx]^+)||^2
 *   rd2 = ||c - K'y - lambda||^2
 *   pobj = c'x,  dobj = q'y + l'lambda^+ - u'lambda^-
 * With a diagonal Q (qd != NULL, the QP extension) the gradient of the
 * objective replaces c: lambda = proj_Lambda(c + Qx - K'y),
 * rd2 = ||c + Qx - K'y - lambda||^2, pobj = c'x + x'Qx / 2 and
 * dobj = q'y + l'lambda^+ - u'lambda^- - x'Qx / 2 (the QP's dual objective). */
static void kkt_pieces(int32_t m, int32_t n, int32_t n_eq, const double *c, const double *q,
                       const double *l, const double *u, const double *qd, const double *x, const double *y,
                       const double *Kx, const double *KTy, double *rp2, double *rd2, double *pobj,
                       double *dobj) {
  double sp = 0.0;
  for (int32_t i = 0; i < m; ++i) {
    double r = q[i] - Kx[i];
    if (i >= n_eq) r = r > 0.0 ? r : 0.0;
    sp += r * r;
  }
  double sd = 0.0, lu = 0.0, xqx = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    double d = qd ? c[j] + qd[j] * x[j] - KTy[j] : c[j] - KTy[j];
    double lam = proj_lambda(d, l[j], u[j]);
    double r = d - lam;
    sd += r * r;
    if (lam > 0.0) lu += l[j] * lam;
    if (lam < 0.0) lu -= u[j] * (-lam);
    if (qd) xqx += qd[j] * x[j] * x[j];
  }
  *rp2 = sp;
  *rd2 = sd;
  *pobj = dot(n, c, x) + 0.5 * xqx;
  *dobj = dot(m, q, y) + lu - 0.5 * xqx;
}

/* eq. (kkt): KKT_omega from its pieces. */
static double kkt_omega_from(double rp2, double rd2, double pobj, double dobj, double omega) {
  double gap = dobj - pobj;
  return sqrt(omega * omega * rp2 + rd2 / (omega * omega) + gap * gap);
}

/* Sec. 4.1 termination quantities on the LP as given:
 * out = {pobj, dobj, ||r_p||, ||r_d||, ||q||, ||c||}.  Exported for tests. */
int orc_kkt_terms(const orc_lp *lp, const double *x, const double *y, double *out) {
  int32_t m = lp->m, n = lp->n;
  double *Kx = (double *)calloc((size_t)m + 1, sizeof(double));
  double *KTy = (double *)calloc((size_t)n + 1, sizeof(double));
  if (!Kx || !KTy) {
    free(Kx);
    free(KTy);
    return ORC_ERR_NOMEM;
  }
  spmv(m, lp->row_ptr, lp->col_idx, lp->val, x, Kx);
  /* K'y by scattering rows (plain definition (K'y)_j = sum_i K_ij y_i). */
  for (int32_t i = 0; i < m; ++i)
    for (int32_t e = lp->row_ptr[i]; e < lp->row_ptr[i + 1]; ++e) KTy[lp->col_idx[e]] += lp->val[e] * y[i];
  double rp2, rd2, pobj, dobj;
  kkt_pieces(m, n, lp->n_eq, lp->c, lp->q, lp->l, lp->u, lp->qd, x, y, Kx, KTy, &rp2, &rd2, &pobj, &dobj);
  out[0] = pobj;
  out[1] = dobj;
  out[2] = sqrt(rp2);
  out[3] = sqrt(rd2);
  out[4] = norm2(m, lp->q);
  out[5] = norm2(n, lp->c);
  free(Kx);
  free(KTy);
  return ORC_OK;
}

/* eq. (kkt) on the LP as given.  Exported for tests. */
double orc_kkt_omega(const orc_lp *lp, const double *x, const double *y, double omega) {
  double t[6];
  if (orc_kkt_terms(lp, x, y, t) != ORC_OK) return NAN;
  return kkt_omega_from(t[2] * t[2], t[3] * t[3], t[0], t[1], omega);
}

/* Infeasibility certificates of the LP as given, for a primal ray xr (n)
 * and a dual ray yr (m), by LP duality:
 *   dual ray (certifies primal infeasibility): lambda = proj_Lambda(-K'yr),
 *     out[0] = q'yr + l'lambda+ - u'lambda-   (must be > 0),
 *     out[1] = ||(-K'yr - lambda, min(yr_i, 0) on ">=" rows)||_2;
 *   primal ray (certifies dual infeasibility):
 *     out[2] = -c'xr                          (must be > 0),
 *     out[3] = ||(K_E xr, min(K_G xr, 0), distance of xr to the recession
 *              cone of X: xr_j >= 0 where l_j is finite, <= 0 where u_j is
 *              finite)||_2.
 * Lambda_j is the cone of the header's lambda reading, so lambda_j > 0 only
 * where l_j is finite and lambda_j < 0 only where u_j is finite.  Exported
 * for tests. */
int orc_infeas_terms(const orc_lp *lp, const double *xr, const double *yr, double *out) {
  int32_t m = lp->m, n = lp->n;
  double *Kx = (double *)calloc((size_t)m + 1, sizeof(double));
  double *KTy = (double *)calloc((size_t)n + 1, sizeof(double));
  if (!Kx || !KTy) {
    free(Kx);
    free(KTy);
    return ORC_ERR_NOMEM;
  }
  spmv(m, lp->row_ptr, lp->col_idx, lp->val, xr, Kx);
  for (int32_t i = 0; i < m; ++i)
    for (int32_t e = lp->row_ptr[i]; e < lp->row_ptr[i + 1]; ++e) KTy[lp->col_idx[e]] += lp->val[e] * yr[i];
  double obj_d = 0.0, res_d = 0.0, obj_p = 0.0, res_p = 0.0;
  for (int32_t i = 0; i < m; ++i) {
    obj_d += lp->q[i] * yr[i];
    if (i >= lp->n_eq) {
      double v = yr[i] < 0.0 ? yr[i] : 0.0;
      res_d += v * v;
      double r = Kx[i] < 0.0 ? Kx[i] : 0.0;
      res_p += r * r;
    } else {
      res_p += Kx[i] * Kx[i];
    }
  }
  for (int32_t j = 0; j < n; ++j) {
    double a = -KTy[j];
    double lam = proj_lambda(a, lp->l[j], lp->u[j]);
    double r = a - lam;
    res_d += r * r;
    if (lam > 0.0) obj_d += lp->l[j] * lam;
    if (lam < 0.0) obj_d -= lp->u[j] * (-lam);
    obj_p -= lp->c[j] * xr[j];
    double v = 0.0;
    if (isfinite(lp->l[j]) && xr[j] < 0.0) v += xr[j] * xr[j];
    if (isfinite(lp->u[j]) && xr[j] > 0.0) v += xr[j] * xr[j];
    res_p += v;
  }
  out[0] = obj_d;
  out[1] = sqrt(res_d);
  out[2] = obj_p;
  out[3] = sqrt(res_p);
  free(Kx);
  free(KTy);
  return ORC_OK;
}

/* Status certified by orc_infeas_terms' output t at tolerance eps: primal
 * infeasible (dual ray) first, then dual infeasible (primal ray), else -1. */
static int infeas_status(const double *t, double eps) {
  if (t[0] > 0.0 && t[1] <= eps * t[0]) return ORC_PRIMAL_INFEASIBLE;
  if (t[2] > 0.0 && t[3] <= eps * t[2]) return ORC_DUAL_INFEASIBLE;
  return -1;
}
int orc_infeas_status(const double *t, double eps) { return infeas_status(t, eps); }

/* Sec. 4.1: all three relative inequalities hold with epsilon = tol. */
static int terms_pass(const double *t, double tol) {
  double pobj = t[0], dobj = t[1];
  if (!(fabs(dobj - pobj) <= tol * (1.0 + fabs(dobj) + fabs(pobj)))) return 0;
  if (!(t[2] <= tol * (1.0 + t[4]))) return 0;
  if (!(t[3] <= tol * (1.0 + t[5]))) return 0;
  return 1;
}

int orc_terms_pass(const double *t, double tol) { return terms_pass(t, tol); }

/* ------------------------------------------------------------------------ */
/* small scalar rules, exported so tests can pin them one by one             */
/* ------------------------------------------------------------------------ */

/* Sec. 2.2 InitializePrimalWeight. */
double orc_primal_weight_init(double c_norm, double q_norm, double eps_zero) {
  if (c_norm > eps_zero && q_norm > eps_zero) return c_norm / q_norm;
  return 1.0;
}

/* Sec. 2.2 PrimalWeightUpdate (log-space smoothing reading). */
double orc_primal_weight_update(double dx, double dy, double omega, double theta, double eps_zero) {
  if (dx > eps_zero && dy > eps_zero) return exp(theta * log(dy / dx) + (1.0 - theta) * log(omega));
  return omega;
}

/* Algorithm 2: eta_bar from the step's pieces (eq. step-size), with the
 * interaction term taken in absolute value: for the Lagrangian of eq.
 * (primal-dual) the PDHG metric's cross term is +2 dy'K dx, so the printed
 * sign alone would accept divergent steps; |dy'K dx| is safe for either sign
 * convention.  eta_bar = +inf when the interaction is exactly zero. */
double orc_eta_bar(double dx2, double dy2, double cross, double omega) {
  double a = fabs(cross);
  if (!(a > 0.0)) return INFINITY;
  return (omega * dx2 + dy2 / omega) / (2.0 * a);
}

/* Algorithm 2: next trial step size.  k = accepted steps before this call;
 * the exponent base is the 1-based number of the step being taken plus one,
 * k + 2 (read literally with k = 0 the printed (k+1)^-0.3 = 1 makes the
 * first factor 0 and the step size collapses to zero). */
double orc_eta_next(double eta, double eta_bar, int64_t k) {
  double kk = (double)(k + 2);
  double a = (1.0 - pow(kk, -0.3)) * eta_bar;
  double b = (1.0 + pow(kk, -0.6)) * eta;
  return a < b ? a : b;
}

/* Sec. 3.4 restart criteria; returns a bit mask of the criteria that hold. */
int32_t orc_restart_mask(double kkt_cand, double kkt_start, double kkt_prev_cand, int64_t t, int64_t k,
                         double beta_suff, double beta_nec, double beta_art) {
  int32_t mask = 0;
  if (kkt_cand <= beta_suff * kkt_start) mask |= 1;
  if (kkt_cand <= beta_nec * kkt_start && kkt_cand > kkt_prev_cand) mask |= 2;
  if ((double)t >= beta_art * (double)k) mask |= 4;
  return mask;
}

/* eq. (pdhg): one vanilla PDHG step with explicit tau, sigma on the LP as
 * given.  Exported for the hand-computed test. */
int orc_pdhg_step(const orc_lp *lp, const double *x, const double *y, double tau, double sigma,
                  double *x_out, double *y_out) {
  int32_t m = lp->m, n = lp->n;
  double *KTy = (double *)calloc((size_t)n + 1, sizeof(double));
  double *v = (double *)calloc((size_t)n + 1, sizeof(double));
  double *Kv = (double *)calloc((size_t)m + 1, sizeof(double));
  if (!KTy || !v || !Kv) {
    free(KTy);
    free(v);
    free(Kv);
    return ORC_ERR_NOMEM;
  }
  for (int32_t i = 0; i < m; ++i)
    for (int32_t e = lp->row_ptr[i]; e < lp->row_ptr[i + 1]; ++e) KTy[lp->col_idx[e]] += lp->val[e] * y[i];
  for (int32_t j = 0; j < n; ++j) x_out[j] = clamp(x[j] - tau * (lp->c[j] - KTy[j]), lp->l[j], lp->u[j]);
  for (int32_t j = 0; j < n; ++j) v[j] = 2.0 * x_out[j] - x[j];
  spmv(m, lp->row_ptr, lp->col_idx, lp->val, v, Kv);
  for (int32_t i = 0; i < m; ++i) {
    double yn = y[i] + sigma * (lp->q[i] - Kv[i]);
    if (i >= lp->n_eq && yn < 0.0) yn = 0.0;
    y_out[i] = yn;
  }
  free(KTy);
  free(v);
  free(Kv);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* normalized duality gap (restart-metric ablation, not the paper's metric)  */
/* ------------------------------------------------------------------------ */

/* Normalized duality gap of z = (x, y) on the scaled LP with radius r in the
 * primal-weight norm ||(dx, dy)||_omega^2 = omega ||dx||^2 + ||dy||^2 / omega:
 *   rho_r(z) = (1/r) max { L(x, y^) - L(x^, y) : z^ in X x Y, ||z^ - z||_omega <= r },
 * the restart metric of the CPU PDLP restart scheme that Sec. 3.4 replaces
 * by the KKT error (Sec. 2.2 "Adaptive restarts"; Appendix A).  With
 * L(x, y) = c'x - y'Kx + q'y the objective is linear in d = z^ - z:
 *   L(x, y^) - L(x^, y) = -(c - K'y)'dx + (q - Kx)'dy   (zero at d = 0).
 * In e = (sqrt(omega) dx, dy / sqrt(omega)) the ball is ||e|| <= r, the
 * objective is h'e with h = (-(c - K'y) / sqrt(omega), sqrt(omega)(q - Kx)),
 * and X x Y becomes a box B around 0 (lower bound -y / sqrt(omega) on ">="
 * rows).  A linear function over a ball cut by a box is maximised by
 * e(t) = proj_B(t h) with t >= 0 the largest at which ||e(t)|| <= r
 * (||e(t)|| does not decrease in t); t is found by bisection.  r = 0 or
 * h = 0 gives 0.  Kx = K x, KTy = K' y. */
static double box_step(double t, double h, double lo, double hi) {
  double v = t * h;
  if (v < lo) v = lo;
  if (v > hi) v = hi;
  return v;
}

/* ||e(t)||^2 and h'e(t) at the multiplier t (one pass over the coordinates). */
static void gap_eval(double t, int32_t m, int32_t n, int32_t n_eq, const double *c, const double *q,
                     const double *l, const double *u, const double *x, const double *y, const double *Kx,
                     const double *KTy, double so, double *norm2, double *value) {
  double n2 = 0.0, v = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    const double h = -(c[j] - KTy[j]) / so;
    const double e = box_step(t, h, so * (l[j] - x[j]), so * (u[j] - x[j]));
    n2 += e * e;
    v += h * e;
  }
  for (int32_t i = 0; i < m; ++i) {
    const double h = so * (q[i] - Kx[i]);
    const double e = box_step(t, h, i >= n_eq ? -y[i] / so : -INFINITY, INFINITY);
    n2 += e * e;
    v += h * e;
  }
  *norm2 = n2;
  *value = v;
}

static double normalized_gap(int32_t m, int32_t n, int32_t n_eq, const double *c, const double *q,
                             const double *l, const double *u, const double *x, const double *y,
                             const double *Kx, const double *KTy, double omega, double r) {
  if (!(r > 0.0)) return 0.0;
  const double so = sqrt(omega);
  double n2, val, prev = -1.0, hi = 1.0;
  gap_eval(hi, m, n, n_eq, c, q, l, u, x, y, Kx, KTy, so, &n2, &val);
  /* grow t until the ball binds, or until the box alone bounds e */
  while (n2 < r * r) {
    if (n2 == prev || !(hi < 1e300)) return val / r; /* every coordinate at its bound */
    prev = n2;
    hi *= 2.0;
    gap_eval(hi, m, n, n_eq, c, q, l, u, x, y, Kx, KTy, so, &n2, &val);
  }
  double lo = 0.0;
  for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    gap_eval(mid, m, n, n_eq, c, q, l, u, x, y, Kx, KTy, so, &n2, &val);
    if (n2 <= r * r)
      lo = mid;
    else
      hi = mid;
  }
  gap_eval(lo, m, n, n_eq, c, q, l, u, x, y, Kx, KTy, so, &n2, &val);
  return val / r;
}

/* rho_r(z) for the tests, on the LP as given (no scaling). */
double orc_normalized_gap(const orc_lp *lp, const double *x, const double *y, double omega, double r) {
  double *Kx = (double *)calloc((size_t)lp->m + 1, sizeof(double));
  double *KTy = (double *)calloc((size_t)lp->n + 1, sizeof(double));
  if (!Kx || !KTy) {
    free(Kx);
    free(KTy);
    return NAN;
  }
  spmv(lp->m, lp->row_ptr, lp->col_idx, lp->val, x, Kx);
  for (int32_t i = 0; i < lp->m; ++i)
    for (int32_t e = lp->row_ptr[i]; e < lp->row_ptr[i + 1]; ++e) KTy[lp->col_idx[e]] += lp->val[e] * y[i];
  const double g = normalized_gap(lp->m, lp->n, lp->n_eq, lp->c, lp->q, lp->l, lp->u, x, y, Kx, KTy, omega, r);
  free(Kx);
  free(KTy);
  return g;
}

/* ||(x - xr, y - yr)||_omega */
static double wdist(int32_t m, int32_t n, const double *x, const double *y, const double *xr, const double *yr,
                    double omega) {
  double a = 0.0, b = 0.0;
  for (int32_t j = 0; j < n; ++j) a += (x[j] - xr[j]) * (x[j] - xr[j]);
  for (int32_t i = 0; i < m; ++i) b += (y[i] - yr[i]) * (y[i] - yr[i]);
  return sqrt(omega * a + b / omega);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 + Algorithm 2 (restarted PDHG with adaptive steps)            */
/* ------------------------------------------------------------------------ */

typedef struct {
  /* scaled problem */
  double *sv, *D1, *D2, *sc, *sq, *sl, *su;
  double *sqd; /* QP: the scaled diagonal D2 Q D2 (NULL for an LP) */
  int32_t *tp, *ti;
  double *tv;
  double *sv32, *tv32; /* K~ and K~' rounded to FP32 (step_value_bits = 32) */
  int64_t *perm;
  /* iterates and products */
  double *x, *y, *Kx, *KTy, *xp, *yp, *v, *Kv, *dxv, *Kdx;
  double *sum_x, *sum_y, *xb, *yb, *Kxb, *KTyb, *x_last, *y_last;
  double *xo, *yo;
  double *x_prev, *y_prev; /* the accepted iterate before the last one */
} orc_work;

static void free_work(orc_work *w) {
  double **d[] = {&w->sv, &w->D1, &w->D2, &w->sc, &w->sq, &w->sl, &w->su, &w->tv,
                  &w->x, &w->y, &w->Kx, &w->KTy, &w->xp, &w->yp, &w->v, &w->Kv,
                  &w->dxv, &w->Kdx, &w->sum_x, &w->sum_y, &w->xb, &w->yb, &w->Kxb,
                  &w->KTyb, &w->x_last, &w->y_last, &w->xo, &w->yo, &w->x_prev, &w->y_prev, &w->sqd,
                  &w->sv32, &w->tv32};
  for (size_t i = 0; i < sizeof(d) / sizeof(d[0]); ++i) {
    free(*d[i]);
    *d[i] = NULL;
  }
  free(w->tp);
  free(w->ti);
  free(w->perm);
}

/* v rounded to the nearest FP32 value; below the smallest normal float the
 * signed zero (the FP32-values mode's copy of K~). */
static double round_f32(double v) {
  float f = (float)v;
  if (fabsf(f) < FLT_MIN) f = copysignf(0.0f, f);
  return (double)f;
}

static int validate(const orc_lp *lp) {
  if (lp->m < 0 || lp->n < 0 || lp->n_eq < 0 || lp->n_eq > lp->m) return ORC_ERR_INVALID;
  if (lp->row_ptr[0] != 0) return ORC_ERR_INVALID;
  for (int32_t i = 0; i < lp->m; ++i)
    if (lp->row_ptr[i + 1] < lp->row_ptr[i]) return ORC_ERR_INVALID;
  for (int32_t i = 0; i < lp->m; ++i)
    for (int32_t e = lp->row_ptr[i]; e < lp->row_ptr[i + 1]; ++e)
      if (lp->col_idx[e] < 0 || lp->col_idx[e] >= lp->n || !isfinite(lp->val[e])) return ORC_ERR_INVALID;
  for (int32_t j = 0; j < lp->n; ++j)
    if (!isfinite(lp->c[j]) || isnan(lp->l[j]) || isnan(lp->u[j]) || lp->l[j] > lp->u[j] ||
        lp->l[j] == INFINITY || lp->u[j] == -INFINITY)
      return ORC_ERR_INVALID;
  for (int32_t i = 0; i < lp->m; ++i)
    if (!isfinite(lp->q[i])) return ORC_ERR_INVALID;
  if (lp->qd)
    for (int32_t j = 0; j < lp->n; ++j)
      if (!isfinite(lp->qd[j]) || lp->qd[j] < 0.0) return ORC_ERR_INVALID;
  return ORC_OK;
}

/* Termination test (Sec. 4.1) of a scaled-space point: unscale to the
 * original LP (x = D2 x^, y = D1 y~) and evaluate there. */
static int check_original(const orc_lp *lp, const orc_work *w, const double *xs, const double *ys,
                          double tol, double *terms) {
  for (int32_t j = 0; j < lp->n; ++j) w->xo[j] = w->D2[j] * xs[j];
  for (int32_t i = 0; i < lp->m; ++i) w->yo[i] = w->D1[i] * ys[i];
  orc_kkt_terms(lp, w->xo, w->yo, terms);
  return terms_pass(terms, tol);
}

int orc_solve(const orc_lp *lp, const orc_params *p, const double *x0, const double *y0, double *x_out,
              double *y_out, orc_info *info, orc_check *trace, int32_t trace_cap) {
  if (!lp || !p || !x_out || !y_out || !info) return ORC_ERR_INVALID;
  if (validate(lp) != ORC_OK) return ORC_ERR_INVALID;
  if (p->check_period < 1 || p->max_iter < 1 || !(p->tol >= 0.0) || !(p->eps_infeas >= 0.0)) return ORC_ERR_INVALID;
  if (p->step_value_bits != 0 && p->step_value_bits != 64 && p->step_value_bits != 32) return ORC_ERR_INVALID;
  const int32_t m = lp->m, n = lp->n, n_eq = lp->n_eq;
  const int32_t *rp = lp->row_ptr, *ci = lp->col_idx;
  const int64_t nnz = m > 0 ? rp[m] : 0;
  size_t M = (size_t)m + 1, N = (size_t)n + 1, Z = (size_t)nnz + 1;
  orc_work w;
  memset(&w, 0, sizeof(w));
#define ALLOC(ptr, cnt, T)                          \
  do {                                              \
    (ptr) = (T *)calloc((cnt), sizeof(T));          \
    if (!(ptr)) {                                   \
      free_work(&w);                                \
      return ORC_ERR_NOMEM;                         \
    }                                               \
  } while (0)
  ALLOC(w.sv, Z, double);
  ALLOC(w.D1, M, double);
  ALLOC(w.D2, N, double);
  ALLOC(w.sc, N, double);
  ALLOC(w.sq, M, double);
  ALLOC(w.sl, N, double);
  ALLOC(w.su, N, double);
  ALLOC(w.tp, N, int32_t);
  ALLOC(w.ti, Z, int32_t);
  ALLOC(w.tv, Z, double);
  ALLOC(w.perm, Z, int64_t);
  ALLOC(w.x, N, double);
  ALLOC(w.y, M, double);
  ALLOC(w.Kx, M, double);
  ALLOC(w.KTy, N, double);
  ALLOC(w.xp, N, double);
  ALLOC(w.yp, M, double);
  ALLOC(w.v, N, double);
  ALLOC(w.Kv, M, double);
  ALLOC(w.dxv, N, double);
  ALLOC(w.Kdx, M, double);
  ALLOC(w.sum_x, N, double);
  ALLOC(w.sum_y, M, double);
  ALLOC(w.xb, N, double);
  ALLOC(w.yb, M, double);
  ALLOC(w.Kxb, M, double);
  ALLOC(w.KTyb, N, double);
  ALLOC(w.x_last, N, double);
  ALLOC(w.y_last, M, double);
  ALLOC(w.xo, N, double);
  ALLOC(w.yo, M, double);
  ALLOC(w.x_prev, N, double);
  ALLOC(w.y_prev, M, double);
#undef ALLOC

  /* ---- Sec. 2.2 preconditioning ---- */
  for (int64_t e = 0; e < nnz; ++e) w.sv[e] = lp->val[e];
  orc_precondition(m, n, rp, ci, w.sv, p->ruiz_iters, p->pc_alpha, w.D1, w.D2);
  for (int32_t j = 0; j < n; ++j) {
    w.sc[j] = w.D2[j] * lp->c[j];
    w.sl[j] = lp->l[j] / w.D2[j];
    w.su[j] = lp->u[j] / w.D2[j];
  }
  for (int32_t i = 0; i < m; ++i) w.sq[i] = w.D1[i] * lp->q[i];
  if (lp->qd) { /* QP: x = D2 x~ turns x'Qx into x~'(D2 Q D2)x~ */
    w.sqd = (double *)calloc(N, sizeof(double));
    if (!w.sqd) {
      free_work(&w);
      return ORC_ERR_NOMEM;
    }
    for (int32_t j = 0; j < n; ++j) w.sqd[j] = w.D2[j] * lp->qd[j] * w.D2[j];
  }
  if (transpose_pattern(m, n, rp, ci, w.tp, w.ti, w.perm) != ORC_OK) {
    free_work(&w);
    return ORC_ERR_NOMEM;
  }
  for (int64_t e = 0; e < nnz; ++e) w.tv[e] = w.sv[w.perm[e]];
  /* the steps' copy of K~ and K~' (FP32 values, widened exactly) */
  const double *ssv = w.sv, *stv = w.tv;
  if (p->step_value_bits == 32) {
    w.sv32 = (double *)calloc(Z, sizeof(double));
    w.tv32 = (double *)calloc(Z, sizeof(double));
    if (!w.sv32 || !w.tv32) {
      free_work(&w);
      return ORC_ERR_NOMEM;
    }
    for (int64_t e = 0; e < nnz; ++e) w.sv32[e] = round_f32(w.sv[e]);
    for (int64_t e = 0; e < nnz; ++e) w.tv32[e] = round_f32(w.tv[e]);
    ssv = w.sv32;
    stv = w.tv32;
  }

  /* ---- Algorithm 1, initialisation ---- */
  double kmax = 0.0;
  for (int64_t e = 0; e < nnz; ++e)
    if (fabs(w.sv[e]) > kmax) kmax = fabs(w.sv[e]);
  double eta_hat = kmax > 0.0 ? 1.0 / kmax : 1.0;
  double omega = orc_primal_weight_init(norm2(n, w.sc), norm2(m, w.sq), p->eps_zero);
  for (int32_t j = 0; j < n; ++j) w.x[j] = x0 ? x0[j] / w.D2[j] : 0.0;
  for (int32_t i = 0; i < m; ++i) w.y[i] = y0 ? y0[i] / w.D1[i] : 0.0;
  spmv(m, rp, ci, w.sv, w.x, w.Kx);
  spmv(n, w.tp, w.ti, w.tv, w.y, w.KTy);
  memcpy(w.x_last, w.x, sizeof(double) * (size_t)n);
  memcpy(w.y_last, w.y, sizeof(double) * (size_t)m);
  double rp2, rd2, pobj, dobj;
  kkt_pieces(m, n, n_eq, w.sc, w.sq, w.sl, w.su, w.sqd, w.x, w.y, w.Kx, w.KTy, &rp2, &rd2, &pobj, &dobj);
  double kkt_start = kkt_omega_from(rp2, rd2, pobj, dobj, omega);
  double kkt_prev = kkt_start;
  double W = 0.0;
  int64_t k = 0, t = 0, attempts = 0, restarts = 0, checks = 0;
  int status = -1, which = 0;
  double terms[6] = {0, 0, 0, 0, 0, 0};
  double ray[2] = {0.0, 0.0};
  int32_t ntrace = 0;
  int gap_start_pending = p->restart_metric == 1;

  while (status < 0) {
    /* ---- Algorithm 2: AdaptiveStepPDHG(z, omega, eta_hat, k) ---- */
    double eta = eta_hat, eta_next = eta_hat;
    for (;;) {
      ++attempts;
      double tau = eta / omega, sigma = eta * omega;
      if (w.sqd) /* QP: the exact proximal step of x'Qx/2 + (c - K'y)'x over X (Q diagonal) */
        for (int32_t j = 0; j < n; ++j)
          w.xp[j] = clamp((w.x[j] - tau * (w.sc[j] - w.KTy[j])) / (1.0 + tau * w.sqd[j]), w.sl[j], w.su[j]);
      else
        for (int32_t j = 0; j < n; ++j) w.xp[j] = clamp(w.x[j] - tau * (w.sc[j] - w.KTy[j]), w.sl[j], w.su[j]);
      for (int32_t j = 0; j < n; ++j) w.v[j] = 2.0 * w.xp[j] - w.x[j];
      spmv(m, rp, ci, ssv, w.v, w.Kv);
      for (int32_t i = 0; i < m; ++i) {
        double yn = w.y[i] + sigma * (w.sq[i] - w.Kv[i]);
        if (i >= n_eq && yn < 0.0) yn = 0.0;
        w.yp[i] = yn;
      }
      for (int32_t j = 0; j < n; ++j) w.dxv[j] = w.xp[j] - w.x[j];
      spmv(m, rp, ci, ssv, w.dxv, w.Kdx);
      double dx2 = dot(n, w.dxv, w.dxv);
      double dy2 = 0.0, cross = 0.0;
      for (int32_t i = 0; i < m; ++i) {
        double d = w.yp[i] - w.y[i];
        dy2 += d * d;
        cross += d * w.Kdx[i];
      }
      double eta_bar = orc_eta_bar(dx2, dy2, cross, omega);
      eta_next = orc_eta_next(eta, eta_bar, k);
      if (!isfinite(dx2) || !isfinite(dy2) || !isfinite(cross) || isnan(eta_bar) || !(eta_next > 0.0)) {
        status = ORC_NUMERICAL;
        break;
      }
      if (eta <= eta_bar) break; /* accept */
      eta = eta_next;
    }
    if (status >= 0) break;
    /* accepted step: z <- (x', y') */
    memcpy(w.x_prev, w.x, sizeof(double) * (size_t)n);
    memcpy(w.y_prev, w.y, sizeof(double) * (size_t)m);
    memcpy(w.x, w.xp, sizeof(double) * (size_t)n);
    memcpy(w.y, w.yp, sizeof(double) * (size_t)m);
    spmv(m, rp, ci, ssv, w.x, w.Kx);
    spmv(n, w.tp, w.ti, stv, w.y, w.KTy);
    eta_hat = eta_next;
    /* Algorithm 1, average of the epoch weighted by accepted step sizes */
    for (int32_t j = 0; j < n; ++j) w.sum_x[j] += eta * w.x[j];
    for (int32_t i = 0; i < m; ++i) w.sum_y[i] += eta * w.y[i];
    W += eta;
    ++k;
    ++t;
    if (k % p->check_period != 0 && k < p->max_iter) continue;

    /* ---- restart / termination check ---- */
    ++checks;
    double invW = 1.0 / W;
    for (int32_t j = 0; j < n; ++j) w.xb[j] = invW * w.sum_x[j];
    for (int32_t i = 0; i < m; ++i) w.yb[i] = invW * w.sum_y[i];
    spmv(m, rp, ci, w.sv, w.xb, w.Kxb);
    spmv(n, w.tp, w.ti, w.tv, w.yb, w.KTyb);
    /* Sec. 4.1 on the original LP: current first, then average */
    if (check_original(lp, &w, w.x, w.y, p->tol, terms)) {
      status = ORC_OPTIMAL;
      which = 0;
      break;
    }
    const double rel_gap = fabs(terms[0] - terms[1]) / (1.0 + fabs(terms[0]) + fabs(terms[1]));
    const double rel_primal = terms[2] / (1.0 + terms[4]), rel_dual = terms[3] / (1.0 + terms[5]);
    if (check_original(lp, &w, w.xb, w.yb, p->tol, terms)) {
      status = ORC_OPTIMAL;
      which = 1;
      break;
    }
    /* Sec. 2.2 infeasibility detection: difference ray, then normalised-
     * iterate ray, both unscaled to the original LP */
    if (p->eps_infeas > 0.0 && !lp->qd) { /* LP only: the certificates below are the LP's */
      for (int seq = 0; seq < 2 && status < 0; ++seq) {
        const double *xr0 = seq == 0 ? w.x_prev : w.x_last, *yr0 = seq == 0 ? w.y_prev : w.y_last;
        for (int32_t j = 0; j < n; ++j) w.xo[j] = w.D2[j] * (w.x[j] - xr0[j]);
        for (int32_t i = 0; i < m; ++i) w.yo[i] = w.D1[i] * (w.y[i] - yr0[i]);
        double it[4];
        if (orc_infeas_terms(lp, w.xo, w.yo, it) != ORC_OK) {
          free_work(&w);
          return ORC_ERR_NOMEM;
        }
        int st = infeas_status(it, p->eps_infeas);
        if (st >= 0) {
          status = st;
          which = 2 + seq;
          ray[0] = st == ORC_PRIMAL_INFEASIBLE ? it[0] : it[2];
          ray[1] = st == ORC_PRIMAL_INFEASIBLE ? it[1] : it[3];
        }
      }
      if (status >= 0) {
        check_original(lp, &w, w.x, w.y, p->tol, terms);
        break;
      }
    }
    if (k >= p->max_iter) {
      check_original(lp, &w, w.x, w.y, p->tol, terms);
      status = ORC_ITER_LIMIT;
      which = 0;
      break;
    }
    /* Sec. 3.4 GetRestartCandidate on the scaled LP */
    double rpc, rdc, pc, dc, rpa, rda, pa, da;
    kkt_pieces(m, n, n_eq, w.sc, w.sq, w.sl, w.su, w.sqd, w.x, w.y, w.Kx, w.KTy, &rpc, &rdc, &pc, &dc);
    kkt_pieces(m, n, n_eq, w.sc, w.sq, w.sl, w.su, w.sqd, w.xb, w.yb, w.Kxb, w.KTyb, &rpa, &rda, &pa, &da);
    double kc = kkt_omega_from(rpc, rdc, pc, dc, omega);
    double ka = kkt_omega_from(rpa, rda, pa, da, omega);
    if (p->restart_metric == 1) {
      /* the normalized duality gap of each point over the ball reaching back
       * to the epoch's restart point z^{n,0} (kept in x_last, y_last) */
      const double rc = wdist(m, n, w.x, w.y, w.x_last, w.y_last, omega);
      const double ra = wdist(m, n, w.xb, w.yb, w.x_last, w.y_last, omega);
      kc = normalized_gap(m, n, n_eq, w.sc, w.sq, w.sl, w.su, w.x, w.y, w.Kx, w.KTy, omega, rc);
      ka = normalized_gap(m, n, n_eq, w.sc, w.sq, w.sl, w.su, w.xb, w.yb, w.Kxb, w.KTyb, omega, ra);
      if (restarts == 0 && gap_start_pending) {
        /* z^{0,0} has no earlier restart point: its gap is taken over the
         * first candidate's radius */
        const double r0 = !(kc < ka) ? ra : rc;
        spmv(m, rp, ci, w.sv, w.x_last, w.Kv);
        spmv(n, w.tp, w.ti, w.tv, w.y_last, w.v);
        kkt_start = normalized_gap(m, n, n_eq, w.sc, w.sq, w.sl, w.su, w.x_last, w.y_last, w.Kv, w.v, omega, r0);
        kkt_prev = kkt_start;
        gap_start_pending = 0;
      }
    }
    int cand_avg = !(kc < ka);
    double kcand = cand_avg ? ka : kc;
    int32_t mask = orc_restart_mask(kcand, kkt_start, kkt_prev, t, k, p->beta_suff, p->beta_nec, p->beta_art);
    if (mask) {
      if (cand_avg) {
        memcpy(w.x, w.xb, sizeof(double) * (size_t)n);
        memcpy(w.y, w.yb, sizeof(double) * (size_t)m);
        memcpy(w.Kx, w.Kxb, sizeof(double) * (size_t)m);
        memcpy(w.KTy, w.KTyb, sizeof(double) * (size_t)n);
      }
      double ddx = 0.0, ddy = 0.0;
      for (int32_t j = 0; j < n; ++j) ddx += (w.x[j] - w.x_last[j]) * (w.x[j] - w.x_last[j]);
      for (int32_t i = 0; i < m; ++i) ddy += (w.y[i] - w.y_last[i]) * (w.y[i] - w.y_last[i]);
      omega = orc_primal_weight_update(sqrt(ddx), sqrt(ddy), omega, p->theta, p->eps_zero);
      memcpy(w.x_last, w.x, sizeof(double) * (size_t)n);
      memcpy(w.y_last, w.y, sizeof(double) * (size_t)m);
      memset(w.sum_x, 0, sizeof(double) * (size_t)n);
      memset(w.sum_y, 0, sizeof(double) * (size_t)m);
      W = 0.0;
      t = 0;
      ++restarts;
      if (p->restart_metric == 1)
        kkt_start = normalized_gap(m, n, n_eq, w.sc, w.sq, w.sl, w.su, w.x, w.y, w.Kx, w.KTy, omega,
                                   sqrt(omega * ddx + ddy / omega));
      else if (cand_avg)
        kkt_start = kkt_omega_from(rpa, rda, pa, da, omega);
      else
        kkt_start = kkt_omega_from(rpc, rdc, pc, dc, omega);
      kkt_prev = kkt_start;
    } else {
      kkt_prev = kcand;
    }
    if (trace && ntrace < trace_cap) {
      orc_check *r = &trace[ntrace++];
      r->k = k;
      r->attempts = attempts;
      r->restarts = restarts;
      r->restart = mask;
      r->cand_avg = cand_avg;
      r->kkt_cur = kc;
      r->kkt_avg = ka;
      r->kkt_start = kkt_start;
      r->omega = omega;
      r->eta_hat = eta_hat;
      r->rel_gap = rel_gap;
      r->rel_primal = rel_primal;
      r->rel_dual = rel_dual;
    }
  }

  /* output in the original space; x = D2 x^ is projected onto X so that the
   * rounding of l / D2 * D2 cannot leave it an ulp outside its bounds */
  const double *xs = which == 1 ? w.xb : w.x;
  const double *ys = which == 1 ? w.yb : w.y;
  for (int32_t j = 0; j < n; ++j) x_out[j] = clamp(w.D2[j] * xs[j], lp->l[j], lp->u[j]);
  for (int32_t i = 0; i < m; ++i) y_out[i] = w.D1[i] * ys[i];
  /* an infeasibility certificate is returned in place of the iterate it
   * concerns: the dual ray in y (primal infeasible), the primal ray in x
   * (dual infeasible), unprojected */
  if (status == ORC_PRIMAL_INFEASIBLE || status == ORC_DUAL_INFEASIBLE) {
    const double *xr0 = which == 2 ? w.x_prev : w.x_last, *yr0 = which == 2 ? w.y_prev : w.y_last;
    if (status == ORC_PRIMAL_INFEASIBLE)
      for (int32_t i = 0; i < m; ++i) y_out[i] = w.D1[i] * (w.y[i] - yr0[i]);
    else
      for (int32_t j = 0; j < n; ++j) x_out[j] = w.D2[j] * (w.x[j] - xr0[j]);
  }
  if (status == ORC_NUMERICAL) orc_kkt_terms(lp, x_out, y_out, terms);
  info->status = status;
  info->which = which;
  info->iters = k;
  info->attempts = attempts;
  info->restarts = restarts;
  info->checks = checks;
  info->pobj = terms[0];
  info->dobj = terms[1];
  info->rp_norm = terms[2];
  info->rd_norm = terms[3];
  info->q_norm = terms[4];
  info->c_norm = terms[5];
  info->omega = omega;
  info->eta_hat = eta_hat;
  info->ray_obj = ray[0];
  info->ray_res = ray[1];
  free_work(&w);
  return ntrace;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3 (Appendix A): standard-form LP, fixed step, uniform average   */
/* ------------------------------------------------------------------------ */

/* Appendix A KKT error of min c'x s.t. Ax = b, x >= 0:
 * ||(Ax - b, [-x]^+, [A'y - c]^+, [c'x - b'y]^+)||_2 */
double orc_kkt_standard(int32_t m, int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                        const double *b, const double *c, const double *x, const double *y) {
  double s = 0.0;
  for (int32_t i = 0; i < m; ++i) {
    double ax = 0.0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) ax += v[e] * x[ci[e]];
    s += (ax - b[i]) * (ax - b[i]);
  }
  double *aty = (double *)calloc((size_t)n + 1, sizeof(double));
  if (!aty) return NAN;
  for (int32_t i = 0; i < m; ++i)
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) aty[ci[e]] += v[e] * y[i];
  for (int32_t j = 0; j < n; ++j) {
    double nx = -x[j] > 0.0 ? -x[j] : 0.0;
    double d = aty[j] - c[j] > 0.0 ? aty[j] - c[j] : 0.0;
    s += nx * nx + d * d;
  }
  double g = dot(n, c, x) - dot(m, b, y);
  if (g > 0.0) s += g * g;
  free(aty);
  return sqrt(s);
}

/* Runs Algorithm 3 with tau = sigma = s for at most max_iter inner steps in
 * total; records KKT(z^{n,0}) for every restart point (kkt_rec[0] is the
 * start) and the length of every completed inner loop.  Returns the number
 * of completed restarts, or < 0 on error. */
int32_t orc_alg3(int32_t m, int32_t n, const int32_t *rp, const int32_t *ci, const double *v,
                 const double *b, const double *c, double s, double beta, int64_t max_iter, double *x,
                 double *y, double *kkt_rec, int64_t *len_rec, int32_t cap) {
  double *xp = (double *)calloc((size_t)n + 1, sizeof(double));
  double *xb = (double *)calloc((size_t)n + 1, sizeof(double));
  double *yb = (double *)calloc((size_t)m + 1, sizeof(double));
  double *aty = (double *)calloc((size_t)n + 1, sizeof(double));
  double *vv = (double *)calloc((size_t)n + 1, sizeof(double));
  double *av = (double *)calloc((size_t)m + 1, sizeof(double));
  if (!xp || !xb || !yb || !aty || !vv || !av) {
    free(xp);
    free(xb);
    free(yb);
    free(aty);
    free(vv);
    free(av);
    return -3;
  }
  int32_t nrest = 0;
  double kkt0 = orc_kkt_standard(m, n, rp, ci, v, b, c, x, y);
  if (cap > 0) kkt_rec[0] = kkt0;
  int64_t total = 0;
  while (total < max_iter) {
    int64_t kin = 0;
    int done = 0;
    for (int32_t j = 0; j < n; ++j) xb[j] = 0.0;
    for (int32_t i = 0; i < m; ++i) yb[i] = 0.0;
    while (total < max_iter) {
      for (int32_t j = 0; j < n; ++j) aty[j] = 0.0;
      for (int32_t i = 0; i < m; ++i)
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) aty[ci[e]] += v[e] * y[i];
      for (int32_t j = 0; j < n; ++j) {
        double z = x[j] - s * (c[j] - aty[j]);
        xp[j] = z > 0.0 ? z : 0.0;
      }
      for (int32_t j = 0; j < n; ++j) vv[j] = 2.0 * xp[j] - x[j];
      spmv(m, rp, ci, v, vv, av);
      for (int32_t i = 0; i < m; ++i) y[i] = y[i] + s * (b[i] - av[i]);
      for (int32_t j = 0; j < n; ++j) x[j] = xp[j];
      double kk = (double)kin;
      for (int32_t j = 0; j < n; ++j) xb[j] = kk / (kk + 1.0) * xb[j] + 1.0 / (kk + 1.0) * x[j];
      for (int32_t i = 0; i < m; ++i) yb[i] = kk / (kk + 1.0) * yb[i] + 1.0 / (kk + 1.0) * y[i];
      ++kin;
      ++total;
      double kb = orc_kkt_standard(m, n, rp, ci, v, b, c, xb, yb);
      if (kb <= beta * kkt0) {
        done = 1;
        kkt0 = kb;
        break;
      }
    }
    if (!done) break;
    for (int32_t j = 0; j < n; ++j) x[j] = xb[j];
    for (int32_t i = 0; i < m; ++i) y[i] = yb[i];
    if (nrest + 1 < cap) kkt_rec[nrest + 1] = kkt0;
    if (nrest < cap) len_rec[nrest] = kin;
    ++nrest;
  }
  free(xp);
  free(xb);
  free(yb);
  free(aty);
  free(vv);
  free(av);
  return nrest;
}
