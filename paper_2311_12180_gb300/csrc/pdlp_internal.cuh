// Internal declarations shared by the solver's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pdlp {

// Thread-block geometry of the step and check kernels (see pdlp_kernels.cu).
constexpr int NT = 256;
constexpr int NW = NT / 32;

// Sliced-ELL storage of K and K' (see pdlp_kernels.cu and pdlp_sell.h).
// Rows are renumbered (the solver's internal order): within each group
// (the equality rows of K, then its ">=" rows; all rows of K') by length,
// longest first.  Rows of at most SELL_LONG entries are stored in slices of
// 32 consecutive internal rows, entry k of the slice's lane-th row at
// off + 32 k + lane (L = the slice's longest row; shorter rows padded); a
// longer row is stored contiguously from off, padded to a multiple of 32.
// Padding entries hold column -1 and value 0.  Every item starts at a
// multiple of 32 entries.
constexpr int SELL_LONG = 48;
// strides of 32 entries loaded per batch: primal step (K'), dual step (K),
// check passes
constexpr int SELL_U_P = 2;
constexpr int SELL_U_D = 2;
constexpr int SELL_U_C = 4;
// CTAs per SM the two-vector check pass over K' is compiled for
constexpr int CHECK_MINB = 2;
// CTAs per SM the step kernels are compiled for (registers per thread:
// 65536 / (256 x this))
constexpr int STEP_MINB = 4;

// One unit of work for one warp: a slice {first row, rows (1..32), L, off}
// or a long row {row, -1, length, off}.
struct SellMat {
  int32_t rows;
  int32_t nitems;
  const int4 *items;    // in schedule order (cost, longest first)
  const int32_t *idx;   // internal column of each stored entry, -1 for padding
  const double *val;    // FP64 values (scaled)
  const float *val32;   // FP32 copy of val (or null)
};

constexpr int ST_RUNNING = -1;
constexpr int ST_OPTIMAL = 0;
constexpr int ST_ITER_LIMIT = 1;
constexpr int ST_TIME_LIMIT = 2;
constexpr int ST_NUMERICAL = 3;
constexpr int ST_PRIMAL_INFEASIBLE = 4;
constexpr int ST_DUAL_INFEASIBLE = 5;

constexpr int MODE_CHECK = 0;
constexpr int MODE_INIT = 1;

// Last-block counters, one per kernel class.
enum { CNT_DUAL = 0, CNT_R1 = 1, CNT_R2 = 2, CNT_R3 = 3, CNT_NUM = 8 };

// Partial-sum slots per block.
constexpr int NV_A = 1;   // ||x'-x||^2
constexpr int NV_B = 2;   // ||y'-y||^2, (y'-y)'(Kx'-Kx)
constexpr int NV_R1 = 8;  // per point (cur, avg): rd2 scaled, rd2 original, c'x, l'lam+ - u'lam-
constexpr int NV_R2 = 6;  // per point: rp2 scaled, rp2 original, q'y
constexpr int NV_R3 = 2;  // ||x_new - x_last||^2, ||y_new - y_last||^2
// Infeasibility pieces per ray (difference, normalised iterate), original LP:
// ||-K'yr - lam||^2, l'lam+ - u'lam-, c'xr, ||bound-cone violation of xr||^2,
// ||(K_E xr, min(K_G xr, 0))||^2, q'yr, ||min(yr_G, 0)||^2.
constexpr int NV_I1 = 7;
constexpr int NV_I = 2 * NV_I1;

// Device-resident solver state: read by every kernel at entry, written only
// by one thread of the last block of a kernel (or by the host between solves).
struct DevState {
  double eta;        // step size of the next Algorithm 2 trial
  double omega;      // primal weight
  double W;          // sum of accepted step sizes in the current epoch
  double kkt_start;  // KKT_omega(z^{n,0})
  double kkt_prev;   // KKT_omega of the previous restart candidate
  double tol;
  double q_norm, c_norm;  // original-space norms (Sec. 4.1)
  double theta, eps_zero, beta_suff, beta_nec, beta_art;
  double cand[4];    // candidate pieces: rp2, rd2, pobj, dobj (scaled)
  double term[4];    // original-space pobj, dobj, ||rp||, ||rd|| at the last check
  double rel_kkt_best;     // FP32 polish: best original relative KKT seen at a restart
  double eps_infeas;       // relative tolerance of the infeasibility certificates (0: off)
  double ray[2];           // certificate found: its objective and residual norm
  long long k, t, attempts, restarts, checks, max_iter, f64_switch_k;
  int cur;           // which of the two buffers holds the accepted iterate
  int need_g;        // 1: g = K'y is stale (y changed since it was computed)
  int check_pending; // 1: a restart / termination check is due
  int status;        // ST_*
  int which;         // 0: output the current iterate, 1: the average; infeasible:
                     // 2: difference ray, 3: normalised-iterate ray
  int restart_to;    // 0: none, 1: restart to current, 2: to average
  int mode;          // MODE_CHECK / MODE_INIT
  int P;
  int ntrace, trace_cap;
  int use_f32;       // 1: the step kernels read the FP32 values
  int polish, stall; // FP32 polish switch and its stall counter
  unsigned int cnt[CNT_NUM];
};

// One check's record in the device ring (trace_cap records, written at
// ntrace mod trace_cap; ntrace counts every record ever written).
struct TraceRec {
  long long k;
  long long attempts;  // Algorithm 2 trials so far (rejections = attempts - k)
  long long restarts;  // restarts so far, this check's included
  int restart;
  int cand_avg;
  double kkt_cur, kkt_avg, kkt_start, omega, eta_hat;
  double rel_gap, rel_primal, rel_dual;  // Sec. 4.1 measures of the current iterate, original LP
};

struct Vecs {
  int n, m, n_eq;
  int gridA, gridR1;
  // scaled problem data
  const double *c, *l, *u, *D2, *rD2;  // n (rD2 = 1 / D2)
  const double *l0, *u0;         // n, original bounds (output projection)
  const double *q, *D1, *rD1;    // m (rD1 = 1 / D1)
  // iterates (two buffers, DevState::cur selects the accepted one)
  double *x[2], *sx[2];          // n: iterate, epoch sum of eta * x
  double *y[2], *sy[2], *Kx[2];  // m
  double *g, *gbar, *xlast, *xout;  // n
  double *Kxbar, *ylast, *yout;     // m
  // infeasibility detection: K'y at the epoch start and at the previous
  // accepted iterate (n), K x at the epoch start (m)
  double *g0, *gprev, *kx0;
  int gridI;
  double *partA, *partB, *partR1, *partR2, *partR3, *partI;
  TraceRec *trace;
  // (k + 2)^-0.3 at pw[k] and (k + 2)^-0.6 at pw[npw + k] for k < npw
  const double *pw;
  long long npw;
  // internal -> original row of K (m) and column (n); every vector above is
  // in the internal order, k_output writes the original order
  const int32_t *perm_r, *perm_c;
  // QP extension: the scaled diagonal D2 Q D2 of the objective's Hessian
  // (n, internal order), or null for an LP
  const double *qd;
};

// ---- kernel launchers (pdlp_kernels.cu) ----
// KC_PRIMAL_REUSE: a k_primal launch that reuses the stored g = K'y (after a
// rejected trial or a check) instead of recomputing it; timed separately.
enum KernelClass { KC_PRIMAL = 0, KC_DUAL, KC_R1, KC_R2, KC_R3, KC_OUTPUT, KC_PRIMAL_REUSE, KC_INFEAS, KC_NUM };
const char *kernel_class_name(int kc);

struct LaunchCfg {
  int gridA, gridB, gridR1, gridR2, gridR3;
};

cudaError_t launch_primal(const SellMat &KT, const Vecs &V, DevState *st, int grid, cudaStream_t s);
cudaError_t launch_dual(const SellMat &K, const Vecs &V, DevState *st, int grid, cudaStream_t s);
cudaError_t launch_check_primal(const SellMat &KT, const Vecs &V, DevState *st, int grid, cudaStream_t s);
cudaError_t launch_check_dual(const SellMat &K, const Vecs &V, DevState *st, int grid, cudaStream_t s);
cudaError_t launch_restart(const Vecs &V, DevState *st, int grid, cudaStream_t s);
cudaError_t launch_infeas(const Vecs &V, DevState *st, int grid, cudaStream_t s);
cudaError_t launch_output(const Vecs &V, DevState *st, cudaStream_t s);
cudaError_t launch_time_limit(DevState *st, cudaStream_t s);
int occupancy_grid(int kc, int num_sms);
cudaError_t kernels_init();  // one-time kernel attributes (none needed at present)

// Records `msg` as the calling thread's pdlp_last_error() and returns `code`.
int set_error(int code, const char *msg);

// Order-preserving integer key of an IEEE double (sign-magnitude -> two's
// complement): a < b  <=>  key(a) < key(b) for non-NaN values (with -0 < +0).
__device__ __forceinline__ long long dkey(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

// proj onto [l, u] with integer compares, keeping the clamp off the FP64 pipe.
// A NaN input maps to u (positive NaN) or l (negative NaN); with infinite
// bounds it becomes +-inf and the step test flags it.
__device__ __forceinline__ double clamp_bits(double v, double l, double u) {
  const long long kv = dkey(v);
  double r = v;
  if (kv < dkey(l)) r = l;
  if (kv > dkey(u)) r = u;
  return r;
}


}  // namespace pdlp
