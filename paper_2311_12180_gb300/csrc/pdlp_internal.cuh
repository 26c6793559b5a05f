// Internal declarations shared by the solver's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pdlp {

// Tile-SpMV geometry (see pdlp_kernels.cu).  A tile is a run of consecutive
// CSR rows holding at most TILE_NNZ nonzeros and TILE_ROWS rows, or a single
// row longer than TILE_NNZ.  One CTA of NT threads processes one tile at a
// time, one row per thread in the epilogue.
constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr int EPT = 8;                   // consecutive entries per thread
constexpr int TILE_NNZ = NT * EPT - EPT;  // 2040: the EPT-aligned span of a tile fits NT * EPT
constexpr int TILE_ROWS = 256;

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

struct Csr {
  int32_t rows;
  int32_t ntiles;
  const int32_t *ptr;    // rows + 1
  const int32_t *idx;    // nnz
  const double *val;     // nnz, FP64 (scaled)
  const float *val32;    // nnz, FP32 copy of val (or null)
  const int2 *tmeta;     // ntiles + 1: {first row, first nonzero} of each tile; last = {rows, nnz}
};

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

struct TraceRec {
  long long k;
  int restart;
  int cand_avg;
  double kkt_cur, kkt_avg, kkt_start, omega, eta_hat;
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
};

// ---- kernel launchers (pdlp_kernels.cu) ----
// KC_PRIMAL_REUSE: a k_primal launch that reuses the stored g = K'y (after a
// rejected trial or a check) instead of recomputing it; timed separately.
enum KernelClass { KC_PRIMAL = 0, KC_DUAL, KC_R1, KC_R2, KC_R3, KC_OUTPUT, KC_PRIMAL_REUSE, KC_INFEAS, KC_NUM };
const char *kernel_class_name(int kc);

struct LaunchCfg {
  int gridA, gridB, gridR1, gridR2, gridR3;
};

cudaError_t launch_primal(const Csr &KT, const Vecs &V, DevState *st, int grid, cudaStream_t s);
cudaError_t launch_dual(const Csr &K, const Vecs &V, DevState *st, int grid, cudaStream_t s);
cudaError_t launch_check_primal(const Csr &KT, const Vecs &V, DevState *st, int grid, cudaStream_t s);
cudaError_t launch_check_dual(const Csr &K, const Vecs &V, DevState *st, int grid, cudaStream_t s);
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
