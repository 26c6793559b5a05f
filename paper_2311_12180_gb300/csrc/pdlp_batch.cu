// Batched restarted PDHG: many independent LPs of uneven size in one
// persistent launch (cuPDLP.jl paper, Algorithms 1 and 2, eq. (kkt),
// Sec. 3.4, Sec. 4.1, Sec. 2.2 preconditioning).
//
// One CTA of NTB threads solves one instance from start to finish: every
// half-step is a CTA-wide pass over the instance's K' or K separated by
// __syncthreads, so no grid-wide synchronisation or inter-CTA wait exists.
// CTAs take instances from a device queue in decreasing order of nonzeros
// (longest first keeps the tail short).  Each instance carries its own step
// size, primal weight, restart, termination and infeasibility state in
// registers (identical in every thread: all of them read the same
// block-reduced sums).  Its SpMVs
// map G lanes to a row (G a power of two <= 32: autotuned per instance in
// pdlp_batch_create for the LPs solved by teams, a fixed rule for the
// others); a team LP's row sums have one order whatever G is and its sums
// over rows are taken by element passes (rows_spmv), so results are the same
// for every schedule and every create.
//
// Arithmetic matches the single-instance kernels in pdlp_kernels.cu (same
// formulas and readings of the paper); only the summation order differs.

#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "pdlp.h"
#include "pdlp_host.h"
#include "pdlp_internal.cuh"
#include "pdlp_setup.cuh"

namespace pdlp {
namespace batch {

constexpr int NTB = 512;
// dynamic shared memory of k_batch_solve: an LP with resident_bytes() up to
// this is solved from shared memory (one CTA per SM either way: the kernel
// runs 512 threads at > 64 registers)
constexpr int RESIDENT_MAX = 200 * 1024;
constexpr int NWB = NTB / 32;
// shared reduction buffer: NV partials per warp, NV results, 4 broadcast slots
constexpr int RED_BCAST = 16 * NWB + 16;
constexpr int RED_TEAM = RED_BCAST + 8;  // 16 slots: team-reduction results
constexpr int RED_SIZE = RED_TEAM + 16;

// per-instance vector blocks
// (VM_KXS / VN_GS: K x and K'y at the epoch start, VN_GP: K'y of the
// previous accepted iterate, kept for infeasibility detection; touched only
// at checks, they stay in global memory when the rest of an LP is resident
// in shared memory: VM_RES / VN_RES blocks are copied in)
enum { VM_Q = 0, VM_D1, VM_Y0, VM_Y1, VM_SY0, VM_SY1, VM_KX0, VM_KX1, VM_KXB, VM_YL, VM_YOUT, VM_Q0, VM_KXS,
       VM_COUNT };
enum { VN_C = 0, VN_L, VN_U, VN_D2, VN_L0, VN_U0, VN_X0, VN_X1, VN_SX0, VN_SX1, VN_G, VN_GB, VN_XL, VN_XOUT, VN_C0,
       VN_GS, VN_GP, VN_COUNT };
constexpr int VM_RES = VM_KXS, VN_RES = VN_GS;

struct Inst {
  int m, n, n_eq, gk, gt;  // gk / gt: lanes per row for K / K' (the schedule)
  int sk, st;              // sk / st: slots of the canonical row-sum order for K / K'
  int pad;
  long long kp, ke, tp, te;  // offsets of K row_ptr / nonzeros, K' row_ptr / nonzeros
  long long om, on;          // offsets of the m- and n-vector blocks
  long long okm, okn;        // the same offsets, kept when om / on point into shared memory
  long long xo, yo;          // offsets in the packed outputs (sum of n / sum of m)
  double eta0, omega0, qn, cn;
};

struct Params {
  double tol, theta, eps_zero, beta_suff, beta_nec, beta_art;
  double eps_infeas;  // relative tolerance of the infeasibility certificates (0: off)
  long long max_iter;
  int P, warm;
  // Algorithm 2 exponent factors, built once per solve by setup_pow_table
  // (the same pow() the step test would call): (k + 2)^-0.3 at pw[k] and
  // (k + 2)^-0.6 at pw[npw + k] for k < npw.  Two FP64 powers per step are
  // a large part of a small LP's step on GB300's narrow FP64 pipe.
  const double *pw;
  long long npw;
  // test hook for the barrier timeout (environment PDLP_TEST_TEAM_STALL=1):
  // rank 1 of team 0 leaves at once, so its team's first barrier runs out
  int stall;
};

struct Arrays {
  const int *kptr, *kidx, *tptr, *tidx;
  double *kval, *tval;
  double *vm, *vn;
  double *vmk, *vnk;      // global bases of the vector blocks (the kept vectors live there)
  const double *x0, *y0;  // packed warm start (or null)
  double *xout, *yout;
  int *status;
  long long *iters;
  unsigned long long *t_start, *t_end;  // per-LP global-timer stamps (ns) of the last solve
};

// ---------------------------------------------------------------- CTA helpers

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// CTA-wide sums of NV values, result in every thread (fixed order).  A warp
// whose values are all zero (no rows of a small LP) skips its FP64 shuffle
// tree: GB300 issues FP64 at a small fraction of the FP32 rate, so the trees
// of idle warps would dominate a small LP's iteration.
template <int NV>
__device__ __forceinline__ void allsum(double (&v)[NV], double *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  bool any = false;
#pragma unroll
  for (int a = 0; a < NV; ++a) any |= __double_as_longlong(v[a]) != 0;
  if (__any_sync(0xffffffffu, any)) {
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = wsum(v[a]);
  }
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) red[a * NWB + wid] = v[a];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      const double s = wsum(lane < NWB ? red[a * NWB + lane] : 0.0);
      if (lane == 0) red[16 * NWB + a] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = red[16 * NWB + a];
  __syncthreads();
}

__device__ __forceinline__ double allmax(double v, double *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = wmax(v);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const double s = wmax(lane < NWB ? red[lane] : 0.0);
    if (lane == 0) red[16 * NWB] = s;
  }
  __syncthreads();
  v = red[16 * NWB];
  __syncthreads();
  return v;
}

// Warp sums of NV values (warps whose values are all zero skip the FP64
// shuffle tree, as in allsum), written per warp to red[a * NWB + warp];
// ends with a CTA barrier.
template <int NV>
__device__ __forceinline__ void warp_partials(double (&v)[NV], double *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  bool any = false;
#pragma unroll
  for (int a = 0; a < NV; ++a) any |= __double_as_longlong(v[a]) != 0;
  if (__any_sync(0xffffffffu, any)) {
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = wsum(v[a]);
  }
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) red[a * NWB + wid] = v[a];
  }
  __syncthreads();
}

// Loads of vectors that the solve itself writes.  A team of CTAs (below)
// reads entries that other SMs wrote inside this kernel, so those loads go
// to the L2 (ld.cg), past the SM's non-coherent L1.
template <bool CG>
__device__ __forceinline__ double ldv(const double *p) {
  if constexpr (CG)
    return __ldcg(p);
  else
    return *p;
}

__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// An LP solved by one CTA: every loop covers all rows, syncs are CTA barriers.
struct Solo {
  static constexpr bool kTeam = false;
  __device__ __forceinline__ int rank() const { return 0; }
  __device__ __forceinline__ int size() const { return 1; }
  __device__ __forceinline__ bool sync() {
    __syncthreads();
    return true;
  }
  template <int NV>
  __device__ __forceinline__ bool reduce(double (&v)[NV], double *red) {
    allsum<NV>(v, red);
    return true;
  }
  // The sums (same order as allsum) go to f in thread 0 only; whatever f
  // writes to red[RED_BCAST..] is visible to every thread on return.  Two
  // barriers instead of allsum's three plus one for the broadcast.
  template <int NV, class F>
  __device__ __forceinline__ bool reduce_apply(double (&v)[NV], double *red, F &&f) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    warp_partials<NV>(v, red);
    if (wid == 0) {
      double t[NV];
#pragma unroll
      for (int a = 0; a < NV; ++a) t[a] = wsum(lane < NWB ? red[a * NWB + lane] : 0.0);
      if (lane == 0) f(t);
    }
    __syncthreads();
    return true;
  }
};

// Team-barrier and reduction state in global memory (one entry per team).
struct TeamState {
  unsigned *cnt, *gen;  // barrier arrival counter and generation
  int *q;               // queue position broadcast by the team leader
  double *slots;        // [team][2][TEAM][16] partial sums
  int *abort;           // set when a barrier wait times out
  int teams;
};
constexpr int TEAM = 4;                 // CTAs per team
constexpr int BACK_CTAS = 16;           // CTAs that start from the small end of the queue
constexpr long long TEAM_MIN_NNZ = 32768;  // LPs at least this large are solved by a team
// lanes-per-row rule of an LP solved by one CTA: SOLO_FILL = false: the
// smallest power of two G with (mean row length) / G <= SOLO_TARGET;
// SOLO_FILL = true: the largest power of two G <= 32 with rows * G <= the
// CTA's threads (one round of rows fills the CTA), at most the rule's G for
// SOLO_TARGET = 1
constexpr double SOLO_TARGET = 4.0;
constexpr bool SOLO_FILL = false;
constexpr unsigned long long TEAM_WAIT_NS = 2000000000ull;

// An LP solved by TEAM CTAs (one per SM): rows and vector entries are dealt
// round-robin in chunks, partial sums meet in global slots read in rank order
// (every CTA obtains bitwise the same sums and therefore takes the same
// decisions), and phases are separated by a sense-reversing barrier on a
// global counter whose spin is bounded: a wait longer than TEAM_WAIT_NS sets
// the abort flag, and every CTA of the batch then leaves its loops.
struct Team {
  static constexpr bool kTeam = true;
  int r;
  unsigned *cnt, *gen;
  double *slots;
  int *abort;
  int buf;
  __device__ __forceinline__ int rank() const { return r; }
  __device__ __forceinline__ int size() const { return TEAM; }
  __device__ bool sync() {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
      int ok = 1;
      unsigned g, old;
      asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(gen) : "memory");
      // arrival (acquire-release): the CTA's writes, ordered before this
      // thread by the barrier above, are released; the last arrival acquires
      // everything the earlier arrivals released and passes it on through the
      // generation, which the waiting CTAs acquire
      asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(cnt) : "memory");
      if (old == TEAM - 1) {
        asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(cnt) : "memory");
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(gen) : "memory");
      } else {
        const unsigned long long t0 = gtimer_ns();
        for (;;) {
          unsigned cur;
          asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(gen) : "memory");
          if (cur != g) break;
          if (*(volatile int *)abort || gtimer_ns() - t0 > TEAM_WAIT_NS) {
            atomicExch(abort, 1);
            ok = 0;
            break;
          }
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
  }
  template <int NV>
  __device__ bool reduce(double (&v)[NV], double *red) {
    static_assert(NV <= 16, "16 slots per rank");
    allsum<NV>(v, red);
    double *sl = slots + (size_t)buf * TEAM * 16;
    if (threadIdx.x == 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) sl[r * 16 + a] = v[a];
    }
    const bool ok = sync();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        double t = 0.0;
        for (int k = 0; k < TEAM; ++k) t += __ldcg(sl + k * 16 + a);
        red[RED_TEAM + a] = t;
      }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = red[RED_TEAM + a];
    __syncthreads();
    buf ^= 1;  // the other buffer: a rank rewrites this one only after the next barrier
    return ok;
  }
  // As Solo::reduce_apply over the whole team: every CTA's thread 0 gets the
  // same team sums (rank order) and runs f.
  template <int NV, class F>
  __device__ bool reduce_apply(double (&v)[NV], double *red, F &&f) {
    static_assert(NV <= 16, "16 slots per rank");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    warp_partials<NV>(v, red);
    double *sl = slots + (size_t)buf * TEAM * 16;
    if (wid == 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        const double c = wsum(lane < NWB ? red[a * NWB + lane] : 0.0);
        if (lane == 0) sl[r * 16 + a] = c;
      }
    }
    const bool ok = sync();
    if (threadIdx.x == 0) {
      double t[NV];
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        t[a] = 0.0;
        for (int k = 0; k < TEAM; ++k) t[a] += __ldcg(sl + k * 16 + a);
      }
      f(t);
    }
    __syncthreads();
    buf ^= 1;
    return ok;
  }
};

// Rows of a CSR block with G lanes per row: for each row, f(row, sums) runs
// in the group's first lane.  Every lane of a warp takes part in each round,
// so the shuffles are always full-warp.  For an LP solved by a team, f only
// stores: its sums over rows (step-test and KKT pieces) are taken afterwards
// by an elementwise pass with a fixed thread per element, so which thread
// finished a row never matters and the autotuned G cannot change them.  On
// one CTA (fixed G) f also keeps those sums, saving the pass.
//
// A row's sum has one order whatever G is (G a power of two dividing S, S / G
// in {1, 2, 4}): S slots, slot s taking the row's entries e with
// e mod S = s in increasing order (an FMA chain), and the slots added by the
// xor butterfly S/2, S/4, ..., 1.  Lane li of a group holds the R = S / G
// slots li + G j: slot pairs at offsets >= G are added in registers (in
// butterfly order), the rest by shuffles.  So the schedule (G) changes
// speed, never results: the autotuner may pick any G per LP.
template <int R, int NV, bool SCALED, bool CG, class F>
__device__ __forceinline__ void rows_spmv_r(const int *__restrict__ ptr, const int *__restrict__ idx,
                                            const double *__restrict__ val, int rows, int G,
                                            const double *const (&xs)[NV], const double (&sc)[NV], F &f, int part,
                                            int parts) {
  const int gid = threadIdx.x / G, li = threadIdx.x % G, ngroups = NTB / G, S = G * R;
  for (int base = part * ngroups; base < rows; base += parts * ngroups) {
    const int r = base + gid;
    double s[R][NV];
#pragma unroll
    for (int j = 0; j < R; ++j)
#pragma unroll
      for (int a = 0; a < NV; ++a) s[j][a] = 0.0;
    if (r < rows) {
      const int e1 = ptr[r + 1];
      for (int b0 = ptr[r] + li; b0 < e1; b0 += S) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int e = b0 + G * j;
          if (e < e1) {
            const double v = val[e];
            const int c = idx[e];
#pragma unroll
            for (int a = 0; a < NV; ++a) {
              const double xv = ldv<CG>(xs[a] + c);
              s[j][a] = fma(v, SCALED ? sc[a] * xv : xv, s[j][a]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int b = R / 2; b >= 1; b >>= 1)
#pragma unroll
      for (int j = 0; j < b; ++j)
#pragma unroll
        for (int a = 0; a < NV; ++a) s[j][a] += s[j + b][a];
    for (int o = G >> 1; o > 0; o >>= 1) {
#pragma unroll
      for (int a = 0; a < NV; ++a) s[0][a] += __shfl_xor_sync(0xffffffffu, s[0][a], o, G);
    }
    if (r < rows && li == 0) f(r, s[0]);
  }
}

template <int NV, bool SCALED, bool CG = false, class F>
__device__ __forceinline__ void rows_spmv(const int *__restrict__ ptr, const int *__restrict__ idx,
                                          const double *__restrict__ val, int rows, int G, int S,
                                          const double *const (&xs)[NV], const double (&sc)[NV], F &f,
                                          int part, int parts) {
  const int R = S / G;
  if (R == 1)
    rows_spmv_r<1, NV, SCALED, CG>(ptr, idx, val, rows, G, xs, sc, f, part, parts);
  else if (R == 2)
    rows_spmv_r<2, NV, SCALED, CG>(ptr, idx, val, rows, G, xs, sc, f, part, parts);
  else
    rows_spmv_r<4, NV, SCALED, CG>(ptr, idx, val, rows, G, xs, sc, f, part, parts);
}

__device__ __forceinline__ double proj_lambda(double d, double l, double u) {
  const bool lf = isfinite(l), uf = isfinite(u);
  if (lf && uf) return d;
  if (lf) return d > 0.0 ? d : 0.0;
  if (uf) return d < 0.0 ? d : 0.0;
  return 0.0;
}

__device__ __forceinline__ double kkt_omega(double rp2, double rd2, double pobj, double dobj, double w) {
  const double gap = dobj - pobj;
  return sqrt(w * w * rp2 + rd2 / (w * w) + gap * gap);
}

__device__ __forceinline__ bool sec41_pass(double pobj, double dobj, double rp, double rd, double tol, double qn,
                                           double cn) {
  return fabs(dobj - pobj) <= tol * (1.0 + fabs(dobj) + fabs(pobj)) && rp <= tol * (1.0 + qn) &&
         rd <= tol * (1.0 + cn);
}

// ---------------------------------------------------------------- batched scaling (Sec. 2.2)

__global__ void __launch_bounds__(NTB) k_batch_scale(Arrays A, Inst *inst, int count, int ruiz_iters,
                                                     double pc_alpha, double eps_zero) {
  __shared__ double red[RED_SIZE];
  const int id = blockIdx.x;
  if (id >= count) return;
  Inst I = inst[id];
  const int *kp = A.kptr + I.kp, *ki = A.kidx + I.ke, *tp = A.tptr + I.tp, *ti = A.tidx + I.te;
  double *kv = A.kval + I.ke, *tv = A.tval + I.te;
  double *vm = A.vm + I.om, *vn = A.vn + I.on;
  const int m = I.m, n = I.n;
  double *D1 = vm + (long long)VM_D1 * m, *D2 = vn + (long long)VN_D2 * n;
  double *r = vm + (long long)VM_KXB * m, *s = vn + (long long)VN_GB * n;  // per-pass factors (scratch)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < m; i += NTB) D1[i] = 1.0;
  for (int j = threadIdx.x; j < n; j += NTB) D2[j] = 1.0;
  const int passes = ruiz_iters + (pc_alpha >= 0.0 ? 1 : 0);
  for (int it = 0; it < passes; ++it) {
    const bool ruiz = it < ruiz_iters;
    for (int i = wid; i < m; i += NWB) {
      double acc = 0.0;
      for (int e = kp[i] + lane; e < kp[i + 1]; e += 32) {
        const double a = fabs(kv[e]);
        acc = ruiz ? fmax(acc, a) : acc + (pc_alpha == 1.0 ? a : pow(a, 2.0 - pc_alpha));
      }
      acc = ruiz ? wmax(acc) : wsum(acc);
      if (lane == 0) r[i] = acc > 0.0 ? sqrt(acc) : 1.0;
    }
    for (int j = wid; j < n; j += NWB) {
      double acc = 0.0;
      for (int e = tp[j] + lane; e < tp[j + 1]; e += 32) {
        const double a = fabs(tv[e]);
        acc = ruiz ? fmax(acc, a) : acc + (pc_alpha == 1.0 ? a : pow(a, pc_alpha));
      }
      acc = ruiz ? wmax(acc) : wsum(acc);
      if (lane == 0) s[j] = acc > 0.0 ? sqrt(acc) : 1.0;
    }
    __syncthreads();
    for (int i = wid; i < m; i += NWB)
      for (int e = kp[i] + lane; e < kp[i + 1]; e += 32) kv[e] = kv[e] / r[i] / s[ki[e]];
    for (int j = wid; j < n; j += NWB)
      for (int e = tp[j] + lane; e < tp[j + 1]; e += 32) tv[e] = tv[e] / r[ti[e]] / s[j];
    for (int i = threadIdx.x; i < m; i += NTB) D1[i] = D1[i] / r[i];
    for (int j = threadIdx.x; j < n; j += NTB) D2[j] = D2[j] / s[j];
    __syncthreads();
  }
  // scaled vectors, norms, initial step size and primal weight
  double cc[1] = {0.0}, qq[1] = {0.0}, kmax = 0.0;
  for (int j = threadIdx.x; j < n; j += NTB) {
    const double c = D2[j] * vn[(long long)VN_C0 * n + j];
    vn[(long long)VN_C * n + j] = c;
    vn[(long long)VN_L * n + j] = vn[(long long)VN_L0 * n + j] / D2[j];
    vn[(long long)VN_U * n + j] = vn[(long long)VN_U0 * n + j] / D2[j];
    cc[0] = fma(c, c, cc[0]);
  }
  for (int i = threadIdx.x; i < m; i += NTB) {
    const double q = D1[i] * vm[(long long)VM_Q0 * m + i];
    vm[(long long)VM_Q * m + i] = q;
    qq[0] = fma(q, q, qq[0]);
  }
  for (long long e = kp[0] + threadIdx.x; e < kp[m]; e += NTB) kmax = fmax(kmax, fabs(kv[e]));
  allsum<1>(cc, red);
  allsum<1>(qq, red);
  kmax = allmax(kmax, red);
  if (threadIdx.x == 0) {
    const double cn = sqrt(cc[0]), qn = sqrt(qq[0]);
    inst[id].eta0 = kmax > 0.0 ? 1.0 / kmax : 1.0;
    inst[id].omega0 = (cn > eps_zero && qn > eps_zero) ? cn / qn : 1.0;
  }
}

// ---------------------------------------------------------------- one instance, one CTA

template <bool CG>
struct PrimalRow {
  const double *c, *l, *u, *x, *sx;
  double *g, *xn, *sxn;
  double tau, eta;
  bool store_g;
  double dx2 = 0.0;  // one CTA per LP (fixed schedule): ||x' - x||^2 kept here
  __device__ __forceinline__ void operator()(int j, const double (&s)[1]) { apply(j, s[0]); }
  __device__ __forceinline__ void apply(int j, double gj) {
    if (store_g) g[j] = gj;
    const double xj = ldv<CG>(x + j);
    const double v = clamp_bits(fma(-tau, c[j] - gj, xj), l[j], u[j]);  // integer compares, off the FP64 pipe
    xn[j] = v;
    sxn[j] = fma(eta, v, ldv<CG>(sx + j));
    if (!CG) {
      const double d = v - xj;
      dx2 = fma(d, d, dx2);
    }
  }
};

template <bool CG>
struct DualRow {
  const double *q, *y, *kx, *sy;
  double *yn, *kxn, *syn;
  double sigma, eta;
  int n_eq;
  double dy2 = 0.0, cross = 0.0;  // one CTA per LP: the step-test pieces kept here
  __device__ __forceinline__ void operator()(int i, const double (&s)[1]) {
    const double kn = s[0], kxi = ldv<CG>(kx + i), yi = ldv<CG>(y + i);
    double v = fma(sigma, q[i] - fma(2.0, kn, -kxi), yi);
    if (i >= n_eq && __double_as_longlong(v) < 0) v = 0.0;  // proj_Y by the sign bit
    yn[i] = v;
    kxn[i] = kn;
    syn[i] = fma(eta, v, ldv<CG>(sy + i));
    if (!CG) {
      const double d = v - yi;
      dy2 = fma(d, d, dy2);
      cross = fma(d, kn - kxi, cross);
    }
  }
};

// Dual-side KKT pieces for the current (and, with avg, the average) point.
template <bool CG>
struct CheckT {
  const double *c, *l, *u, *d2, *x, *sx;
  double *g, *gbar;
  double invW;
  int kind;  // 0: start point {g}; 1: {g, gbar}; 2: {gbar}, g current
  double acc[8];
  // infeasibility detection (keep): K'y at the epoch start (kind 0) and of
  // the previous accepted iterate (kind 1, the value this pass overwrites)
  bool keep = false;
  double *gs = nullptr, *gp = nullptr;
  __device__ __forceinline__ void piece(double cj, double gj, double lj, double uj, double dj, double xj, double *a) {
    const double d = cj - gj;
    const double lam = proj_lambda(d, lj, uj);
    const double r = d - lam;
    a[0] = fma(r, r, a[0]);
    const double ro = r / dj;
    a[1] = fma(ro, ro, a[1]);
    a[2] = fma(cj, xj, a[2]);
    if (lam > 0.0) a[3] = fma(lj, lam, a[3]);
    if (lam < 0.0) a[3] = a[3] - uj * (-lam);
  }
  template <int NV>
  __device__ __forceinline__ void operator()(int j, const double (&s)[NV]) {
    double gj = kind == 2 ? ldv<CG>(g + j) : 0.0, gb = 0.0;
    if (kind == 0) {
      gj = s[0];
      g[j] = gj;
      if (keep) gs[j] = gj;
    } else if (kind == 1) {
      gj = s[0];
      gb = s[NV - 1];
      if (keep) gp[j] = ldv<CG>(g + j);
      g[j] = gj;
    } else {
      gb = s[0];
    }
    if (kind) gbar[j] = gb;
    if (!CG) {  // one CTA per LP: the pieces here (a team takes them in sums())
      piece(c[j], gj, l[j], u[j], d2[j], ldv<CG>(x + j), acc);
      if (kind) piece(c[j], gb, l[j], u[j], d2[j], invW * ldv<CG>(sx + j), acc + 4);
    }
  }
  // this element's pieces, from the stored K'y (and K'ybar)
  __device__ __forceinline__ void sums(int j) {
    piece(c[j], ldv<CG>(g + j), l[j], u[j], d2[j], ldv<CG>(x + j), acc);
    if (kind) piece(c[j], ldv<CG>(gbar + j), l[j], u[j], d2[j], invW * ldv<CG>(sx + j), acc + 4);
  }
};

template <bool CG>
struct CheckK {
  const double *q, *d1, *y, *sy;
  double *kx, *kxbar;
  double invW;
  int check, n_eq;
  double acc[6];
  // infeasibility detection (keep): K x at the epoch start (start pass)
  bool keep = false;
  double *kxs = nullptr;
  __device__ __forceinline__ void piece(double qi, double kxi, bool ineq, double di, double yi, double *a) {
    double r = qi - kxi;
    if (ineq && r < 0.0) r = 0.0;
    a[0] = fma(r, r, a[0]);
    const double ro = r / di;
    a[1] = fma(ro, ro, a[1]);
    a[2] = fma(qi, yi, a[2]);
  }
  __device__ __forceinline__ void operator()(int i, const double (&s)[1]) {
    if (!check) {
      kx[i] = s[0];
      if (keep) kxs[i] = s[0];
    } else {
      kxbar[i] = s[0];
    }
    if (!CG) {  // one CTA per LP: the pieces here (a team takes them in sums())
      const bool ineq = i >= n_eq;
      piece(q[i], check ? ldv<CG>(kx + i) : s[0], ineq, d1[i], ldv<CG>(y + i), acc);
      if (check) piece(q[i], s[0], ineq, d1[i], invW * ldv<CG>(sy + i), acc + 3);
    }
  }
  // this element's pieces, from the stored K x (and K xbar)
  __device__ __forceinline__ void sums(int i) {
    const bool ineq = i >= n_eq;
    piece(q[i], ldv<CG>(kx + i), ineq, d1[i], ldv<CG>(y + i), acc);
    if (check) piece(q[i], ldv<CG>(kxbar + i), ineq, d1[i], invW * ldv<CG>(sy + i), acc + 3);
  }
};

// This thread's share of the Sec. 2.2 infeasibility pieces for one ray,
// z - z_prev (difference of the last two accepted iterates) or z - z^{n,0}
// (the normalised iterate times t), unscaled to the original LP from the
// stored products: xr = D2 dx^, yr = D1 dy^, K'yr = (K~' dy^) / D2,
// K xr = (K~ dx^) / D1, c'xr = c~'dx^, q'yr = q~'dy^; with D2 > 0,
// lambda = proj_Lambda(-K'yr) = pp / D2 for pp = proj_Lambda(-K~' dy^), so
// l'lambda+ - u'lambda- = l~'pp+ - u~'pp- in scaled terms.  Layout:
// {||-K'yr - lambda||^2, l'lambda+ - u'lambda-, c'xr, cone violation of xr
// squared, ||(K_E xr, min(K_G xr, 0))||^2, q'yr, ||min(yr_G, 0)||^2}.
template <bool CG>
__device__ __forceinline__ void infeas_pieces(double (&f)[7], int n, int m, int n_eq, int e0, int es,
                                              const double *g, const double *gref, const double *x,
                                              const double *xref, const double *c, const double *l, const double *u,
                                              const double *D2, const double *kx, const double *kxref,
                                              const double *y, const double *yref, const double *q,
                                              const double *D1) {
#pragma unroll
  for (int a = 0; a < 7; ++a) f[a] = 0.0;
  for (int j = e0; j < n; j += es) {
    const double lj = l[j], uj = u[j], dj = D2[j];
    const bool lf = isfinite(lj), uf = isfinite(uj);
    const double mg = ldv<CG>(gref + j) - ldv<CG>(g + j);  // -(K~' dy^)_j
    const double pp = proj_lambda(mg, lj, uj);
    const double res = (mg - pp) / dj;
    f[0] = fma(res, res, f[0]);
    if (pp > 0.0) f[1] = fma(lj, pp, f[1]);
    if (pp < 0.0) f[1] = fma(uj, pp, f[1]);
    const double dx = ldv<CG>(x + j) - ldv<CG>(xref + j);
    f[2] = fma(c[j], dx, f[2]);
    if ((lf && dx < 0.0) || (uf && dx > 0.0)) {
      const double xo = dj * dx;
      f[3] = fma(xo, xo, f[3]);
    }
  }
  for (int i = e0; i < m; i += es) {
    const bool ineq = i >= n_eq;
    double kr = (ldv<CG>(kx + i) - ldv<CG>(kxref + i)) / D1[i];
    if (ineq && kr > 0.0) kr = 0.0;
    f[4] = fma(kr, kr, f[4]);
    const double dy = ldv<CG>(y + i) - ldv<CG>(yref + i);
    f[5] = fma(q[i], dy, f[5]);
    if (ineq && dy < 0.0) {
      const double yo = D1[i] * dy;
      f[6] = fma(yo, yo, f[6]);
    }
  }
}

// Sec. 2.2 infeasibility tests on one ray's reduced pieces, the dual-ray
// (primal infeasibility) test first; the same rule as the single-LP check.
// Returns the status, ST_RUNNING if neither certificate holds.
__device__ __forceinline__ int infeas_decide(const double (&a)[7], double eps) {
  const double obj_d = a[5] + a[1], res_d = sqrt(a[0] + a[6]);
  if (obj_d > 0.0 && res_d <= eps * obj_d) return ST_PRIMAL_INFEASIBLE;
  const double obj_p = -a[2], res_p = sqrt(a[4] + a[3]);
  if (obj_p > 0.0 && res_p <= eps * obj_p) return ST_DUAL_INFEASIBLE;
  return ST_RUNNING;
}

template <class Grp>
__device__ void solve_instance(const Arrays &A, const Inst &I, const Params &p, int id, double *red, Grp &grp) {
  constexpr bool CG = Grp::kTeam;
  const int m = I.m, n = I.n, tid = threadIdx.x;
  // this CTA's share of the element loops and of the row loops
  const int part = grp.rank(), parts = grp.size(), e0 = part * NTB + tid, es = parts * NTB;
  const int *kp = A.kptr + I.kp, *ki = A.kidx + I.ke, *tp = A.tptr + I.tp, *ti = A.tidx + I.te;
  const double *kv = A.kval + I.ke, *tv = A.tval + I.te;
  double *vm = A.vm + I.om, *vn = A.vn + I.on;
  auto VM = [&](int k) { return vm + (long long)k * m; };
  auto VN = [&](int k) { return vn + (long long)k * n; };
  double *x[2] = {VN(VN_X0), VN(VN_X1)}, *sx[2] = {VN(VN_SX0), VN(VN_SX1)};
  double *y[2] = {VM(VM_Y0), VM(VM_Y1)}, *sy[2] = {VM(VM_SY0), VM(VM_SY1)}, *kx[2] = {VM(VM_KX0), VM(VM_KX1)};
  double *g = VN(VN_G), *gbar = VN(VN_GB), *xl = VN(VN_XL), *yl = VM(VM_YL), *kxb = VM(VM_KXB);
  const double *c = VN(VN_C), *l = VN(VN_L), *u = VN(VN_U), *D2 = VN(VN_D2), *q = VM(VM_Q), *D1 = VM(VM_D1);
  const bool keep = p.eps_infeas > 0.0;  // infeasibility detection (vectors VN_GS, VN_GP, VM_KXS)
  auto VMK = [&](int k) { return A.vmk + I.okm + (long long)k * m; };  // global memory always
  auto VNK = [&](int k) { return A.vnk + I.okn + (long long)k * n; };
  // ---- start point (Sec. 4.1 "Initialization", or the warm start) ----
  for (int j = e0; j < n; j += es) {
    const double v = (p.warm && A.x0) ? A.x0[I.xo + j] / D2[j] : 0.0;
    x[0][j] = v;
    xl[j] = v;
    sx[0][j] = 0.0;
  }
  for (int i = e0; i < m; i += es) {
    const double v = (p.warm && A.y0) ? A.y0[I.yo + i] / D1[i] : 0.0;
    y[0][i] = v;
    yl[i] = v;
    sy[0][i] = 0.0;
  }
  bool ok = grp.sync();
  double eta = I.eta0, omega = I.omega0, W = 0.0, kkt_start, kkt_prev;
  double tau = eta / omega, sigma = eta * omega;  // primal / dual step sizes
  long long k = 0, t = 0;
  int cur = 0, need_g = 0, status = ST_RUNNING, which = 0;
  // KKT(z^{0,0}) with omega^0
  {
    CheckT<CG> ct{c, l, u, D2, x[0], sx[0], g, gbar, 0.0, 0, {0, 0, 0, 0, 0, 0, 0, 0}};
    ct.keep = keep;
    ct.gs = VNK(VN_GS);
    const double *const xs[1] = {y[0]};
    const double sc[1] = {1.0};
    rows_spmv<1, false, CG>(tp, ti, tv, n, I.gt, I.st, xs, sc, ct, part, parts);
    CheckK<CG> ck{q, D1, y[0], sy[0], kx[0], kxb, 0.0, 0, I.n_eq, {0, 0, 0, 0, 0, 0}};
    ck.keep = keep;
    ck.kxs = VMK(VM_KXS);
    const double *const xs2[1] = {x[0]};
    rows_spmv<1, false, CG>(kp, ki, kv, m, I.gk, I.sk, xs2, sc, ck, part, parts);
    if (CG) {  // a team: the stored products, then their pieces element by element
      ok = grp.sync() && ok;
      for (int j = e0; j < n; j += es) ct.sums(j);
      for (int i = e0; i < m; i += es) ck.sums(i);
    }
    double s[5] = {ct.acc[0], ct.acc[2], ct.acc[3], ck.acc[0], ck.acc[2]};
    ok = grp.template reduce<5>(s, red) && ok;
    if (!ok) status = ST_NUMERICAL;
    kkt_start = kkt_omega(s[3], s[0], s[1], s[4] + s[2], omega);
    kkt_prev = kkt_start;
  }
  while (status == ST_RUNNING) {
    const int nxt = cur ^ 1;
    // ---- Algorithm 2 trial: primal half-step ----
    PrimalRow<CG> pr{c, l, u, x[cur], sx[cur], g, x[nxt], sx[nxt], tau, eta, need_g != 0};
    if (need_g) {
      const double *const xs[1] = {y[cur]};
      const double sc[1] = {1.0};
      rows_spmv<1, false, CG>(tp, ti, tv, n, I.gt, I.st, xs, sc, pr, part, parts);
    } else {
      for (int j = e0; j < n; j += es) pr.apply(j, ldv<CG>(g + j));
    }
    if (!grp.sync()) {
      status = ST_NUMERICAL;
      break;
    }
    // ---- dual half-step ----
    DualRow<CG> dr{q, y[cur], kx[cur], sy[cur], y[nxt], kx[nxt], sy[nxt], sigma, eta, I.n_eq};
    {
      const double *const xs[1] = {x[nxt]};
      const double sc[1] = {1.0};
      rows_spmv<1, false, CG>(kp, ki, kv, m, I.gk, I.sk, xs, sc, dr, part, parts);
    }
    double s3[3] = {pr.dx2, dr.dy2, dr.cross};
    if (CG) {
      // a team (autotuned schedule): ||x' - x||^2, ||y' - y||^2 and
      // (y' - y)'(Kx' - Kx) from the stored vectors, one fixed thread per element
      if (!grp.sync()) {
        status = ST_NUMERICAL;
        break;
      }
      for (int j = e0; j < n; j += es) {
        const double d = ldv<CG>(x[nxt] + j) - ldv<CG>(x[cur] + j);
        s3[0] = fma(d, d, s3[0]);
      }
      for (int i = e0; i < m; i += es) {
        const double kn = ldv<CG>(kx[nxt] + i), d = ldv<CG>(y[nxt] + i) - ldv<CG>(y[cur] + i);
        s3[1] = fma(d, d, s3[1]);
        s3[2] = fma(d, kn - ldv<CG>(kx[cur] + i), s3[2]);
      }
    }
    // ---- step-size test (eq. step-size with |interaction|; exponent base k + 2) ----
    // one thread evaluates it and broadcasts: the FP64 divisions and powers,
    // run by every warp, would cost more than the whole iteration of a small
    // LP on GB300's narrow FP64 pipe
    auto step = [&](const double (&q3)[3]) {
      const double ia = fabs(q3[2]);
      const double eb = ia > 0.0 ? (omega * q3[0] + q3[1] / omega) / (2.0 * ia) : CUDART_INF;
      const double kk = (double)(k + 2);
      const double p3 = k < p.npw ? p.pw[k] : pow(kk, -0.3), p6 = k < p.npw ? p.pw[p.npw + k] : pow(kk, -0.6);
      const double e1 = (1.0 - p3) * eb, e2 = (1.0 + p6) * eta;
      const double en = e1 < e2 ? e1 : e2;
      const bool accept = eta <= eb;
      red[RED_BCAST] = en;
      red[RED_BCAST + 1] = en / omega;
      red[RED_BCAST + 2] = en * omega;
      red[RED_BCAST + 3] =
          (!isfinite(q3[0]) || !isfinite(q3[1]) || !isfinite(q3[2]) || isnan(eb) || !(en > 0.0)) ? 1.0 : 0.0;
      red[RED_BCAST + 4] = accept ? 1.0 : 0.0;
      red[RED_BCAST + 5] = accept ? W + eta : W;
    };
    if (!grp.template reduce_apply<3>(s3, red, step)) {
      status = ST_NUMERICAL;
      break;
    }
    // (the slots are rewritten only after the next iteration's barriers)
    if (red[RED_BCAST + 3] != 0.0) {
      status = ST_NUMERICAL;
      break;
    }
    eta = red[RED_BCAST];
    tau = red[RED_BCAST + 1];
    sigma = red[RED_BCAST + 2];
    W = red[RED_BCAST + 5];
    if (red[RED_BCAST + 4] == 0.0) {
      need_g = 0;
      continue;
    }
    cur = nxt;
    ++k;
    ++t;
    need_g = 1;
    if (k % p.P != 0 && k < p.max_iter) continue;
    // ---- restart / termination check (Sec. 3.4 / Sec. 4.1) ----
    const double invW = 1.0 / W;
    CheckT<CG> ct{c, l, u, D2, x[cur], sx[cur], g, gbar, invW, 1, {0, 0, 0, 0, 0, 0, 0, 0}};
    ct.keep = keep;
    ct.gs = VNK(VN_GS);
    ct.gp = VNK(VN_GP);
    {
      const double *const xs[2] = {y[cur], sy[cur]};
      const double sc[2] = {1.0, invW};
      rows_spmv<2, true, CG>(tp, ti, tv, n, I.gt, I.st, xs, sc, ct, part, parts);
    }
    CheckK<CG> ck{q, D1, y[cur], sy[cur], kx[cur], kxb, invW, 1, I.n_eq, {0, 0, 0, 0, 0, 0}};
    ck.keep = keep;
    ck.kxs = VMK(VM_KXS);
    {
      const double *const xs[1] = {sx[cur]};
      const double sc[1] = {invW};
      rows_spmv<1, true, CG>(kp, ki, kv, m, I.gk, I.sk, xs, sc, ck, part, parts);
    }
    need_g = 0;
    if (CG) {
      if (!grp.sync()) {
        status = ST_NUMERICAL;
        break;
      }
      for (int j = e0; j < n; j += es) ct.sums(j);
      for (int i = e0; i < m; i += es) ck.sums(i);
    }
    double s[14];
#pragma unroll
    for (int a = 0; a < 8; ++a) s[a] = ct.acc[a];
#pragma unroll
    for (int a = 0; a < 6; ++a) s[8 + a] = ck.acc[a];
    if (!grp.template reduce<14>(s, red)) {
      status = ST_NUMERICAL;
      break;
    }
    // Sec. 2.2 infeasibility: the difference ray, then the normalised one
    // (after the reduction's barriers: g, the kept K'y and Kx are written)
    int istat = ST_RUNNING, iray = 0;
    for (int r = 0; keep && r < 2 && istat == ST_RUNNING; ++r) {
      double f[7];
      infeas_pieces<CG>(f, n, m, I.n_eq, e0, es, g, VNK(r == 0 ? VN_GP : VN_GS), x[cur], r == 0 ? x[cur ^ 1] : xl,
                        c, l, u, D2, kx[cur], r == 0 ? kx[cur ^ 1] : VMK(VM_KXS), y[cur], r == 0 ? y[cur ^ 1] : yl,
                        q, D1);
      if (!grp.template reduce<7>(f, red)) {
        istat = ST_NUMERICAL;
        break;
      }
      istat = infeas_decide(f, p.eps_infeas);
      iray = 2 + r;
    }
    if (istat == ST_NUMERICAL) {
      status = ST_NUMERICAL;
      break;
    }
    // Sec. 4.1 termination, Sec. 2.2 infeasibility, GetRestartCandidate and
    // the criteria of Sec. 3.4: scalar work, evaluated by one thread and
    // broadcast (decision 0 / 1: optimal at the current / average point,
    // 2: iteration limit, 3: go on, 4: restart, 5: infeasible)
    if (tid == 0) {
      const double pc = s[2], dc = s[10] + s[3], rpc = sqrt(s[9]), rdc = sqrt(s[1]);
      const double pa = s[6], da = s[13] + s[7], rpa = sqrt(s[12]), rda = sqrt(s[5]);
      double dec = 3.0, kcand = 0.0;
      bool cand_avg = false;
      if (sec41_pass(pc, dc, rpc, rdc, p.tol, I.qn, I.cn)) {
        dec = 0.0;
      } else if (sec41_pass(pa, da, rpa, rda, p.tol, I.qn, I.cn)) {
        dec = 1.0;
      } else if (istat != ST_RUNNING) {
        dec = 5.0;
        red[RED_BCAST + 3] = (double)istat;
        red[RED_BCAST + 4] = (double)iray;
      } else if (k >= p.max_iter) {
        dec = 2.0;
      } else {
        const double kc = kkt_omega(s[8], s[0], pc, dc, omega);
        const double ka = kkt_omega(s[11], s[4], pa, da, omega);
        cand_avg = !(kc < ka);
        kcand = cand_avg ? ka : kc;
        const bool restart = kcand <= p.beta_suff * kkt_start ||
                             (kcand <= p.beta_nec * kkt_start && kcand > kkt_prev) ||
                             (double)t >= p.beta_art * (double)k;
        dec = restart ? 4.0 : 3.0;
      }
      red[RED_BCAST] = dec;
      red[RED_BCAST + 1] = cand_avg ? 1.0 : 0.0;
      red[RED_BCAST + 2] = kcand;
    }
    __syncthreads();
    const int dec = (int)red[RED_BCAST];
    if (dec <= 2) {
      status = dec == 2 ? ST_ITER_LIMIT : ST_OPTIMAL;
      which = dec == 1 ? 1 : 0;
      break;
    }
    if (dec == 5) {
      status = (int)red[RED_BCAST + 3];
      which = (int)red[RED_BCAST + 4];
      break;
    }
    if (dec == 3) {
      kkt_prev = red[RED_BCAST + 2];
      continue;
    }
    const bool cand_avg = red[RED_BCAST + 1] != 0.0;
    double dd[2] = {0.0, 0.0};
    for (int j = e0; j < n; j += es) {
      double xn = ldv<CG>(x[cur] + j);
      if (cand_avg) {
        xn = invW * ldv<CG>(sx[cur] + j);
        x[cur][j] = xn;
        g[j] = ldv<CG>(gbar + j);
      }
      if (keep) VNK(VN_GS)[j] = cand_avg ? ldv<CG>(gbar + j) : ldv<CG>(g + j);  // K'y at the new epoch start
      const double d = xn - ldv<CG>(xl + j);
      dd[0] = fma(d, d, dd[0]);
      xl[j] = xn;
      sx[cur][j] = 0.0;
    }
    for (int i = e0; i < m; i += es) {
      double yn = ldv<CG>(y[cur] + i);
      if (cand_avg) {
        yn = invW * ldv<CG>(sy[cur] + i);
        y[cur][i] = yn;
        kx[cur][i] = ldv<CG>(kxb + i);
      }
      if (keep) VMK(VM_KXS)[i] = cand_avg ? ldv<CG>(kxb + i) : ldv<CG>(kx[cur] + i);  // K x at the new epoch start
      const double d = yn - ldv<CG>(yl + i);
      dd[1] = fma(d, d, dd[1]);
      yl[i] = yn;
      sy[cur][i] = 0.0;
    }
    if (!grp.template reduce<2>(dd, red)) {
      status = ST_NUMERICAL;
      break;
    }
    // PrimalWeightUpdate and KKT of the new start point with the new omega
    if (tid == 0) {
      const double dx = sqrt(dd[0]), dy = sqrt(dd[1]);
      double om = omega;
      if (dx > p.eps_zero && dy > p.eps_zero) om = exp(p.theta * log(dy / dx) + (1.0 - p.theta) * log(om));
      const double pc = s[2], dc = s[10] + s[3], pa = s[6], da = s[13] + s[7];
      red[RED_BCAST + 3] = om;
      red[RED_BCAST + 4] = cand_avg ? kkt_omega(s[11], s[4], pa, da, om) : kkt_omega(s[8], s[0], pc, dc, om);
      red[RED_BCAST + 5] = eta / om;
      red[RED_BCAST + 6] = eta * om;
    }
    __syncthreads();
    omega = red[RED_BCAST + 3];
    kkt_start = red[RED_BCAST + 4];
    kkt_prev = kkt_start;
    tau = red[RED_BCAST + 5];
    sigma = red[RED_BCAST + 6];
    W = 0.0;
    t = 0;
  }
  // ---- output in the original space (an infeasibility certificate in place
  // of the iterate it concerns: y for primal, x for dual infeasibility) ----
  __syncthreads();
  const bool avg = which == 1;
  const bool xray = status == ST_DUAL_INFEASIBLE, yray = status == ST_PRIMAL_INFEASIBLE;
  const double invW = avg ? 1.0 / W : 0.0;
  for (int j = e0; j < n; j += es) {
    if (xray) {
      A.xout[I.xo + j] = D2[j] * (ldv<CG>(x[cur] + j) - ldv<CG>((which == 2 ? x[cur ^ 1] : xl) + j));
      continue;
    }
    const double xs = avg ? invW * ldv<CG>(sx[cur] + j) : ldv<CG>(x[cur] + j);
    double v = D2[j] * xs;
    const double l0 = vn[(long long)VN_L0 * n + j], u0 = vn[(long long)VN_U0 * n + j];
    if (v < l0) v = l0;
    if (v > u0) v = u0;
    A.xout[I.xo + j] = v;
  }
  for (int i = e0; i < m; i += es) {
    if (yray) {
      A.yout[I.yo + i] = D1[i] * (ldv<CG>(y[cur] + i) - ldv<CG>((which == 2 ? y[cur ^ 1] : yl) + i));
      continue;
    }
    const double ys = avg ? invW * ldv<CG>(sy[cur] + i) : ldv<CG>(y[cur] + i);
    A.yout[I.yo + i] = D1[i] * ys;
  }
  if (tid == 0 && part == 0) {
    A.status[id] = status;
    A.iters[id] = k;
    unsigned long long tn;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tn));
    A.t_end[id] = tn;
  }
  __syncthreads();
}

// Shared-memory bytes an LP needs to run resident (K, K', and every m- and
// n-vector block; each array 16-byte aligned).
__host__ __device__ inline long long resident_bytes(int m, int n, long long nnz) {
  auto a16 = [](long long b) { return (b + 15) & ~15LL; };
  return a16(4LL * (m + 1)) + a16(4LL * (n + 1)) + 2 * a16(4 * nnz) + 2 * a16(8 * nnz) +
         a16(8LL * VM_RES * m) + a16(8LL * VN_RES * n);
}

template <typename T>
__device__ __forceinline__ T *carve(unsigned char *&p, long long count) {
  T *r = reinterpret_cast<T *>(p);
  p += (sizeof(T) * count + 15) & ~15LL;
  return r;
}
template <typename T>
__device__ __forceinline__ void copy_in(T *dst, const T *src, long long count) {
  for (long long i = threadIdx.x; i < count; i += NTB) dst[i] = src[i];
}

// Solves the LP at queue position q with this CTA alone: from shared memory
// when its data fits in `resident_max` bytes of the CTA's dynamic shared
// memory (scaled K, K' and vectors copied in; read-only data is never copied
// back, the outputs go straight to global memory), else from global memory.
// The small LPs, which need the most iterations, thus run at shared-memory
// latency.
__device__ void solve_alone(const Arrays &A, const Inst *__restrict__ inst, int id, const Params &p,
                            long long resident_max, double *red, unsigned char *bsm) {
  const Inst I = inst[id];
  if (threadIdx.x == 0) A.t_start[id] = gtimer_ns();
  Solo solo;
  const long long nnz = A.kptr[I.kp + I.m] - A.kptr[I.kp];
  if (resident_bytes(I.m, I.n, nnz) <= resident_max) {
    unsigned char *cur = bsm;
    Arrays R = A;
    Inst J = I;
    int *kptr = carve<int>(cur, I.m + 1), *tptr = carve<int>(cur, I.n + 1);
    int *kidx = carve<int>(cur, nnz), *tidx = carve<int>(cur, nnz);
    double *kval = carve<double>(cur, nnz), *tval = carve<double>(cur, nnz);
    double *vm = carve<double>(cur, (long long)VM_RES * I.m), *vn = carve<double>(cur, (long long)VN_RES * I.n);
    // row pointers relative to the LP's first nonzero
    const int k0 = A.kptr[I.kp], t0 = A.tptr[I.tp];
    for (int i = threadIdx.x; i <= I.m; i += NTB) kptr[i] = A.kptr[I.kp + i] - k0;
    for (int j = threadIdx.x; j <= I.n; j += NTB) tptr[j] = A.tptr[I.tp + j] - t0;
    copy_in(kidx, A.kidx + I.ke + k0, nnz);
    copy_in(tidx, A.tidx + I.te + t0, nnz);
    copy_in(kval, A.kval + I.ke + k0, nnz);
    copy_in(tval, A.tval + I.te + t0, nnz);
    copy_in(vm, A.vm + I.om, (long long)VM_RES * I.m);
    copy_in(vn, A.vn + I.on, (long long)VN_RES * I.n);
    __syncthreads();
    R.kptr = kptr;
    R.tptr = tptr;
    R.kidx = kidx;
    R.tidx = tidx;
    R.kval = kval;
    R.tval = tval;
    R.vm = vm;
    R.vn = vn;
    J.kp = J.ke = J.tp = J.te = J.om = J.on = 0;
    solve_instance(R, J, p, id, red, solo);
  } else {
    solve_instance(A, I, p, id, red, solo);
  }
}

// Claims of queue positions from either end.  queue[0] counts claims from
// the front (largest LPs), queue[1] from the back (smallest); claimed[q] makes
// each position go to exactly one CTA where the two ends meet.  Returns -1
// when that end is exhausted.  A back claim stops, without claiming, at the
// first LP that a team must take.
__device__ __forceinline__ int claim_front(int *queue, int *claimed, int count) {
  const int q = atomicAdd(queue, 1);
  if (q >= count || atomicExch(claimed + q, 1) != 0) return -1;
  return q;
}
__device__ __forceinline__ int claim_back(const Arrays &A, const Inst *__restrict__ inst, const int *__restrict__ order,
                                          int *queue, int *claimed, int count, bool teams) {
  const int q = count - 1 - atomicAdd(queue + 1, 1);
  if (q < 0) return -1;
  if (teams) {
    const Inst &I = inst[order[q]];
    if (A.kptr[I.kp + I.m] - A.kptr[I.kp] >= TEAM_MIN_NNZ) return -1;
  }
  if (atomicExch(claimed + q, 1) != 0) return -1;
  return q;
}

// Persistent solver over the queue `order` (largest LPs first).  The first
// ts.teams * TEAM CTAs work in teams of TEAM (CTA b in team b / TEAM) from
// the front: the team leader claims the next LP and, while it has at least
// TEAM_MIN_NNZ nonzeros, all TEAM CTAs solve it together, so one large LP
// that needs many iterations no longer holds a single SM for the whole
// batch; from the first smaller LP on, the team disbands and each of its
// CTAs claims LPs alone.  The remaining CTAs start alone from the back, on
// the smallest LPs: those need the most iterations, and starting them first
// keeps them off the end of the schedule.  Large LPs are always solved by a
// team and small ones always by one CTA, so results do not depend on timing.
__global__ void __launch_bounds__(NTB) k_batch_solve(Arrays A, const Inst *__restrict__ inst,
                                                     const int *__restrict__ order, int count, int *queue,
                                                     int *claimed, Params p, long long resident_max, TeamState ts) {
  __shared__ double red[RED_SIZE];
  __shared__ int s_id;
  extern __shared__ __align__(16) unsigned char bsm[];
  const int team = blockIdx.x / TEAM;
  if (team < ts.teams) {
    if (p.stall && blockIdx.x == 1) return;
    Team grp{(int)(blockIdx.x % TEAM), ts.cnt + team, ts.gen + team, ts.slots + (size_t)team * 2 * TEAM * 16,
             ts.abort, 0};
    for (;;) {
      if (grp.rank() == 0 && threadIdx.x == 0) ts.q[team] = claim_front(queue, claimed, count);
      if (!grp.sync()) return;
      if (threadIdx.x == 0) s_id = __ldcg(ts.q + team);
      __syncthreads();
      const int q = s_id;
      // every rank has read the position before the leader may overwrite it
      if (!grp.sync()) return;
      if (q < 0) return;
      const int id = order[q];
      const Inst I = inst[id];
      const long long nnz = A.kptr[I.kp + I.m] - A.kptr[I.kp];
      if (nnz >= TEAM_MIN_NNZ) {
        if (grp.rank() == 0 && threadIdx.x == 0) A.t_start[id] = gtimer_ns();
        solve_instance(A, I, p, id, red, grp);
        if (*(volatile int *)ts.abort) return;
        continue;
      }
      // the first smaller LP: the leader solves it, and the team disbands
      if (grp.rank() == 0) solve_alone(A, inst, id, p, resident_max, red, bsm);
      break;
    }
    for (;;) {
      if (threadIdx.x == 0) s_id = claim_front(queue, claimed, count);
      __syncthreads();
      const int q = s_id;
      __syncthreads();
      if (q < 0) return;
      solve_alone(A, inst, order[q], p, resident_max, red, bsm);
    }
  }
  for (;;) {
    if (threadIdx.x == 0) s_id = claim_back(A, inst, order, queue, claimed, count, ts.teams > 0);
    __syncthreads();
    const int q = s_id;
    __syncthreads();
    if (q < 0) return;
    solve_alone(A, inst, order[q], p, resident_max, red, bsm);
  }
}

}  // namespace batch
}  // namespace pdlp

// ================================================================ host side

using namespace pdlp;
using namespace pdlp::batch;

struct pdlp_batch {
  int device = 0, count = 0, num_sms = 0, grid = 0;
  pdlp_params prm{};
  cudaStream_t stream = nullptr, cap = nullptr;
  bool own_stream = false;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  Arrays A{};
  Inst *d_inst = nullptr;
  int *d_order = nullptr, *d_queue = nullptr;
  double *d_x0 = nullptr, *d_y0 = nullptr;
  std::vector<Inst> h_inst;
  long long sum_m = 0, sum_n = 0, sum_nnz = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  Params gp{};  // parameters baked into the graph
  const double *g_x0 = nullptr, *g_y0 = nullptr;
  double solve_ms = 0.0, setup_ms = 0.0, tune_ms = 0.0;
  double lanes_target = 4.0;
  int resident = 0;  // LPs that fit the shared-memory budget
  int team_lps = 0;  // LPs solved by a team
  double *pw = nullptr;  // exponent-factor table (k_pow_table)
  long long npw = 0;
  TeamState ts{};               // team barriers / reductions (in the arena)
  void *team_words = nullptr;   // counters, generations, positions, abort flag
  size_t team_words_bytes = 0;
};

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int lanes_for(double mean_len, double target) {
  int g = 1;
  while (g < 32 && mean_len / g > target) g <<= 1;
  return g;
}

// the fixed lanes-per-row rule of an LP solved by one CTA (SOLO_FILL)
int solo_lanes(int rows, double mean_len) {
  if (!SOLO_FILL) return lanes_for(mean_len, SOLO_TARGET);
  int g = 1;
  while (g < 32 && (long long)rows * (2 * g) <= NTB) g <<= 1;
  return std::min(g, lanes_for(mean_len, 1.0));
}

void free_batch(pdlp_batch *b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->arena) cudaFree(b->arena);
  if (b->pw) cudaFree(b->pw);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

#define BCK(call)                                                                                              \
  do {                                                                                                         \
    cudaError_t e_ = (call);                                                                                   \
    if (e_ != cudaSuccess) return set_error(PDLP_ERR_CUDA, (std::string(#call) + ": " + cudaGetErrorString(e_)).c_str()); \
  } while (0)

int launch_solve(pdlp_batch *b, const Arrays &A, const Params &p, cudaStream_t s) {
  BCK(cudaMemsetAsync(b->d_queue, 0, 8 + 4 * (size_t)b->count, s));
  // team barrier counters and the abort flag start at zero
  BCK(cudaMemsetAsync(b->team_words, 0, b->team_words_bytes, s));
  k_batch_solve<<<b->grid, NTB, RESIDENT_MAX, s>>>(A, b->d_inst, b->d_order, b->count, b->d_queue,
                                                  b->d_queue + 2, p, (long long)RESIDENT_MAX, b->ts);
  BCK(cudaGetLastError());
  return PDLP_OK;
}

}  // namespace

extern "C" {

int pdlp_batch_create(pdlp_batch **out, int32_t count, const pdlp_lp *lps, const pdlp_params *params,
                      void *stream) {
  if (!out || count < 1 || !lps) return set_error(PDLP_ERR_INVALID, "pdlp_batch_create: need out, count >= 1, lps");
  pdlp_params prm;
  if (params)
    prm = *params;
  else
    pdlp_default_params(&prm);
  if (prm.check_period < 1 || prm.ruiz_iters < 0 || !(prm.pc_alpha <= 2.0) || prm.value_bits != 64)
    return set_error(PDLP_ERR_INVALID, "pdlp_batch_create: invalid parameters (batched solves use value_bits 64)");
  const double t0 = now_ms();
  pdlp_batch *b = new pdlp_batch();
  b->count = count;
  b->prm = prm;
  b->h_inst.resize(count);
  // ---- validate and lay out ----
  long long KP = 0, KE = 0, TP = 0, TE = 0, OM = 0, ON = 0, XO = 0, YO = 0;
  for (int i = 0; i < count; ++i) {
    const pdlp_lp &L = lps[i];
    if (L.m < 0 || L.n < 1 || L.n_eq < 0 || L.n_eq > L.m || !L.c || !L.row_ptr || !L.l || !L.u ||
        (L.m > 0 && !L.q) || L.row_ptr[0] != 0) {
      delete b;
      return set_error(PDLP_ERR_INVALID, ("pdlp_batch_create: bad dimensions or null array in LP " + std::to_string(i)).c_str());
    }
    for (int r = 0; r < L.m; ++r)
      if (L.row_ptr[r + 1] < L.row_ptr[r]) {
        delete b;
        return set_error(PDLP_ERR_INVALID, ("pdlp_batch_create: row_ptr not non-decreasing in LP " + std::to_string(i)).c_str());
      }
    const long long nnz = L.row_ptr[L.m];
    for (long long e = 0; e < nnz; ++e)
      if (L.col_idx[e] < 0 || L.col_idx[e] >= L.n || !std::isfinite(L.val[e])) {
        delete b;
        return set_error(PDLP_ERR_INVALID, ("pdlp_batch_create: bad column index or value in LP " + std::to_string(i)).c_str());
      }
    for (int j = 0; j < L.n; ++j)
      if (!std::isfinite(L.c[j]) || std::isnan(L.l[j]) || std::isnan(L.u[j]) || L.l[j] > L.u[j] || L.l[j] == INFINITY ||
          L.u[j] == -INFINITY) {
        delete b;
        return set_error(PDLP_ERR_INVALID, ("pdlp_batch_create: bad c or bounds in LP " + std::to_string(i)).c_str());
      }
    for (int r = 0; r < L.m; ++r)
      if (!std::isfinite(L.q[r])) {
        delete b;
        return set_error(PDLP_ERR_INVALID, ("pdlp_batch_create: non-finite q in LP " + std::to_string(i)).c_str());
      }
    Inst &I = b->h_inst[i];
    std::memset(&I, 0, sizeof(I));
    I.m = L.m;
    I.n = L.n;
    I.n_eq = L.n_eq;
    I.kp = KP;
    I.ke = KE;
    I.tp = TP;
    I.te = TE;
    I.om = I.okm = OM;
    I.on = I.okn = ON;
    I.xo = XO;
    I.yo = YO;
    KP += L.m + 1;
    TP += L.n + 1;
    if (resident_bytes(L.m, L.n, nnz) <= RESIDENT_MAX) ++b->resident;
    if (nnz >= TEAM_MIN_NNZ) ++b->team_lps;
    KE += nnz;
    TE += nnz;
    OM += (long long)VM_COUNT * L.m;
    ON += (long long)VN_COUNT * L.n;
    XO += L.n;
    YO += L.m;
    double qn = 0.0, cn = 0.0;
    for (int r = 0; r < L.m; ++r) qn += L.q[r] * L.q[r];
    for (int j = 0; j < L.n; ++j) cn += L.c[j] * L.c[j];
    I.qn = std::sqrt(qn);
    I.cn = std::sqrt(cn);
  }
  b->sum_m = YO;
  b->sum_n = XO;
  b->sum_nnz = KE;
  // ---- device ----
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) {
    if (stream) {
      b->stream = (cudaStream_t)stream;
    } else {
      e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
      b->own_stream = true;
    }
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  int per_sm = 1;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batch_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, RESIDENT_MAX);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_solve, NTB, RESIDENT_MAX);
  if (e != cudaSuccess) {
    free_batch(b);
    return set_error(PDLP_ERR_CUDA, cudaGetErrorString(e));
  }
  b->grid = std::max(1, std::min(count, per_sm * b->num_sms));
  // with room for a team: whole teams plus BACK_CTAS CTAs that start from
  // the small end of the queue
  const int teams = b->grid >= BACK_CTAS + TEAM ? (b->grid - BACK_CTAS) / TEAM : 0;
  if (teams) b->grid = teams * TEAM + BACK_CTAS;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  const size_t o_kptr = off; off += al(4 * KP);
  const size_t o_kidx = off; off += al(4 * KE + 16);
  const size_t o_kval = off; off += al(8 * KE + 16);
  const size_t o_tptr = off; off += al(4 * TP);
  const size_t o_tidx = off; off += al(4 * TE + 16);
  const size_t o_tval = off; off += al(8 * TE + 16);
  const size_t o_vm = off; off += al(8 * std::max<long long>(OM, 1));
  const size_t o_vn = off; off += al(8 * ON);
  const size_t o_xo = off; off += al(8 * XO);
  const size_t o_yo = off; off += al(8 * std::max<long long>(YO, 1));
  const size_t o_x0 = off; off += al(8 * XO);
  const size_t o_y0 = off; off += al(8 * std::max<long long>(YO, 1));
  const size_t o_st = off; off += al(4 * count);
  const size_t o_it = off; off += al(8 * count);
  const size_t o_ts = off; off += al(16 * (size_t)count);
  const size_t o_in = off; off += al(sizeof(Inst) * count);
  const size_t o_or = off; off += al(4 * count);
  const size_t o_q = off; off += al(8 + 4 * (size_t)count);  // front / back counters, claim flags
  const size_t o_tw = off; off += al(4 * (3 * (size_t)teams + 1));
  const size_t o_tsl = off; off += al(8 * (size_t)std::max(teams, 1) * 2 * TEAM * 16);
  b->arena_bytes = off;
  e = cudaMalloc((void **)&b->arena, b->arena_bytes);
  if (e != cudaSuccess) {
    free_batch(b);
    return set_error(e == cudaErrorMemoryAllocation ? PDLP_ERR_OOM : PDLP_ERR_CUDA, cudaGetErrorString(e));
  }
  char *Ar = b->arena;
  b->A.kptr = (int *)(Ar + o_kptr);
  b->A.kidx = (int *)(Ar + o_kidx);
  b->A.kval = (double *)(Ar + o_kval);
  b->A.tptr = (int *)(Ar + o_tptr);
  b->A.tidx = (int *)(Ar + o_tidx);
  b->A.tval = (double *)(Ar + o_tval);
  b->A.vm = b->A.vmk = (double *)(Ar + o_vm);
  b->A.vn = b->A.vnk = (double *)(Ar + o_vn);
  b->A.xout = (double *)(Ar + o_xo);
  b->A.yout = (double *)(Ar + o_yo);
  b->d_x0 = (double *)(Ar + o_x0);
  b->d_y0 = (double *)(Ar + o_y0);
  b->A.status = (int *)(Ar + o_st);
  b->A.iters = (long long *)(Ar + o_it);
  b->A.t_start = (unsigned long long *)(Ar + o_ts);
  b->A.t_end = b->A.t_start + count;
  b->d_inst = (Inst *)(Ar + o_in);
  b->d_order = (int *)(Ar + o_or);
  b->d_queue = (int *)(Ar + o_q);
  {
    unsigned *w = (unsigned *)(Ar + o_tw);
    b->ts.cnt = w;
    b->ts.gen = w + teams;
    b->ts.q = (int *)(w + 2 * teams);
    b->ts.abort = (int *)(w + 3 * teams);
    b->ts.slots = (double *)(Ar + o_tsl);
    b->ts.teams = teams;
    b->team_words = w;
    b->team_words_bytes = 4 * (3 * (size_t)teams + 1);
  }
  // longest instances first
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    const long long na = lps[a].row_ptr[lps[a].m], nc = lps[c].row_ptr[lps[c].m];
    return na + lps[a].m + lps[a].n > nc + lps[c].m + lps[c].n;
  });
  cudaStream_t st = b->stream;
#define BCKS(call)                                                                             \
  do {                                                                                         \
    cudaError_t e2_ = (call);                                                                  \
    if (e2_ != cudaSuccess) {                                                                  \
      std::string msg_ = std::string(#call) + ": " + cudaGetErrorString(e2_);                   \
      free_batch(b);                                                                           \
      return set_error(PDLP_ERR_CUDA, msg_.c_str());                                           \
    }                                                                                          \
  } while (0)
  BCKS(cudaMemsetAsync(b->arena, 0, b->arena_bytes, st));
  // per LP: K straight from the caller's arrays, K' by a stable counting sort
  // into a host buffer of the worker thread that handles the LP, and the
  // input vectors into their blocks.  The sources are pageable: each copy has
  // read its source when the call returns, so a buffer is reused at once.
  {
    long long max_n = 1, max_nnz = 1, tot_nnz = 0;
    for (int i = 0; i < count; ++i) {
      max_n = std::max<long long>(max_n, lps[i].n);
      max_nnz = std::max<long long>(max_nnz, lps[i].row_ptr[lps[i].m]);
      tot_nnz += lps[i].row_ptr[lps[i].m];
    }
    const int T = std::min(host_threads(tot_nnz), count);
    std::vector<cudaError_t> errs(T, cudaSuccess);
    parallel_for(T, [&](int w) {
      std::vector<int> tp((size_t)max_n + 1), ti((size_t)max_nnz);
      std::vector<double> tv((size_t)max_nnz);
      cudaError_t e = cudaSetDevice(b->device);
      for (int i = w; i < count && e == cudaSuccess; i += T) {
        const pdlp_lp &L = lps[i];
        const Inst &I = b->h_inst[i];
        const long long nnz = L.row_ptr[L.m];
        csr_transpose(L.m, L.n, L.row_ptr, L.col_idx, L.val, tp.data(), ti.data(), tv.data());
        auto cp = [&](void *dst, const void *src, size_t bytes) {
          if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
        };
        cp((void *)(b->A.kptr + I.kp), L.row_ptr, 4 * (size_t)(L.m + 1));
        cp((void *)(b->A.tptr + I.tp), tp.data(), 4 * (size_t)(L.n + 1));
        cp((void *)(b->A.kidx + I.ke), L.col_idx, 4 * (size_t)nnz);
        cp(b->A.kval + I.ke, L.val, 8 * (size_t)nnz);
        cp((void *)(b->A.tidx + I.te), ti.data(), 4 * (size_t)nnz);
        cp(b->A.tval + I.te, tv.data(), 8 * (size_t)nnz);
        cp(b->A.vm + I.om + (long long)VM_Q0 * L.m, L.q, 8 * (size_t)L.m);
        cp(b->A.vn + I.on + (long long)VN_C0 * L.n, L.c, 8 * (size_t)L.n);
        cp(b->A.vn + I.on + (long long)VN_L0 * L.n, L.l, 8 * (size_t)L.n);
        cp(b->A.vn + I.on + (long long)VN_U0 * L.n, L.u, 8 * (size_t)L.n);
      }
      errs[w] = e;
    });
    for (cudaError_t e : errs) BCKS(e);
  }
  BCKS(cudaMemcpyAsync(b->d_order, order.data(), 4 * count, cudaMemcpyHostToDevice, st));
  BCKS(cudaMemcpyAsync(b->d_inst, b->h_inst.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice, st));
  k_batch_scale<<<count, NTB, 0, st>>>(b->A, b->d_inst, count, prm.ruiz_iters, prm.pc_alpha, prm.eps_zero);
  BCKS(cudaGetLastError());
  BCKS(cudaMemcpyAsync(b->h_inst.data(), b->d_inst, sizeof(Inst) * count, cudaMemcpyDeviceToHost, st));
  BCKS(cudaStreamSynchronize(st));
  b->setup_ms = now_ms() - t0;
  // ---- schedule: lanes per row (G) for each LP's K and K'.  An LP solved
  // by a team is autotuned: candidates are the rules "smallest power of two
  // G <= 32 with mean row length / G <= t" for t in {4, 8, 16} (warp-per-row
  // for the longest rows, several rows per warp for short ones); every
  // candidate is timed on short solves of the whole batch (2P iterations)
  // and each LP keeps the one under which it finished fastest.  Its row sums
  // do not depend on G (the slot order of rows_spmv, S = the t = 4 rule) and
  // its sums over rows are taken by element passes, so the choice, and any
  // timing noise behind it, changes speed only, never results.  An LP on one
  // CTA (latency-bound: an element pass would cost it more than tuning
  // gains) keeps the fixed rule t = SOLO_TARGET. ----
  std::vector<double> mean_k(count), mean_t(count);
  std::vector<char> team(count);
  for (int i = 0; i < count; ++i) {
    Inst &I = b->h_inst[i];
    const double nnz = (double)lps[i].row_ptr[lps[i].m];
    mean_k[i] = I.m ? nnz / I.m : 0.0;
    mean_t[i] = nnz / I.n;
    team[i] = nnz >= (double)TEAM_MIN_NNZ;
    // a team's rows may take any tuned G (S from the t = 4 rule); an LP on
    // one CTA keeps the fixed rule t = SOLO_TARGET (S = G: the plain order)
    I.sk = team[i] ? lanes_for(mean_k[i], 4.0) : solo_lanes(I.m, mean_k[i]);
    I.st = team[i] ? lanes_for(mean_t[i], 4.0) : solo_lanes(I.n, mean_t[i]);
  }
  const double cands[3] = {4.0, 8.0, 16.0};
  auto lanes_of = [&](int i, double target, int *gk, int *gt) {
    const Inst &I = b->h_inst[i];
    if (!team[i]) {
      *gk = I.sk;
      *gt = I.st;
      return;
    }
    *gk = std::max(lanes_for(mean_k[i], target), std::max(1, I.sk / 4));
    *gt = std::max(lanes_for(mean_t[i], target), std::max(1, I.st / 4));
  };
  auto set_lanes = [&](const std::vector<int> &choice) -> int {
    for (int i = 0; i < count; ++i) lanes_of(i, cands[choice[i]], &b->h_inst[i].gk, &b->h_inst[i].gt);
    cudaError_t e3 = cudaMemcpyAsync(b->d_inst, b->h_inst.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice, st);
    return e3 == cudaSuccess ? PDLP_OK : set_error(PDLP_ERR_CUDA, cudaGetErrorString(e3));
  };
  const double t1 = now_ms();
  Params tp{};
  tp.tol = 0.0;
  tp.theta = prm.theta;
  tp.eps_zero = prm.eps_zero;
  tp.eps_infeas = prm.eps_infeas;
  tp.beta_suff = prm.beta_suff;
  tp.beta_nec = prm.beta_nec;
  tp.beta_art = prm.beta_art;
  tp.max_iter = 2 * prm.check_period;
  tp.P = prm.check_period;
  tp.warm = 0;
  std::vector<int> choice(count, 0);
  std::vector<double> best(count, INFINITY);
  std::vector<unsigned long long> stamps(2 * (size_t)count);
  for (int ci = -1; ci < 3; ++ci) {  // ci = -1: an untimed warm-up launch
    std::vector<int> all(count, ci < 0 ? 0 : ci);
    int rc = set_lanes(all);
    if (!rc) rc = launch_solve(b, b->A, tp, st);
    if (rc) {
      free_batch(b);
      return rc;
    }
    BCKS(cudaMemcpyAsync(stamps.data(), b->A.t_start, 16 * (size_t)count, cudaMemcpyDeviceToHost, st));
    BCKS(cudaStreamSynchronize(st));
    if (ci < 0) continue;
    for (int i = 0; i < count; ++i) {
      const double d = (double)(stamps[count + i] - stamps[i]);
      if (d < best[i]) {
        best[i] = d;
        choice[i] = ci;
      }
    }
  }
  // test hook (environment PDLP_TEST_BATCH_TARGET = 4, 8 or 16): every LP
  // gets that candidate, so tests can compare results across schedules
  if (const char *force = std::getenv("PDLP_TEST_BATCH_TARGET")) {
    const double f = std::atof(force);
    for (int k = 0; k < 3; ++k)
      if (f == cands[k]) std::fill(choice.begin(), choice.end(), k);
  }
  int rc = set_lanes(choice);
  if (rc) {
    free_batch(b);
    return rc;
  }
  BCKS(cudaStreamSynchronize(st));
  {
    int votes[3] = {0, 0, 0};
    for (int i = 0; i < count; ++i) votes[choice[i]]++;
    const int top = (int)(std::max_element(votes, votes + 3) - votes);
    b->lanes_target = cands[top];
  }
  b->tune_ms = now_ms() - t1;
#undef BCKS
  *out = b;
  return PDLP_OK;
}

int pdlp_batch_solve(pdlp_batch *b, const double *x0, const double *y0, double tol, int64_t max_iter, double *x_out,
                     double *y_out, int32_t *status, int64_t *iters) {
  if (!b) return set_error(PDLP_ERR_INVALID, "pdlp_batch_solve: batch is NULL");
  if (!(tol >= 0.0) || max_iter < 1) return set_error(PDLP_ERR_INVALID, "pdlp_batch_solve: need tol >= 0, max_iter >= 1");
  BCK(cudaSetDevice(b->device));
  const double t0 = now_ms();
  cudaStream_t st = b->stream;
  Params p{};
  p.tol = tol;
  p.theta = b->prm.theta;
  p.eps_zero = b->prm.eps_zero;
  p.eps_infeas = b->prm.eps_infeas;
  p.beta_suff = b->prm.beta_suff;
  p.beta_nec = b->prm.beta_nec;
  p.beta_art = b->prm.beta_art;
  p.max_iter = max_iter;
  p.P = b->prm.check_period;
  p.warm = (x0 || y0) ? 1 : 0;
  {
    const char *ev = std::getenv("PDLP_TEST_TEAM_STALL");
    p.stall = (ev && ev[0] == '1' && b->ts.teams > 0) ? 1 : 0;
  }
  {
    const long long need = std::min<long long>(max_iter, 1LL << 22);
    if (need > b->npw) {
      if (b->pw) cudaFree(b->pw);
      b->pw = nullptr;
      b->npw = 0;
      BCK(cudaMalloc(&b->pw, 2 * sizeof(double) * (size_t)need));
      BCK(setup_pow_table(b->pw, need, st));
      b->npw = need;
    }
    p.pw = b->pw;
    p.npw = b->npw;
  }
  Arrays A = b->A;
  A.x0 = x0 ? b->d_x0 : nullptr;
  A.y0 = y0 ? b->d_y0 : nullptr;
  if (x0) BCK(cudaMemcpyAsync(b->d_x0, x0, 8 * b->sum_n, cudaMemcpyHostToDevice, st));
  if (y0 && b->sum_m) BCK(cudaMemcpyAsync(b->d_y0, y0, 8 * b->sum_m, cudaMemcpyHostToDevice, st));
  // one CUDA graph per (parameters, warm start) combination, rebuilt when they change
  const bool same = b->gexec && std::memcmp(&b->gp, &p, sizeof(Params)) == 0 && b->g_x0 == A.x0 && b->g_y0 == A.y0;
  if (!same) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    const int rc = launch_solve(b, A, p, b->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e2 != cudaSuccess) return set_error(PDLP_ERR_CUDA, cudaGetErrorString(e2));
    b->graph = g;
    BCK(cudaGraphInstantiate(&b->gexec, b->graph, 0));
    b->gp = p;
    b->g_x0 = A.x0;
    b->g_y0 = A.y0;
  }
  BCK(cudaGraphLaunch(b->gexec, st));
  if (x_out) BCK(cudaMemcpyAsync(x_out, b->A.xout, 8 * b->sum_n, cudaMemcpyDeviceToHost, st));
  if (y_out && b->sum_m) BCK(cudaMemcpyAsync(y_out, b->A.yout, 8 * b->sum_m, cudaMemcpyDeviceToHost, st));
  if (status) BCK(cudaMemcpyAsync(status, b->A.status, 4 * (size_t)b->count, cudaMemcpyDeviceToHost, st));
  if (iters) BCK(cudaMemcpyAsync(iters, b->A.iters, 8 * (size_t)b->count, cudaMemcpyDeviceToHost, st));
  int aborted = 0;
  BCK(cudaMemcpyAsync(&aborted, b->ts.abort, sizeof(int), cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  if (aborted)
    return set_error(PDLP_ERR_CUDA, "pdlp_batch_solve: a team of CTAs timed out at a barrier (another kernel holding "
                                    "SMs?); the results are incomplete");
  b->solve_ms = now_ms() - t0;
  return PDLP_OK;
}

int pdlp_batch_info(const pdlp_batch *b, pdlp_batch_stats *s) {
  if (!b || !s) return set_error(PDLP_ERR_INVALID, "pdlp_batch_info: null argument");
  std::memset(s, 0, sizeof(*s));
  s->count = b->count;
  s->grid = b->grid;
  s->sum_m = b->sum_m;
  s->sum_n = b->sum_n;
  s->sum_nnz = b->sum_nnz;
  s->setup_ms = b->setup_ms;
  s->tune_ms = b->tune_ms;
  s->solve_ms = b->solve_ms;
  s->entries_per_lane = b->lanes_target;
  s->device_bytes = b->arena_bytes;
  s->resident = b->resident;
  s->resident_max_bytes = RESIDENT_MAX;
  s->team_lps = b->ts.teams > 0 ? b->team_lps : 0;
  s->team_size = TEAM;
  s->team_min_nnz = (int32_t)TEAM_MIN_NNZ;
  return PDLP_OK;
}

int pdlp_batch_times(const pdlp_batch *b, double *start_s, double *end_s) {
  if (!b) return set_error(PDLP_ERR_INVALID, "pdlp_batch_times: batch is NULL");
  BCK(cudaSetDevice(b->device));
  std::vector<unsigned long long> h(2 * (size_t)b->count);
  BCK(cudaMemcpy(h.data(), b->A.t_start, 16 * (size_t)b->count, cudaMemcpyDeviceToHost));
  unsigned long long t0 = ~0ull;
  for (int i = 0; i < b->count; ++i) t0 = std::min(t0, h[i]);
  for (int i = 0; i < b->count; ++i) {
    if (start_s) start_s[i] = 1e-9 * (double)(h[i] - t0);
    if (end_s) end_s[i] = 1e-9 * (double)(h[b->count + i] - t0);
  }
  return PDLP_OK;
}

int pdlp_batch_lanes(const pdlp_batch *b, int32_t *lanes_K, int32_t *lanes_KT) {
  if (!b) return set_error(PDLP_ERR_INVALID, "pdlp_batch_lanes: batch is NULL");
  for (int i = 0; i < b->count; ++i) {
    if (lanes_K) lanes_K[i] = b->h_inst[i].gk;
    if (lanes_KT) lanes_KT[i] = b->h_inst[i].gt;
  }
  return PDLP_OK;
}

void pdlp_batch_destroy(pdlp_batch *b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

}  // extern "C"
