// Hot-path kernels of restarted PDHG (cuPDLP.jl paper, Algorithms 1 and 2,
// eq. (pdhg), eq. (step-size), eq. (kkt), Sec. 3.4 and Sec. 4.1).
//
// One accepted PDHG iteration is two kernels:
//   k_primal  (rows of K'):  g = K'y (only when y changed), then
//             x' = proj_X(x - (eta/omega)(c - g)),  sx' = sx + eta x',
//             block partial of ||x' - x||^2.
//   k_dual    (rows of K):   Kx', then
//             y' = proj_Y(y + eta*omega (q - (2 Kx' - Kx))),  sy' = sy + eta y',
//             partials of ||y'-y||^2 and (y'-y)'(Kx' - Kx) = (y'-y)'K(x'-x);
//             its last CTA finishes all partials in a fixed order and runs the
//             Algorithm 2 test (accept: flip the buffer parity; reject: retry
//             with eta').
// Every P accepted steps the check kernels run:
//   k_check_primal (rows of K'):  K'y (if stale) and K'ybar in one pass over
//             K', dual residual / objective pieces for the current and the
//             average iterate, scaled (restart) and original (termination).
//   k_check_dual   (rows of K):   K xbar, primal residual pieces; its last CTA
//             applies Sec. 4.1 termination, GetRestartCandidate and the three
//             restart criteria of Sec. 3.4.
//   k_infeas (elementwise, between the two):  pieces of the infeasibility
//             certificates (Sec. 2.2, last bullet) for the difference of the
//             last two accepted iterates and for the normalised iterate,
//             from stored products (no SpMV).
//   k_restart (elementwise):      moves the candidate into the iterate, resets
//             the epoch average, and (last CTA) PrimalWeightUpdate.
// Every kernel reads the device state at entry and returns at once when it
// has nothing to do, so a fixed CUDA graph of P + E trial slots followed by the
// check kernels advances the solve by exactly one check period.
//
// SpMV (sliced ELL, see SellMat): rows are renumbered by length within
// their group at create, so that 32 consecutive internal rows have nearly
// equal lengths; such a slice is stored column-major (entry k of lane l at
// off + 32 k + l) and one warp computes it with one row per lane: coalesced
// 4-byte index loads, 8-byte value loads, random gathers of x / y straight
// into registers, FMAs in the row's own order, and the row's epilogue in the
// same lane -- no shared memory, no barriers, no cross-lane reduction.  The
// random gathers bind on GB300 (about 0.85 per clock per SM whatever the
// cache qualifier; 2e7 of them take ~74 us), then the narrow FP64 pipe
// (~1.6 DFMA per clock per SM), so the layout spends one FMA per stored
// entry and one epilogue per 32 rows.  Rows longer than SELL_LONG are stored
// contiguously and taken by a whole warp (lane-strided partial sums); their
// totals come out of a butterfly over 32 such rows at a time, followed by
// one vectorised epilogue.  Warps walk a cost-sorted item list in a snake
// order, independently: every warp keeps its own loads and gathers in
// flight.  Reductions are deterministic: fixed per-lane order, fixed
// butterfly and shuffle trees, fixed block order in the last CTA.  No
// atomics touch floating point.

#include <math.h>
#include <math_constants.h>

#include "pdlp_internal.cuh"

namespace pdlp {

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA-wide sums of NV values in a fixed order; totals land in every lane of
// warp 0.  s_red holds NV * NW doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *s_red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = warp_sum(v[a]);
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) s_red[a * NW + wid] = v[a];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = warp_sum(lane < NW ? s_red[a * NW + lane] : 0.0);
  }
  __syncthreads();
}

// Writes this CTA's NV partial sums, and returns true in every thread of the
// CTA that finishes last; there `tot` holds the grid totals summed in block
// order (deterministic for a fixed grid).  The counter is reset for the next
// launch by that CTA.
template <int NV>
__device__ __forceinline__ bool grid_finish(double (&v)[NV], double *part, unsigned int *counter, double *s_red,
                                            int *s_flag, double (&tot)[NV]) {
  block_sum<NV>(v, s_red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) part[(size_t)blockIdx.x * NV + a] = v[a];
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    *s_flag = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!*s_flag) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) acc[a] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) {
#pragma unroll
    for (int a = 0; a < NV; ++a) acc[a] += __ldcg(part + (size_t)b * NV + a);
  }
  block_sum<NV>(acc, s_red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) s_red[a] = acc[a];
    *counter = 0u;
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NV; ++a) tot[a] = s_red[a];
  __syncthreads();
  return true;
}

// Sums a partial array of `count` blocks x NV values written by an earlier
// kernel, in block order.  Totals valid in every lane of warp 0.
template <int NV>
__device__ __forceinline__ void sum_partials(const double *part, int count, double *s_red, double (&tot)[NV]) {
#pragma unroll
  for (int a = 0; a < NV; ++a) tot[a] = 0.0;
  for (int b = threadIdx.x; b < count; b += NT) {
#pragma unroll
    for (int a = 0; a < NV; ++a) tot[a] += __ldcg(part + (size_t)b * NV + a);
  }
  block_sum<NV>(tot, s_red);
}

// ---------------------------------------------------------------- sliced-ELL SpMV

// float -> double from the IEEE bits with integer operations, exact for
// every normal float and for zero: with t the magnitude bits, the high word
// is the sign | ((t >> 3) + (896 << 20)) (exponent re-biased by 1023 - 127,
// top 20 mantissa bits), the low word the last 3 mantissa bits << 29, and
// t = 0 gives the signed zero.  The FP32 copies the step kernels read hold
// only normal floats and zeros (setup_f32 flushes the subnormals, and the
// scaled matrix is finite), so no hardware conversion and no branch: the
// widening stays off GB300's narrow FP64 pipe.
__device__ __forceinline__ double f2d(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int t = b & 0x7fffffffu;
  const unsigned int hi = (b ^ t) | (t ? (t >> 3) + 0x38000000u : 0u);
  return __hiloint2double((int)hi, (int)(b << 29));
}
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return f2d(v); }

// Sum over `cnt` strides of 32 stored entries, this lane's entry of each
// stride: acc[a] += val * xs[a][col] in stride order (FMA), padding (column
// -1) skipped.  U strides are loaded (streaming, coalesced across the
// warp) before their gathers are issued, and all gathers before the FMAs.
template <int U, typename VT, int NV, bool SCALED>
__device__ __forceinline__ void strided_dot(const int32_t *__restrict__ ip, const VT *__restrict__ vp, int cnt,
                                            const double *const (&xs)[NV], const double (&sc)[NV],
                                            double (&acc)[NV]) {
  int k = 0;
  for (; k + U <= cnt; k += U) {
    int c[U];
    VT v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = __ldcs(ip + 32 * (k + u));
      v[u] = __ldcs(vp + 32 * (k + u));
    }
    double g[NV][U];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        const double xv = c[u] >= 0 ? __ldg(xs[a] + c[u]) : 0.0;
        g[a][u] = SCALED ? sc[a] * xv : xv;
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int a = 0; a < NV; ++a) acc[a] = fma(widen(v[u]), g[a][u], acc[a]);
  }
  for (; k < cnt; ++k) {
    const int c = __ldcs(ip + 32 * k);
    const VT v = __ldcs(vp + 32 * k);
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      const double xv = c >= 0 ? __ldg(xs[a] + c) : 0.0;
      acc[a] = fma(widen(v), SCALED ? sc[a] * xv : xv, acc[a]);
    }
  }
}

// One butterfly level: lanes with the `off` bit clear keep row a's pair sum,
// lanes with it set keep row b's.
__device__ __forceinline__ double bfly(double a, double b, int off, int lane) {
  const bool hi = (lane & off) != 0;
  const double recv = __shfl_xor_sync(0xffffffffu, hi ? a : b, off);
  return (hi ? b : a) + recv;
}

// Long rows (whole warp per row) are reduced 32 at a time: the per-lane
// partial sums of the batch's rows go through a five-level butterfly
// (31 additions per lane for 32 rows instead of 5 per row), after which
// lane l holds the total of the batch's row rev5(l), and one vectorised
// epilogue finishes all 32 rows.  The tree is fixed, so the sums are too.
template <int NV>
struct LongRows {
  double buf[5][NV];
  int t;        // rows in the current batch (warp-uniform)
  int *rows;    // this warp's 32 row slots in shared memory
  double *tot;  // this warp's 32 x NV totals in shared memory (partial batch)
};

template <int NV, class Epi>
__device__ __forceinline__ void long_push(LongRows<NV> &lr, const double (&p)[NV], int row, Epi &ep) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) lr.rows[lr.t] = row;
  const int t = lr.t;
  double v[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = p[a];
  bool done = false;
  if (!(t & 1)) {
#pragma unroll
    for (int a = 0; a < NV; ++a) lr.buf[0][a] = v[a];
  } else {
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = bfly(lr.buf[0][a], v[a], 16, lane);
    if (!(t & 2)) {
#pragma unroll
      for (int a = 0; a < NV; ++a) lr.buf[1][a] = v[a];
    } else {
#pragma unroll
      for (int a = 0; a < NV; ++a) v[a] = bfly(lr.buf[1][a], v[a], 8, lane);
      if (!(t & 4)) {
#pragma unroll
        for (int a = 0; a < NV; ++a) lr.buf[2][a] = v[a];
      } else {
#pragma unroll
        for (int a = 0; a < NV; ++a) v[a] = bfly(lr.buf[2][a], v[a], 4, lane);
        if (!(t & 8)) {
#pragma unroll
          for (int a = 0; a < NV; ++a) lr.buf[3][a] = v[a];
        } else {
#pragma unroll
          for (int a = 0; a < NV; ++a) v[a] = bfly(lr.buf[3][a], v[a], 2, lane);
          if (!(t & 16)) {
#pragma unroll
            for (int a = 0; a < NV; ++a) lr.buf[4][a] = v[a];
          } else {
#pragma unroll
            for (int a = 0; a < NV; ++a) v[a] = bfly(lr.buf[4][a], v[a], 1, lane);
            done = true;
          }
        }
      }
    }
  }
  lr.t = t + 1;
  if (done) {
    __syncwarp();
    const int r = lr.rows[__brev(lane) >> 27];
    __syncwarp();
    if (r >= 0) {
      ep.prefetch(r);
      ep.finish(r, v);
    }
    lr.t = 0;
  }
}

// Finishes a partial batch of t < 32 long rows without padding it: buf[k]
// (present when bit k of t is set) holds slots [t & ~(2^(k+1) - 1), +2^k)
// after k butterfly levels, lane l carrying a partial of the block's slot
// rev_k(l >> (5 - k)); the remaining 5 - k levels are a plain xor reduction,
// after which the first lane of every group of 32 >> k holds its row's
// total.  The totals go through shared memory so that lane s finishes slot
// s: one epilogue (one round of operand loads) for the whole batch.
template <int NV, class Epi>
__device__ __forceinline__ void long_flush(LongRows<NV> &lr, Epi &ep) {
  const int lane = threadIdx.x & 31, t = lr.t;
  __syncwarp();
#pragma unroll
  for (int k = 4; k >= 0; --k) {
    if (!(t & (1 << k))) continue;
    const int start = t & ~((2 << k) - 1);
    double v[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = lr.buf[k][a];
#pragma unroll
    for (int off = 16 >> k; off >= 1; off >>= 1)
#pragma unroll
      for (int a = 0; a < NV; ++a) v[a] += __shfl_xor_sync(0xffffffffu, v[a], off);
    if ((lane & ((32 >> k) - 1)) == 0) {
      const int slot = start + (k ? (int)(__brev((unsigned)(lane >> (5 - k))) >> (32 - k)) : 0);
#pragma unroll
      for (int a = 0; a < NV; ++a) lr.tot[slot * NV + a] = v[a];
    }
  }
  __syncwarp();
  if (lane < t) {
    const int r = lr.rows[lane];
    double v[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = lr.tot[lane * NV + a];
    ep.prefetch(r);
    ep.finish(r, v);
  }
  __syncwarp();
  lr.t = 0;
}

// y = A x for NV (1 or 2) gathered vectors, each finished row r passed to
// ep.finish(r, sums) after ep.prefetch(r).  With SCALED, gathered entries of
// vector a are multiplied by sc[a] (the epoch average (1/W) sum).  Warp w of
// the grid takes items w, 2G - 1 - w, 2G + w, ... of the schedule (G warps):
// a snake over the cost-sorted items, so every warp gets about the same work.
template <int U, typename VT, int NV, bool SCALED, class Epi>
__device__ __forceinline__ void spmv_sell(const SellMat &A, const VT *__restrict__ val,
                                          const double *const (&xs)[NV], const double (&sc)[NV], Epi &ep,
                                          int *warp_rows, double *warp_tot) {
  const int lane = threadIdx.x & 31;
  const int nw = (int)((gridDim.x * (unsigned)NT) >> 5);
  const int gw = (int)((blockIdx.x * (unsigned)NT + threadIdx.x) >> 5);
  LongRows<NV> lr;
  lr.t = 0;
  lr.rows = warp_rows;
  lr.tot = warp_tot;
  // the warp's b-th item of the snake order (-1: none)
  auto item_of = [&](int b) -> long long {
    const long long first = (long long)b * nw;
    if (first >= A.nitems) return -1;
    const long long it = first + ((b & 1) ? nw - 1 - gw : gw);
    return it < A.nitems ? it : -1;
  };
  long long it = item_of(0);
  int4 d = it >= 0 ? __ldg(A.items + it) : make_int4(0, 0, 0, 0);
  for (int b = 0; it >= 0; ++b) {
    const long long itn = item_of(b + 1);
    int4 dn = make_int4(0, 0, 0, 0);
    double acc[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) acc[a] = 0.0;
    if (d.y > 0) {  // slice: one row per lane
      const bool has = lane < d.y;
      const int row = d.x + lane;
      if (has) ep.prefetch(row);
      strided_dot<U, VT, NV, SCALED>(A.idx + d.w + lane, val + d.w + lane, d.z, xs, sc, acc);
      if (has) ep.finish(row, acc);
    } else {  // long row: the whole warp
      strided_dot<U, VT, NV, SCALED>(A.idx + d.w + lane, val + d.w + lane, (d.z + 31) >> 5, xs, sc, acc);
      long_push(lr, acc, d.x, ep);
    }
    if (itn >= 0) dn = __ldg(A.items + itn);  // the next item's descriptor
    it = itn;
    d = dn;
  }
  if (lr.t > 0) long_flush(lr, ep);
}

// ---------------------------------------------------------------- primal step

// QP: qd (the scaled diagonal of Q) non-null, and the primal step is the
// exact proximal step of x'Qx/2 + (c - K'y)'x over X, coordinate by
// coordinate: x' = proj_X((x - tau (c - g)) / (1 + tau Q_jj)).
template <bool QP>
struct PrimalEpi {
  const double *__restrict__ c, *__restrict__ l, *__restrict__ u, *__restrict__ x, *__restrict__ sx;
  const double *__restrict__ qd;
  double *__restrict__ g, *__restrict__ xn, *__restrict__ sxn;
  double tau, eta, dx2;
  double pc, pl, pu, px, psx, pq;
  __device__ __forceinline__ void prefetch(int j) {
    pc = c[j];
    pl = l[j];
    pu = u[j];
    px = x[j];
    psx = sx[j];
    if (QP) pq = qd[j];
  }
  __device__ __forceinline__ void finish(int j, const double (&gs)[1]) { apply(j, gs[0], true); }
  __device__ __forceinline__ void apply(int j, double gj, bool store_g) {
    if (store_g) g[j] = gj;
    const double v = QP ? clamp_bits(fma(-tau, pc - gj, px) / fma(tau, pq, 1.0), pl, pu)
                        : clamp_bits(fma(-tau, pc - gj, px), pl, pu);
    xn[j] = v;
    sxn[j] = fma(eta, v, psx);
    const double d = v - px;
    dx2 = fma(d, d, dx2);
  }
};

template <bool QP>
__device__ __forceinline__ void primal_step(const SellMat &KT, const Vecs &V, const DevState *st, double *s_red,
                                            int (*s_rows)[32], double (*s_tot)[64]) {
  const int cur = st->cur, nxt = cur ^ 1, need_g = st->need_g, f32 = st->use_f32;
  const double eta = st->eta, omega = st->omega;
  PrimalEpi<QP> ep;
  ep.c = V.c;
  ep.l = V.l;
  ep.u = V.u;
  ep.qd = V.qd;
  ep.x = V.x[cur];
  ep.sx = V.sx[cur];
  ep.g = V.g;
  ep.xn = V.x[nxt];
  ep.sxn = V.sx[nxt];
  ep.tau = eta / omega;
  ep.eta = eta;
  ep.dx2 = 0.0;
  if (need_g) {
    const double *const xs[1] = {V.y[cur]};
    const double sc[1] = {1.0};
    if (f32)
      spmv_sell<SELL_U_P, float, 1, false>(KT, KT.val32, xs, sc, ep, s_rows[threadIdx.x >> 5], s_tot[threadIdx.x >> 5]);
    else
      spmv_sell<SELL_U_P, double, 1, false>(KT, KT.val, xs, sc, ep, s_rows[threadIdx.x >> 5], s_tot[threadIdx.x >> 5]);
  } else {
    // rejected trial: g = K'y is unchanged, only the projection reruns
    for (int j = blockIdx.x * NT + threadIdx.x; j < V.n; j += gridDim.x * NT) {
      ep.prefetch(j);
      ep.apply(j, V.g[j], false);
    }
  }
  double acc[1] = {ep.dx2};
  block_sum<1>(acc, s_red);
  if (threadIdx.x == 0) V.partA[blockIdx.x] = acc[0];
}

// STEP_MINB CTAs per SM: as many warps (gathers in flight) as the registers allow
__global__ void __launch_bounds__(NT, STEP_MINB) k_primal(SellMat KT, Vecs V, DevState *__restrict__ st) {
  __shared__ double s_red[16 * NW];
  __shared__ int s_rows[NW][32];
  __shared__ double s_tot[NW][64];
  if (st->status != ST_RUNNING || st->check_pending) return;
  primal_step<false>(KT, V, st, s_red, s_rows, s_tot);
}

// The QP's primal step (V.qd set), a kernel of its own so that the LP's
// keeps its register budget.
__global__ void __launch_bounds__(NT, STEP_MINB) k_primal_qp(SellMat KT, Vecs V, DevState *__restrict__ st) {
  __shared__ double s_red[16 * NW];
  __shared__ int s_rows[NW][32];
  __shared__ double s_tot[NW][64];
  if (st->status != ST_RUNNING || st->check_pending) return;
  primal_step<true>(KT, V, st, s_red, s_rows, s_tot);
}

// ---------------------------------------------------------------- dual step + Algorithm 2 test

struct DualEpi {
  const double *__restrict__ q, *__restrict__ y, *__restrict__ kx, *__restrict__ sy;
  double *__restrict__ yn, *__restrict__ kxn, *__restrict__ syn;
  double sigma, eta, dy2, cross;
  int n_eq;
  double pq, py, pkx, psy;
  __device__ __forceinline__ void prefetch(int i) {
    pq = q[i];
    py = y[i];
    pkx = kx[i];
    psy = sy[i];
  }
  __device__ __forceinline__ void finish(int i, const double (&ks)[1]) {
    const double kn = ks[0];
    double v = fma(sigma, pq - fma(2.0, kn, -pkx), py);
    if (i >= n_eq && __double_as_longlong(v) < 0) v = 0.0;  // proj_Y: sign bit test
    yn[i] = v;
    kxn[i] = kn;
    syn[i] = fma(eta, v, psy);
    const double d = v - py;
    dy2 = fma(d, d, dy2);
    cross = fma(d, kn - pkx, cross);
  }
};

// Algorithm 2 acceptance test (one thread).  eq. (step-size) with the
// interaction taken in absolute value; the exponent base counts the step
// being taken from 1 (k + 2 for k accepted steps so far).
__device__ void step_test(DevState *st, const Vecs &V, double dx2, double dy2, double cross) {
  const double eta = st->eta, omega = st->omega;
  const long long k = st->k;
  const double ia = fabs(cross);
  const double eta_bar = ia > 0.0 ? (omega * dx2 + dy2 / omega) / (2.0 * ia) : CUDART_INF;
  const double kk = (double)(k + 2);
  // the exponent factors come from a table built at create by the same pow()
  // (two FP64 powers are microseconds of serial latency on GB300's FP64 pipe,
  // on the critical path of every step)
  const double p3 = k < V.npw ? V.pw[k] : pow(kk, -0.3), p6 = k < V.npw ? V.pw[V.npw + k] : pow(kk, -0.6);
  const double e1 = (1.0 - p3) * eta_bar;
  const double e2 = (1.0 + p6) * eta;
  const double eta_next = e1 < e2 ? e1 : e2;
  st->attempts += 1;
  if (!isfinite(dx2) || !isfinite(dy2) || !isfinite(cross) || isnan(eta_bar) || !(eta_next > 0.0)) {
    st->status = ST_NUMERICAL;
    return;
  }
  st->eta = eta_next;
  if (eta <= eta_bar) {
    st->cur ^= 1;
    st->k = k + 1;
    st->t += 1;
    st->W += eta;
    st->need_g = 1;
    if ((k + 1) % st->P == 0 || k + 1 >= st->max_iter) st->check_pending = 1;
  } else {
    st->need_g = 0;  // g = K'y was refreshed by this trial's primal kernel
  }
}

__global__ void __launch_bounds__(NT, STEP_MINB) k_dual(SellMat K, Vecs V, DevState *__restrict__ st) {
  __shared__ double s_red[16 * NW];
  __shared__ int s_flag;
  __shared__ int s_rows[NW][32];
  __shared__ double s_tot[NW][64];
  if (st->status != ST_RUNNING || st->check_pending) return;
  const int cur = st->cur, nxt = cur ^ 1, f32 = st->use_f32;
  const double eta = st->eta, omega = st->omega;
  DualEpi ep;
  ep.q = V.q;
  ep.y = V.y[cur];
  ep.kx = V.Kx[cur];
  ep.sy = V.sy[cur];
  ep.yn = V.y[nxt];
  ep.kxn = V.Kx[nxt];
  ep.syn = V.sy[nxt];
  ep.sigma = eta * omega;
  ep.eta = eta;
  ep.dy2 = 0.0;
  ep.cross = 0.0;
  ep.n_eq = V.n_eq;
  const double *const xs[1] = {V.x[nxt]};
  const double sc[1] = {1.0};
  if (f32)
    spmv_sell<SELL_U_D, float, 1, false, DualEpi>(K, K.val32, xs, sc, ep, s_rows[threadIdx.x >> 5], s_tot[threadIdx.x >> 5]);
  else
    spmv_sell<SELL_U_D, double, 1, false, DualEpi>(K, K.val, xs, sc, ep, s_rows[threadIdx.x >> 5], s_tot[threadIdx.x >> 5]);
  double acc[2] = {ep.dy2, ep.cross};
  double tot[2];
  if (!grid_finish<2>(acc, V.partB, &st->cnt[CNT_DUAL], s_red, &s_flag, tot)) return;
  double dx[1];
  sum_partials<1>(V.partA, V.gridA, s_red, dx);
  if (threadIdx.x == 0) step_test(st, V, dx[0], tot[0], tot[1]);
}

// ---------------------------------------------------------------- restart / termination check

// IEEE-bit tests (integer pipe): sign of a nonzero, finiteness
__device__ __forceinline__ bool neg_bits(double v) { return __double_as_longlong(v) < 0; }
__device__ __forceinline__ bool pos_bits(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ bool finite_bits(double v) {
  return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// proj_Lambda (reading 5 of the paper's lambda): every test on the IEEE
// bits, so GB300's narrow FP64 pipe does none of it.  -0.0 maps to -0.0 or
// +0.0, which no sum below can tell from 0.
__device__ __forceinline__ double proj_lambda(double d, double l, double u) {
  const bool lf = finite_bits(l), uf = finite_bits(u);
  if (lf && uf) return d;
  if (lf) return pos_bits(d) ? d : 0.0;
  if (uf) return neg_bits(d) ? d : 0.0;
  return 0.0;
}

// Dual-side pieces of eq. (kkt) / Sec. 4.1 for one variable.
// With qp (Q_jj = qdj), the objective's gradient c + Qx replaces c in the
// reduced cost, and x'Qx/2 is added to the primal objective c'x and taken
// from the dual one (the QP's objectives).
// The original-space residual is r / D2, taken as r times the stored 1/D2
// (rd2): no FP64 division on the hot check path.
__device__ __forceinline__ void dual_piece(double c, double g, double l, double u, double rd2, double x,
                                           double *acc, bool qp = false, double qdj = 0.0) {
  const double d = qp ? fma(qdj, x, c) - g : c - g;
  const double lam = proj_lambda(d, l, u);
  const double r = d - lam;
  acc[0] = fma(r, r, acc[0]);
  const double ro = r * rd2;
  acc[1] = fma(ro, ro, acc[1]);
  acc[2] = fma(c, x, acc[2]);
  if (pos_bits(lam)) acc[3] = fma(l, lam, acc[3]);
  if (neg_bits(lam) && (__double_as_longlong(lam) << 1) != 0) acc[3] = acc[3] - u * (-lam);
  if (qp) {
    const double h = 0.5 * qdj * x * x;
    acc[2] += h;
    acc[3] -= h;
  }
}

// Epilogue of the dual-side check pass.  kind 0: start point (sums = {K'y});
// kind 1: check with stale g (sums = {K'y, K'ybar}); kind 2: check with g
// current (sums = {K'ybar}, g loaded).
struct CheckPrimalEpi {
  const double *__restrict__ c, *__restrict__ l, *__restrict__ u, *__restrict__ rd2, *__restrict__ x,
      *__restrict__ sx;
  double *__restrict__ g, *__restrict__ gbar;
  double *__restrict__ g0, *__restrict__ gprev;  // kept for infeasibility detection when keep
  const double *__restrict__ qd;                 // QP: the scaled diagonal of Q (else null)
  double invW;
  int kind, keep;
  double acc[NV_R1];
  double pc, pl, pu, pd2, px, psx, pg, pq;
  __device__ __forceinline__ void prefetch(int j) {
    pc = c[j];
    pl = l[j];
    pu = u[j];
    pd2 = rd2[j];
    px = x[j];
    psx = kind ? sx[j] : 0.0;
    pg = (kind == 2 || (kind == 1 && keep)) ? g[j] : 0.0;
    pq = qd ? qd[j] : 0.0;
  }
  template <int NV>
  __device__ __forceinline__ void finish(int j, const double (&s)[NV]) {
    double gj = pg, gb = 0.0;
    if (kind == 0) {
      gj = s[0];
      g[j] = gj;
      if (keep) g0[j] = gj;  // K'y at the epoch start
    } else if (kind == 1) {
      gj = s[0];
      gb = s[NV - 1];
      if (keep) gprev[j] = pg;  // K'y of the previous accepted iterate
      g[j] = gj;
    } else {
      gb = s[0];
    }
    const bool qp = qd != nullptr;
    dual_piece(pc, gj, pl, pu, pd2, px, acc, qp, pq);
    if (kind) {
      gbar[j] = gb;
      dual_piece(pc, gb, pl, pu, pd2, invW * psx, acc + 4, qp, pq);
    }
  }
};

__global__ void __launch_bounds__(NT, CHECK_MINB) k_check_primal(SellMat KT, Vecs V, DevState *__restrict__ st) {
  __shared__ double s_red[16 * NW];
  __shared__ int s_rows[NW][32];
  __shared__ double s_tot[NW][64];
  if (st->status != ST_RUNNING || !st->check_pending) return;
  const int mode = st->mode, cur = st->cur, need_g = st->need_g;
  const bool check = mode == MODE_CHECK;
  CheckPrimalEpi ep;
  ep.c = V.c;
  ep.l = V.l;
  ep.u = V.u;
  ep.rd2 = V.rD2;
  ep.x = V.x[cur];
  ep.sx = V.sx[cur];
  ep.g = V.g;
  ep.gbar = V.gbar;
  ep.g0 = V.g0;
  ep.gprev = V.gprev;
  ep.qd = V.qd;
  ep.invW = check ? 1.0 / st->W : 0.0;
  ep.kind = !check ? 0 : (need_g ? 1 : 2);
  ep.keep = st->eps_infeas > 0.0;
#pragma unroll
  for (int a = 0; a < NV_R1; ++a) ep.acc[a] = 0.0;
  if (ep.kind == 0) {
    const double *const xs[1] = {V.y[cur]};
    const double sc[1] = {1.0};
    spmv_sell<SELL_U_C, double, 1, false>(KT, KT.val, xs, sc, ep, s_rows[threadIdx.x >> 5], s_tot[threadIdx.x >> 5]);
  } else if (ep.kind == 1) {
    const double *const xs[2] = {V.y[cur], V.sy[cur]};
    const double sc[2] = {1.0, ep.invW};
    spmv_sell<SELL_U_C, double, 2, true>(KT, KT.val, xs, sc, ep, s_rows[threadIdx.x >> 5], s_tot[threadIdx.x >> 5]);
  } else {
    const double *const xs[1] = {V.sy[cur]};
    const double sc[1] = {ep.invW};
    spmv_sell<SELL_U_C, double, 1, true>(KT, KT.val, xs, sc, ep, s_rows[threadIdx.x >> 5], s_tot[threadIdx.x >> 5]);
  }
  block_sum<NV_R1>(ep.acc, s_red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV_R1; ++a) V.partR1[(size_t)blockIdx.x * NV_R1 + a] = ep.acc[a];
  }
}

// The original-space residual is r / D1, taken as r times the stored 1/D1.
__device__ __forceinline__ void primal_piece(double q, double kx, bool ineq, double rd1, double y, double *acc) {
  double r = q - kx;
  if (ineq && neg_bits(r)) r = 0.0;
  acc[0] = fma(r, r, acc[0]);
  const double ro = r * rd1;
  acc[1] = fma(ro, ro, acc[1]);
  acc[2] = fma(q, y, acc[2]);
}

__device__ __forceinline__ double kkt_omega(double rp2, double rd2, double pobj, double dobj, double omega) {
  const double gap = dobj - pobj;
  return sqrt(omega * omega * rp2 + rd2 / (omega * omega) + gap * gap);
}

__device__ __forceinline__ bool sec41_pass(double pobj, double dobj, double rp, double rd, double tol, double qn,
                                           double cn) {
  if (!(fabs(dobj - pobj) <= tol * (1.0 + fabs(dobj) + fabs(pobj)))) return false;
  if (!(rp <= tol * (1.0 + qn))) return false;
  if (!(rd <= tol * (1.0 + cn))) return false;
  return true;
}

__device__ __forceinline__ double sec41_rel(double pobj, double dobj, double rp, double rd, double qn, double cn) {
  const double a = fabs(dobj - pobj) / (1.0 + fabs(dobj) + fabs(pobj));
  const double b = rp / (1.0 + qn);
  const double c = rd / (1.0 + cn);
  return fmax(a, fmax(b, c));
}

// p: the 8 dual-side sums (current 0..3, average 4..7); d: the 6 primal-side
// sums (current 0..2, average 3..5).
// Sec. 2.2 infeasibility detection on k_infeas' sums for one ray (original
// LP): the dual ray certifies primal infeasibility when its objective
// q'yr + l'lam+ - u'lam- is positive and ||(-K'yr - lam, min(yr_G, 0))||
// is at most eps times it; the primal ray certifies dual infeasibility when
// -c'xr is positive and ||(K_E xr, min(K_G xr, 0), cone violation)|| is at
// most eps times it.  Returns the status, or ST_RUNNING.
__device__ int infeas_status(const double *a, double eps, double *ray) {
  const double obj_d = a[5] + a[1], res_d = sqrt(a[0] + a[6]);
  if (obj_d > 0.0 && res_d <= eps * obj_d) {
    ray[0] = obj_d;
    ray[1] = res_d;
    return ST_PRIMAL_INFEASIBLE;
  }
  const double obj_p = -a[2], res_p = sqrt(a[4] + a[3]);
  if (obj_p > 0.0 && res_p <= eps * obj_p) {
    ray[0] = obj_p;
    ray[1] = res_p;
    return ST_DUAL_INFEASIBLE;
  }
  return ST_RUNNING;
}

__device__ void check_decide(DevState *st, TraceRec *trace, const double *p, const double *d, const double *inf) {
  const double omega = st->omega;
  if (st->mode == MODE_INIT) {
    const double k0 = kkt_omega(d[0], p[0], p[2], d[2] + p[3], omega);
    st->kkt_start = k0;
    st->kkt_prev = k0;
    st->mode = MODE_CHECK;
    st->need_g = 0;
    st->check_pending = 0;
    return;
  }
  st->checks += 1;
  st->need_g = 0;
  const double pc = p[2], dc = d[2] + p[3], rpc = sqrt(d[1]), rdc = sqrt(p[1]);
  const double pa = p[6], da = d[5] + p[7], rpa = sqrt(d[4]), rda = sqrt(p[5]);
  const double tol = st->tol, qn = st->q_norm, cn = st->c_norm;
  st->term[0] = pc;
  st->term[1] = dc;
  st->term[2] = rpc;
  st->term[3] = rdc;
  if (sec41_pass(pc, dc, rpc, rdc, tol, qn, cn)) {
    st->status = ST_OPTIMAL;
    st->which = 0;
    return;
  }
  if (sec41_pass(pa, da, rpa, rda, tol, qn, cn)) {
    st->term[0] = pa;
    st->term[1] = da;
    st->term[2] = rpa;
    st->term[3] = rda;
    st->status = ST_OPTIMAL;
    st->which = 1;
    return;
  }
  if (inf) {  // difference ray, then normalised-iterate ray
    for (int r = 0; r < 2; ++r) {
      const int stt = infeas_status(inf + r * NV_I1, st->eps_infeas, st->ray);
      if (stt != ST_RUNNING) {
        st->status = stt;
        st->which = 2 + r;
        return;
      }
    }
  }
  if (st->k >= st->max_iter) {
    st->status = ST_ITER_LIMIT;
    st->which = 0;
    return;
  }
  const double kc = kkt_omega(d[0], p[0], pc, dc, omega);
  const double ka = kkt_omega(d[3], p[4], pa, da, omega);
  const int cand_avg = !(kc < ka);
  const double kcand = cand_avg ? ka : kc;
  const double ks = st->kkt_start;
  int mask = 0;
  if (kcand <= st->beta_suff * ks) mask |= 1;
  if (kcand <= st->beta_nec * ks && kcand > st->kkt_prev) mask |= 2;
  if ((double)st->t >= st->beta_art * (double)st->k) mask |= 4;
  if (mask) {
    st->restart_to = cand_avg ? 2 : 1;
    if (cand_avg) {
      st->cand[0] = d[3];
      st->cand[1] = p[4];
      st->cand[2] = pa;
      st->cand[3] = da;
    } else {
      st->cand[0] = d[0];
      st->cand[1] = p[0];
      st->cand[2] = pc;
      st->cand[3] = dc;
    }
    if (st->use_f32 && st->polish) {
      // FP32-values mode: move the steps to the FP64 K once the original-space
      // relative KKT of the restart point stops improving for two restarts.
      const double rel = cand_avg ? sec41_rel(pa, da, rpa, rda, qn, cn) : sec41_rel(pc, dc, rpc, rdc, qn, cn);
      if (rel < st->rel_kkt_best) {
        st->rel_kkt_best = rel;
        st->stall = 0;
      } else if (++st->stall >= 2) {
        st->use_f32 = 0;
        st->f64_switch_k = st->k;
      }
    }
  } else {
    st->kkt_prev = kcand;
    st->check_pending = 0;
  }
  {  // the check's record, into the ring
    TraceRec &r = trace[st->ntrace % st->trace_cap];
    r.k = st->k;
    r.attempts = st->attempts;
    r.restarts = st->restarts + (mask ? 1 : 0);
    r.restart = mask;
    r.cand_avg = cand_avg;
    r.kkt_cur = kc;
    r.kkt_avg = ka;
    r.kkt_start = st->kkt_start;
    r.omega = omega;
    r.eta_hat = st->eta;
    r.rel_gap = fabs(pc - dc) / (1.0 + fabs(pc) + fabs(dc));
    r.rel_primal = rpc / (1.0 + qn);
    r.rel_dual = rdc / (1.0 + cn);
    st->ntrace += 1;
  }
}

// Epilogue of the primal-side check pass.  check = 0: start point (sums =
// {Kx}, stored as Kx); check = 1: sums = {K xbar}.
struct CheckDualEpi {
  const double *__restrict__ q, *__restrict__ rd1, *__restrict__ y, *__restrict__ sy;
  double *__restrict__ kx, *__restrict__ kxbar, *__restrict__ kx0;
  double invW;
  int check, n_eq, keep;
  double acc[NV_R2];
  double pq, pd1, py, psy, pkx;
  __device__ __forceinline__ void prefetch(int i) {
    pq = q[i];
    pd1 = rd1[i];
    py = y[i];
    psy = check ? sy[i] : 0.0;
    pkx = check ? kx[i] : 0.0;
  }
  __device__ __forceinline__ void finish(int i, const double (&s)[1]) {
    const bool ineq = i >= n_eq;
    double kxi = pkx;
    if (!check) {
      kxi = s[0];
      kx[i] = kxi;
      if (keep) kx0[i] = kxi;  // K x at the epoch start
    }
    primal_piece(pq, kxi, ineq, pd1, py, acc);
    if (check) {
      kxbar[i] = s[0];
      primal_piece(pq, s[0], ineq, pd1, invW * psy, acc + 3);
    }
  }
};

__global__ void __launch_bounds__(NT) k_check_dual(SellMat K, Vecs V, DevState *__restrict__ st) {
  __shared__ double s_red[16 * NW];
  __shared__ int s_flag;
  __shared__ int s_rows[NW][32];
  __shared__ double s_tot[NW][64];
  if (st->status != ST_RUNNING || !st->check_pending) return;
  const int mode = st->mode, cur = st->cur;
  const bool check = mode == MODE_CHECK;
  CheckDualEpi ep;
  ep.q = V.q;
  ep.rd1 = V.rD1;
  ep.y = V.y[cur];
  ep.sy = V.sy[cur];
  ep.kx = V.Kx[cur];
  ep.kxbar = V.Kxbar;
  ep.kx0 = V.kx0;
  ep.invW = check ? 1.0 / st->W : 0.0;
  ep.check = check ? 1 : 0;
  ep.n_eq = V.n_eq;
  ep.keep = st->eps_infeas > 0.0;
#pragma unroll
  for (int a = 0; a < NV_R2; ++a) ep.acc[a] = 0.0;
  if (!check) {
    const double *const xs[1] = {V.x[cur]};
    const double sc[1] = {1.0};
    spmv_sell<SELL_U_C, double, 1, false>(K, K.val, xs, sc, ep, s_rows[threadIdx.x >> 5], s_tot[threadIdx.x >> 5]);
  } else {
    const double *const xs[1] = {V.sx[cur]};
    const double sc[1] = {ep.invW};
    spmv_sell<SELL_U_C, double, 1, true>(K, K.val, xs, sc, ep, s_rows[threadIdx.x >> 5], s_tot[threadIdx.x >> 5]);
  }
  double tot[NV_R2];
  if (!grid_finish<NV_R2>(ep.acc, V.partR2, &st->cnt[CNT_R2], s_red, &s_flag, tot)) return;
  double p[NV_R1];
  sum_partials<NV_R1>(V.partR1, V.gridR1, s_red, p);
  double inf[NV_I];
  const bool infeas = check && st->eps_infeas > 0.0;
  if (infeas) sum_partials<NV_I>(V.partI, V.gridI, s_red, inf);
  if (threadIdx.x == 0) check_decide(st, V.trace, p, tot, infeas ? inf : nullptr);
}

// ---------------------------------------------------------------- infeasibility detection

// Pieces of the two certificates (NV_I1 each, layout of NV_I1) for the rays
// z - z_prev (difference of the last two accepted iterates; only when this
// check's K'y pass stored K'y_prev) and z - z^{n,0} (the normalised iterate
// times t: the tests are invariant to positive scaling), unscaled to the
// original LP: xr = D2 dx^, yr = D1 dy^, K xr = (K~ dx^) / D1 and
// K'yr = (K~' dy^) / D2 from the stored products, c'xr = c~'dx^ and
// q'yr = q~'dy^.  Since D2 > 0, lambda = proj_Lambda(-K'yr) = p / D2 with
// p = proj_Lambda(-K~' dy^), so l'lambda+ - u'lambda- = sum of l~ p (p > 0)
// and u~ p (p < 0) in scaled terms.  Sign and finiteness tests read the IEEE
// bits (integer pipe); GB300's FP64 pipe does only the arithmetic.  Runs
// between k_check_primal (which refreshed g = K'y) and k_check_dual, whose
// last CTA sums the block partials and decides.
__global__ void __launch_bounds__(NT) k_infeas(Vecs V, DevState *__restrict__ st) {
  __shared__ double s_red[16 * NW];
  if (st->status != ST_RUNNING || !st->check_pending || st->mode != MODE_CHECK || !(st->eps_infeas > 0.0)) return;
  const int cur = st->cur, prv = cur ^ 1;
  const int r0 = st->need_g ? 0 : 1;  // the difference ray needs this check's stored K'y_prev
  double a[NV_I];
#pragma unroll
  for (int k = 0; k < NV_I; ++k) a[k] = 0.0;
  const int stride = gridDim.x * NT;
  for (int j = blockIdx.x * NT + threadIdx.x; j < V.n; j += stride) {
    const double d2 = V.D2[j], rd2 = V.rD2[j], lt = V.l[j], ut = V.u[j], cj = V.c[j], gj = V.g[j];
    const double xj = V.x[cur][j];
    const bool lf = finite_bits(lt), uf = finite_bits(ut);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (r < r0) continue;
      double *b = a + r * NV_I1;
      const double mg = (r == 0 ? V.gprev[j] : V.g0[j]) - gj;  // -(K~' dy^)_j
      double p = mg;                                             // proj onto the cone of the bounds
      if (!lf && !uf) p = 0.0;
      else if (!uf && neg_bits(p)) p = 0.0;
      else if (!lf && pos_bits(p)) p = 0.0;
      const double res = (mg - p) * rd2;
      b[0] = fma(res, res, b[0]);
      if (pos_bits(p)) b[1] = fma(lt, p, b[1]);
      else if (neg_bits(p)) b[1] = fma(ut, p, b[1]);
      const double dx = xj - (r == 0 ? V.x[prv][j] : V.xlast[j]);
      b[2] = fma(cj, dx, b[2]);
      if ((lf && neg_bits(dx)) || (uf && pos_bits(dx))) {
        const double xo = d2 * dx;
        b[3] = fma(xo, xo, b[3]);
      }
    }
  }
  for (int i = blockIdx.x * NT + threadIdx.x; i < V.m; i += stride) {
    const double d1 = V.D1[i], rd1 = V.rD1[i], qi = V.q[i], yi = V.y[cur][i], kxi = V.Kx[cur][i];
    const bool ineq = i >= V.n_eq;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (r < r0) continue;
      double *b = a + r * NV_I1;
      double kr = (kxi - (r == 0 ? V.Kx[prv][i] : V.kx0[i])) * rd1;
      if (ineq && pos_bits(kr)) kr = 0.0;
      b[4] = fma(kr, kr, b[4]);
      const double dy = yi - (r == 0 ? V.y[prv][i] : V.ylast[i]);
      b[5] = fma(qi, dy, b[5]);
      if (ineq && neg_bits(dy)) {
        const double yo = d1 * dy;
        b[6] = fma(yo, yo, b[6]);
      }
    }
  }
  block_sum<NV_I>(a, s_red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV_I; ++k) V.partI[(size_t)blockIdx.x * NV_I + k] = a[k];
  }
}

// ---------------------------------------------------------------- restart

__global__ void __launch_bounds__(NT) k_restart(Vecs V, DevState *__restrict__ st) {
  __shared__ double s_red[16 * NW];
  __shared__ int s_flag;
  if (st->status != ST_RUNNING || !st->check_pending || st->restart_to == 0) return;
  const bool avg = st->restart_to == 2;
  const bool keep = st->eps_infeas > 0.0;
  const int cur = st->cur;
  const double invW = 1.0 / st->W;
  double acc[2] = {0.0, 0.0};
  const int stride = gridDim.x * NT;
  double *__restrict__ x = V.x[cur];
  double *__restrict__ sx = V.sx[cur];
  for (int j = blockIdx.x * NT + threadIdx.x; j < V.n; j += stride) {
    double xn;
    if (avg) {
      xn = invW * sx[j];
      x[j] = xn;
      V.g[j] = V.gbar[j];
    } else {
      xn = x[j];
    }
    if (keep) V.g0[j] = V.g[j];  // K'y at the new epoch start
    const double d = xn - V.xlast[j];
    acc[0] = fma(d, d, acc[0]);
    V.xlast[j] = xn;
    sx[j] = 0.0;
  }
  double *__restrict__ y = V.y[cur];
  double *__restrict__ sy = V.sy[cur];
  double *__restrict__ kx = V.Kx[cur];
  for (int i = blockIdx.x * NT + threadIdx.x; i < V.m; i += stride) {
    double yn;
    if (avg) {
      yn = invW * sy[i];
      y[i] = yn;
      kx[i] = V.Kxbar[i];
    } else {
      yn = y[i];
    }
    if (keep) V.kx0[i] = kx[i];  // K x at the new epoch start
    const double d = yn - V.ylast[i];
    acc[1] = fma(d, d, acc[1]);
    V.ylast[i] = yn;
    sy[i] = 0.0;
  }
  double tot[2];
  if (!grid_finish<2>(acc, V.partR3, &st->cnt[CNT_R3], s_red, &s_flag, tot)) return;
  if (threadIdx.x == 0) {
    // Sec. 2.2 PrimalWeightUpdate, read in log space
    const double dx = sqrt(tot[0]), dy = sqrt(tot[1]);
    double omega = st->omega;
    if (dx > st->eps_zero && dy > st->eps_zero)
      omega = exp(st->theta * log(dy / dx) + (1.0 - st->theta) * log(omega));
    st->omega = omega;
    st->W = 0.0;
    st->t = 0;
    st->restarts += 1;
    const double k0 = kkt_omega(st->cand[0], st->cand[1], st->cand[2], st->cand[3], omega);
    st->kkt_start = k0;
    st->kkt_prev = k0;
    st->restart_to = 0;
    st->check_pending = 0;
    if (st->ntrace > 0 && V.trace[(st->ntrace - 1) % st->trace_cap].k == st->k) {
      V.trace[(st->ntrace - 1) % st->trace_cap].omega = omega;
      V.trace[(st->ntrace - 1) % st->trace_cap].kkt_start = k0;
    }
  }
}

// ---------------------------------------------------------------- output

// Original-space output, written in the original order of rows and
// columns: the current iterate or the average (projected onto X), or, for an
// infeasibility status, the certificate ray in place of the
// iterate it concerns (y for primal infeasibility, x for dual
// infeasibility; unprojected).
__global__ void __launch_bounds__(NT) k_output(Vecs V, DevState *__restrict__ st) {
  const int which = st->which, cur = st->cur, prv = cur ^ 1, status = st->status;
  const bool avg = which == 1;
  const bool xray = status == ST_DUAL_INFEASIBLE, yray = status == ST_PRIMAL_INFEASIBLE;
  const double invW = avg ? 1.0 / st->W : 0.0;
  const int stride = gridDim.x * NT;
  for (int j = blockIdx.x * NT + threadIdx.x; j < V.n; j += stride) {
    if (xray) {
      V.xout[V.perm_c[j]] = V.D2[j] * (V.x[cur][j] - (which == 2 ? V.x[prv][j] : V.xlast[j]));
      continue;
    }
    const double xs = avg ? invW * V.sx[cur][j] : V.x[cur][j];
    double v = V.D2[j] * xs;
    if (v < V.l0[j]) v = V.l0[j];
    if (v > V.u0[j]) v = V.u0[j];
    V.xout[V.perm_c[j]] = v;
  }
  for (int i = blockIdx.x * NT + threadIdx.x; i < V.m; i += stride) {
    if (yray) {
      V.yout[V.perm_r[i]] = V.D1[i] * (V.y[cur][i] - (which == 2 ? V.y[prv][i] : V.ylast[i]));
      continue;
    }
    const double ys = avg ? invW * V.sy[cur][i] : V.y[cur][i];
    V.yout[V.perm_r[i]] = V.D1[i] * ys;
  }
}

__global__ void k_time_limit(DevState *st) {
  if (st->status == ST_RUNNING) st->status = ST_TIME_LIMIT;
}

// ---------------------------------------------------------------- launchers

const char *kernel_class_name(int kc) {
  static const char *names[KC_NUM] = {"k_primal", "k_dual", "k_check_primal", "k_check_dual", "k_restart",
                                      "k_output", "k_primal_reuse_g", "k_infeas"};
  return (kc >= 0 && kc < KC_NUM) ? names[kc] : "";
}

int occupancy_grid(int kc, int num_sms) {
  int nb = 1;
  switch (kc) {
    case KC_PRIMAL: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_primal, NT, 0); break;
    case KC_DUAL: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_dual, NT, 0); break;
    case KC_R1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_check_primal, NT, 0); break;
    case KC_R2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_check_dual, NT, 0); break;
    case KC_R3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_restart, NT, 0); break;
    case KC_INFEAS: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_infeas, NT, 0); break;
    default: nb = 4;
  }
  if (nb < 1) nb = 1;
  return nb * num_sms;
}

// Preferred shared-memory carveout of the step kernels, in percent of the
// largest configuration: 8 % is the smallest that holds four CTAs' static
// shared memory, so the L1 keeps the rest.  Every in-flight gather of x or y
// holds an L1 line until it returns, so the L1's size bounds the gathers in
// flight (measured on the 1e6 x 2e6 LP: 8 % 83.5 / 117.9 us per k_primal /
// k_dual launch, the driver's default 86.2 / 119.0, 28 % 92.1 / 120.4,
// 58 % 112.5 / 132.9).
#ifndef PDLP_STEP_CARVEOUT
#define PDLP_STEP_CARVEOUT 8
#endif
cudaError_t kernels_init() {
  if (PDLP_STEP_CARVEOUT < 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_primal, cudaFuncAttributePreferredSharedMemoryCarveout, PDLP_STEP_CARVEOUT);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_primal_qp, cudaFuncAttributePreferredSharedMemoryCarveout, PDLP_STEP_CARVEOUT);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dual, cudaFuncAttributePreferredSharedMemoryCarveout, PDLP_STEP_CARVEOUT);
  return e;
}
cudaError_t launch_primal(const SellMat &KT, const Vecs &V, DevState *st, int grid, cudaStream_t s) {
  if (V.qd)
    k_primal_qp<<<grid, NT, 0, s>>>(KT, V, st);
  else
    k_primal<<<grid, NT, 0, s>>>(KT, V, st);
  return cudaGetLastError();
}
cudaError_t launch_dual(const SellMat &K, const Vecs &V, DevState *st, int grid, cudaStream_t s) {
  k_dual<<<grid, NT, 0, s>>>(K, V, st);
  return cudaGetLastError();
}
cudaError_t launch_check_primal(const SellMat &KT, const Vecs &V, DevState *st, int grid, cudaStream_t s) {
  k_check_primal<<<grid, NT, 0, s>>>(KT, V, st);
  return cudaGetLastError();
}
cudaError_t launch_check_dual(const SellMat &K, const Vecs &V, DevState *st, int grid, cudaStream_t s) {
  k_check_dual<<<grid, NT, 0, s>>>(K, V, st);
  return cudaGetLastError();
}
cudaError_t launch_restart(const Vecs &V, DevState *st, int grid, cudaStream_t s) {
  k_restart<<<grid, NT, 0, s>>>(V, st);
  return cudaGetLastError();
}
cudaError_t launch_infeas(const Vecs &V, DevState *st, int grid, cudaStream_t s) {
  k_infeas<<<grid, NT, 0, s>>>(V, st);
  return cudaGetLastError();
}
cudaError_t launch_output(const Vecs &V, DevState *st, cudaStream_t s) {
  const int n = V.n > V.m ? V.n : V.m;
  int grid = (n + NT - 1) / NT;
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  k_output<<<grid, NT, 0, s>>>(V, st);
  return cudaGetLastError();
}
cudaError_t launch_time_limit(DevState *st, cudaStream_t s) {
  k_time_limit<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

}  // namespace pdlp
