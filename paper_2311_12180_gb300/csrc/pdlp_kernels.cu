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
//   k_restart (elementwise):      moves the candidate into the iterate, resets
//             the epoch average, and (last CTA) PrimalWeightUpdate.
// Every kernel reads the device state at entry and returns at once when it
// has nothing to do, so a fixed CUDA graph of P + E trial slots followed by the
// check kernels advances the solve by exactly one check period.
//
// SpMV: a tile is a run of consecutive rows with <= TILE_NNZ nonzeros and
// <= TILE_ROWS rows (or one longer row).  The random 8-byte gathers of x / y
// are the binding resource on GB300 (each is a distinct cache line for the
// SM's L1TEX tag stage, ~0.9 lines per clock per SM), so the two hot kernels
// run a persistent per-CTA software pipeline of cp.async copies: while tile k
// is reduced, the gathers of tile k+1 and the index / value / row-pointer
// copies of tile k+2 are in flight, landing directly in shared memory.  The
// reduction keeps every lane busy (GB300 issues FP64 at ~1.6 DFMA per clock
// per SM and a warp-wide FP64 instruction costs the same however many lanes
// are active): thread t sums EPT consecutive entries with FMA, and rows that
// cross thread boundaries are completed from per-thread carries.  The
// epilogue runs one row per thread on operands prefetched into registers
// before the reduction.  Reductions are deterministic: fixed per-thread
// order, fixed shuffle trees, fixed block order in the last CTA.  No atomics
// touch floating point.

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

// ---------------------------------------------------------------- tile SpMV

// Balanced tile SpMV.  GB300 issues FP64 at ~1.6 DFMA per clock per SM, and
// a warp-wide FP64 instruction costs the same issue slots however many lanes
// are active, so the reduction must keep every lane busy:
//   phase A  coalesced streaming loads of the tile's indices and values, the
//            gathers, and staging of (value, entry) pairs in shared memory;
//   phase B  thread t sums the EPT consecutive entries [EPT t, EPT t + EPT)
//            with full-lane FMAs, writing rows that start and end in its range
//            directly, keeping the partial of the row it enters ("head") and
//            of the row it leaves open ("carry");
//   phase C  the thread holding a row's last entry adds the carries of the
//            threads the row crossed: serially for up to CHAIN_MAX of them,
//            otherwise with a warp-strided sum.
// The staging arrays are padded by one slot per EPT entries so phase B reads
// (stride EPT + 1 = 5 doubles across lanes) are free of bank conflicts.
constexpr int EPT = TILE_NNZ / NT;  // 4
static_assert(EPT >= 2 && (EPT & (EPT - 1)) == 0, "EPT must be a power of two");
constexpr int PADDED = TILE_NNZ + TILE_NNZ / EPT;
constexpr int CHAIN_MAX = 8;
__device__ __forceinline__ int pidx(int o) { return o + o / EPT; }

// With one gathered vector a[] holds values and b[] gathered entries (summed
// with FMA); with two vectors a[] and b[] hold the two products.
template <int NVS>
struct TileSmem {
  double a[PADDED];
  double b[PADDED];
  double rowsum[NVS][TILE_ROWS];
  double carry[NVS][NT];
  int off[TILE_ROWS + 1];
  double red[16 * NW];
  int flag;
};

__device__ __forceinline__ double ld_val(const double *p) { return __ldcs(p); }
__device__ __forceinline__ double ld_val(const float *p) { return (double)__ldcs(p); }

// Row sums of one tile against NV (1 or 2) gathered vectors: out[a] of thread
// t holds the sum for row r0 + t (t < r1 - r0).  With SCALED, vector a is
// multiplied by sc[a] entry by entry before use (the epoch average 1/W * sum).
template <typename VT, int NV, bool SCALED, int NVS>
__device__ __forceinline__ void tile_spmv(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                          const VT *__restrict__ val, const double *const (&xs)[NV],
                                          const double (&sc)[NV], int r0, int r1, TileSmem<NVS> &sm,
                                          double (&out)[NV]) {
  static_assert(NV == 1 || NV == 2, "one or two gathered vectors");
  static_assert(NV <= NVS, "tile shared memory too small");
  const int tid = threadIdx.x;
  const int e0 = ptr[r0], e1 = ptr[r1];
  const int nz = e1 - e0, nrows = r1 - r0;
#pragma unroll
  for (int a = 0; a < NV; ++a) out[a] = 0.0;
  if (nz > TILE_NNZ) {  // one row longer than a tile: the whole CTA strides over it
    double acc[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) acc[a] = 0.0;
    for (int e = e0 + tid; e < e1; e += NT) {
      const int col = __ldcs(idx + e);
      const double v = ld_val(val + e);
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        const double xv = __ldg(xs[a] + col);
        acc[a] = fma(v, SCALED ? sc[a] * xv : xv, acc[a]);
      }
    }
    block_sum<NV>(acc, sm.red);
    if (tid == 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) out[a] = acc[a];
    }
    return;
  }
  // ---- phase A ----
  int cols[EPT];
  double vals[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int o = tid + k * NT;
    cols[k] = o < nz ? __ldcs(idx + e0 + o) : 0;
    vals[k] = o < nz ? ld_val(val + e0 + o) : 0.0;
  }
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int o = tid + k * NT;
    if (o < nz) {
      const int p = pidx(o);
      const double x0 = __ldg(xs[0] + cols[k]);
      if (NV == 1) {
        sm.a[p] = vals[k];
        sm.b[p] = SCALED ? sc[0] * x0 : x0;
      } else {
        const double x1 = __ldg(xs[NV - 1] + cols[k]);
        sm.a[p] = vals[k] * (SCALED ? sc[0] * x0 : x0);
        sm.b[p] = vals[k] * (SCALED ? sc[NV - 1] * x1 : x1);
      }
    }
  }
  if (tid < nrows) {
    sm.off[tid] = ptr[r0 + tid] - e0;
#pragma unroll
    for (int a = 0; a < NV; ++a) sm.rowsum[a][tid] = 0.0;
  }
  if (tid == 0) sm.off[nrows] = nz;
  __syncthreads();
  // ---- phase B ----
  const int s0 = tid * EPT;
  double acc[NV], carry[NV], head[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) acc[a] = carry[a] = head[a] = 0.0;
  bool has_head = false;
  int head_row = 0;
  if (s0 < nz) {
    int lo = 0, hi = nrows;  // largest row with off[row] <= s0 (a nonempty row holding entry s0)
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (sm.off[mid] <= s0)
        lo = mid;
      else
        hi = mid;
    }
    int r = lo, rstart = sm.off[lo], rend = sm.off[lo + 1];
    const int s1 = min(s0 + EPT, nz);
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = s0 + i;
      if (e < s1) {
        const int p = pidx(e);
        if (NV == 1) {
          acc[0] = fma(sm.a[p], sm.b[p], acc[0]);
        } else {
          acc[0] += sm.a[p];
          acc[NV - 1] += sm.b[p];
        }
        if (e + 1 == rend) {
          if (rstart >= s0) {
#pragma unroll
            for (int a = 0; a < NV; ++a) sm.rowsum[a][r] = acc[a];
          } else {
            has_head = true;
            head_row = r;
#pragma unroll
            for (int a = 0; a < NV; ++a) head[a] = acc[a];
          }
#pragma unroll
          for (int a = 0; a < NV; ++a) acc[a] = 0.0;
          if (e + 1 < nz) {
            do {
              ++r;
            } while (sm.off[r + 1] == e + 1);
            rstart = e + 1;
            rend = sm.off[r + 1];
          }
        }
      }
    }
    if (rend > s1) {
#pragma unroll
      for (int a = 0; a < NV; ++a) carry[a] = acc[a];
    }
  }
#pragma unroll
  for (int a = 0; a < NV; ++a) sm.carry[a][tid] = carry[a];
  __syncthreads();
  // ---- phase C ----
  bool longchain = false;
  int ts = 0;
  if (has_head) {
    ts = sm.off[head_row] / EPT;  // thread holding the row's first entry
    if (tid - ts <= CHAIN_MAX) {
      double s[NV];
#pragma unroll
      for (int a = 0; a < NV; ++a) s[a] = head[a];
      for (int t2 = tid - 1; t2 >= ts; --t2) {
#pragma unroll
        for (int a = 0; a < NV; ++a) s[a] += sm.carry[a][t2];
      }
#pragma unroll
      for (int a = 0; a < NV; ++a) sm.rowsum[a][head_row] = s[a];
    } else {
      longchain = true;
    }
  }
  const int lane = tid & 31;
  unsigned int msk = __ballot_sync(0xffffffffu, longchain);
  while (msk) {
    const int src = __ffs(msk) - 1;
    msk &= msk - 1;
    const int row = __shfl_sync(0xffffffffu, head_row, src);
    const int t0 = __shfl_sync(0xffffffffu, ts, src);
    const int tend = (tid & ~31) + src;
    double s[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) s[a] = 0.0;
    for (int t2 = t0 + lane; t2 < tend; t2 += 32) {
#pragma unroll
      for (int a = 0; a < NV; ++a) s[a] += sm.carry[a][t2];
    }
#pragma unroll
    for (int a = 0; a < NV; ++a) s[a] = warp_sum(s[a]);
    if (lane == src) {
#pragma unroll
      for (int a = 0; a < NV; ++a) sm.rowsum[a][row] = s[a] + head[a];
    }
  }
  __syncthreads();
  if (tid < nrows) {
#pragma unroll
    for (int a = 0; a < NV; ++a) out[a] = sm.rowsum[a][tid];
  }
  __syncthreads();
}

// ---------------------------------------------------------------- primal step

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

// ---------------------------------------------------------------- pipelined tile SpMV (hot kernels)

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_val(double *dst, const double *src) { cp8(dst, src); }
__device__ __forceinline__ void cp_val(float *dst, const float *src) { cp4(dst, src); }
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Three copy stages (tile k being reduced, k+1 being gathered, k+2 loading)
// and two gather buffers.  Values are stored in the padded layout of pidx()
// (as VT; a float stage uses the first half of its slot).
struct PipeSmem {
  int cols[3][TILE_NNZ];
  double vals[3][PADDED];
  int ptr[3][TILE_ROWS + 1];
  double xg[2][PADDED];
  double rowsum[TILE_ROWS];
  double carry[NT];
  double red[16 * NW];
  int flag;
};

__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return (double)v; }

template <typename VT>
__device__ __forceinline__ void stage_load(const Csr &A, const VT *__restrict__ val, int2 m0, int2 m1, int s,
                                           PipeSmem &sm) {
  const int nz = m1.y - m0.y, nrows = m1.x - m0.x;
  if (nz > TILE_NNZ) return;  // a long row is streamed directly by tile_long
  VT *sv = reinterpret_cast<VT *>(sm.vals[s]);
  for (int o = threadIdx.x; o < nz; o += NT) {
    cp4(&sm.cols[s][o], A.idx + m0.y + o);
    cp_val(sv + pidx(o), val + m0.y + o);
  }
  for (int r = threadIdx.x; r <= nrows; r += NT) cp4(&sm.ptr[s][r], A.ptr + m0.x + r);
}

__device__ __forceinline__ void gather_issue(const double *__restrict__ xg, int2 m0, int2 m1, int s, int bb,
                                             PipeSmem &sm) {
  const int nz = m1.y - m0.y;
  if (nz > TILE_NNZ) return;
  for (int o = threadIdx.x; o < nz; o += NT) cp8(&sm.xg[bb][pidx(o)], xg + sm.cols[s][o]);
}

// Reduce one staged tile (phases B and C of the balanced scheme) and run the
// epilogue for row r0 + threadIdx.x.
template <typename VT, class Epi>
__device__ __forceinline__ void tile_compute(int2 m0, int2 m1, int s, int bb, PipeSmem &sm, Epi &ep) {
  const int tid = threadIdx.x;
  const int r0 = m0.x, e0 = m0.y;
  const int nrows = m1.x - m0.x, nz = m1.y - m0.y;
  const bool has_row = tid < nrows;
  if (has_row) ep.prefetch(r0 + tid);
  const VT *__restrict__ sv = reinterpret_cast<const VT *>(sm.vals[s]);
  const double *__restrict__ sx = sm.xg[bb];
  const int *__restrict__ sp = sm.ptr[s];  // raw row pointers; local offset = sp[r] - e0
  const int s0 = tid * EPT;
  double acc = 0.0, carry = 0.0, head = 0.0;
  bool has_head = false;
  int head_row = 0;
  if (s0 < nz) {
    int lo = 0, hi = nrows;  // largest row with offset <= s0: the nonempty row holding entry s0
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (sp[mid] - e0 <= s0)
        lo = mid;
      else
        hi = mid;
    }
    int r = lo, rstart = sp[lo] - e0, rend = sp[lo + 1] - e0;
    const int s1 = min(s0 + EPT, nz);
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = s0 + i;
      if (e < s1) {
        const int p = pidx(e);
        acc = fma(to_f64(sv[p]), sx[p], acc);
        if (e + 1 == rend) {
          if (rstart >= s0) {
            sm.rowsum[r] = acc;
          } else {
            has_head = true;
            head_row = r;
            head = acc;
          }
          acc = 0.0;
          if (e + 1 < nz) {
            do {
              ++r;
            } while (sp[r + 1] - e0 == e + 1);
            rstart = e + 1;
            rend = sp[r + 1] - e0;
          }
        }
      }
    }
    if (rend > s1) carry = acc;
  }
  sm.carry[tid] = carry;
  __syncthreads();
  bool longchain = false;
  int ts = 0;
  if (has_head) {
    ts = (sp[head_row] - e0) / EPT;  // thread holding the row's first entry
    if (tid - ts <= CHAIN_MAX) {
      double sum = head;
      for (int t2 = tid - 1; t2 >= ts; --t2) sum += sm.carry[t2];
      sm.rowsum[head_row] = sum;
    } else {
      longchain = true;
    }
  }
  const int lane = tid & 31;
  unsigned int msk = __ballot_sync(0xffffffffu, longchain);
  while (msk) {
    const int src = __ffs(msk) - 1;
    msk &= msk - 1;
    const int row = __shfl_sync(0xffffffffu, head_row, src);
    const int t0 = __shfl_sync(0xffffffffu, ts, src);
    const int tend = (tid & ~31) + src;
    double sum = 0.0;
    for (int t2 = t0 + lane; t2 < tend; t2 += 32) sum += sm.carry[t2];
    sum = warp_sum(sum);
    if (lane == src) sm.rowsum[row] = sum + head;
  }
  __syncthreads();
  if (has_row) ep.finish(r0 + tid, sp[tid] == sp[tid + 1] ? 0.0 : sm.rowsum[tid]);
}

// A single row longer than a tile: the whole CTA streams it directly.
template <typename VT, class Epi>
__device__ __forceinline__ void tile_long(const Csr &A, const VT *__restrict__ val, const double *__restrict__ xg,
                                          int2 m0, int2 m1, PipeSmem &sm, Epi &ep) {
  if (threadIdx.x == 0) ep.prefetch(m0.x);
  double acc[1] = {0.0};
  for (int e = m0.y + threadIdx.x; e < m1.y; e += NT) acc[0] = fma(ld_val(val + e), __ldg(xg + __ldcs(A.idx + e)), acc[0]);
  block_sum<1>(acc, sm.red);
  if (threadIdx.x == 0) ep.finish(m0.x, acc[0]);
}

// Persistent loop over tiles blockIdx.x + k * gridDim.x with the copy
// pipeline described at the top of the file.
template <typename VT, class Epi>
__device__ __forceinline__ void spmv_pipeline(const Csr &A, const VT *__restrict__ val, const double *__restrict__ xg,
                                              PipeSmem &sm, Epi &ep) {
  const int G = gridDim.x, T = A.ntiles;
  int t = blockIdx.x;
  if (t >= T) return;
  int2 a0 = A.tmeta[t], a1 = A.tmeta[t + 1];  // tile k
  int2 b0 = make_int2(0, 0), b1 = b0;         // tile k+1
  if (t + G < T) {
    b0 = A.tmeta[t + G];
    b1 = A.tmeta[t + G + 1];
  }
  stage_load<VT>(A, val, a0, a1, 0, sm);
  cp_commit();
  if (t + G < T) stage_load<VT>(A, val, b0, b1, 1, sm);
  cp_commit();
  cp_wait_all_but_one();
  __syncthreads();
  gather_issue(xg, a0, a1, 0, 0, sm);
  cp_commit();
  for (int k = 0; t < T; ++k, t += G) {
    int2 c0 = make_int2(0, 0), c1 = c0;  // tile k+2
    const bool has1 = t + G < T, has2 = t + 2 * G < T;
    if (has2) {
      c0 = A.tmeta[t + 2 * G];
      c1 = A.tmeta[t + 2 * G + 1];
    }
    cp_wait_all();
    __syncthreads();  // stage of tile k+1 and the gathers of tile k have landed
    if (has1) gather_issue(xg, b0, b1, (k + 1) % 3, (k + 1) & 1, sm);
    cp_commit();
    if (has2) stage_load<VT>(A, val, c0, c1, (k + 2) % 3, sm);
    cp_commit();
    if (a1.y - a0.y > TILE_NNZ)
      tile_long<VT>(A, val, xg, a0, a1, sm, ep);
    else
      tile_compute<VT>(a0, a1, k % 3, k & 1, sm, ep);
    a0 = b0;
    a1 = b1;
    b0 = c0;
    b1 = c1;
  }
  cp_wait_all();
  __syncthreads();
}

// ---------------------------------------------------------------- primal step

struct PrimalEpi {
  const double *__restrict__ c, *__restrict__ l, *__restrict__ u, *__restrict__ x, *__restrict__ sx;
  double *__restrict__ g, *__restrict__ xn, *__restrict__ sxn;
  double tau, eta, dx2;
  double pc, pl, pu, px, psx;
  __device__ __forceinline__ void prefetch(int j) {
    pc = c[j];
    pl = l[j];
    pu = u[j];
    px = x[j];
    psx = sx[j];
  }
  __device__ __forceinline__ void finish(int j, double gj) {
    g[j] = gj;
    const double v = clamp_bits(fma(-tau, pc - gj, px), pl, pu);
    xn[j] = v;
    sxn[j] = fma(eta, v, psx);
    const double d = v - px;
    dx2 = fma(d, d, dx2);
  }
};

extern __shared__ __align__(16) unsigned char g_dsmem[];

__global__ void __launch_bounds__(NT) k_primal(Csr KT, Vecs V, DevState *__restrict__ st) {
  PipeSmem &sm = *reinterpret_cast<PipeSmem *>(g_dsmem);
  if (st->status != ST_RUNNING || st->check_pending) return;
  const int cur = st->cur, nxt = cur ^ 1, need_g = st->need_g, f32 = st->use_f32;
  const double eta = st->eta, omega = st->omega;
  PrimalEpi ep;
  ep.c = V.c;
  ep.l = V.l;
  ep.u = V.u;
  ep.x = V.x[cur];
  ep.sx = V.sx[cur];
  ep.g = V.g;
  ep.xn = V.x[nxt];
  ep.sxn = V.sx[nxt];
  ep.tau = eta / omega;
  ep.eta = eta;
  ep.dx2 = 0.0;
  if (need_g) {
    if (f32)
      spmv_pipeline<float>(KT, KT.val32, V.y[cur], sm, ep);
    else
      spmv_pipeline<double>(KT, KT.val, V.y[cur], sm, ep);
  } else {
    // rejected trial: g = K'y is unchanged, only the projection reruns
    for (int j = blockIdx.x * NT + threadIdx.x; j < V.n; j += gridDim.x * NT) {
      ep.prefetch(j);
      ep.finish(j, V.g[j]);
    }
  }
  double acc[1] = {ep.dx2};
  block_sum<1>(acc, sm.red);
  if (threadIdx.x == 0) V.partA[blockIdx.x] = acc[0];
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
  __device__ __forceinline__ void finish(int i, double kn) {
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
__device__ void step_test(DevState *st, double dx2, double dy2, double cross) {
  const double eta = st->eta, omega = st->omega;
  const long long k = st->k;
  const double ia = fabs(cross);
  const double eta_bar = ia > 0.0 ? (omega * dx2 + dy2 / omega) / (2.0 * ia) : CUDART_INF;
  const double kk = (double)(k + 2);
  const double e1 = (1.0 - pow(kk, -0.3)) * eta_bar;
  const double e2 = (1.0 + pow(kk, -0.6)) * eta;
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

__global__ void __launch_bounds__(NT) k_dual(Csr K, Vecs V, DevState *__restrict__ st) {
  PipeSmem &sm = *reinterpret_cast<PipeSmem *>(g_dsmem);
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
  if (f32)
    spmv_pipeline<float>(K, K.val32, V.x[nxt], sm, ep);
  else
    spmv_pipeline<double>(K, K.val, V.x[nxt], sm, ep);
  double acc[2] = {ep.dy2, ep.cross};
  double tot[2];
  if (!grid_finish<2>(acc, V.partB, &st->cnt[CNT_DUAL], sm.red, &sm.flag, tot)) return;
  double dx[1];
  sum_partials<1>(V.partA, V.gridA, sm.red, dx);
  if (threadIdx.x == 0) step_test(st, dx[0], tot[0], tot[1]);
}

// ---------------------------------------------------------------- restart / termination check

__device__ __forceinline__ double proj_lambda(double d, double l, double u) {
  const bool lf = isfinite(l), uf = isfinite(u);
  if (lf && uf) return d;
  if (lf) return d > 0.0 ? d : 0.0;
  if (uf) return d < 0.0 ? d : 0.0;
  return 0.0;
}

// Dual-side pieces of eq. (kkt) / Sec. 4.1 for one variable.
__device__ __forceinline__ void dual_piece(double c, double g, double l, double u, double d2, double x,
                                           double *acc) {
  const double d = c - g;
  const double lam = proj_lambda(d, l, u);
  const double r = d - lam;
  acc[0] = fma(r, r, acc[0]);
  const double ro = r / d2;
  acc[1] = fma(ro, ro, acc[1]);
  acc[2] = fma(c, x, acc[2]);
  if (lam > 0.0) acc[3] = fma(l, lam, acc[3]);
  if (lam < 0.0) acc[3] = acc[3] - u * (-lam);
}

__global__ void __launch_bounds__(NT) k_check_primal(Csr KT, Vecs V, DevState *__restrict__ st) {
  __shared__ TileSmem<2> sm;
  if (st->status != ST_RUNNING || !st->check_pending) return;
  const int mode = st->mode, cur = st->cur, need_g = st->need_g;
  const bool check = mode == MODE_CHECK;
  const double invW = check ? 1.0 / st->W : 0.0;
  const double *__restrict__ x = V.x[cur];
  const double *__restrict__ sx = V.sx[cur];
  double acc[NV_R1];
#pragma unroll
  for (int a = 0; a < NV_R1; ++a) acc[a] = 0.0;
  for (int t = blockIdx.x; t < KT.ntiles; t += gridDim.x) {
    const int r0 = KT.tmeta[t].x, r1 = KT.tmeta[t + 1].x;
    double g = 0.0, gb = 0.0;
    double s2[2];
    double s1[1];
    if (!check) {
      const double *const xs[1] = {V.y[cur]};
      const double sc[1] = {1.0};
      tile_spmv<double, 1, false>(KT.ptr, KT.idx, KT.val, xs, sc, r0, r1, sm, s1);
      g = s1[0];
    } else if (need_g) {
      const double *const xs[2] = {V.y[cur], V.sy[cur]};
      const double sc[2] = {1.0, invW};
      tile_spmv<double, 2, true>(KT.ptr, KT.idx, KT.val, xs, sc, r0, r1, sm, s2);
      g = s2[0];
      gb = s2[1];
    } else {
      const double *const xs[1] = {V.sy[cur]};
      const double sc[1] = {invW};
      tile_spmv<double, 1, true>(KT.ptr, KT.idx, KT.val, xs, sc, r0, r1, sm, s1);
      gb = s1[0];
    }
    if ((int)threadIdx.x < r1 - r0) {
      const int j = r0 + threadIdx.x;
      if (!check || need_g)
        V.g[j] = g;
      else
        g = V.g[j];
      const double c = V.c[j], l = V.l[j], u = V.u[j], d2 = V.D2[j];
      dual_piece(c, g, l, u, d2, x[j], acc);
      if (check) {
        V.gbar[j] = gb;
        dual_piece(c, gb, l, u, d2, invW * sx[j], acc + 4);
      }
    }
  }
  block_sum<NV_R1>(acc, sm.red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV_R1; ++a) V.partR1[(size_t)blockIdx.x * NV_R1 + a] = acc[a];
  }
}

__device__ __forceinline__ void primal_piece(double q, double kx, bool ineq, double d1, double y, double *acc) {
  double r = q - kx;
  if (ineq && r < 0.0) r = 0.0;
  acc[0] = fma(r, r, acc[0]);
  const double ro = r / d1;
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
__device__ void check_decide(DevState *st, TraceRec *trace, const double *p, const double *d) {
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
  if (st->ntrace < st->trace_cap) {
    TraceRec &r = trace[st->ntrace];
    r.k = st->k;
    r.restart = mask;
    r.cand_avg = cand_avg;
    r.kkt_cur = kc;
    r.kkt_avg = ka;
    r.kkt_start = st->kkt_start;
    r.omega = omega;
    r.eta_hat = st->eta;
    st->ntrace += 1;
  }
}

__global__ void __launch_bounds__(NT) k_check_dual(Csr K, Vecs V, DevState *__restrict__ st) {
  __shared__ TileSmem<1> sm;
  if (st->status != ST_RUNNING || !st->check_pending) return;
  const int mode = st->mode, cur = st->cur;
  const bool check = mode == MODE_CHECK;
  const double invW = check ? 1.0 / st->W : 0.0;
  const double *__restrict__ y = V.y[cur];
  const double *__restrict__ sy = V.sy[cur];
  double acc[NV_R2];
#pragma unroll
  for (int a = 0; a < NV_R2; ++a) acc[a] = 0.0;
  for (int t = blockIdx.x; t < K.ntiles; t += gridDim.x) {
    const int r0 = K.tmeta[t].x, r1 = K.tmeta[t + 1].x;
    double s1[1];
    if (!check) {
      const double *const xs[1] = {V.x[cur]};
      const double sc[1] = {1.0};
      tile_spmv<double, 1, false>(K.ptr, K.idx, K.val, xs, sc, r0, r1, sm, s1);
    } else {
      const double *const xs[1] = {V.sx[cur]};
      const double sc[1] = {invW};
      tile_spmv<double, 1, true>(K.ptr, K.idx, K.val, xs, sc, r0, r1, sm, s1);
    }
    if ((int)threadIdx.x < r1 - r0) {
      const int i = r0 + threadIdx.x;
      const bool ineq = i >= V.n_eq;
      const double q = V.q[i], d1 = V.D1[i];
      double kx;
      if (!check) {
        kx = s1[0];
        V.Kx[cur][i] = kx;
      } else {
        kx = V.Kx[cur][i];
      }
      primal_piece(q, kx, ineq, d1, y[i], acc);
      if (check) {
        V.Kxbar[i] = s1[0];
        primal_piece(q, s1[0], ineq, d1, invW * sy[i], acc + 3);
      }
    }
  }
  double tot[NV_R2];
  if (!grid_finish<NV_R2>(acc, V.partR2, &st->cnt[CNT_R2], sm.red, &sm.flag, tot)) return;
  double p[NV_R1];
  sum_partials<NV_R1>(V.partR1, V.gridR1, sm.red, p);
  if (threadIdx.x == 0) check_decide(st, V.trace, p, tot);
}

// ---------------------------------------------------------------- restart

__global__ void __launch_bounds__(NT) k_restart(Vecs V, DevState *__restrict__ st) {
  __shared__ double s_red[16 * NW];
  __shared__ int s_flag;
  if (st->status != ST_RUNNING || !st->check_pending || st->restart_to == 0) return;
  const bool avg = st->restart_to == 2;
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
    if (st->ntrace > 0 && V.trace[st->ntrace - 1].k == st->k) {
      V.trace[st->ntrace - 1].omega = omega;
      V.trace[st->ntrace - 1].kkt_start = k0;
    }
  }
}

// ---------------------------------------------------------------- output

__global__ void __launch_bounds__(NT) k_output(Vecs V, DevState *__restrict__ st) {
  const int which = st->which, cur = st->cur;
  const double invW = which ? 1.0 / st->W : 0.0;
  const int stride = gridDim.x * NT;
  for (int j = blockIdx.x * NT + threadIdx.x; j < V.n; j += stride) {
    const double xs = which ? invW * V.sx[cur][j] : V.x[cur][j];
    double v = V.D2[j] * xs;
    if (v < V.l0[j]) v = V.l0[j];
    if (v > V.u0[j]) v = V.u0[j];
    V.xout[j] = v;
  }
  for (int i = blockIdx.x * NT + threadIdx.x; i < V.m; i += stride) {
    const double ys = which ? invW * V.sy[cur][i] : V.y[cur][i];
    V.yout[i] = V.D1[i] * ys;
  }
}

__global__ void k_time_limit(DevState *st) {
  if (st->status == ST_RUNNING) st->status = ST_TIME_LIMIT;
}

// ---------------------------------------------------------------- launchers

const char *kernel_class_name(int kc) {
  static const char *names[KC_NUM] = {"k_primal", "k_dual", "k_check_primal", "k_check_dual", "k_restart",
                                      "k_output", "k_primal_reuse_g"};
  return (kc >= 0 && kc < KC_NUM) ? names[kc] : "";
}

int occupancy_grid(int kc, int num_sms) {
  int nb = 1;
  switch (kc) {
    case KC_PRIMAL: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_primal, NT, sizeof(PipeSmem)); break;
    case KC_DUAL: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_dual, NT, sizeof(PipeSmem)); break;
    case KC_R1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_check_primal, NT, 0); break;
    case KC_R2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_check_dual, NT, 0); break;
    case KC_R3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_restart, NT, 0); break;
    default: nb = 4;
  }
  if (nb < 1) nb = 1;
  return nb * num_sms;
}

cudaError_t kernels_init() {
  cudaError_t e = cudaFuncSetAttribute(k_primal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PipeSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PipeSmem));
  return e;
}
cudaError_t launch_primal(const Csr &KT, const Vecs &V, DevState *st, int grid, cudaStream_t s) {
  k_primal<<<grid, NT, sizeof(PipeSmem), s>>>(KT, V, st);
  return cudaGetLastError();
}
cudaError_t launch_dual(const Csr &K, const Vecs &V, DevState *st, int grid, cudaStream_t s) {
  k_dual<<<grid, NT, sizeof(PipeSmem), s>>>(K, V, st);
  return cudaGetLastError();
}
cudaError_t launch_check_primal(const Csr &KT, const Vecs &V, DevState *st, int grid, cudaStream_t s) {
  k_check_primal<<<grid, NT, 0, s>>>(KT, V, st);
  return cudaGetLastError();
}
cudaError_t launch_check_dual(const Csr &K, const Vecs &V, DevState *st, int grid, cudaStream_t s) {
  k_check_dual<<<grid, NT, 0, s>>>(K, V, st);
  return cudaGetLastError();
}
cudaError_t launch_restart(const Vecs &V, DevState *st, int grid, cudaStream_t s) {
  k_restart<<<grid, NT, 0, s>>>(V, st);
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
