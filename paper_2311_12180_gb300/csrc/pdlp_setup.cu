// Setup-time kernels: Sec. 2.2 diagonal preconditioning on the GPU (Ruiz
// l_inf passes, then one Pock-Chambolle pass), scaling of c, q, l, u, the
// FP32 value copy, the scalar reductions behind Algorithm 1's initial step
// size and InitializePrimalWeight, and the scaled warm-start point.
//
// K and K' are scaled in place with the same two divisions in the same order
// for every entry, (v / r_i) / s_j with r the row factor of K and s its column
// factor, so the two copies stay exact transposes of each other.

#include <math.h>

#include <mutex>
#include <string>

#include "pdlp.h"
#include "pdlp_internal.cuh"
#include "pdlp_setup.cuh"

namespace pdlp {

namespace {

constexpr int ST = 256;

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_add(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per row: out[r] = max_e |val[e]| (kind 0) or sum_e |val[e]|^p (kind 1).
__global__ void k_row_norm(const int32_t *__restrict__ ptr, const double *__restrict__ val, int32_t rows,
                           double *__restrict__ out, int kind, double p) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * ST + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * ST) >> 5;
  for (long long r = warp; r < rows; r += nwarps) {
    const int e0 = ptr[r], e1 = ptr[r + 1];
    double acc = 0.0;
    for (int e = e0 + lane; e < e1; e += 32) {
      const double a = fabs(val[e]);
      if (kind == 0)
        acc = fmax(acc, a);
      else
        acc += (p == 1.0) ? a : pow(a, p);
    }
    acc = kind == 0 ? warp_max(acc) : warp_add(acc);
    if (lane == 0) out[r] = acc;
  }
}

// f <- sqrt(f), or 1 where the line is empty (norm 0).
__global__ void k_factor(double *__restrict__ f, int32_t n) {
  for (int i = blockIdx.x * ST + threadIdx.x; i < n; i += gridDim.x * ST) f[i] = f[i] > 0.0 ? sqrt(f[i]) : 1.0;
}

// K (row_is_kmajor = 1): val[e] = (val[e] / r[i]) / s[idx[e]] for row i.
// K' (row_is_kmajor = 0): row j of K', idx = row of K: (val / r[idx]) / s[j].
__global__ void k_scale(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx, double *__restrict__ val,
                        int32_t rows, const double *__restrict__ r, const double *__restrict__ s,
                        int row_is_kmajor) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * ST + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * ST) >> 5;
  for (long long row = warp; row < rows; row += nwarps) {
    const int e0 = ptr[row], e1 = ptr[row + 1];
    for (int e = e0 + lane; e < e1; e += 32) {
      const int o = idx[e];
      if (row_is_kmajor)
        val[e] = val[e] / r[row] / s[o];
      else
        val[e] = val[e] / r[o] / s[row];
    }
  }
}

__global__ void k_div(double *__restrict__ D, const double *__restrict__ f, int32_t n) {
  for (int i = blockIdx.x * ST + threadIdx.x; i < n; i += gridDim.x * ST) D[i] = D[i] / f[i];
}

// Ruiz maxima in one pass over K's entries: the IEEE bits of |v| are
// ordered like the values, so an integer atomicMax per entry on the row's
// and the column's slot gives max |K~_ij| exactly (order-independent).
__global__ void k_entry_max(const int32_t *__restrict__ idx, const int32_t *__restrict__ rowid,
                            const double *__restrict__ val, int64_t nnz, unsigned long long *__restrict__ rmax,
                            unsigned long long *__restrict__ cmax) {
  for (int64_t e = (int64_t)blockIdx.x * ST + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * ST) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(val[e]) & 0x7fffffffffffffffull;
    atomicMax(rmax + rowid[e], bits);
    atomicMax(cmax + idx[e], bits);
  }
}

// rD[i] = 1 / D[i], correctly rounded (IEEE division).
__global__ void k_recip(int32_t count, const double *D, double *rD) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) rD[i] = 1.0 / D[i];
}

// RN(a / b) from y = RN(1 / b) by one correction step (Markstein, IBM J. Res.
// Dev. 34(1), 1990; Handbook of Floating-Point Arithmetic, the theorem on
// division by an FMA correction): q = RN(a y) is within one ulp of a / b,
// the remainder a - b q is exact with an FMA, and RN(q + (a - b q) y) is the
// correctly rounded quotient when nothing underflows or overflows.  Where a
// or q is outside [2^-900, 2^900] (or zero, or not finite) the plain
// division runs instead.  Three FP64 operations instead of a division
// routine: the Ruiz passes divide every entry twice, on GB300's narrow FP64
// pipe.
__device__ __forceinline__ unsigned int exp_bits(double v) {
  return (unsigned int)((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ffu;
}
__device__ __forceinline__ double div_rn(double a, double b, double y) {
  const double q = a * y;
  const unsigned int ea = exp_bits(a), eq = exp_bits(q);
  if (ea < 1023u - 900u || ea > 1023u + 900u || eq < 1023u - 900u || eq > 1023u + 900u) return a / b;
  const double r = fma(-b, q, a);
  return fma(r, y, q);
}

// K's entries in storage order: val[e] = (val[e] / r[row]) / s[column], the
// same two correctly rounded divisions in the same order as the row-wise
// k_scale (the reciprocals rr, rs of the factors make each one three FP64
// operations, div_rn).
__global__ void k_scale_entries(const int32_t *__restrict__ idx, const int32_t *__restrict__ rowid,
                                double *__restrict__ val, int64_t nnz, const double *__restrict__ r,
                                const double *__restrict__ s, const double *__restrict__ rr,
                                const double *__restrict__ rs) {
  for (int64_t e = (int64_t)blockIdx.x * ST + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * ST) {
    const int32_t i = rowid[e], j = idx[e];
    val[e] = div_rn(div_rn(val[e], r[i], rr[i]), s[j], rs[j]);
  }
}

// K' values as a copy of K's through the transpose permutation.
__global__ void k_copy_perm(const int32_t *__restrict__ perm, const double *__restrict__ kval, int64_t nnz,
                            double *__restrict__ tval) {
  for (int64_t p = (int64_t)blockIdx.x * ST + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * ST)
    tval[p] = kval[perm[p]];
}

__global__ void k_fill(double *__restrict__ a, int32_t n, double v) {
  for (int i = blockIdx.x * ST + threadIdx.x; i < n; i += gridDim.x * ST) a[i] = v;
}

__global__ void k_vectors(int32_t m, int32_t n, const double *__restrict__ c0, const double *__restrict__ q0,
                          const double *__restrict__ l0, const double *__restrict__ u0, const double *__restrict__ D1,
                          const double *__restrict__ D2, double *__restrict__ c, double *__restrict__ q,
                          double *__restrict__ l, double *__restrict__ u) {
  for (int j = blockIdx.x * ST + threadIdx.x; j < n; j += gridDim.x * ST) {
    c[j] = D2[j] * c0[j];
    l[j] = l0[j] / D2[j];
    u[j] = u0[j] / D2[j];
  }
  for (int i = blockIdx.x * ST + threadIdx.x; i < m; i += gridDim.x * ST) q[i] = D1[i] * q0[i];
}

// FP32 copy of the scaled values (round to nearest); a value below the
// smallest normal float is stored as a signed zero, so the step kernels'
// integer widening sees only normal floats and zeros.
__global__ void k_f32(long long nnz, const double *__restrict__ v, float *__restrict__ f) {
  for (long long e = (long long)blockIdx.x * ST + threadIdx.x; e < nnz; e += (long long)gridDim.x * ST) {
    const float x = (float)v[e];
    f[e] = (__float_as_uint(x) & 0x7f800000u) ? x : __uint_as_float(__float_as_uint(x) & 0x80000000u);
  }
}

// out = {sum c^2, sum q^2, max |val|} in two steps with a fixed order for a
// fixed grid: SCAL_BLOCKS block partials (grid-strided shares, block tree),
// then one block adds them in block order.  The maximum is taken on the
// IEEE bits of |val| (integer compares, exact, off the FP64 pipe).
constexpr int SCAL_BLOCKS = 256;

__device__ __forceinline__ unsigned long long warp_umax(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

__global__ void __launch_bounds__(ST) k_scalars_part(int32_t m, int32_t n, long long nnz,
                                                     const double *__restrict__ c, const double *__restrict__ q,
                                                     const double *__restrict__ val, double *__restrict__ part) {
  __shared__ double red[2][ST / 32];
  __shared__ unsigned long long rmx[ST / 32];
  double a = 0.0, b = 0.0;
  unsigned long long mx = 0;
  const long long t0 = (long long)blockIdx.x * ST + threadIdx.x, stride = (long long)gridDim.x * ST;
  for (long long j = t0; j < n; j += stride) a = fma(c[j], c[j], a);
  for (long long i = t0; i < m; i += stride) b = fma(q[i], q[i], b);
  for (long long e = t0; e < nnz; e += stride) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(val[e]) & 0x7fffffffffffffffull;
    mx = bits > mx ? bits : mx;
  }
  a = warp_add(a);
  b = warp_add(b);
  mx = warp_umax(mx);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
    rmx[wid] = mx;
  }
  __syncthreads();
  if (wid == 0) {
    a = warp_add(lane < ST / 32 ? red[0][lane] : 0.0);
    b = warp_add(lane < ST / 32 ? red[1][lane] : 0.0);
    mx = warp_umax(lane < ST / 32 ? rmx[lane] : 0ull);
    if (lane == 0) {
      part[3 * blockIdx.x] = a;
      part[3 * blockIdx.x + 1] = b;
      part[3 * blockIdx.x + 2] = __longlong_as_double((long long)mx);
    }
  }
}

__global__ void __launch_bounds__(32) k_scalars_final(const double *__restrict__ part, int blocks,
                                                      double *__restrict__ out) {
  const int lane = threadIdx.x;
  double a = 0.0, b = 0.0;
  unsigned long long mx = 0;
  for (int k = lane; k < blocks; k += 32) {
    a += part[3 * k];
    b += part[3 * k + 1];
    const unsigned long long bits = (unsigned long long)__double_as_longlong(part[3 * k + 2]);
    mx = bits > mx ? bits : mx;
  }
  a = warp_add(a);
  b = warp_add(b);
  mx = warp_umax(mx);
  if (lane == 0) {
    out[0] = a;
    out[1] = b;
    out[2] = __longlong_as_double((long long)mx);
  }
}

__global__ void k_warm(int32_t m, int32_t n, const double *__restrict__ x0, const double *__restrict__ y0,
                       const double *__restrict__ D1, const double *__restrict__ D2, double *__restrict__ x,
                       double *__restrict__ y) {
  for (int j = blockIdx.x * ST + threadIdx.x; j < n; j += gridDim.x * ST) x[j] = x0 ? x0[j] / D2[j] : 0.0;
  for (int i = blockIdx.x * ST + threadIdx.x; i < m; i += gridDim.x * ST) y[i] = y0 ? y0[i] / D1[i] : 0.0;
}

int grid_for(long long n) {
  long long g = (n + ST - 1) / ST;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t setup_scale(int32_t m, int32_t n, int64_t nnz, int32_t *K_ptr, int32_t *K_idx, double *K_val,
                        int32_t *T_ptr, int32_t *T_idx, double *T_val, double *D1, double *D2, double *work_m,
                        double *work_n, int ruiz_iters, double pc_alpha, cudaStream_t s) {
  (void)nnz;
  if (m > 0) k_fill<<<grid_for(m), ST, 0, s>>>(D1, m, 1.0);
  k_fill<<<grid_for(n), ST, 0, s>>>(D2, n, 1.0);
  const int passes = ruiz_iters + (pc_alpha >= 0.0 ? 1 : 0);
  for (int it = 0; it < passes; ++it) {
    const bool ruiz = it < ruiz_iters;
    const int kind = ruiz ? 0 : 1;
    // row factors of K (one warp per row of K), column factors (rows of K')
    if (m > 0) k_row_norm<<<grid_for((long long)m * 32), ST, 0, s>>>(K_ptr, K_val, m, work_m, kind, 2.0 - pc_alpha);
    k_row_norm<<<grid_for((long long)n * 32), ST, 0, s>>>(T_ptr, T_val, n, work_n, kind, pc_alpha);
    if (m > 0) k_factor<<<grid_for(m), ST, 0, s>>>(work_m, m);
    k_factor<<<grid_for(n), ST, 0, s>>>(work_n, n);
    if (m > 0) k_scale<<<grid_for((long long)m * 32), ST, 0, s>>>(K_ptr, K_idx, K_val, m, work_m, work_n, 1);
    k_scale<<<grid_for((long long)n * 32), ST, 0, s>>>(T_ptr, T_idx, T_val, n, work_m, work_n, 0);
    if (m > 0) k_div<<<grid_for(m), ST, 0, s>>>(D1, work_m, m);
    k_div<<<grid_for(n), ST, 0, s>>>(D2, work_n, n);
  }
  return cudaGetLastError();
}

cudaError_t setup_scale_perm(int32_t m, int32_t n, int64_t nnz, const int32_t *K_ptr, const int32_t *K_idx,
                             double *K_val, const int32_t *T_ptr, double *T_val, const int32_t *rowid,
                             const int32_t *perm, double *D1, double *D2, double *work_m, double *work_n,
                             double *rcp_m, double *rcp_n, int ruiz_iters, double pc_alpha, cudaStream_t s) {
  if (m > 0) k_fill<<<grid_for(m), ST, 0, s>>>(D1, m, 1.0);
  k_fill<<<grid_for(n), ST, 0, s>>>(D2, n, 1.0);
  const int eg = grid_for(nnz);
  for (int it = 0; it < ruiz_iters; ++it) {
    cudaError_t e = cudaMemsetAsync(work_m, 0, sizeof(double) * (size_t)m, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(work_n, 0, sizeof(double) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    if (nnz > 0)
      k_entry_max<<<eg, ST, 0, s>>>(K_idx, rowid, K_val, nnz, reinterpret_cast<unsigned long long *>(work_m),
                                    reinterpret_cast<unsigned long long *>(work_n));
    if (m > 0) k_factor<<<grid_for(m), ST, 0, s>>>(work_m, m);
    k_factor<<<grid_for(n), ST, 0, s>>>(work_n, n);
    if (m > 0) k_recip<<<grid_for(m), ST, 0, s>>>(m, work_m, rcp_m);
    k_recip<<<grid_for(n), ST, 0, s>>>(n, work_n, rcp_n);
    if (nnz > 0) k_scale_entries<<<eg, ST, 0, s>>>(K_idx, rowid, K_val, nnz, work_m, work_n, rcp_m, rcp_n);
    if (m > 0) k_div<<<grid_for(m), ST, 0, s>>>(D1, work_m, m);
    k_div<<<grid_for(n), ST, 0, s>>>(D2, work_n, n);
  }
  if (nnz > 0) k_copy_perm<<<eg, ST, 0, s>>>(perm, K_val, nnz, T_val);
  if (pc_alpha >= 0.0) {  // Pock-Chambolle: row sums over K, column sums over K' (fixed order)
    if (m > 0) k_row_norm<<<grid_for((long long)m * 32), ST, 0, s>>>(K_ptr, K_val, m, work_m, 1, 2.0 - pc_alpha);
    k_row_norm<<<grid_for((long long)n * 32), ST, 0, s>>>(T_ptr, T_val, n, work_n, 1, pc_alpha);
    if (m > 0) k_factor<<<grid_for(m), ST, 0, s>>>(work_m, m);
    k_factor<<<grid_for(n), ST, 0, s>>>(work_n, n);
    if (m > 0) k_recip<<<grid_for(m), ST, 0, s>>>(m, work_m, rcp_m);
    k_recip<<<grid_for(n), ST, 0, s>>>(n, work_n, rcp_n);
    if (nnz > 0) k_scale_entries<<<eg, ST, 0, s>>>(K_idx, rowid, K_val, nnz, work_m, work_n, rcp_m, rcp_n);
    if (m > 0) k_div<<<grid_for(m), ST, 0, s>>>(D1, work_m, m);
    k_div<<<grid_for(n), ST, 0, s>>>(D2, work_n, n);
    if (nnz > 0) k_copy_perm<<<eg, ST, 0, s>>>(perm, K_val, nnz, T_val);
  }
  return cudaGetLastError();
}

cudaError_t setup_vectors(int32_t m, int32_t n, const double *c0, const double *q0, const double *l0,
                          const double *u0, const double *D1, const double *D2, double *c, double *q, double *l,
                          double *u, cudaStream_t s) {
  k_vectors<<<grid_for(n > m ? n : m), ST, 0, s>>>(m, n, c0, q0, l0, u0, D1, D2, c, q, l, u);
  return cudaGetLastError();
}

cudaError_t setup_recip(int32_t count, const double *D, double *rD, cudaStream_t s) {
  if (count > 0) k_recip<<<grid_for(count), ST, 0, s>>>(count, D, rD);
  return cudaGetLastError();
}

cudaError_t setup_f32(int64_t nnz, const double *val, float *val32, cudaStream_t s) {
  if (nnz > 0) k_f32<<<grid_for(nnz), ST, 0, s>>>(nnz, val, val32);
  return cudaGetLastError();
}

size_t scalars_work_doubles() { return 3 * (size_t)SCAL_BLOCKS; }

cudaError_t setup_scalars(int32_t m, int32_t n, int64_t nnz, const double *c, const double *q, const double *val,
                          double *out, double *work, cudaStream_t s) {
  k_scalars_part<<<SCAL_BLOCKS, ST, 0, s>>>(m, n, nnz, c, q, val, work);
  k_scalars_final<<<1, 32, 0, s>>>(work, SCAL_BLOCKS, out);
  return cudaGetLastError();
}

cudaError_t setup_warm(int32_t m, int32_t n, const double *x0, const double *y0, const double *D1,
                       const double *D2, double *x, double *y, cudaStream_t s) {
  k_warm<<<grid_for(n > m ? n : m), ST, 0, s>>>(m, n, x0, y0, D1, D2, x, y);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- K' row starts on the device
//
// Column counts of K (atomic increments into T_ptr[1 + column]), then an
// inclusive scan of T_ptr[1..n] in place: T_ptr becomes the row starts of K'.
// The scan is per 1024-element block (warp shuffles, then the warp totals),
// an exclusive scan of the block totals, and a final add; the largest column
// count is kept for the choice between the device and the host transpose.

namespace {

constexpr int SCAN_B = 1024;

__global__ void k_col_count(const int32_t *__restrict__ idx, int64_t nnz, int32_t *__restrict__ cnt1) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt1 + idx[e], 1);
}

// Inclusive scan of x over the SCAN_B threads of the block (every thread
// gets its prefix); sh holds 32 ints.
__device__ __forceinline__ int32_t block_incl_scan(int32_t x, int32_t *sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = sh[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  if (warp > 0) x += sh[warp - 1];
  __syncthreads();  // sh is reused by the caller's next scan
  return x;
}

__global__ void __launch_bounds__(SCAN_B) k_scan_local(int32_t *__restrict__ a, int32_t count,
                                                       int32_t *__restrict__ bsum, int32_t *__restrict__ mx) {
  __shared__ int32_t sh[32];
  const int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  const int32_t v = i < count ? a[i] : 0;
  int32_t m = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
  const int32_t x = block_incl_scan(v, sh);
  if (i < count) a[i] = x;
  if (threadIdx.x == SCAN_B - 1) bsum[blockIdx.x] = x;
}

// Exclusive scan of the nb block totals in place (one block, chunks of SCAN_B).
__global__ void __launch_bounds__(SCAN_B) k_scan_blocks(int32_t *__restrict__ bsum, int32_t nb) {
  __shared__ int32_t sh[32];
  __shared__ int32_t total;
  int32_t carry = 0;  // sum of the earlier chunks, the same in every thread
  for (int32_t base = 0; base < nb; base += SCAN_B) {
    const int32_t i = base + threadIdx.x;
    const int32_t v = i < nb ? bsum[i] : 0;
    const int32_t x = block_incl_scan(v, sh);
    if (i < nb) bsum[i] = carry + x - v;
    if (threadIdx.x == SCAN_B - 1) total = x;
    __syncthreads();
    carry += total;
    __syncthreads();
  }
}

__global__ void k_scan_add(int32_t *__restrict__ a, int32_t count, const int32_t *__restrict__ bsum) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    a[i] += bsum[i / SCAN_B];
}

}  // namespace

size_t col_starts_work_ints(int32_t n) { return 4 + ((size_t)n + SCAN_B - 1) / SCAN_B; }

cudaError_t setup_col_starts(int32_t n, int64_t nnz, const int32_t *K_idx, int32_t *T_ptr, int32_t *work,
                             cudaStream_t s) {
  // work: the largest column count (work[0]), block totals (work + 4)
  const int32_t nb = (int32_t)(((int64_t)n + SCAN_B - 1) / SCAN_B);
  cudaError_t e = cudaMemsetAsync(T_ptr, 0, sizeof(int32_t) * ((size_t)n + 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(work, 0, sizeof(int32_t) * 4, s);
  if (e != cudaSuccess) return e;
  if (nnz > 0) {
    int64_t g = (nnz + 255) / 256;
    if (g > 152 * 64) g = 152 * 64;
    k_col_count<<<(int)g, 256, 0, s>>>(K_idx, nnz, T_ptr + 1);
  }
  k_scan_local<<<nb, SCAN_B, 0, s>>>(T_ptr + 1, n, work + 4, work);
  k_scan_blocks<<<1, SCAN_B, 0, s>>>(work + 4, nb);
  int64_t g = ((int64_t)n + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  k_scan_add<<<(int)g, 256, 0, s>>>(T_ptr + 1, n, work + 4);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- K' on the device
//
// Stable transpose, given K' row starts (setup_col_starts): a
// scatter of entry numbers into their columns (atomic cursors: arbitrary
// order), a sort of each column's entry numbers (which restores the row
// order, since K's entries are numbered row by row), and a gather of rows and
// values.  The result equals the host counting sort.  Columns longer than
// TRANSPOSE_MAX_SEG entries are left to the host sort.

namespace {

__global__ void k_scatter_entries(const int32_t *__restrict__ idx, int64_t nnz, const int32_t *__restrict__ tp,
                                  int32_t *__restrict__ cursor, int32_t *__restrict__ perm) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = idx[e];
    perm[tp[c] + atomicAdd(cursor + c, 1)] = (int32_t)e;
  }
}

// One warp per column of at most 32 entries: bitonic sort of the entry
// numbers across the lanes (padding INT_MAX).
__global__ void k_sort_short(const int32_t *__restrict__ tp, int32_t n, int32_t *__restrict__ perm) {
  const int lane = threadIdx.x & 31;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t b = tp[w], len = tp[w + 1] - b;
    if (len <= 1 || len > 32) continue;
    int32_t v = lane < len ? perm[b + lane] : INT32_MAX;
    for (int k = 2; k <= 32; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        const int32_t o = __shfl_xor_sync(0xffffffffu, v, j);
        const bool up = (lane & k) == 0, lower = (lane & j) == 0;
        v = (lower == up) ? min(v, o) : max(v, o);
      }
    if (lane < len) perm[b + lane] = v;
  }
}

// One CTA per column of 33..TRANSPOSE_MAX_SEG entries: bitonic sort in
// shared memory.
constexpr int TRANSPOSE_MAX_SEG = 4096;
__global__ void k_sort_long(const int32_t *__restrict__ tp, int32_t n, int32_t *__restrict__ perm) {
  __shared__ int32_t sh[TRANSPOSE_MAX_SEG];
  for (int32_t c = blockIdx.x; c < n; c += gridDim.x) {
    const int32_t b = tp[c], len = tp[c + 1] - b;
    if (len <= 32) continue;  // uniform across the CTA
    int P2 = 64;
    while (P2 < len) P2 <<= 1;
    for (int t = threadIdx.x; t < P2; t += blockDim.x) sh[t] = t < len ? perm[b + t] : INT32_MAX;
    __syncthreads();
    for (int k = 2; k <= P2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < P2; t += blockDim.x) {
          const int u = t ^ j;
          if (u > t) {
            const bool up = (t & k) == 0;
            const int32_t a = sh[t], d = sh[u];
            if ((a > d) == up) {
              sh[t] = d;
              sh[u] = a;
            }
          }
        }
        __syncthreads();
      }
    for (int t = threadIdx.x; t < len; t += blockDim.x) perm[b + t] = sh[t];
    __syncthreads();
  }
}

// row number of every entry of K (one warp per row)
__global__ void k_entry_rows(const int32_t *__restrict__ ptr, int32_t rows, int32_t *__restrict__ rowid) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5)
    for (int32_t e = ptr[r] + lane; e < ptr[r + 1]; e += 32) rowid[e] = (int32_t)r;
}

__global__ void k_gather_entries(const int32_t *__restrict__ perm, int64_t nnz, const int32_t *__restrict__ rowid,
                                 const double *__restrict__ val, int32_t *__restrict__ ti, double *__restrict__ tv) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = perm[p];
    ti[p] = rowid[e];
    tv[p] = val[e];
  }
}

int tgrid(int64_t work, int per = 256) {
  int64_t g = (work + per - 1) / per;
  if (g > 152 * 64) g = 152 * 64;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t setup_transpose(int32_t m, int32_t n, int64_t nnz, const int32_t *K_ptr, const int32_t *K_idx,
                            const double *K_val, const int32_t *T_ptr, int32_t *T_idx, double *T_val, int32_t *work,
                            cudaStream_t s) {
  // work: cursor (n), perm (nnz), rowid (nnz)
  int32_t *cursor = work, *perm = cursor + n, *rowid = perm + nnz;
  cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)n, s);
  if (e != cudaSuccess) return e;
  if (nnz) {
    k_scatter_entries<<<tgrid(nnz), 256, 0, s>>>(K_idx, nnz, T_ptr, cursor, perm);
    k_sort_short<<<tgrid((int64_t)n * 32), 256, 0, s>>>(T_ptr, n, perm);
    k_sort_long<<<tgrid(n, 1), 1024, 0, s>>>(T_ptr, n, perm);
    k_entry_rows<<<tgrid((int64_t)m * 32), 256, 0, s>>>(K_ptr, m, rowid);
    k_gather_entries<<<tgrid(nnz), 256, 0, s>>>(perm, nnz, rowid, K_val, T_idx, T_val);
  }
  return cudaGetLastError();
}

size_t transpose_work_ints(int32_t n, int64_t nnz) { return (size_t)n + 2 * (size_t)nnz; }
int transpose_max_segment() { return TRANSPOSE_MAX_SEG; }

__global__ void k_pow_table(double *pw, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const double kk = (double)(i + 2);
    pw[i] = pow(kk, -0.3);
    pw[count + i] = pow(kk, -0.6);
  }
}

cudaError_t setup_pow_table(double *pw, long long count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_pow_table<<<256, 256, 0, s>>>(pw, count);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- sliced-ELL layout

namespace {

// inv[perm[r]] = r
__global__ void k_invert(int32_t rows, const int32_t *__restrict__ perm, int32_t *__restrict__ inv) {
  for (int32_t r = blockIdx.x * ST + threadIdx.x; r < rows; r += gridDim.x * ST) inv[perm[r]] = r;
}

// One warp per internal row r: entry k of original row perm[r] goes to
// base[r] + k (long row) or base[r] + 32 k (slice row), its column renumbered
// through inv.  Padding was set beforehand (column -1, value 0).
__global__ void k_sell_fill(int32_t rows, const int32_t *__restrict__ perm, const int32_t *__restrict__ base,
                            const uint8_t *__restrict__ lane, const int32_t *__restrict__ ptr,
                            const int32_t *__restrict__ idx, const double *__restrict__ val,
                            const int32_t *__restrict__ inv, int32_t *__restrict__ sidx,
                            double *__restrict__ sval) {
  const int ln = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * ST + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * ST) >> 5;
  for (long long r = warp; r < rows; r += nwarps) {
    const int32_t i = perm[r], e0 = ptr[i], e1 = ptr[i + 1];
    const int64_t b = base[r], step = lane[r] ? 32 : 1;
    for (int32_t e = e0 + ln; e < e1; e += 32) {
      const int64_t d = b + (int64_t)(e - e0) * step;
      sidx[d] = inv[idx[e]];
      sval[d] = val[e];
    }
  }
}

__global__ void k_warm_perm(int32_t m, int32_t n, const double *__restrict__ x0, const double *__restrict__ y0,
                            const int32_t *__restrict__ perm_r, const int32_t *__restrict__ perm_c,
                            const double *__restrict__ D1, const double *__restrict__ D2, double *__restrict__ x,
                            double *__restrict__ y) {
  for (int j = blockIdx.x * ST + threadIdx.x; j < n; j += gridDim.x * ST) x[j] = x0 ? x0[perm_c[j]] / D2[j] : 0.0;
  for (int i = blockIdx.x * ST + threadIdx.x; i < m; i += gridDim.x * ST) y[i] = y0 ? y0[perm_r[i]] / D1[i] : 0.0;
}

// first[0] = min index e with a column outside [0, n) or a non-finite value
// (unchanged when there is none)
__global__ void k_check_entries(int64_t nnz, const int32_t *__restrict__ idx, const double *__restrict__ val,
                                int32_t n, unsigned long long *__restrict__ first) {
  for (int64_t e = (int64_t)blockIdx.x * ST + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * ST) {
    const int32_t c = idx[e];
    const unsigned long long b = (unsigned long long)__double_as_longlong(val[e]);
    if (c < 0 || c >= n || (b & 0x7ff0000000000000ull) == 0x7ff0000000000000ull) atomicMin(first, (unsigned long long)e);
  }
}

// QP: qd[j] = (D2[j] * q0[perm_c[j]]) * D2[j], the internal-order diagonal of
// D2 Q D2 (D2 internal, q0 the caller's diagonal in the original order)
__global__ void k_qp_diag(int32_t n, const int32_t *__restrict__ perm_c, const double *__restrict__ D2,
                          const double *__restrict__ q0, double *__restrict__ qd) {
  for (int32_t j = blockIdx.x * ST + threadIdx.x; j < n; j += gridDim.x * ST) qd[j] = D2[j] * q0[perm_c[j]] * D2[j];
}

// dst[r] = src[perm[r]]
__global__ void k_permute(int32_t count, const int32_t *__restrict__ perm, const double *__restrict__ src,
                          double *__restrict__ dst) {
  for (int32_t r = blockIdx.x * ST + threadIdx.x; r < count; r += gridDim.x * ST) dst[r] = src[perm[r]];
}

}  // namespace

cudaError_t setup_invert(int32_t rows, const int32_t *perm, int32_t *inv, cudaStream_t s) {
  if (rows > 0) k_invert<<<grid_for(rows), ST, 0, s>>>(rows, perm, inv);
  return cudaGetLastError();
}

cudaError_t setup_sell_fill(int32_t rows, int64_t total, const int32_t *perm, const int32_t *base,
                            const uint8_t *lane, const int32_t *ptr, const int32_t *idx, const double *val,
                            const int32_t *inv, int32_t *sidx, double *sval, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sidx, 0xff, sizeof(int32_t) * (size_t)total, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sval, 0, sizeof(double) * (size_t)total, s);
  if (e != cudaSuccess) return e;
  if (rows > 0)
    k_sell_fill<<<grid_for((long long)rows * 32), ST, 0, s>>>(rows, perm, base, lane, ptr, idx, val, inv, sidx,
                                                              sval);
  return cudaGetLastError();
}

cudaError_t setup_warm_perm(int32_t m, int32_t n, const double *x0, const double *y0, const int32_t *perm_r,
                            const int32_t *perm_c, const double *D1, const double *D2, double *x, double *y,
                            cudaStream_t s) {
  k_warm_perm<<<grid_for(n > m ? n : m), ST, 0, s>>>(m, n, x0, y0, perm_r, perm_c, D1, D2, x, y);
  return cudaGetLastError();
}

cudaError_t setup_check_entries(int64_t nnz, const int32_t *idx, const double *val, int32_t n, int64_t *first,
                                int *col_bad, cudaStream_t s) {
  *first = nnz;
  *col_bad = 0;
  unsigned long long *d = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&d, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  unsigned long long h = ~0ull;
  int32_t c = 0;
  e = cudaMemsetAsync(d, 0xff, sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    k_check_entries<<<grid_for(nnz), ST, 0, s>>>(nnz, idx, val, n, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && h < (unsigned long long)nnz) {
    e = cudaMemcpyAsync(&c, idx + h, sizeof(c), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *first = (int64_t)h;
    *col_bad = (c < 0 || c >= n) ? 1 : 0;
  }
  const cudaError_t ef = cudaFreeAsync(d, s);
  return e != cudaSuccess ? e : ef;
}

namespace {

// Debug checks of a sliced-ELL copy (PDLP_DEBUG_CHECKS=1 at create): the
// step and check kernels gather through these indices and walk these items
// without bounds checks of their own.  Counts go to err[0] (stored entries),
// err[1] (work items), err[2] (rows not covered exactly once).
__global__ void k_check_sell_entries(int64_t total, int32_t cols, const int32_t *__restrict__ sidx,
                                     const double *__restrict__ sval, const float *__restrict__ sval32,
                                     unsigned int *err) {
  for (int64_t e = (int64_t)blockIdx.x * ST + threadIdx.x; e < total; e += (int64_t)gridDim.x * ST) {
    const int32_t c = sidx[e];
    const bool pad = c == -1;
    if (c < -1 || c >= cols || (pad && sval[e] != 0.0) || (pad && sval32 && sval32[e] != 0.0f))
      atomicAdd(err, 1u);
  }
}

__global__ void k_check_sell_items(int32_t nitems, const int4 *__restrict__ items, int32_t rows, int64_t total,
                                   unsigned int *err, unsigned int *cover) {
  for (int32_t it = blockIdx.x * ST + threadIdx.x; it < nitems; it += gridDim.x * ST) {
    const int4 d = items[it];
    bool bad = d.w < 0 || (d.w & 31) != 0 || d.x < 0 || d.z < 0;
    if (!bad && d.y > 0) {  // slice: d.y rows from d.x, d.z strides of 32 entries
      bad = d.y > 32 || d.x + d.y > rows || d.z > SELL_LONG || (int64_t)d.w + 32LL * d.z > total;
      if (!bad)
        for (int r = 0; r < d.y; ++r) atomicAdd(cover + d.x + r, 1u);
    } else if (!bad && d.y == -1) {  // long row d.x of d.z entries
      bad = d.x >= rows || d.z <= SELL_LONG || (int64_t)d.w + 32LL * ((d.z + 31) / 32) > total;
      if (!bad) atomicAdd(cover + d.x, 1u);
    } else {
      bad = true;
    }
    if (bad) atomicAdd(err + 1, 1u);
  }
}

__global__ void k_check_sell_cover(int32_t rows, const unsigned int *__restrict__ cover, unsigned int *err) {
  for (int32_t r = blockIdx.x * ST + threadIdx.x; r < rows; r += gridDim.x * ST)
    if (cover[r] != 1u) atomicAdd(err + 2, 1u);
}

}  // namespace

cudaError_t setup_check_sell(int32_t rows, int32_t cols, int64_t total, int32_t nitems, const int4 *items,
                             const int32_t *sidx, const double *sval, const float *sval32, unsigned int counts[3],
                             cudaStream_t s) {
  counts[0] = counts[1] = counts[2] = 0;
  unsigned int *d = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&d, sizeof(unsigned int) * (3 + (size_t)rows), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(d, 0, sizeof(unsigned int) * (3 + (size_t)rows), s);
  if (e == cudaSuccess && total > 0) k_check_sell_entries<<<grid_for(total), ST, 0, s>>>(total, cols, sidx, sval, sval32, d);
  if (e == cudaSuccess && nitems > 0) k_check_sell_items<<<grid_for(nitems), ST, 0, s>>>(nitems, items, rows, total, d, d + 3);
  if (e == cudaSuccess && rows > 0) k_check_sell_cover<<<grid_for(rows), ST, 0, s>>>(rows, d + 3, d);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(counts, d, sizeof(unsigned int) * 3, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const cudaError_t ef = cudaFreeAsync(d, s);
  return e != cudaSuccess ? e : ef;
}

cudaError_t setup_qp_diag(int32_t n, const int32_t *perm_c, const double *D2, const double *q0, double *qd,
                          cudaStream_t s) {
  k_qp_diag<<<grid_for(n), ST, 0, s>>>(n, perm_c, D2, q0, qd);
  return cudaGetLastError();
}

cudaError_t setup_permute(int32_t count, const int32_t *perm, const double *src, double *dst, cudaStream_t s) {
  if (count > 0) k_permute<<<grid_for(count), ST, 0, s>>>(count, perm, src, dst);
  return cudaGetLastError();
}

}  // namespace pdlp

// ---------------------------------------------------------------------------
// Allocation-free variant of the scaling pass (pdlp_scale_device_noalloc).
//
// The per-pass row and column factors of setup_scale live in this file-scope
// device array instead of in memory the solver allocates.  The array's host
// symbol is only a host-side stand-in: kernels receive the device address
// looked up once per device with cudaGetSymbolAddress (under a lock, with
// that device current) on the first call made on the device.

namespace {

constexpr int32_t NOALLOC_MAX_LINES = 1 << 18;  // rows and columns, each
__device__ __align__(256) double g_scale_scratch[2 * NOALLOC_MAX_LINES];

constexpr int MAX_DEVICES = 256;
std::mutex g_scratch_mu;
double *g_scratch_dev[MAX_DEVICES] = {};

}  // namespace

extern "C" int pdlp_scale_device_noalloc(int32_t m, int32_t n, const int32_t *K_ptr, const int32_t *K_idx,
                                         double *K_val, const int32_t *KT_ptr, const int32_t *KT_idx, double *KT_val,
                                         int32_t ruiz_iters, double pc_alpha, double *D1, double *D2,
                                         void *stream) {
  using namespace pdlp;
  if (m < 0 || n < 1 || m > NOALLOC_MAX_LINES || n > NOALLOC_MAX_LINES)
    return set_error(PDLP_ERR_INVALID,
                     ("pdlp_scale_device_noalloc: need 0 <= m <= 262144 and 1 <= n <= 262144 (got m=" +
                      std::to_string(m) + ", n=" + std::to_string(n) + ")")
                         .c_str());
  if (ruiz_iters < 0 || !(pc_alpha <= 2.0))
    return set_error(PDLP_ERR_INVALID, "pdlp_scale_device_noalloc: need ruiz_iters >= 0 and pc_alpha <= 2");
  // K' rows always exist (n >= 1); entries, and so K and the entry arrays of
  // both matrices, exist only when m > 0
  if (!KT_ptr || !D2 || (m > 0 && (!K_ptr || !K_idx || !K_val || !KT_idx || !KT_val || !D1)))
    return set_error(PDLP_ERR_INVALID, "pdlp_scale_device_noalloc: null pointer argument");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(PDLP_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= MAX_DEVICES) return set_error(PDLP_ERR_INVALID, "pdlp_scale_device_noalloc: device ordinal");
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scale_scratch);
      if (e != cudaSuccess) return set_error(PDLP_ERR_CUDA, cudaGetErrorString(e));
      g_scratch_dev[dev] = static_cast<double *>(p);
    }
    scratch = g_scratch_dev[dev];
  }
  double *work_m = scratch, *work_n = scratch + NOALLOC_MAX_LINES;
  e = setup_scale(m, n, 0, const_cast<int32_t *>(K_ptr), const_cast<int32_t *>(K_idx), K_val,
                  const_cast<int32_t *>(KT_ptr), const_cast<int32_t *>(KT_idx), KT_val, D1, D2, work_m, work_n,
                  ruiz_iters, pc_alpha, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return set_error(PDLP_ERR_CUDA, cudaGetErrorString(e));
  return PDLP_OK;
}

