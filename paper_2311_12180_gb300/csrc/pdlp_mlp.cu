// BF16 multilayer perceptron for learned warm starts of parametric LPs:
// theta (in) -> hidden -> ReLU -> hidden -> ReLU -> out, trained with MSE on
// per-output standardised targets by Adam with FP32 master weights.
//
// Every GEMM runs on the 5th-generation tensor cores: C = A Bt', A (M x K)
// and Bt (N x K) BF16 in global memory with K contiguous, staged into shared
// memory by TMA (128-byte swizzle, a 3-stage mbarrier ring), multiplied by
// tcgen05.mma (kind::f16, M = N = 128 per CTA, K = 16 per instruction)
// issued by one thread, accumulated in FP32 in tensor memory and read back
// with tcgen05.ld by the CTA's eight warps (a TMEM lane quarter and half of
// the columns each) for a fused epilogue.  Because both operands must have K contiguous, every
// tensor that enters a GEMM once as "rows x K" and once as "K x rows" is kept
// in both layouts: the epilogues and elementwise kernels that produce an
// activation or gradient write its transpose too (coalesced across the warp,
// whose lanes hold consecutive rows), and the BF16 weight copies are rebuilt
// in both layouts from the FP32 masters after each Adam step.
//
// Mixed precision: weights and activations enter the GEMMs as BF16, the
// output layer, the loss, all gradients and the Adam state stay FP32, and the
// output gradient is rounded to BF16 only as a GEMM operand.  The loss is
// fused into the output-layer GEMM's epilogue.  Split-K partial sums, column
// sums and the loss are reduced in a fixed order, so training is
// deterministic.  Every wait on an mbarrier is bounded (2 s); a GEMM that
// times out records an error that the host call returns.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pdlp.h"
#include "pdlp_internal.cuh"

namespace pdlp {
namespace mlp {

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------- tcgen05 GEMM

constexpr int TBM = 128, TBN = 128, TBK = 64, STAGES = 3;
constexpr int GEMM_THREADS = 256;  // 8 warps: warp w reads TMEM lanes 32 (w % 4).., columns 64 (w / 4)..
constexpr int A_BYTES = TBM * TBK * 2, B_BYTES = TBN * TBK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int GEMM_SMEM = STAGES * STAGE_BYTES + 1024 + 128;  // + alignment slack + barriers
constexpr uint32_t TMEM_COLS = TBN;                           // FP32 accumulator: 128 lanes x 128 columns
// instruction descriptor: D F32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N / 8 at bits 17-22, M / 16 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                           ((uint32_t)(TBM >> 4) << 24);
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;

enum { GEMM_ERR_FULL = 1, GEMM_ERR_EMPTY = 2, GEMM_ERR_DONE = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of the mbarrier; false after WAIT_LIMIT_NS.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  const unsigned long long t0 = gtimer();
  while (!mbar_try(a, parity))
    if (gtimer() - t0 > WAIT_LIMIT_NS) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// start address / 16 (bits 0-13), leading offset 16 B (unused by this
// layout), stride between 8-row groups 1024 B (bits 32-45), descriptor
// version 1 (bits 46-47), layout SWIZZLE_128B = 2 (bits 61-63).
__device__ __forceinline__ unsigned long long sw128_desc(uint32_t addr) {
  unsigned long long d = (unsigned long long)((addr & 0x3FFFF) >> 4);
  d |= (unsigned long long)(16 >> 4) << 16;
  d |= (unsigned long long)(1024 >> 4) << 32;
  d |= 1ull << 46;
  d |= 2ull << 61;
  return d;
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, unsigned long long a, unsigned long long b,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// C(m, n) = sum_k A(m, k) Bt(n, k) over split z = blockIdx.z's K range
// [z kchunk, min(K, (z + 1) kchunk)) (kchunk a multiple of TBK), A and Bt
// described by the tensor maps (box TBK x 128, 128-byte swizzle).  Thread 0
// issues the TMA loads and the MMAs; the finished tile passes through
// epi.chunk(m, n, values, count, split) -- 16 consecutive columns n.. of
// row m, count of them inside the matrix -- for m < M, then epi.finish()
// runs in every thread.  A wait that exceeds its limit sets *err and skips the epilogue.
template <class Epi>
__global__ void __launch_bounds__(GEMM_THREADS) k_tc_gemm(const __grid_constant__ CUtensorMap ma,
                                                 const __grid_constant__ CUtensorMap mb, int M, int N, int K,
                                                 int kchunk, Epi epi, int *err, int stall) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~static_cast<uintptr_t>(1023));
  unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + STAGES * STAGE_BYTES);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  const int nk = ke > kb ? (ke - kb + TBK - 1) / TBK : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (threadIdx.x == 0) {
    bool ok = true;
    for (int s = 0; s < STAGES && s < nk; ++s) {
      // test hook: CTA 0 never loads stage 0, so its first wait runs out
      if (stall && s == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) continue;
      const uint32_t a = smem_u32(smem + s * STAGE_BYTES);
      mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
      tma_load_2d(a, &ma, kb + s * TBK, m0, full0 + 8 * s);
      tma_load_2d(a + A_BYTES, &mb, kb + s * TBK, n0, full0 + 8 * s);
    }
    for (int k = 0; k < nk && ok; ++k) {
      const int s = k % STAGES;
      const uint32_t ph = (uint32_t)(k / STAGES) & 1u;
      if (!mbar_wait(full0 + 8 * s, ph)) {
        atomicExch(err, GEMM_ERR_FULL);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a = smem_u32(smem + s * STAGE_BYTES), b = a + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < TBK / 16; ++kk)
        umma_bf16(tmem, sw128_desc(a + kk * 32), sw128_desc(b + kk * 32), (k | kk) != 0 ? 1u : 0u);
      umma_commit(empty0 + 8 * s);
      if (k + STAGES < nk) {
        // the stage is refilled once the MMAs just issued have read it
        if (!mbar_wait(empty0 + 8 * s, ph)) {
          atomicExch(err, GEMM_ERR_EMPTY);
          ok = false;
          break;
        }
        mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
        tma_load_2d(a, &ma, kb + (k + STAGES) * TBK, m0, full0 + 8 * s);
        tma_load_2d(b, &mb, kb + (k + STAGES) * TBK, n0, full0 + 8 * s);
      }
    }
    umma_commit(done);  // arrives when every MMA issued above has completed
  }
  __syncthreads();
  const bool ok = mbar_wait(done, 0);
  if (!ok) atomicExch(err, GEMM_ERR_DONE);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // a split with an empty K range never wrote its accumulator: its tile is zero
  const int quarter = warp & 3, half = warp >> 2;
  const int row = m0 + quarter * 32 + lane;
#pragma unroll 1
  for (int c0 = half * (TBN / 2); c0 < (half + 1) * (TBN / 2) && ok; c0 += 16) {
    float v[16];
    tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
    if (!nk) {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = 0.0f;
    }
    if (row < M && n0 + c0 < N) epi.chunk(row, n0 + c0, v, min(16, N - n0 - c0), (int)blockIdx.z);
  }
  epi.finish();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ---------------------------------------------------------------- epilogues
//
// Each thread holds 16 consecutive columns of one row.  Row-major outputs are
// written with 16-byte vector stores when the row stride and base allow it
// (`vec`, decided on the host), transposed outputs element by element (the
// 32 lanes of a warp hold 32 consecutive rows, so those stores coalesce).

__device__ __forceinline__ void st16_f32(float *p, const float (&v)[16]) {
  float4 *q = reinterpret_cast<float4 *>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k) q[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}
__device__ __forceinline__ void ld16_f32(const float *p, float (&v)[16]) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 a = q[k];
    v[4 * k] = a.x;
    v[4 * k + 1] = a.y;
    v[4 * k + 2] = a.z;
    v[4 * k + 3] = a.w;
  }
}
__device__ __forceinline__ void st16_bf16(bf16 *p, const bf16 (&h)[16]) {
  uint4 *q = reinterpret_cast<uint4 *>(p);
  const uint4 *src = reinterpret_cast<const uint4 *>(h);
  q[0] = src[0];
  q[1] = src[1];
}

struct EpiBase {
  __device__ __forceinline__ void finish() {}
};
// hidden layer: H = bf16(relu(z + b)), stored as H (rows x hidden, ld a
// multiple of 8: vector stores) and H'
struct EpiHidden : EpiBase {
  const float *bias;
  bf16 *out, *outT;
  int ld, ldT;
  __device__ __forceinline__ void chunk(int m, int n, const float (&v)[16], int cnt, int) const {
    __align__(16) bf16 h[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float z = j < cnt ? v[j] + bias[n + j] : 0.0f;
      h[j] = __float2bfloat16(z > 0.0f ? z : 0.0f);
    }
    if (cnt == 16) {
      st16_bf16(out + (size_t)m * ld + n, h);
    } else {
      for (int j = 0; j < cnt; ++j) out[(size_t)m * ld + n + j] = h[j];
    }
    for (int j = 0; j < cnt; ++j) outT[(size_t)(n + j) * ldT + m] = h[j];
  }
};
// output layer for prediction: Y = z + b (standardised units)
struct EpiOut : EpiBase {
  const float *bias;
  float *y;
  int ld;
  bool vec;
  __device__ __forceinline__ void chunk(int m, int n, const float (&v)[16], int cnt, int) const {
    float o[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) o[j] = j < cnt ? v[j] + bias[n + j] : 0.0f;
    if (vec && cnt == 16) {
      st16_f32(y + (size_t)m * ld + n, o);
    } else {
      for (int j = 0; j < cnt; ++j) y[(size_t)m * ld + n + j] = o[j];
    }
  }
};
// output layer for training, with the loss fused: d = z + b - (t - mu) / sigma,
// dY = 2 d / (B N) in FP32 (for the bias gradient) and as BF16 GEMM operand
// in both layouts; each CTA writes its partial sum of d^2 (fixed order:
// FP32 over a thread's 16 columns, FP64 across chunks and threads).
struct EpiLoss {
  const float *bias, *t, *mu, *sigma;
  const int *rows;  // batch row m's target is row rows[m] of the data set t
  float *dy;
  bf16 *dyh, *dyhT;
  double *part;
  float scale;
  int ldt, ldh, ldT;
  bool vec;  // t / dy rows allow 16-byte accesses
  double acc;
  __device__ __forceinline__ void chunk(int m, int n, const float (&v)[16], int cnt, int) {
    float tv[16];
    const float *tr = t + (size_t)rows[m] * ldt;
    if (vec && cnt == 16) {
      ld16_f32(tr + n, tv);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) tv[j] = j < cnt ? tr[n + j] : 0.0f;
    }
    float g[16];
    __align__(16) bf16 gh[16];
    float sq = 0.0f;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      float d = 0.0f;
      if (j < cnt) d = v[j] + bias[n + j] - (tv[j] - mu[n + j]) / sigma[n + j];
      sq = fmaf(d, d, sq);
      g[j] = scale * d;
      gh[j] = __float2bfloat16(g[j]);
    }
    acc += (double)sq;
    if (vec && cnt == 16) {
      st16_f32(dy + (size_t)m * ldt + n, g);
      st16_bf16(dyh + (size_t)m * ldh + n, gh);
    } else {
      for (int j = 0; j < cnt; ++j) {
        dy[(size_t)m * ldt + n + j] = g[j];
        dyh[(size_t)m * ldh + n + j] = gh[j];
      }
    }
    for (int j = 0; j < cnt; ++j) dyhT[(size_t)(n + j) * ldT + m] = gh[j];
  }
  __device__ __forceinline__ void finish() {
    __shared__ double red[GEMM_THREADS / 32];
    double s = acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < GEMM_THREADS / 32; ++w) t += red[w];
      part[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
  }
};
// plain FP32 store (weight gradients, dH1)
struct EpiStore : EpiBase {
  float *out;
  int ld;
  bool vec;
  __device__ __forceinline__ void chunk(int m, int n, const float (&v)[16], int cnt, int) const {
    if (vec && cnt == 16) {
      st16_f32(out + (size_t)m * ld + n, v);
    } else {
      for (int j = 0; j < cnt; ++j) out[(size_t)m * ld + n + j] = v[j];
    }
  }
};
// split-K partial sums, summed later in split order
struct EpiPartial : EpiBase {
  float *part;
  int ld;
  size_t stride;
  bool vec;
  __device__ __forceinline__ void chunk(int m, int n, const float (&v)[16], int cnt, int s) const {
    float *p = part + s * stride + (size_t)m * ld + n;
    if (vec && cnt == 16) {
      st16_f32(p, v);
    } else {
      for (int j = 0; j < cnt; ++j) p[j] = v[j];
    }
  }
};

// ---------------------------------------------------------------- elementwise kernels

// dZ2 = (sum of split partials, in split order) masked by H2 > 0: FP32 rows
// (bias gradient) and BF16 in both layouts (GEMM operands).
__global__ void k_splitk_relu_grad(const float *__restrict__ part, int splits, int B, int H,
                                   const bf16 *__restrict__ h, int ldh, float *__restrict__ dz,
                                   bf16 *__restrict__ dzh, bf16 *__restrict__ dzhT, int ldT) {
  const size_t count = (size_t)B * H;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / H), j = (int)(i % H);
    float s = 0.0f;
    for (int k = 0; k < splits; ++k) s += part[k * count + i];
    const float g = __bfloat162float(h[(size_t)b * ldh + j]) > 0.0f ? s : 0.0f;
    dz[i] = g;
    const bf16 gh = __float2bfloat16(g);
    dzh[(size_t)b * ldh + j] = gh;
    dzhT[(size_t)j * ldT + b] = gh;
  }
}

// Mini-batch gather: inputs to BF16 in both layouts, targets (FP32) of the
// sampled rows.
__global__ void k_gather(const float *__restrict__ X, const int *__restrict__ idx, int batch, int in_dim,
                         bf16 *__restrict__ xb, int ldx, bf16 *__restrict__ xbT, int ldT) {
  const int b = blockIdx.x;
  if (b >= batch) return;
  const size_t row = (size_t)idx[b];
  for (int i = threadIdx.x; i < in_dim; i += blockDim.x) {
    const bf16 v = __float2bfloat16(X[row * in_dim + i]);
    xb[(size_t)b * ldx + i] = v;
    xbT[(size_t)i * ldT + b] = v;
  }
}

// prediction input: X (count x in, FP32) -> BF16 rows
__global__ void k_input_bf16(const float *__restrict__ x, int count, int in_dim, bf16 *__restrict__ xb, int ldx) {
  const size_t total = (size_t)count * in_dim;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    xb[(i / in_dim) * ldx + i % in_dim] = __float2bfloat16(x[i]);
}

// mean of the per-CTA partial sums (one block of 256 threads: strided sums,
// then a fixed tree)
__global__ void k_loss_finish(const double *__restrict__ part, int nparts, size_t count, float *__restrict__ out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    *out = (float)(t / (double)count);
  }
}

// out[c] = sum over rows of X[rows x cols] (fixed row order): bias gradients.
// Column sums of X (rows x cols, FP32): a block of 32 columns x 8 row
// groups; group g adds rows g, g + 8, ... in order, then the eight partial
// sums are added in group order (a fixed order, whatever the grid).
constexpr int COLSUM_GROUPS = 8;
__global__ void k_colsum(const float *__restrict__ X, int rows, int cols, float *__restrict__ out) {
  __shared__ float part[COLSUM_GROUPS][32];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  for (int c0 = blockIdx.x * 32; c0 < cols; c0 += gridDim.x * 32) {
    const int c = c0 + lane;
    float s = 0.0f;
    if (c < cols)
      for (int r = grp; r < rows; r += COLSUM_GROUPS) s += X[(size_t)r * cols + c];
    part[grp][lane] = s;
    __syncthreads();
    if (grp == 0 && c < cols) {
      float t = 0.0f;
#pragma unroll
      for (int g = 0; g < COLSUM_GROUPS; ++g) t += part[g][lane];
      out[c] = t;
    }
    __syncthreads();
  }
}

// dZ1 = dH1 masked by H1 > 0: FP32 rows (bias gradient) and BF16 transposed
// (operand of the first layer's weight gradient).
__global__ void k_relu_grad(const float *__restrict__ dh, int B, int H, const bf16 *__restrict__ h, int ldh,
                            float *__restrict__ dz, bf16 *__restrict__ dzhT, int ldT) {
  const size_t count = (size_t)B * H;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / H), j = (int)(i % H);
    const float g = __bfloat162float(h[(size_t)b * ldh + j]) > 0.0f ? dh[i] : 0.0f;
    dz[i] = g;
    dzhT[(size_t)j * ldT + b] = __float2bfloat16(g);
  }
}

// Per-output mean and standard deviation of the targets (two passes, FP64).
__global__ void k_mean_std(const float *__restrict__ T, int samples, int out_dim, float *__restrict__ mu,
                           float *__restrict__ sigma) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < out_dim; o += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < samples; ++r) s += T[(size_t)r * out_dim + o];
    const double mean = s / samples;
    double v = 0.0;
    for (int r = 0; r < samples; ++r) {
      const double d = T[(size_t)r * out_dim + o] - mean;
      v += d * d;
    }
    const double sd = sqrt(v / samples);
    mu[o] = (float)mean;
    sigma[o] = (float)(sd > 1e-6 ? sd : 1e-6);
  }
}

__global__ void k_unstandardize(const float *__restrict__ y, size_t count, int out_dim, const float *__restrict__ mu,
                                const float *__restrict__ sigma, float *__restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(i % out_dim);
    out[i] = y[i] * sigma[o] + mu[o];
  }
}

// Adam on the FP32 master copy.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, size_t count, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float mh = a / c1, vh = b / c2;
    p[i] = p[i] - lr * mh / (sqrtf(vh) + eps);
  }
}

// BF16 copies of a weight matrix W (rows x cols, FP32, row-major) as W
// (ld ldw; skipped when wb is null) and W' (cols x rows, ld ldt), through
// 32 x 32 shared tiles so that the reads and both writes are coalesced.
__global__ void k_weight_bf16(const float *__restrict__ w, int rows, int cols, bf16 *__restrict__ wb, int ldw,
                              bf16 *__restrict__ wt, int ldt) {
  __shared__ float tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = ty; k < 32; k += 8) {
    const int r = r0 + k, c = c0 + tx;
    if (r < rows && c < cols) {
      const float v = w[(size_t)r * cols + c];
      tile[k][tx] = v;
      if (wb) wb[(size_t)r * ldw + c] = __float2bfloat16(v);
    }
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int c = c0 + k, r = r0 + tx;
    if (r < rows && c < cols) wt[(size_t)c * ldt + r] = __float2bfloat16(tile[tx][k]);
  }
}

int grid1(size_t n, int bs = 256) {
  size_t g = (n + bs - 1) / bs;
  if (g > 65535 * 4) g = 65535 * 4;
  return (int)(g < 1 ? 1 : g);
}
// k_colsum: one block per 32 columns
int colsum_grid(int cols) { return cols > 0 ? (cols + 31) / 32 : 1; }

}  // namespace mlp
}  // namespace pdlp

// ================================================================ host side

using namespace pdlp;
using namespace pdlp::mlp;

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Tensor map of a BF16 matrix (rows x cols, row stride ld elements, ld a
// multiple of 8) read in TBK x 128 boxes with the 128-byte swizzle; rows and
// columns past the extents read as zero.
bool make_map(CUtensorMap *m, const bf16 *base, int rows, int cols, int ld) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {TBK, 128};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int pad8(int x) { return (x + 7) / 8 * 8; }

// rows of ld floats starting at p allow 16-byte accesses at 16-column offsets
bool vec4(const float *p, int ld) { return reinterpret_cast<uintptr_t>(p) % 16 == 0 && ld % 4 == 0; }

}  // namespace

struct pdlp_mlp {
  int device = 0;
  int in = 0, hid = 0, out = 0, maxb = 0, splits = 1;
  int ldi = 0, ldh = 0, ldo = 0, ldb = 0;  // padded leading dimensions (multiples of 8)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t nparam = 0, oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
  // BF16 weights: W1' (hid x in), W2 (hid x hid) and W2', W3 (hid x out) and W3' (out x hid)
  bf16 *w1t = nullptr, *w2 = nullptr, *w2t = nullptr, *w3 = nullptr, *w3t = nullptr;
  // one mini-batch: BF16 GEMM operands in both layouts, FP32 loss path
  bf16 *xb = nullptr, *xbT = nullptr, *h1 = nullptr, *h1T = nullptr, *h2 = nullptr, *h2T = nullptr;
  bf16 *dyh = nullptr, *dyhT = nullptr, *dz2h = nullptr, *dz2hT = nullptr, *dz1hT = nullptr;
  float *xin = nullptr, *y = nullptr, *dy = nullptr, *dz2 = nullptr, *dz1 = nullptr, *dh1 = nullptr,
        *part = nullptr;
  double *lpart = nullptr;
  int lparts = 0;
  float *loss_dev = nullptr, *mu = nullptr, *sigma = nullptr;
  int *err = nullptr;
  // data set
  float *X = nullptr, *T = nullptr;
  int samples = 0;
  int *idx = nullptr;
  size_t idx_cap = 0;
  long long adam_t = 0;
  // test hook for the bounded waits (environment PDLP_TEST_GEMM_STALL=1 at a
  // call): the call's first GEMM starves one CTA of its first stage
  int stall_next = 0;
  std::vector<void *> allocs;
};

namespace {

#define MCK(...)                                                                                             \
  do {                                                                                                       \
    cudaError_t e_ = (__VA_ARGS__);                                                                          \
    if (e_ != cudaSuccess) return set_error(PDLP_ERR_CUDA, (std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)).c_str()); \
  } while (0)

template <class T>
int dalloc(pdlp_mlp *M, T **p, size_t count) {
  void *q = nullptr;
  const cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess)
    return set_error(e == cudaErrorMemoryAllocation ? PDLP_ERR_OOM : PDLP_ERR_CUDA, cudaGetErrorString(e));
  M->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return PDLP_OK;
}

void free_mlp(pdlp_mlp *M) {
  if (!M) return;
  for (void *q : M->allocs) cudaFree(q);
  if (M->own_stream && M->stream) cudaStreamDestroy(M->stream);
  delete M;
}

// C (M x N) = A (M x K, ld lda) Bt' (Bt: N x K, ld ldb) through epi.
template <class Epi>
int gemm(pdlp_mlp *Mn, int M, int N, int K, int splits, const bf16 *A, int lda, const bf16 *Bt, int ldb,
         const Epi &epi) {
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, K, lda) || !make_map(&mb, Bt, N, K, ldb))
    return set_error(PDLP_ERR_CUDA, "MLP GEMM: cuTensorMapEncodeTiled unavailable or rejected the operand");
  const int kchunk = ((K + splits - 1) / splits + TBK - 1) / TBK * TBK;
  dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM, splits);
  const int stall = Mn->stall_next;
  Mn->stall_next = 0;
  k_tc_gemm<Epi><<<grid, GEMM_THREADS, GEMM_SMEM, Mn->stream>>>(ma, mb, M, N, K, kchunk, epi, Mn->err, stall);
  MCK(cudaGetLastError());
  return PDLP_OK;
}

template <class Epi>
cudaError_t allow_smem() {
  return cudaFuncSetAttribute(k_tc_gemm<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
}

// BF16 copies of the weights from the FP32 masters.
int refresh_weights(pdlp_mlp *M) {
  cudaStream_t s = M->stream;
  auto grid2 = [](int rows, int cols) { return dim3((cols + 31) / 32, (rows + 31) / 32); };
  k_weight_bf16<<<grid2(M->in, M->hid), 256, 0, s>>>(M->p + M->oW1, M->in, M->hid, nullptr, 0, M->w1t, M->ldi);
  k_weight_bf16<<<grid2(M->hid, M->hid), 256, 0, s>>>(M->p + M->oW2, M->hid, M->hid, M->w2, M->ldh, M->w2t, M->ldh);
  k_weight_bf16<<<grid2(M->hid, M->out), 256, 0, s>>>(M->p + M->oW3, M->hid, M->out, M->w3, M->ldo, M->w3t, M->ldh);
  MCK(cudaGetLastError());
  return PDLP_OK;
}

// hidden layers for rows [0, B) of xb
int forward_hidden(pdlp_mlp *M, int B) {
  int rc = gemm(M, B, M->hid, M->in, 1, M->xb, M->ldi, M->w1t, M->ldi,
                EpiHidden{{}, M->p + M->ob1, M->h1, M->h1T, M->ldh, M->ldb});
  if (!rc)
    rc = gemm(M, B, M->hid, M->hid, 1, M->h1, M->ldh, M->w2t, M->ldh,
              EpiHidden{{}, M->p + M->ob2, M->h2, M->h2T, M->ldh, M->ldb});
  return rc;
}

// loss (fused into the output layer) and every gradient into M->g for the
// batch in xb / tb
int forward_backward(pdlp_mlp *M, int B, const int *rows) {
  cudaStream_t s = M->stream;
  int rc = forward_hidden(M, B);
  if (rc) return rc;
  const size_t BO = (size_t)B * M->out, BH = (size_t)B * M->hid;
  const int tiles = ((M->out + TBN - 1) / TBN) * ((B + TBM - 1) / TBM);
  EpiLoss el{M->p + M->ob3, M->T, M->mu, M->sigma, rows, M->dy, M->dyh, M->dyhT, M->lpart, 2.0f / (float)BO,
             M->out, M->ldo, M->ldb, vec4(M->T, M->out) && vec4(M->dy, M->out), 0.0};
  rc = gemm(M, B, M->out, M->hid, 1, M->h2, M->ldh, M->w3t, M->ldh, el);
  if (rc) return rc;
  k_loss_finish<<<1, 256, 0, s>>>(M->lpart, tiles, BO, M->loss_dev);
  // output layer: gW3 = H2' dY, gb3 = column sums of dY, dH2 = dY W3'
  rc = gemm(M, M->hid, M->out, B, 1, M->h2T, M->ldb, M->dyhT, M->ldb, EpiStore{{}, M->g + M->oW3, M->out, vec4(M->g + M->oW3, M->out)});
  if (rc) return rc;
  k_colsum<<<colsum_grid(M->out), 256, 0, s>>>(M->dy, B, M->out, M->g + M->ob3);
  rc = gemm(M, B, M->hid, M->out, M->splits, M->dyh, M->ldo, M->w3, M->ldo, EpiPartial{{}, M->part, M->hid, BH, vec4(M->part, M->hid) && BH % 4 == 0});
  if (rc) return rc;
  k_splitk_relu_grad<<<grid1(BH), 256, 0, s>>>(M->part, M->splits, B, M->hid, M->h2, M->ldh, M->dz2, M->dz2h,
                                               M->dz2hT, M->ldb);
  // second layer
  rc = gemm(M, M->hid, M->hid, B, 1, M->h1T, M->ldb, M->dz2hT, M->ldb, EpiStore{{}, M->g + M->oW2, M->hid, vec4(M->g + M->oW2, M->hid)});
  if (rc) return rc;
  k_colsum<<<colsum_grid(M->hid), 256, 0, s>>>(M->dz2, B, M->hid, M->g + M->ob2);
  rc = gemm(M, B, M->hid, M->hid, 1, M->dz2h, M->ldh, M->w2, M->ldh, EpiStore{{}, M->dh1, M->hid, vec4(M->dh1, M->hid)});
  if (rc) return rc;
  k_relu_grad<<<grid1(BH), 256, 0, s>>>(M->dh1, B, M->hid, M->h1, M->ldh, M->dz1, M->dz1hT, M->ldb);
  // first layer
  rc = gemm(M, M->in, M->hid, B, 1, M->xbT, M->ldb, M->dz1hT, M->ldb, EpiStore{{}, M->g + M->oW1, M->hid, vec4(M->g + M->oW1, M->hid)});
  if (rc) return rc;
  k_colsum<<<colsum_grid(M->hid), 256, 0, s>>>(M->dz1, B, M->hid, M->g + M->ob1);
  MCK(cudaGetLastError());
  return PDLP_OK;
}

int ensure_idx(pdlp_mlp *M, size_t count) {
  if (count <= M->idx_cap) return PDLP_OK;
  int *p = nullptr;
  int rc = dalloc(M, &p, count);
  if (rc) return rc;
  M->idx = p;
  M->idx_cap = count;
  return PDLP_OK;
}

// after a synchronisation: a GEMM whose wait timed out fails the call
int check_err(pdlp_mlp *M) {
  int e = 0;
  MCK(cudaMemcpy(&e, M->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    cudaMemset(M->err, 0, sizeof(int));
    return set_error(PDLP_ERR_CUDA,
                     ("MLP GEMM: a tensor-core pipeline wait timed out (stage " + std::to_string(e) + ")").c_str());
  }
  return PDLP_OK;
}

}  // namespace

extern "C" {

int pdlp_mlp_create(pdlp_mlp **out, int32_t in_dim, int32_t hidden, int32_t out_dim, int32_t max_batch, void *stream) {
  if (!out || in_dim < 1 || hidden < 1 || out_dim < 1 || max_batch < 1)
    return set_error(PDLP_ERR_INVALID, "pdlp_mlp_create: dimensions and max_batch must be >= 1");
  if (max_batch > 65535 || (int64_t)in_dim * hidden > INT32_MAX || (int64_t)hidden * out_dim > INT32_MAX)
    return set_error(PDLP_ERR_INVALID, "pdlp_mlp_create: max_batch above 65535 or a weight matrix above 2^31 entries");
  *out = nullptr;
  pdlp_mlp *M = new pdlp_mlp();
  M->in = in_dim;
  M->hid = hidden;
  M->out = out_dim;
  M->maxb = max_batch;
  M->ldi = pad8(in_dim);
  M->ldh = pad8(hidden);
  M->ldo = pad8(out_dim);
  M->ldb = pad8(max_batch);
  size_t o = 0;
  M->oW1 = o; o += (size_t)in_dim * hidden;
  M->ob1 = o; o += hidden;
  M->oW2 = o; o += (size_t)hidden * hidden;
  M->ob2 = o; o += hidden;
  M->oW3 = o; o += (size_t)hidden * out_dim;
  M->ob3 = o; o += out_dim;
  M->nparam = o;
  cudaError_t e = cudaGetDevice(&M->device);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, M->device);
  if (e == cudaSuccess) {
    if (stream) {
      M->stream = (cudaStream_t)stream;
    } else {
      e = cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking);
      M->own_stream = true;
    }
  }
  if (e == cudaSuccess) e = allow_smem<EpiHidden>();
  if (e == cudaSuccess) e = allow_smem<EpiOut>();
  if (e == cudaSuccess) e = allow_smem<EpiLoss>();
  if (e == cudaSuccess) e = allow_smem<EpiStore>();
  if (e == cudaSuccess) e = allow_smem<EpiPartial>();
  if (e != cudaSuccess) {
    free_mlp(M);
    return set_error(PDLP_ERR_CUDA, cudaGetErrorString(e));
  }
  if (!encode_fn()) {
    free_mlp(M);
    return set_error(PDLP_ERR_CUDA, "pdlp_mlp_create: the driver offers no cuTensorMapEncodeTiled");
  }
  // split the long reduction of dH2 = dY W3' over the outputs so that the
  // batch x hidden output tiles fill the SMs: about one CTA per SM, at least
  // four 64-wide K blocks per split
  {
    const int tiles = ((hidden + TBN - 1) / TBN) * ((max_batch + TBM - 1) / TBM);
    const int by_sm = std::max(1, sms / std::max(1, tiles));
    const int by_k = std::max(1, out_dim / (4 * TBK));
    M->splits = std::max(1, std::min(std::min(by_sm, by_k), 64));
  }
  const size_t B = max_batch, BH = B * hidden, BO = B * out_dim;
  const size_t LB = M->ldb;
  M->lparts = ((out_dim + TBN - 1) / TBN) * ((max_batch + TBM - 1) / TBM);
  int rc = 0;
  rc = rc ? rc : dalloc(M, &M->p, M->nparam);
  rc = rc ? rc : dalloc(M, &M->g, M->nparam);
  rc = rc ? rc : dalloc(M, &M->m1, M->nparam);
  rc = rc ? rc : dalloc(M, &M->m2, M->nparam);
  rc = rc ? rc : dalloc(M, &M->w1t, (size_t)hidden * M->ldi);
  rc = rc ? rc : dalloc(M, &M->w2, (size_t)hidden * M->ldh);
  rc = rc ? rc : dalloc(M, &M->w2t, (size_t)hidden * M->ldh);
  rc = rc ? rc : dalloc(M, &M->w3, (size_t)hidden * M->ldo);
  rc = rc ? rc : dalloc(M, &M->w3t, (size_t)out_dim * M->ldh);
  rc = rc ? rc : dalloc(M, &M->xb, B * M->ldi);
  rc = rc ? rc : dalloc(M, &M->xbT, (size_t)in_dim * LB);
  rc = rc ? rc : dalloc(M, &M->h1, B * M->ldh);
  rc = rc ? rc : dalloc(M, &M->h1T, (size_t)hidden * LB);
  rc = rc ? rc : dalloc(M, &M->h2, B * M->ldh);
  rc = rc ? rc : dalloc(M, &M->h2T, (size_t)hidden * LB);
  rc = rc ? rc : dalloc(M, &M->dyh, B * M->ldo);
  rc = rc ? rc : dalloc(M, &M->dyhT, (size_t)out_dim * LB);
  rc = rc ? rc : dalloc(M, &M->dz2h, B * M->ldh);
  rc = rc ? rc : dalloc(M, &M->dz2hT, (size_t)hidden * LB);
  rc = rc ? rc : dalloc(M, &M->dz1hT, (size_t)hidden * LB);
  rc = rc ? rc : dalloc(M, &M->xin, B * in_dim);
  rc = rc ? rc : dalloc(M, &M->y, BO);
  rc = rc ? rc : dalloc(M, &M->dy, BO);
  rc = rc ? rc : dalloc(M, &M->dz2, BH);
  rc = rc ? rc : dalloc(M, &M->dz1, BH);
  rc = rc ? rc : dalloc(M, &M->dh1, BH);
  rc = rc ? rc : dalloc(M, &M->part, BH * M->splits);
  rc = rc ? rc : dalloc(M, &M->lpart, (size_t)M->lparts);
  rc = rc ? rc : dalloc(M, &M->loss_dev, 1);
  rc = rc ? rc : dalloc(M, &M->mu, out_dim);
  rc = rc ? rc : dalloc(M, &M->sigma, out_dim);
  rc = rc ? rc : dalloc(M, &M->err, 1);
  if (rc) {
    free_mlp(M);
    return rc;
  }
  cudaMemsetAsync(M->m1, 0, sizeof(float) * M->nparam, M->stream);
  cudaMemsetAsync(M->m2, 0, sizeof(float) * M->nparam, M->stream);
  cudaMemsetAsync(M->p, 0, sizeof(float) * M->nparam, M->stream);
  cudaMemsetAsync(M->err, 0, sizeof(int), M->stream);
  // identity standardisation until data is set
  std::vector<float> zeros(out_dim, 0.0f), ones(out_dim, 1.0f);
  cudaMemcpyAsync(M->mu, zeros.data(), sizeof(float) * out_dim, cudaMemcpyHostToDevice, M->stream);
  cudaMemcpyAsync(M->sigma, ones.data(), sizeof(float) * out_dim, cudaMemcpyHostToDevice, M->stream);
  rc = refresh_weights(M);
  e = cudaStreamSynchronize(M->stream);
  if (rc || e != cudaSuccess) {
    free_mlp(M);
    return rc ? rc : set_error(PDLP_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = M;
  return PDLP_OK;
}

int64_t pdlp_mlp_param_count(const pdlp_mlp *M) { return M ? (int64_t)M->nparam : 0; }

int pdlp_mlp_set_params(pdlp_mlp *M, const float *params) {
  if (!M || !params) return set_error(PDLP_ERR_INVALID, "pdlp_mlp_set_params: null argument");
  MCK(cudaSetDevice(M->device));
  MCK(cudaMemcpyAsync(M->p, params, sizeof(float) * M->nparam, cudaMemcpyHostToDevice, M->stream));
  MCK(cudaMemsetAsync(M->m1, 0, sizeof(float) * M->nparam, M->stream));
  MCK(cudaMemsetAsync(M->m2, 0, sizeof(float) * M->nparam, M->stream));
  M->adam_t = 0;
  int rc = refresh_weights(M);
  if (rc) return rc;
  MCK(cudaStreamSynchronize(M->stream));
  return PDLP_OK;
}

int pdlp_mlp_get_params(const pdlp_mlp *M, float *params) {
  if (!M || !params) return set_error(PDLP_ERR_INVALID, "pdlp_mlp_get_params: null argument");
  MCK(cudaSetDevice(M->device));
  MCK(cudaMemcpyAsync(params, M->p, sizeof(float) * M->nparam, cudaMemcpyDeviceToHost, M->stream));
  MCK(cudaStreamSynchronize(M->stream));
  return PDLP_OK;
}

int pdlp_mlp_set_data(pdlp_mlp *M, int32_t samples, const float *X, const float *T) {
  if (!M || samples < 1 || !X || !T) return set_error(PDLP_ERR_INVALID, "pdlp_mlp_set_data: need samples >= 1 and data");
  MCK(cudaSetDevice(M->device));
  if (samples > M->samples) {
    int rc = dalloc(M, &M->X, (size_t)samples * M->in);
    if (!rc) rc = dalloc(M, &M->T, (size_t)samples * M->out);
    if (rc) return rc;
  }
  M->samples = samples;
  MCK(cudaMemcpyAsync(M->X, X, sizeof(float) * (size_t)samples * M->in, cudaMemcpyHostToDevice, M->stream));
  MCK(cudaMemcpyAsync(M->T, T, sizeof(float) * (size_t)samples * M->out, cudaMemcpyHostToDevice, M->stream));
  k_mean_std<<<grid1(M->out), 256, 0, M->stream>>>(M->T, samples, M->out, M->mu, M->sigma);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(M->stream));
  return PDLP_OK;
}

int pdlp_mlp_train(pdlp_mlp *M, int32_t steps, int32_t batch, const int32_t *idx, float lr, float beta1, float beta2,
                   float eps, float *losses) {
  if (!M || steps < 1 || batch < 1 || batch > M->maxb || !idx || M->samples < 1)
    return set_error(PDLP_ERR_INVALID, "pdlp_mlp_train: need data, steps >= 1, 1 <= batch <= max_batch, indices");
  for (long long i = 0; i < (long long)steps * batch; ++i)
    if (idx[i] < 0 || idx[i] >= M->samples) return set_error(PDLP_ERR_INVALID, "pdlp_mlp_train: index out of range");
  MCK(cudaSetDevice(M->device));
  int rc = ensure_idx(M, (size_t)steps * batch);
  if (rc) return rc;
  float *dloss = nullptr;
  rc = dalloc(M, &dloss, steps);
  if (rc) return rc;
  cudaStream_t s = M->stream;
  MCK(cudaMemcpyAsync(M->idx, idx, sizeof(int) * (size_t)steps * batch, cudaMemcpyHostToDevice, s));
  for (int st = 0; st < steps; ++st) {
    const int *rows = M->idx + (size_t)st * batch;
    k_gather<<<batch, 64, 0, s>>>(M->X, rows, batch, M->in, M->xb, M->ldi, M->xbT, M->ldb);
    MCK(cudaGetLastError());
    rc = forward_backward(M, batch, rows);
    if (rc) return rc;
    MCK(cudaMemcpyAsync(dloss + st, M->loss_dev, sizeof(float), cudaMemcpyDeviceToDevice, s));
    ++M->adam_t;
    const float c1 = 1.0f - powf(beta1, (float)M->adam_t), c2 = 1.0f - powf(beta2, (float)M->adam_t);
    k_adam<<<grid1(M->nparam), 256, 0, s>>>(M->p, M->g, M->m1, M->m2, M->nparam, lr, beta1, beta2, eps, c1, c2);
    MCK(cudaGetLastError());
    rc = refresh_weights(M);
    if (rc) return rc;
  }
  if (losses) MCK(cudaMemcpyAsync(losses, dloss, sizeof(float) * steps, cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  // free the per-call loss buffer
  cudaFree(dloss);
  M->allocs.pop_back();
  return check_err(M);
}

int pdlp_mlp_predict(pdlp_mlp *M, int32_t count, const float *X, float *Y) {
  if (!M || count < 1 || !X || !Y) return set_error(PDLP_ERR_INVALID, "pdlp_mlp_predict: null argument or count < 1");
  MCK(cudaSetDevice(M->device));
  cudaStream_t s = M->stream;
  for (int b0 = 0; b0 < count; b0 += M->maxb) {
    const int B = std::min(M->maxb, count - b0);
    MCK(cudaMemcpyAsync(M->xin, X + (size_t)b0 * M->in, sizeof(float) * (size_t)B * M->in, cudaMemcpyHostToDevice, s));
    k_input_bf16<<<grid1((size_t)B * M->in), 256, 0, s>>>(M->xin, B, M->in, M->xb, M->ldi);
    int rc = forward_hidden(M, B);
    if (!rc)
      rc = gemm(M, B, M->out, M->hid, 1, M->h2, M->ldh, M->w3t, M->ldh, EpiOut{{}, M->p + M->ob3, M->y, M->out, vec4(M->y, M->out)});
    if (rc) return rc;
    k_unstandardize<<<grid1((size_t)B * M->out), 256, 0, s>>>(M->y, (size_t)B * M->out, M->out, M->mu, M->sigma,
                                                               M->dy);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(Y + (size_t)b0 * M->out, M->dy, sizeof(float) * (size_t)B * M->out, cudaMemcpyDeviceToHost,
                        s));
  }
  MCK(cudaStreamSynchronize(s));
  return check_err(M);
}

int pdlp_mlp_gradients(pdlp_mlp *M, int32_t batch, const int32_t *idx, float *loss, float *grads) {
  if (M) {
    const char *ev = std::getenv("PDLP_TEST_GEMM_STALL");
    M->stall_next = (ev && ev[0] == '1') ? 1 : 0;
  }
  if (!M || batch < 1 || batch > M->maxb || !idx || M->samples < 1)
    return set_error(PDLP_ERR_INVALID, "pdlp_mlp_gradients: need data and 1 <= batch <= max_batch");
  for (int i = 0; i < batch; ++i)
    if (idx[i] < 0 || idx[i] >= M->samples) return set_error(PDLP_ERR_INVALID, "pdlp_mlp_gradients: index out of range");
  MCK(cudaSetDevice(M->device));
  int rc = ensure_idx(M, batch);
  if (rc) return rc;
  cudaStream_t s = M->stream;
  MCK(cudaMemcpyAsync(M->idx, idx, sizeof(int) * batch, cudaMemcpyHostToDevice, s));
  k_gather<<<batch, 64, 0, s>>>(M->X, M->idx, batch, M->in, M->xb, M->ldi, M->xbT, M->ldb);
  rc = forward_backward(M, batch, M->idx);
  if (rc) return rc;
  if (loss) MCK(cudaMemcpyAsync(loss, M->loss_dev, sizeof(float), cudaMemcpyDeviceToHost, s));
  if (grads) MCK(cudaMemcpyAsync(grads, M->g, sizeof(float) * M->nparam, cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  return check_err(M);
}

int pdlp_mlp_stats(const pdlp_mlp *M, float *mu, float *sigma) {
  if (!M) return set_error(PDLP_ERR_INVALID, "pdlp_mlp_stats: null argument");
  MCK(cudaSetDevice(M->device));
  if (mu) MCK(cudaMemcpy(mu, M->mu, sizeof(float) * M->out, cudaMemcpyDeviceToHost));
  if (sigma) MCK(cudaMemcpy(sigma, M->sigma, sizeof(float) * M->out, cudaMemcpyDeviceToHost));
  return PDLP_OK;
}

void pdlp_mlp_destroy(pdlp_mlp *M) {
  if (!M) return;
  cudaSetDevice(M->device);
  cudaStreamSynchronize(M->stream);
  free_mlp(M);
}

}  // extern "C"
