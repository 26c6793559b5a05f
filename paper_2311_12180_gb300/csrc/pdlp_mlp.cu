// BF16 multilayer perceptron for learned warm starts of parametric LPs:
// theta (in) -> hidden -> ReLU -> hidden -> ReLU -> out, trained with MSE on
// per-output standardised targets by Adam with FP32 master weights.
//
// Mixed precision: weights and activations feed the GEMMs in BF16, products
// accumulate in FP32 on the tensor cores (wmma m16n16k16 BF16 -> FP32), the
// output layer, the loss, all gradients and the Adam state stay FP32, and the
// output gradient is rounded to BF16 only as a GEMM operand.  Every step
// (gather of a mini-batch, forward, loss, backward, Adam) is a kernel here;
// the host only passes the mini-batch indices (random numbers drawn by the
// caller) and launches.  Split-K partial sums and column sums are reduced in
// a fixed order, so training is deterministic.

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pdlp.h"
#include "pdlp_internal.cuh"

namespace pdlp {
namespace mlp {

using bf16 = __nv_bfloat16;
namespace wm = nvcuda::wmma;

constexpr int BM = 64, BN = 64, BK = 32, GT = 128;  // GEMM tile, 4 warps of 32 x 32
constexpr int LDA_S = BK + 8, LDB_S = BN + 8, LDC_S = BN + 4;

// C(m, n) = sum_k A(m, k) B(k, n) over k in [k0, k1), A / B in BF16, FP32
// accumulation; A(m, k) at A[m * lda + k] (row) or A[k * lda + m] (A_COL);
// B(k, n) at B[k * ldb + n] (row) or B[n * ldb + k] (B_COL).  The K range of
// split s = blockIdx.z is [s * kchunk, min(K, (s + 1) * kchunk)).  The
// finished tile goes through epi(m, n, value, split).
template <bool A_COL, bool B_COL, class Epi>
__global__ void __launch_bounds__(GT) k_gemm(int M, int N, int K, int kchunk, const bf16 *__restrict__ A, int lda,
                                             const bf16 *__restrict__ B, int ldb, Epi epi) {
  __shared__ __align__(32) bf16 As[BM][LDA_S];
  __shared__ __align__(32) bf16 Bs[BK][LDB_S];
  __shared__ __align__(32) float Cs[BM][LDC_S];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  const int warp = threadIdx.x >> 5, wm_ = warp >> 1, wn_ = warp & 1;
  wm::fragment<wm::accumulator, 16, 16, 16, float> acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) wm::fill_fragment(acc[i][j], 0.0f);
  const bf16 zero = __float2bfloat16(0.0f);
  for (int k0 = kb; k0 < ke; k0 += BK) {
    // A tile: BM x BK
    for (int t = threadIdx.x; t < BM * BK; t += GT) {
      int r, c;
      if (A_COL) {
        r = t % BM;
        c = t / BM;
      } else {
        r = t / BK;
        c = t % BK;
      }
      const int m = m0 + r, k = k0 + c;
      bf16 v = zero;
      if (m < M && k < ke) v = A_COL ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
      As[r][c] = v;
    }
    // B tile: BK x BN
    for (int t = threadIdx.x; t < BK * BN; t += GT) {
      int r, c;
      if (B_COL) {
        r = t % BK;
        c = t / BK;
      } else {
        r = t / BN;
        c = t % BN;
      }
      const int k = k0 + r, n = n0 + c;
      bf16 v = zero;
      if (k < ke && n < N) v = B_COL ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
      Bs[r][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      wm::fragment<wm::matrix_a, 16, 16, 16, bf16, wm::row_major> fa[2];
      wm::fragment<wm::matrix_b, 16, 16, 16, bf16, wm::row_major> fb[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) wm::load_matrix_sync(fa[i], &As[wm_ * 32 + i * 16][kk], LDA_S);
#pragma unroll
      for (int j = 0; j < 2; ++j) wm::load_matrix_sync(fb[j], &Bs[kk][wn_ * 32 + j * 16], LDB_S);
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) wm::mma_sync(acc[i][j], fa[i], fb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
      wm::store_matrix_sync(&Cs[wm_ * 32 + i * 16][wn_ * 32 + j * 16], acc[i][j], LDC_S, wm::mem_row_major);
  __syncthreads();
  for (int t = threadIdx.x; t < BM * BN; t += GT) {
    const int r = t / BN, c = t % BN;
    const int m = m0 + r, n = n0 + c;
    if (m < M && n < N) epi(m, n, Cs[r][c], blockIdx.z);
  }
}

// ---- epilogues ----
struct EpiBiasReluBF16 {  // hidden layer: H = bf16(relu(z + b))
  const float *bias;
  bf16 *out;
  int ld;
  __device__ void operator()(int m, int n, float v, int) const {
    const float z = v + bias[n];
    out[(size_t)m * ld + n] = __float2bfloat16(z > 0.0f ? z : 0.0f);
  }
};
struct EpiBiasF32 {  // output layer: Y = z + b
  const float *bias;
  float *out;
  int ld;
  __device__ void operator()(int m, int n, float v, int) const { out[(size_t)m * ld + n] = v + bias[n]; }
};
struct EpiStoreF32 {  // weight gradient
  float *out;
  int ld;
  __device__ void operator()(int m, int n, float v, int) const { out[(size_t)m * ld + n] = v; }
};
struct EpiPartial {  // split-K partial sums, summed later in split order
  float *part;
  int ld;
  size_t stride;
  __device__ void operator()(int m, int n, float v, int s) const { part[s * stride + (size_t)m * ld + n] = v; }
};

// dH (sum of split partials, in split order), masked by the ReLU of the
// layer's output H: dZ = dH where H > 0.  Writes FP32 and BF16 copies.
__global__ void k_splitk_relu_grad(const float *__restrict__ part, int splits, size_t count,
                                   const bf16 *__restrict__ H, float *__restrict__ dz, bf16 *__restrict__ dzh) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int k = 0; k < splits; ++k) s += part[k * count + i];
    const float g = __bfloat162float(H[i]) > 0.0f ? s : 0.0f;
    dz[i] = g;
    dzh[i] = __float2bfloat16(g);
  }
}

// dH with the mask of H, from a single FP32 product (no split).
__global__ void k_relu_grad(const float *__restrict__ dh, size_t count, const bf16 *__restrict__ H,
                            float *__restrict__ dz, bf16 *__restrict__ dzh) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float g = __bfloat162float(H[i]) > 0.0f ? dh[i] : 0.0f;
    dz[i] = g;
    dzh[i] = __float2bfloat16(g);
  }
}

// Mini-batch gather: inputs to BF16, targets (FP32) of the sampled rows.
__global__ void k_gather(const float *__restrict__ X, const float *__restrict__ T, const int *__restrict__ idx,
                         int batch, int in_dim, int out_dim, bf16 *__restrict__ xb, float *__restrict__ tb) {
  const int b = blockIdx.y;
  if (b >= batch) return;
  const size_t row = (size_t)idx[b];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < out_dim; i += gridDim.x * blockDim.x)
    tb[(size_t)b * out_dim + i] = T[row * out_dim + i];
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < in_dim; i += blockDim.x) xb[(size_t)b * in_dim + i] = __float2bfloat16(X[row * in_dim + i]);
}

__global__ void k_to_bf16(const float *__restrict__ x, size_t count, bf16 *__restrict__ y) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// MSE on standardised targets: d = y - (t - mu) / sigma; dY = 2 d / (B N).
// Per-block partial sums of d^2 (summed in block order by k_loss_finish).
__global__ void k_loss(const float *__restrict__ y, const float *__restrict__ t, const float *__restrict__ mu,
                       const float *__restrict__ sigma, int batch, int out_dim, float *__restrict__ dy,
                       bf16 *__restrict__ dyh, double *__restrict__ part) {
  __shared__ double red[32];
  const size_t count = (size_t)batch * out_dim;
  const float scale = 2.0f / (float)count;
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(i % out_dim);
    const float d = y[i] - (t[i] - mu[o]) / sigma[o];
    acc += (double)d * d;
    const float g = scale * d;
    dy[i] = g;
    dyh[i] = __float2bfloat16(g);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

__global__ void k_loss_finish(const double *__restrict__ part, int nparts, size_t count, float *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += part[i];
    *out = (float)(s / (double)count);
  }
}

// out[n] = sum over rows of X[rows x cols] (fixed row order): bias gradients.
__global__ void k_colsum(const float *__restrict__ X, int rows, int cols, float *__restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += X[(size_t)r * cols + c];
    out[c] = s;
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

// Adam on the FP32 master copy; refreshes the BF16 copy the GEMMs read.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, bf16 *__restrict__ ph, size_t count, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float mh = a / c1, vh = b / c2;
    const float v = p[i] - lr * mh / (sqrtf(vh) + eps);
    p[i] = v;
    ph[i] = __float2bfloat16(v);
  }
}

int grid1(size_t n, int bs = 256) {
  size_t g = (n + bs - 1) / bs;
  if (g > 65535 * 4) g = 65535 * 4;
  return (int)(g < 1 ? 1 : g);
}

template <bool AC, bool BC, class Epi>
cudaError_t gemm(int M, int N, int K, int splits, const bf16 *A, int lda, const bf16 *B, int ldb, Epi epi,
                 cudaStream_t s) {
  const int kchunk = ((K + splits - 1) / splits + BK - 1) / BK * BK;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
  k_gemm<AC, BC, Epi><<<grid, GT, 0, s>>>(M, N, K, kchunk, A, lda, B, ldb, epi);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace pdlp

// ================================================================ host side

using namespace pdlp;
using namespace pdlp::mlp;

struct pdlp_mlp {
  int device = 0;
  int in = 0, hid = 0, out = 0, maxb = 0, splits = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t nparam = 0, oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
  bf16 *ph = nullptr;
  // activations / gradients for one mini-batch
  bf16 *xb = nullptr, *h1 = nullptr, *h2 = nullptr, *dyh = nullptr, *dz2h = nullptr, *dz1h = nullptr;
  float *xin = nullptr, *tb = nullptr, *y = nullptr, *dy = nullptr, *dz2 = nullptr, *dz1 = nullptr, *dh1 = nullptr, *part = nullptr;
  double *lpart = nullptr;
  float *loss_dev = nullptr, *mu = nullptr, *sigma = nullptr;
  // data set
  float *X = nullptr, *T = nullptr;
  int samples = 0;
  int *idx = nullptr;
  size_t idx_cap = 0;
  long long adam_t = 0;
  std::vector<void *> allocs;
};

namespace {

constexpr int LOSS_BLOCKS = 512;

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

// forward of rows [0, B) of xb (BF16 inputs) -> y (FP32, standardised units)
int forward(pdlp_mlp *M, int B) {
  cudaStream_t s = M->stream;
  MCK(gemm<false, false>(B, M->hid, M->in, 1, M->xb, M->in, M->ph + M->oW1, M->hid,
                         EpiBiasReluBF16{M->p + M->ob1, M->h1, M->hid}, s));
  MCK(gemm<false, false>(B, M->hid, M->hid, 1, M->h1, M->hid, M->ph + M->oW2, M->hid,
                         EpiBiasReluBF16{M->p + M->ob2, M->h2, M->hid}, s));
  MCK(gemm<false, false>(B, M->out, M->hid, 1, M->h2, M->hid, M->ph + M->oW3, M->out,
                         EpiBiasF32{M->p + M->ob3, M->y, M->out}, s));
  return PDLP_OK;
}

// loss + gradients of every parameter into M->g for the batch in xb / tb
int backward(pdlp_mlp *M, int B) {
  cudaStream_t s = M->stream;
  const size_t BO = (size_t)B * M->out, BH = (size_t)B * M->hid;
  k_loss<<<LOSS_BLOCKS, 256, 0, s>>>(M->y, M->tb, M->mu, M->sigma, B, M->out, M->dy, M->dyh, M->lpart);
  MCK(cudaGetLastError());
  k_loss_finish<<<1, 32, 0, s>>>(M->lpart, LOSS_BLOCKS, BO, M->loss_dev);
  // output layer
  MCK(gemm<true, false>(M->hid, M->out, B, 1, M->h2, M->hid, M->dyh, M->out, EpiStoreF32{M->g + M->oW3, M->out}, s));
  k_colsum<<<grid1(M->out), 256, 0, s>>>(M->dy, B, M->out, M->g + M->ob3);
  MCK(gemm<false, true>(B, M->hid, M->out, M->splits, M->dyh, M->out, M->ph + M->oW3, M->out,
                        EpiPartial{M->part, M->hid, BH}, s));
  k_splitk_relu_grad<<<grid1(BH), 256, 0, s>>>(M->part, M->splits, BH, M->h2, M->dz2, M->dz2h);
  // second layer
  MCK(gemm<true, false>(M->hid, M->hid, B, 1, M->h1, M->hid, M->dz2h, M->hid, EpiStoreF32{M->g + M->oW2, M->hid}, s));
  k_colsum<<<grid1(M->hid), 256, 0, s>>>(M->dz2, B, M->hid, M->g + M->ob2);
  MCK(gemm<false, true>(B, M->hid, M->hid, 1, M->dz2h, M->hid, M->ph + M->oW2, M->hid, EpiStoreF32{M->dh1, M->hid}, s));
  k_relu_grad<<<grid1(BH), 256, 0, s>>>(M->dh1, BH, M->h1, M->dz1, M->dz1h);
  // first layer
  MCK(gemm<true, false>(M->in, M->hid, B, 1, M->xb, M->in, M->dz1h, M->hid, EpiStoreF32{M->g + M->oW1, M->hid}, s));
  k_colsum<<<grid1(M->hid), 256, 0, s>>>(M->dz1, B, M->hid, M->g + M->ob1);
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

}  // namespace

extern "C" {

int pdlp_mlp_create(pdlp_mlp **out, int32_t in_dim, int32_t hidden, int32_t out_dim, int32_t max_batch, void *stream) {
  if (!out || in_dim < 1 || hidden < 1 || out_dim < 1 || max_batch < 1)
    return set_error(PDLP_ERR_INVALID, "pdlp_mlp_create: dimensions and max_batch must be >= 1");
  if (max_batch > 65535 || (int64_t)in_dim * hidden > INT32_MAX || (int64_t)hidden * out_dim > INT32_MAX)
    return set_error(PDLP_ERR_INVALID, "pdlp_mlp_create: max_batch above 65535 or a weight matrix above 2^31 entries");
  pdlp_mlp *M = new pdlp_mlp();
  M->in = in_dim;
  M->hid = hidden;
  M->out = out_dim;
  M->maxb = max_batch;
  // split the long reduction (over the outputs) of dH2 = dY W3' so the GEMM
  // has enough CTAs: about 4 splits per 2048 outputs, at most 64
  M->splits = std::max(1, std::min(64, out_dim / 512));
  size_t o = 0;
  M->oW1 = o; o += (size_t)in_dim * hidden;
  M->ob1 = o; o += hidden;
  M->oW2 = o; o += (size_t)hidden * hidden;
  M->ob2 = o; o += hidden;
  M->oW3 = o; o += (size_t)hidden * out_dim;
  M->ob3 = o; o += out_dim;
  M->nparam = o;
  cudaError_t e = cudaGetDevice(&M->device);
  if (e == cudaSuccess) {
    if (stream) {
      M->stream = (cudaStream_t)stream;
    } else {
      e = cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking);
      M->own_stream = true;
    }
  }
  if (e != cudaSuccess) {
    free_mlp(M);
    return set_error(PDLP_ERR_CUDA, cudaGetErrorString(e));
  }
  const size_t B = max_batch, BH = B * hidden, BO = B * out_dim;
  int rc = 0;
  rc = rc ? rc : dalloc(M, &M->p, M->nparam);
  rc = rc ? rc : dalloc(M, &M->g, M->nparam);
  rc = rc ? rc : dalloc(M, &M->m1, M->nparam);
  rc = rc ? rc : dalloc(M, &M->m2, M->nparam);
  rc = rc ? rc : dalloc(M, &M->ph, M->nparam);
  rc = rc ? rc : dalloc(M, &M->xb, B * in_dim);
  rc = rc ? rc : dalloc(M, &M->h1, BH);
  rc = rc ? rc : dalloc(M, &M->h2, BH);
  rc = rc ? rc : dalloc(M, &M->dyh, BO);
  rc = rc ? rc : dalloc(M, &M->dz2h, BH);
  rc = rc ? rc : dalloc(M, &M->dz1h, BH);
  rc = rc ? rc : dalloc(M, &M->xin, B * in_dim);
  rc = rc ? rc : dalloc(M, &M->tb, BO);
  rc = rc ? rc : dalloc(M, &M->y, BO);
  rc = rc ? rc : dalloc(M, &M->dy, BO);
  rc = rc ? rc : dalloc(M, &M->dz2, BH);
  rc = rc ? rc : dalloc(M, &M->dz1, BH);
  rc = rc ? rc : dalloc(M, &M->dh1, BH);
  rc = rc ? rc : dalloc(M, &M->part, BH * M->splits);
  rc = rc ? rc : dalloc(M, &M->lpart, LOSS_BLOCKS);
  rc = rc ? rc : dalloc(M, &M->loss_dev, 1);
  rc = rc ? rc : dalloc(M, &M->mu, out_dim);
  rc = rc ? rc : dalloc(M, &M->sigma, out_dim);
  if (rc) {
    free_mlp(M);
    return rc;
  }
  cudaMemsetAsync(M->m1, 0, sizeof(float) * M->nparam, M->stream);
  cudaMemsetAsync(M->m2, 0, sizeof(float) * M->nparam, M->stream);
  cudaMemsetAsync(M->p, 0, sizeof(float) * M->nparam, M->stream);
  cudaMemsetAsync(M->ph, 0, sizeof(bf16) * M->nparam, M->stream);
  // identity standardisation until data is set
  std::vector<float> zeros(out_dim, 0.0f), ones(out_dim, 1.0f);
  cudaMemcpyAsync(M->mu, zeros.data(), sizeof(float) * out_dim, cudaMemcpyHostToDevice, M->stream);
  cudaMemcpyAsync(M->sigma, ones.data(), sizeof(float) * out_dim, cudaMemcpyHostToDevice, M->stream);
  e = cudaStreamSynchronize(M->stream);
  if (e != cudaSuccess) {
    free_mlp(M);
    return set_error(PDLP_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = M;
  return PDLP_OK;
}

int64_t pdlp_mlp_param_count(const pdlp_mlp *M) { return M ? (int64_t)M->nparam : 0; }

int pdlp_mlp_set_params(pdlp_mlp *M, const float *params) {
  if (!M || !params) return set_error(PDLP_ERR_INVALID, "pdlp_mlp_set_params: null argument");
  MCK(cudaSetDevice(M->device));
  MCK(cudaMemcpyAsync(M->p, params, sizeof(float) * M->nparam, cudaMemcpyHostToDevice, M->stream));
  k_to_bf16<<<grid1(M->nparam), 256, 0, M->stream>>>(M->p, M->nparam, M->ph);
  MCK(cudaMemsetAsync(M->m1, 0, sizeof(float) * M->nparam, M->stream));
  MCK(cudaMemsetAsync(M->m2, 0, sizeof(float) * M->nparam, M->stream));
  M->adam_t = 0;
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
    dim3 gg((M->out + 255) / 256 < 64 ? (M->out + 255) / 256 : 64, batch);
    k_gather<<<gg, 256, 0, s>>>(M->X, M->T, M->idx + (size_t)st * batch, batch, M->in, M->out, M->xb, M->tb);
    MCK(cudaGetLastError());
    rc = forward(M, batch);
    if (!rc) rc = backward(M, batch);
    if (rc) return rc;
    MCK(cudaMemcpyAsync(dloss + st, M->loss_dev, sizeof(float), cudaMemcpyDeviceToDevice, s));
    ++M->adam_t;
    const float c1 = 1.0f - powf(beta1, (float)M->adam_t), c2 = 1.0f - powf(beta2, (float)M->adam_t);
    k_adam<<<grid1(M->nparam), 256, 0, s>>>(M->p, M->g, M->m1, M->m2, M->ph, M->nparam, lr, beta1, beta2, eps, c1, c2);
    MCK(cudaGetLastError());
  }
  if (losses) MCK(cudaMemcpyAsync(losses, dloss, sizeof(float) * steps, cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  // free the per-call loss buffer
  cudaFree(dloss);
  M->allocs.pop_back();
  return PDLP_OK;
}

int pdlp_mlp_predict(pdlp_mlp *M, int32_t count, const float *X, float *Y) {
  if (!M || count < 1 || !X || !Y) return set_error(PDLP_ERR_INVALID, "pdlp_mlp_predict: null argument or count < 1");
  MCK(cudaSetDevice(M->device));
  cudaStream_t s = M->stream;
  for (int b0 = 0; b0 < count; b0 += M->maxb) {
    const int B = std::min(M->maxb, count - b0);
    MCK(cudaMemcpyAsync(M->xin, X + (size_t)b0 * M->in, sizeof(float) * (size_t)B * M->in, cudaMemcpyHostToDevice, s));
    k_to_bf16<<<grid1((size_t)B * M->in), 256, 0, s>>>(M->xin, (size_t)B * M->in, M->xb);
    int rc = forward(M, B);
    if (rc) return rc;
    k_unstandardize<<<grid1((size_t)B * M->out), 256, 0, s>>>(M->y, (size_t)B * M->out, M->out, M->mu, M->sigma, M->dy);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(Y + (size_t)b0 * M->out, M->dy, sizeof(float) * (size_t)B * M->out, cudaMemcpyDeviceToHost, s));
  }
  MCK(cudaStreamSynchronize(s));
  return PDLP_OK;
}

int pdlp_mlp_gradients(pdlp_mlp *M, int32_t batch, const int32_t *idx, float *loss, float *grads) {
  if (!M || batch < 1 || batch > M->maxb || !idx || M->samples < 1)
    return set_error(PDLP_ERR_INVALID, "pdlp_mlp_gradients: need data and 1 <= batch <= max_batch");
  for (int i = 0; i < batch; ++i)
    if (idx[i] < 0 || idx[i] >= M->samples) return set_error(PDLP_ERR_INVALID, "pdlp_mlp_gradients: index out of range");
  MCK(cudaSetDevice(M->device));
  int rc = ensure_idx(M, batch);
  if (rc) return rc;
  cudaStream_t s = M->stream;
  MCK(cudaMemcpyAsync(M->idx, idx, sizeof(int) * batch, cudaMemcpyHostToDevice, s));
  dim3 gg((M->out + 255) / 256 < 64 ? (M->out + 255) / 256 : 64, batch);
  k_gather<<<gg, 256, 0, s>>>(M->X, M->T, M->idx, batch, M->in, M->out, M->xb, M->tb);
  rc = forward(M, batch);
  if (!rc) rc = backward(M, batch);
  if (rc) return rc;
  if (loss) MCK(cudaMemcpyAsync(loss, M->loss_dev, sizeof(float), cudaMemcpyDeviceToHost, s));
  if (grads) MCK(cudaMemcpyAsync(grads, M->g, sizeof(float) * M->nparam, cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  return PDLP_OK;
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
