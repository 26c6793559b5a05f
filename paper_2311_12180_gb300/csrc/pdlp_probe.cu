// Device characterisation for the step kernels' rooflines (pdlp_probe_rates):
// the rate of random 8-byte gathers from an L2-resident vector, and the rate
// of FP64 fused multiply-adds.  These are the two on-chip resources the SpMV
// half-steps need besides HBM bandwidth: every stored nonzero costs one
// gather of x or y and one FMA (cuPDLP.jl paper, Sec. 3.3: the iteration is
// dominated by the two matrix-vector products).  Not part of the method.

#include <cuda_runtime.h>

#include "pdlp.h"
#include "pdlp_internal.cuh"

namespace pdlp {
namespace {

constexpr int PT = 256;

// splitmix64 of the counter: the probe's random indices
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void k_probe_fill(int32_t *idx, long long count, int32_t n, double *x) {
  for (long long e = (long long)blockIdx.x * PT + threadIdx.x; e < count; e += (long long)gridDim.x * PT)
    idx[e] = (int32_t)(mix64((unsigned long long)e) % (unsigned long long)n);
  for (long long j = (long long)blockIdx.x * PT + threadIdx.x; j < n; j += (long long)gridDim.x * PT)
    x[j] = (double)(j & 1023);
}

// Each thread takes chunks of 8 consecutive indices (two 16-byte loads) and
// issues their 8 gathers at once; the loaded bits are folded into one word
// per thread so that nothing is optimised away.
__global__ void __launch_bounds__(PT, 4) k_probe_gather(const int32_t *__restrict__ idx, long long chunks,
                                                        const double *__restrict__ x,
                                                        unsigned long long *__restrict__ out) {
  unsigned long long h = 0;
  for (long long ch = (long long)blockIdx.x * PT + threadIdx.x; ch < chunks; ch += (long long)gridDim.x * PT) {
    const int4 a = __ldcs(reinterpret_cast<const int4 *>(idx) + 2 * ch);
    const int4 b = __ldcs(reinterpret_cast<const int4 *>(idx) + 2 * ch + 1);
    const int c[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    double g[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) g[k] = __ldg(x + c[k]);
#pragma unroll
    for (int k = 0; k < 8; ++k) h ^= (unsigned long long)__double_as_longlong(g[k]);
  }
  out[(size_t)blockIdx.x * PT + threadIdx.x] = h;
}

// The same gathers with an SpMV's matrix stream beside them: each thread's
// chunk of 8 entries also streams their 8 FP64 values (4 x 16-byte loads)
// and multiplies-adds them into one FP64 sum, so per entry it moves what a
// sliced-ELL row does -- a 4-byte index, an 8-byte value, a 32-byte sector
// of x -- with one FMA.
__global__ void __launch_bounds__(PT, 4) k_probe_gather_stream(const int32_t *__restrict__ idx,
                                                               const double *__restrict__ val, long long chunks,
                                                               const double *__restrict__ x,
                                                               double *__restrict__ out) {
  double acc = 0.0;
  for (long long ch = (long long)blockIdx.x * PT + threadIdx.x; ch < chunks; ch += (long long)gridDim.x * PT) {
    const int4 a = __ldcs(reinterpret_cast<const int4 *>(idx) + 2 * ch);
    const int4 b = __ldcs(reinterpret_cast<const int4 *>(idx) + 2 * ch + 1);
    const int c[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    double v[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 w = __ldcs(reinterpret_cast<const double2 *>(val) + 4 * ch + k);
      v[2 * k] = w.x;
      v[2 * k + 1] = w.y;
    }
    double g[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) g[k] = __ldg(x + c[k]);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc = fma(v[k], g[k], acc);
  }
  out[(size_t)blockIdx.x * PT + threadIdx.x] = acc;
}

// Eight independent FMA chains per thread.
__global__ void __launch_bounds__(PT) k_probe_fma(double *out, int iters, double a) {
  double r[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) r[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = fma(r[k], a, 0.5);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += r[k];
  out[(size_t)blockIdx.x * PT + threadIdx.x] = s;
}

}  // namespace
}  // namespace pdlp

extern "C" int pdlp_probe_stream_gathers(double *gathers_per_s) {
  using namespace pdlp;
  if (!gathers_per_s) return set_error(PDLP_ERR_INVALID, "pdlp_probe_stream_gathers: null argument");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(PDLP_ERR_CUDA, cudaGetErrorString(e));
  const int32_t n = 1 << 21;         // 16 MB of FP64: L2-resident, far beyond L1
  const long long count = 20000000;  // entries (a multiple of 8)
  const int ggrid = 4 * sms;
  int32_t *idx = nullptr;
  double *x = nullptr, *val = nullptr, *go = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMalloc((void **)&idx, sizeof(int32_t) * count);
  if (e == cudaSuccess) e = cudaMalloc((void **)&val, sizeof(double) * count);
  if (e == cudaSuccess) e = cudaMalloc((void **)&x, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc((void **)&go, sizeof(double) * ggrid * PT);
  if (e == cudaSuccess) {
    k_probe_fill<<<1024, PT, 0, st>>>(idx, count, n, x);
    e = cudaMemsetAsync(val, 0, sizeof(double) * count, st);
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) {  // warm-up
      k_probe_gather_stream<<<ggrid, PT, 0, st>>>(idx, val, count / 8, x, go);
      e = cudaGetLastError();
    }
  }
  const int reps = 10;
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    k_probe_gather_stream<<<ggrid, PT, 0, st>>>(idx, val, count / 8, x, go);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (st) cudaStreamSynchronize(st);
  if (idx) cudaFree(idx);
  if (val) cudaFree(val);
  if (x) cudaFree(x);
  if (go) cudaFree(go);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) return set_error(PDLP_ERR_CUDA, cudaGetErrorString(e));
  *gathers_per_s = (double)count * reps / (1e-3 * ms);
  return PDLP_OK;
}

extern "C" int pdlp_probe_rates(double *gathers_per_s, double *dfma_per_s) {
  using namespace pdlp;
  if (!gathers_per_s || !dfma_per_s) return set_error(PDLP_ERR_INVALID, "pdlp_probe_rates: null argument");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(PDLP_ERR_CUDA, cudaGetErrorString(e));
  const int32_t n = 1 << 21;             // 16 MB of FP64: L2-resident, far beyond L1
  const long long count = 20000000;      // gathers (a multiple of 8)
  const int ggrid = 4 * sms, fgrid = 8 * sms, iters = 4096;
  int32_t *idx = nullptr;
  double *x = nullptr, *fo = nullptr;
  unsigned long long *go = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms_g = 0.f, ms_f = 0.f;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMalloc((void **)&idx, sizeof(int32_t) * count);
  if (e == cudaSuccess) e = cudaMalloc((void **)&x, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc((void **)&go, sizeof(unsigned long long) * ggrid * PT);
  if (e == cudaSuccess) e = cudaMalloc((void **)&fo, sizeof(double) * fgrid * PT);
  if (e == cudaSuccess) {
    k_probe_fill<<<1024, PT, 0, st>>>(idx, count, n, x);
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) {  // warm-up
      k_probe_gather<<<ggrid, PT, 0, st>>>(idx, count / 8, x, go);
      k_probe_fma<<<fgrid, PT, 0, st>>>(fo, 64, 0.999);
      e = cudaGetLastError();
    }
  }
  const int reps = 10;
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    k_probe_gather<<<ggrid, PT, 0, st>>>(idx, count / 8, x, go);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_g, e0, e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) k_probe_fma<<<fgrid, PT, 0, st>>>(fo, iters, 0.999);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_f, e0, e1);
  if (st) cudaStreamSynchronize(st);
  if (idx) cudaFree(idx);
  if (x) cudaFree(x);
  if (go) cudaFree(go);
  if (fo) cudaFree(fo);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) return set_error(PDLP_ERR_CUDA, cudaGetErrorString(e));
  *gathers_per_s = (double)count * reps / (1e-3 * ms_g);
  *dfma_per_s = (double)fgrid * PT * iters * 8.0 / (1e-3 * ms_f);
  return PDLP_OK;
}
