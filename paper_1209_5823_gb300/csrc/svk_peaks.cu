// svk_peaks.cu -- measured FMA throughput of this GPU, the denominators of the rooflines
// of the direct form (FP32 FFMA, scalar or packed f32x2) and of the fit's normal
// equations (FP64 DFMA).
//
// Each thread runs eight independent multiply-add chains x <- x * a + b (|a| < 1, so the
// values stay bounded); 2 FLOP per multiply-add, two multiply-adds per packed f32x2
// instruction.  The grid is 8 blocks of 256 threads per SM, enough warps to cover the
// pipeline latency.
#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T *out, int iters, T a, T b) {
  T x0 = (T)threadIdx.x * (T)1e-6, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b);
    x1 = fma(x1, a, b);
    x2 = fma(x2, a, b);
    x3 = fma(x3, a, b);
    x4 = fma(x4, a, b);
    x5 = fma(x5, a, b);
    x6 = fma(x6, a, b);
    x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

// packed FP32: eight chains of f32x2 pairs, 16 multiply-adds per iteration
__global__ void __launch_bounds__(256) fma2_chains(float *out, int iters, float a, float b) {
  const float t = (float)threadIdx.x * 1e-6f;
  uint64_t x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = f2_pack(t + (float)c, t + (float)c + 0.5f);
  const uint64_t a2 = f2_pack(a, a), b2 = f2_pack(b, b);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = f2_fma(x[c], a2, b2);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float lo, hi;
    f2_unpack(x[c], lo, hi);
    s += lo + hi;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, bool PACKED = false>
int time_fma(int iters, double *flops_per_s, cudaStream_t s) {
  int dev = 0, sms = 0;
  int st = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (st == SVK_OK) st = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  if (st != SVK_OK) return st;
  const int blocks = sms * 8, threads = 256;
  ScopedWorkspace w;
  st = w.acquire((size_t)blocks * threads * sizeof(T), nullptr, 0, s);
  if (st != SVK_OK) return st;
  T *out = static_cast<T *>(w.ptr);
  cudaEvent_t e0, e1;
  if ((st = cuda_status(cudaEventCreate(&e0), "event")) != SVK_OK) return st;
  if ((st = cuda_status(cudaEventCreate(&e1), "event")) != SVK_OK) {
    cudaEventDestroy(e0);
    return st;
  }
  auto run = [&](int n) {
    if constexpr (PACKED) fma2_chains<<<blocks, threads, 0, s>>>(out, n, 0.999999f, 1e-6f);
    else fma_chains<T><<<blocks, threads, 0, s>>>(out, n, (T)0.999999, (T)1e-6);
  };
  run(iters / 4);  // warm-up
  cudaEventRecord(e0, s);
  run(iters);
  cudaEventRecord(e1, s);
  st = cuda_status(cudaEventSynchronize(e1), "FMA timing");
  float ms = 0.0f;
  if (st == SVK_OK) st = cuda_status(cudaEventElapsedTime(&ms, e0, e1), "elapsed time");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SVK_OK) return st;
  *flops_per_s = 2.0 * (PACKED ? 16.0 : 8.0) * (double)iters * blocks * threads / (ms * 1e-3);
  return SVK_OK;
}

}  // namespace

int measure_fma_peak(int kind, double *flops_per_s, cudaStream_t s) {
  // about 30 ms each at the nominal rates
  if (kind == 1) return time_fma<double>(1 << 14, flops_per_s, s);
  if (kind == 2) return time_fma<float, true>(1 << 19, flops_per_s, s);
  return time_fma<float>(1 << 20, flops_per_s, s);
}

}  // namespace svk
