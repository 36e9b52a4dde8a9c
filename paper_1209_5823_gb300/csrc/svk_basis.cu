// svk_basis.cu -- tabulation of the basis stamps B_k of Eq. 2 on the device (FP64
// arithmetic, float32 storage): the Gaussian function basis (Gaussian x monomial
// stamps, Alard & Lupton) and the Dirac delta function basis (one stamp per kernel
// pixel, Miller et al.), Sec. 2.
#include <cuda_fp16.h>

#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
namespace {

constexpr int kMaxGauss = 16;

struct GaussList {
  double sigma[kMaxGauss];
  int deg[kMaxGauss];
  int n;
};

__device__ double ipow_d(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

// Block-wide FP64 sums of two values at once (blockDim.x a multiple of 32, <= 1024): a
// shuffle tree in each warp, the warps' partials added by a shuffle tree in warp 0 (short
// dependent chains: FP64 adds are slow on this part), the result broadcast.
__device__ void block_sum2(double &a, double &b, double (*scratch)[32]) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) {
    scratch[0][w] = a;
    scratch[1][w] = b;
  }
  __syncthreads();
  if (w == 0) {
    double x = l < nw ? scratch[0][l] : 0.0, y = l < nw ? scratch[1][l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    __syncwarp();
    if (l == 0) {
      scratch[0][0] = x;
      scratch[1][0] = y;
    }
  }
  __syncthreads();
  a = scratch[0][0];
  b = scratch[1][0];
  __syncthreads();  // the scratch is reused by the next call
}

constexpr int kBasisThreads = 256, kBasisPer = 16;  // 16 x 256 >= 63 x 63 taps

// One CTA per stamp k, the stamp's taps in registers (tap i = threadIdx.x + 256 j).  For
// SVK_NORM_ALARD every CTA also evaluates B_0 (its sum normalises B_0 and makes the
// even-even stamps zero-sum), so no CTA depends on another; two block reductions: the sums
// of B_0 and B_k, then the squared norm of the corrected B_k.
__global__ void __launch_bounds__(kBasisThreads) gauss_basis_kernel(int L, GaussList gl, int normalize, float *out) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  __shared__ double red[2][32];
  const int LL = L * L, h = (L - 1) / 2;
  const int k = blockIdx.x;
  int g = 0, p = 0, q = 0, idx = k;
  for (g = 0; g < gl.n; ++g) {
    const int nt = (gl.deg[g] + 1) * (gl.deg[g] + 2) / 2;
    if (idx < nt) break;
    idx -= nt;
  }
  for (p = 0; p <= gl.deg[g]; ++p) {
    const int nq = gl.deg[g] - p + 1;
    if (idx < nq) {
      q = idx;
      break;
    }
    idx -= nq;
  }
  // the stamps are separable, exp(-(u^2 + v^2) / s) u^p v^q = fu(u) fv(v): one FP64 exp per
  // offset and Gaussian, and per tap two multiplies (FP64 is GB300's slow pipe)
  __shared__ double e0[64], fu[64], fv[64];
  if (threadIdx.x < 128) {  // warps 0-1 the first Gaussian, warps 2-3 the stamp's (in parallel)
    const int t = threadIdx.x & 63;
    if (t < L) {
      const double u = (double)(t - h);
      if (threadIdx.x < 64) {
        e0[t] = exp(-(u * u) / (2.0 * gl.sigma[0] * gl.sigma[0]));
      } else {
        const double eg = exp(-(u * u) / (2.0 * gl.sigma[g] * gl.sigma[g]));
        fu[t] = eg * ipow_d(u, p);
        fv[t] = eg * ipow_d(u, q);
      }
    }
  }
  __syncthreads();
  double b0[kBasisPer], bk[kBasisPer];
  double sum0 = 0.0, sumk = 0.0;
#pragma unroll
  for (int j = 0; j < kBasisPer; ++j) {
    const int i = threadIdx.x + kBasisThreads * j;
    b0[j] = 0.0;
    bk[j] = 0.0;
    if (i < LL) {
      const int iu = i % L, iv = i / L;
      b0[j] = e0[iu] * e0[iv];
      bk[j] = fu[iu] * fv[iv];
    }
    sum0 += b0[j];
    sumk += bk[j];
  }
  if (normalize == SVK_NORM_ALARD) {
    block_sum2(sum0, sumk, red);
    const double inv0 = 1.0 / sum0;
    if (k == 0) {
#pragma unroll
      for (int j = 0; j < kBasisPer; ++j) {
        const int i = threadIdx.x + kBasisThreads * j;
        if (i < LL) out[i] = (float)(b0[j] * inv0);
      }
      return;
    }
    const bool even = (p % 2) == 0 && (q % 2) == 0;
    double n2 = 0.0, unused = 0.0;
#pragma unroll
    for (int j = 0; j < kBasisPer; ++j) {
      if (even) bk[j] -= sumk * (b0[j] * inv0);
      n2 += bk[j] * bk[j];
    }
    block_sum2(n2, unused, red);
    const double nrm = sqrt(n2);
    const double inv = nrm > 0.0 ? 1.0 / nrm : 1.0;
#pragma unroll
    for (int j = 0; j < kBasisPer; ++j) bk[j] *= inv;
  }
#pragma unroll
  for (int j = 0; j < kBasisPer; ++j) {
    const int i = threadIdx.x + kBasisThreads * j;
    if (i < LL) out[(size_t)k * LL + i] = (float)bk[j];
  }
}

__global__ void delta_basis_kernel(int L, int normalize, float *out) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  const int LL = L * L, c = (LL - 1) / 2;
  const size_t n = (size_t)LL * LL;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / LL), i = (int)(e % LL);
    float v = (i == k) ? 1.0f : 0.0f;
    if (normalize == SVK_NORM_ALARD && k != c && i == c) v = -1.0f;
    out[e] = v;
  }
}

// v <- fp16(1024 v) / 1024 (round to nearest even), so that 1024 v is exactly an FP16 value.
__global__ void round_basis_fp16_kernel(float *__restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __half2float(__float2half_rn(b[i] * 1024.0f)) * (1.0f / 1024.0f);
}

}  // namespace

int launch_round_basis_fp16(float *basis, long long n, cudaStream_t s) {
  if (n <= 0) return SVK_OK;
  const long long blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  round_basis_fp16_kernel<<<(unsigned)blocks, 256, 0, s>>>(basis, n);
  return cuda_status(cudaGetLastError(), "round_basis_fp16_kernel launch");
}

int launch_build_basis(int kind, int L, int n_gauss, const double *sigma, const int *deg, int normalize,
                       float *basis_out, int N, cudaStream_t s) {
  if (kind == SVK_BASIS_DELTA) {
    const size_t n = (size_t)L * L * L * L;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    return cuda_status(launch_dependent(delta_basis_kernel, blocks, 256, 0, s, L, normalize, basis_out),
                       "delta_basis_kernel launch");
  }
  GaussList gl{};
  gl.n = n_gauss;
  for (int g = 0; g < n_gauss; ++g) {
    gl.sigma[g] = sigma[g];
    gl.deg[g] = deg[g];
  }
  if (L * L > kBasisThreads * kBasisPer) return set_error(SVK_ERR_ARG, "basis size %d above %d taps", L, 63);
  return cuda_status(launch_dependent(gauss_basis_kernel, N, kBasisThreads, 0, s, L, gl, normalize, basis_out),
                     "gauss_basis_kernel launch");
}

}  // namespace svk
