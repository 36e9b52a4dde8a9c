// svk_basis.cu -- tabulation of the basis stamps B_k of Eq. 2 on the device (FP64
// arithmetic, float32 storage): the Gaussian function basis (Gaussian x monomial
// stamps, Alard & Lupton) and the Dirac delta function basis (one stamp per kernel
// pixel, Miller et al.), Sec. 2.
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

// Block-wide FP64 sum (blockDim.x multiple of 32, <= 1024).
__device__ double block_sum(double v, double *scratch) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += scratch[i];
  return s;
}

// One CTA per stamp k.  For SVK_NORM_ALARD every CTA also rebuilds B_0 to make the
// even-even stamps zero-sum, so no CTA depends on another.
__global__ void gauss_basis_kernel(int L, GaussList gl, int normalize, float *out) {
  extern __shared__ double sm[];
  const int LL = L * L, h = (L - 1) / 2;
  double *b0 = sm, *bk = sm + LL, *red = sm + 2 * LL;
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
  const double s0 = 2.0 * gl.sigma[0] * gl.sigma[0], sg = 2.0 * gl.sigma[g] * gl.sigma[g];
  for (int i = threadIdx.x; i < LL; i += blockDim.x) {
    const int u = i % L - h, v = i / L - h;
    const double r2 = (double)(u * u + v * v);
    b0[i] = exp(-r2 / s0);
    bk[i] = exp(-r2 / sg) * ipow_d((double)u, p) * ipow_d((double)v, q);
  }
  __syncthreads();
  if (normalize == SVK_NORM_ALARD) {
    double part = 0.0;
    for (int i = threadIdx.x; i < LL; i += blockDim.x) part += b0[i];
    const double sum0 = block_sum(part, red);
    for (int i = threadIdx.x; i < LL; i += blockDim.x) b0[i] = b0[i] / sum0;
    __syncthreads();
    if (k == 0) {
      for (int i = threadIdx.x; i < LL; i += blockDim.x) out[i] = (float)b0[i];
      return;
    }
    if ((p % 2) == 0 && (q % 2) == 0) {
      part = 0.0;
      for (int i = threadIdx.x; i < LL; i += blockDim.x) part += bk[i];
      const double sk = block_sum(part, red);
      for (int i = threadIdx.x; i < LL; i += blockDim.x) bk[i] -= sk * b0[i];
      __syncthreads();
    }
    part = 0.0;
    for (int i = threadIdx.x; i < LL; i += blockDim.x) part += bk[i] * bk[i];
    const double n2 = block_sum(part, red);
    const double nrm = sqrt(n2);
    if (nrm > 0.0)
      for (int i = threadIdx.x; i < LL; i += blockDim.x) bk[i] /= nrm;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < LL; i += blockDim.x) out[(size_t)k * LL + i] = (float)bk[i];
}

__global__ void delta_basis_kernel(int L, int normalize, float *out) {
  const int LL = L * L, c = (LL - 1) / 2;
  const size_t n = (size_t)LL * LL;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / LL), i = (int)(e % LL);
    float v = (i == k) ? 1.0f : 0.0f;
    if (normalize == SVK_NORM_ALARD && k != c && i == c) v = -1.0f;
    out[e] = v;
  }
}

}  // namespace

int launch_build_basis(int kind, int L, int n_gauss, const double *sigma, const int *deg, int normalize,
                       float *basis_out, int N, cudaStream_t s) {
  if (kind == SVK_BASIS_DELTA) {
    const size_t n = (size_t)L * L * L * L;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    delta_basis_kernel<<<blocks, 256, 0, s>>>(L, normalize, basis_out);
    return cuda_status(cudaGetLastError(), "delta_basis_kernel launch");
  }
  GaussList gl{};
  gl.n = n_gauss;
  for (int g = 0; g < n_gauss; ++g) {
    gl.sigma[g] = sigma[g];
    gl.deg[g] = deg[g];
  }
  const size_t smem = (size_t)(2 * L * L + 32) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(gauss_basis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e, "gauss_basis_kernel smem attribute");
  gauss_basis_kernel<<<N, 256, smem, s>>>(L, gl, normalize, basis_out);
  return cuda_status(cudaGetLastError(), "gauss_basis_kernel launch");
}

}  // namespace svk
