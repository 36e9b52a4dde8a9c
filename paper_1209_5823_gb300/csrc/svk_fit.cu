// svk_fit.cu -- Optimal Image Subtraction least-squares fit of the kernel coefficients
// (Sec. 2: least squares on Eq. 1 over isolated-star stamps, the kernel decomposed on the
// basis, each coefficient a polynomial in the frame coordinates).
//
// Model at a stamp pixel p:  sum_k sum_t c[k][t] m_t(p) C_k(p) + sum_j g_j m_j(p),
// C_k = R (x) B_k.  Normal equations A c = b with A = sum w v v^T, b = sum w v I.
//
// 1. fit_ck_kernel     C_k at every stamp pixel, FP32 (one thread per pixel).
// 2. fit_gram_kernel   FP64 weighted moments over the extended columns
//                      E = [C_0 .. C_{N-1}, I, 1]:
//                        S[e1][e2][mu] = sum_p w E_e1 E_e2 mu(p)
//                      for every monomial mu of degree <= 2 max(d, d_bg).  Every entry of
//                      A and b is one of these moments (m_t m_t' = mu_{t+t'}), so the
//                      per-pixel work is (N+2)(N+3)/2 products x n_mu FMAs instead of M^2.
// 3. fit_assemble      A, b from S.
// 4. fit_cholesky      FP64 Cholesky (left-looking, one CTA); the first non-positive pivot
//                      is reported in info and the solve is skipped.
// 5. fit_solve         forward / backward substitution.
// 6. fit_chi2_kernel   chi^2 = sum w (model - I)^2 at the solution, a direct second pass.
#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
namespace {

constexpr int kMaxMu = 28;  // monomials of degree <= 6
constexpr int kChunk = 32;  // pixels staged per step in the moment kernel

__host__ __device__ inline int mono_index(int i, int j, int D) {  // (i outer, j inner)
  return i * (D + 1) - i * (i - 1) / 2 + j;
}

struct FitDims {
  int W, H, pitch, S, n_stamps, N, L, d, bd, T, Tb, M, D, n_mu, NE, P;  // P = stamp pixels
};

__device__ inline double norm_coord(int x, int W) {
  return W > 1 ? (2.0 * (double)x - (double)(W - 1)) / (double)(W - 1) : 0.0;
}

__device__ inline void stamp_pixel(const FitDims &f, const int *stamp_xy, int p, int &x, int &y) {
  const int s = p / (f.S * f.S), q = p % (f.S * f.S), hs = (f.S - 1) / 2;
  x = stamp_xy[2 * s] - hs + q % f.S;
  y = stamp_xy[2 * s + 1] - hs + q / f.S;
}

// C[p][k] = sum_{u,v} B_k(u,v) R(x - u, y - v), zero outside the frame (FP32)
__global__ void fit_ck_kernel(const float *__restrict__ R, const float *__restrict__ basis, const int *stamp_xy,
                              FitDims f, float *__restrict__ C) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= f.P) return;
  int x, y;
  stamp_pixel(f, stamp_xy, p, x, y);
  const int h = (f.L - 1) / 2, LL = f.L * f.L;
  const bool inside = x >= 0 && x < f.W && y >= 0 && y < f.H;
  for (int k = 0; k < f.N; ++k) {
    float acc = 0.0f;
    if (inside) {
      const float *bk = basis + (size_t)k * LL;
      for (int vi = 0; vi < f.L; ++vi) {
        const int yy = y - (vi - h);
        if (yy < 0 || yy >= f.H) continue;
        const float *rrow = R + (size_t)yy * f.pitch;
        for (int ui = 0; ui < f.L; ++ui) {
          const int xx = x - (ui - h);
          if (xx >= 0 && xx < f.W) acc = fmaf(bk[vi * f.L + ui], __ldg(rrow + xx), acc);
        }
      }
    }
    C[(size_t)p * f.N + k] = acc;
  }
}

// S[(e1 * NE + e2) * n_mu + mu] += sum over this CTA's pixels of w E_e1 E_e2 mu(p)
// (e1 <= e2).  Thread = one column pair; CTA = one pixel range x one pair tile.
__global__ void __launch_bounds__(256) fit_gram_kernel(const float *__restrict__ C, const float *__restrict__ I,
                                                       const float *__restrict__ weight, const int *stamp_xy, FitDims f,
                                                       int px_per_cta, double *__restrict__ S) {
  __shared__ float Es[kChunk][66];          // extended columns of the staged pixels (NE <= 66)
  __shared__ double Ms[kChunk][kMaxMu];     // w * mu(p)
  const int npairs = f.NE * (f.NE + 1) / 2;
  const int pair = blockIdx.y * blockDim.x + threadIdx.x;
  int e1 = 0, e2 = 0;
  if (pair < npairs) {  // unrank the pair (e1 <= e2), row-major over e1
    int rem = pair;
    e1 = 0;
    while (rem >= f.NE - e1) {
      rem -= f.NE - e1;
      ++e1;
    }
    e2 = e1 + rem;
  }
  double acc[kMaxMu];
#pragma unroll
  for (int m = 0; m < kMaxMu; ++m) acc[m] = 0.0;
  const int p0 = blockIdx.x * px_per_cta, p1 = min(f.P, p0 + px_per_cta);
  for (int pc = p0; pc < p1; pc += kChunk) {
    __syncthreads();
    for (int i = threadIdx.x; i < kChunk * f.NE; i += blockDim.x) {
      const int q = i / f.NE, e = i % f.NE, p = pc + q;
      float v = 0.0f;
      if (p < p1) {
        int x, y;
        stamp_pixel(f, stamp_xy, p, x, y);
        const bool inside = x >= 0 && x < f.W && y >= 0 && y < f.H;
        if (inside) {
          if (e < f.N) v = C[(size_t)p * f.N + e];
          else if (e == f.N) v = I[(size_t)y * f.pitch + x];
          else v = 1.0f;
        }
      }
      Es[q][e] = v;
    }
    for (int q = threadIdx.x; q < kChunk; q += blockDim.x) {
      const int p = pc + q;
      double w = 0.0, xt = 0.0, yt = 0.0;
      if (p < p1) {
        int x, y;
        stamp_pixel(f, stamp_xy, p, x, y);
        if (x >= 0 && x < f.W && y >= 0 && y < f.H) {
          w = weight ? (double)weight[(size_t)y * f.pitch + x] : 1.0;
          xt = norm_coord(x, f.W);
          yt = norm_coord(y, f.H);
        }
      }
      double xi = w;
      for (int i = 0; i <= f.D; ++i) {
        double v = xi;
        for (int j = 0; j <= f.D - i; ++j) {
          Ms[q][mono_index(i, j, f.D)] = v;
          v *= yt;
        }
        xi *= xt;
      }
    }
    __syncthreads();
    if (pair < npairs) {
      const int nq = min(kChunk, p1 - pc);
      for (int q = 0; q < nq; ++q) {
        const double e = (double)Es[q][e1] * (double)Es[q][e2];
#pragma unroll
        for (int m = 0; m < kMaxMu; ++m)
          if (m < f.n_mu) acc[m] = fma(e, Ms[q][m], acc[m]);
      }
    }
  }
  if (pair < npairs) {
    double *dst = S + ((size_t)e1 * f.NE + e2) * f.n_mu;
#pragma unroll
    for (int m = 0; m < kMaxMu; ++m)
      if (m < f.n_mu) atomicAdd(dst + m, acc[m]);
  }
}

__device__ inline double moment(const double *S, const FitDims &f, int e1, int e2, int mu) {
  if (e1 > e2) {
    const int t = e1;
    e1 = e2;
    e2 = t;
  }
  return S[((size_t)e1 * f.NE + e2) * f.n_mu + mu];
}

// Unknown u -> (column, monomial exponents): kernel terms k*T + t, then background terms.
__device__ inline void unknown(const FitDims &f, int u, int &col, int &ei, int &ej) {
  int t, D;
  if (u < f.N * f.T) {
    col = u / f.T;
    t = u % f.T;
    D = f.d;
  } else {
    col = f.N + 1;  // the constant column
    t = u - f.N * f.T;
    D = f.bd;
  }
  int i = 0;
  while (t > D - i) {
    t -= D - i + 1;
    ++i;
  }
  ei = i;
  ej = t;
}

__global__ void fit_assemble_kernel(const double *S, FitDims f, double *A, double *b) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < f.M * f.M) {
    const int r = idx / f.M, c = idx % f.M;
    int c1, i1, j1, c2, i2, j2;
    unknown(f, r, c1, i1, j1);
    unknown(f, c, c2, i2, j2);
    A[idx] = moment(S, f, c1, c2, mono_index(i1 + i2, j1 + j2, f.D));
  }
  if (idx < f.M) {
    int c1, i1, j1;
    unknown(f, idx, c1, i1, j1);
    b[idx] = moment(S, f, c1, f.N, mono_index(i1, j1, f.D));
  }
}

__device__ double block_sum_d(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// Left-looking Cholesky in place (lower triangle of row-major A), one CTA; *info = -1 on
// success, else the first column whose pivot is not positive.
__global__ void __launch_bounds__(1024) fit_cholesky_kernel(double *A, int M, int *info) {
  __shared__ double red[32];
  __shared__ double piv;
  __shared__ int fail;
  if (threadIdx.x == 0) fail = -1;
  for (int j = 0; j < M; ++j) {
    double part = 0.0;
    const double *rj = A + (size_t)j * M;
    for (int k = threadIdx.x; k < j; k += blockDim.x) part = fma(rj[k], rj[k], part);
    const double s = block_sum_d(part, red);
    if (threadIdx.x == 0) {
      const double dd = rj[j] - s;
      if (!(dd > 0.0)) fail = j;
      else piv = sqrt(dd);
    }
    __syncthreads();
    if (fail >= 0) break;
    const double gjj = piv;
    if (threadIdx.x == 0) A[(size_t)j * M + j] = gjj;
    for (int i = j + 1 + threadIdx.x; i < M; i += blockDim.x) {
      const double *ri = A + (size_t)i * M;
      double acc = ri[j];
      for (int k = 0; k < j; ++k) acc = fma(-ri[k], rj[k], acc);
      A[(size_t)i * M + j] = acc / gjj;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *info = fail;
}

// G G^T x = b (G from fit_cholesky_kernel); skipped, leaving x = 0, when info >= 0.
__global__ void __launch_bounds__(1024) fit_solve_kernel(const double *G, const double *b, int M, const int *info,
                                                         double *x) {
  __shared__ double red[32];
  if (*info >= 0) {
    for (int i = threadIdx.x; i < M; i += blockDim.x) x[i] = 0.0;
    return;
  }
  for (int i = 0; i < M; ++i) {  // forward: G y = b
    double part = 0.0;
    for (int k = threadIdx.x; k < i; k += blockDim.x) part = fma(G[(size_t)i * M + k], x[k], part);
    const double s = block_sum_d(part, red);
    if (threadIdx.x == 0) x[i] = (b[i] - s) / G[(size_t)i * M + i];
    __syncthreads();
  }
  for (int i = M - 1; i >= 0; --i) {  // backward: G^T x = y
    double part = 0.0;
    for (int k = i + 1 + threadIdx.x; k < M; k += blockDim.x) part = fma(G[(size_t)k * M + i], x[k], part);
    const double s = block_sum_d(part, red);
    if (threadIdx.x == 0) x[i] = (x[i] - s) / G[(size_t)i * M + i];
    __syncthreads();
  }
}

__global__ void fit_chi2_kernel(const float *__restrict__ C, const float *__restrict__ I, const float *__restrict__ weight,
                                const int *stamp_xy, FitDims f, const double *coef, const int *info, double *chi2) {
  __shared__ double red[32];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (p < f.P && *info < 0) {
    int x, y;
    stamp_pixel(f, stamp_xy, p, x, y);
    if (x >= 0 && x < f.W && y >= 0 && y < f.H) {
      const double xt = norm_coord(x, f.W), yt = norm_coord(y, f.H);
      double model = 0.0;
      for (int k = 0; k < f.N; ++k) {
        double ak = 0.0, xi = 1.0;
        int t = 0;
        for (int i = 0; i <= f.d; ++i) {
          double yj = 1.0;
          for (int j = 0; j <= f.d - i; ++j, ++t) {
            ak = fma(coef[k * f.T + t], xi * yj, ak);
            yj *= yt;
          }
          xi *= xt;
        }
        model = fma(ak, (double)C[(size_t)p * f.N + k], model);
      }
      double xi = 1.0;
      int t = 0;
      for (int i = 0; i <= f.bd; ++i) {
        double yj = 1.0;
        for (int j = 0; j <= f.bd - i; ++j, ++t) {
          model = fma(coef[f.N * f.T + t], xi * yj, model);
          yj *= yt;
        }
        xi *= xt;
      }
      const double r = model - (double)I[(size_t)y * f.pitch + x];
      r2 = (weight ? (double)weight[(size_t)y * f.pitch + x] : 1.0) * r * r;
    }
  }
  const double s = block_sum_d(r2, red);
  if (threadIdx.x == 0) atomicAdd(chi2, s);
}

FitDims dims(int W, int H, int pitch, int n_stamps, int S, int N, int L, int d, int bd) {
  FitDims f;
  f.W = W;
  f.H = H;
  f.pitch = pitch;
  f.S = S;
  f.n_stamps = n_stamps;
  f.N = N;
  f.L = L;
  f.d = d;
  f.bd = bd;
  f.T = n_terms(d);
  f.Tb = n_terms(bd);
  f.M = N * f.T + f.Tb;
  f.D = 2 * (d > bd ? d : bd);
  f.n_mu = n_terms(f.D);
  f.NE = N + 2;
  f.P = n_stamps * S * S;
  return f;
}

struct FitLayout {
  size_t C, S, A, b, total;
};

FitLayout layout(const FitDims &f) {
  FitLayout l;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 255) & ~size_t(255);
    return at;
  };
  l.C = take((size_t)f.P * f.N * sizeof(float));
  l.S = take((size_t)f.NE * f.NE * f.n_mu * sizeof(double));
  l.A = take((size_t)f.M * f.M * sizeof(double));
  l.b = take((size_t)f.M * sizeof(double));
  l.total = o;
  return l;
}

}  // namespace

size_t fit_workspace_size(int n_stamps, int stamp_size, int N, int L, int degree, int bg_degree) {
  if (n_stamps < 1 || stamp_size < 1 || N < 1 || degree < 0 || degree > 3 || bg_degree < -1 || bg_degree > 3) return 0;
  return layout(dims(1, 1, 1, n_stamps, stamp_size, N, L, degree, bg_degree)).total;
}

int launch_fit(const float *R, const float *I, int W, int H, int pitch, const int *stamp_xy, int n_stamps,
               int stamp_size, const float *basis, int N, int L, int degree, int bg_degree, const float *weight,
               double *coeffs_out, double *chi2_out, int *info_out, void *ws, size_t ws_bytes, cudaStream_t s) {
  const FitDims f = dims(W, H, pitch, n_stamps, stamp_size, N, L, degree, bg_degree);
  if (f.NE > 66) return set_error(SVK_ERR_UNSUPPORTED, "fit supports N <= 64 basis stamps (got %d)", N);
  const FitLayout l = layout(f);
  if (!ws || ws_bytes < l.total) return set_error(SVK_ERR_WORKSPACE, "fit workspace too small");
  unsigned char *w = static_cast<unsigned char *>(ws);
  float *C = reinterpret_cast<float *>(w + l.C);
  double *S = reinterpret_cast<double *>(w + l.S);
  double *A = reinterpret_cast<double *>(w + l.A);
  double *b = reinterpret_cast<double *>(w + l.b);
  cudaError_t e = cudaMemsetAsync(S, 0, (size_t)f.NE * f.NE * f.n_mu * sizeof(double), s);
  if (e == cudaSuccess && chi2_out) e = cudaMemsetAsync(chi2_out, 0, sizeof(double), s);
  if (e != cudaSuccess) return cuda_status(e, "fit memset");
  fit_ck_kernel<<<(f.P + 127) / 128, 128, 0, s>>>(R, basis, stamp_xy, f, C);
  const int npairs = f.NE * (f.NE + 1) / 2;
  const int px_per_cta = 4096;
  dim3 ggrid((f.P + px_per_cta - 1) / px_per_cta, (npairs + 255) / 256);
  fit_gram_kernel<<<ggrid, 256, 0, s>>>(C, I, weight, stamp_xy, f, px_per_cta, S);
  fit_assemble_kernel<<<(f.M * f.M + 255) / 256, 256, 0, s>>>(S, f, A, b);
  fit_cholesky_kernel<<<1, 1024, 0, s>>>(A, f.M, info_out);
  fit_solve_kernel<<<1, 1024, 0, s>>>(A, b, f.M, info_out, coeffs_out);
  if (chi2_out) fit_chi2_kernel<<<(f.P + 255) / 256, 256, 0, s>>>(C, I, weight, stamp_xy, f, coeffs_out, info_out, chi2_out);
  return cuda_status(cudaGetLastError(), "fit kernels launch");
}

}  // namespace svk
