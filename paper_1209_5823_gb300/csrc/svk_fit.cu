// svk_fit.cu -- Optimal Image Subtraction least-squares fit of the kernel coefficients
// (Sec. 2: least squares on Eq. 1 over isolated-star stamps, the kernel decomposed on the
// basis, each coefficient a polynomial in the frame coordinates).
//
// Model at a stamp pixel p:  sum_k sum_t c[k][t] m_t(p) C_k(p) + sum_j g_j m_j(p),
// C_k = R (x) B_k.  Normal equations A c = b with A = sum w v v^T, b = sum w v I.
//
// 1. fit_ck_kernel     C_k at every stamp pixel, FP32 (R patch and basis chunks staged in
//                      shared memory; 4 pixels x 7 stamps per thread).
// 2. fit_gram_kernel   FP64 weighted moments over the extended columns
//                      E = [C_0 .. C_{N-1}, I, 1]:
//                        S[e1][e2][mu] = sum_p w E_e1 E_e2 mu(p)
//                      for every monomial mu of degree <= 2 max(d, d_bg).  Every entry of
//                      A and b is one of these moments (m_t m_t' = mu_{t+t'}), so the
//                      per-pixel work is (N+2)(N+3)/2 products x n_mu FMAs instead of M^2.
// 3. fit_assemble      A, b from S.
// 4. chol_*            FP64 blocked Cholesky over the whole GPU; the first non-positive
//                      pivot is reported in info and the solve is skipped.
// 5. fit_solve         forward / backward substitution (one CTA).
// 6. fit_chi2_kernel   chi^2 = sum w (model - I)^2 at the solution, a direct second pass
//                      in double-float arithmetic.
#include <algorithm>

#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
namespace {

constexpr int kMaxMu = 28;  // monomials of degree <= 6
constexpr int kChunk = 64;  // pixels staged per step in the moment kernel

__host__ __device__ inline int mono_index(int i, int j, int D) {  // (i outer, j inner)
  return i * (D + 1) - i * (i - 1) / 2 + j;
}

struct FitDims {
  int W, H, pitch, S, n_stamps, N, L, d, bd, T, Tb, M, D, n_mu, NE, P;  // P = stamp pixels
  int r0, r1;  // frame rows [r0, r1) held by R, I and weight (row r at (r - r0) * pitch)
};

__device__ inline double norm_coord(int x, int W) {
  return W > 1 ? (2.0 * (double)x - (double)(W - 1)) / (double)(W - 1) : 0.0;
}

__device__ inline void stamp_pixel(const FitDims &f, const int *stamp_xy, int p, int &x, int &y) {
  const int s = p / (f.S * f.S), q = p % (f.S * f.S), hs = (f.S - 1) / 2;
  x = stamp_xy[2 * s] - hs + q % f.S;
  y = stamp_xy[2 * s + 1] - hs + q / f.S;
}

// C[p][k] = sum_{u,v} B_k(u,v) R(x - u, y - v), zero outside the frame (FP32).  CTA =
// one tile of `ty` rows of one stamp: the R patch the tile reads (its pixels plus the
// kernel halo, zero outside the frame) is staged in shared memory, the basis kCkStamps
// stamps at a time ([tap][8] rows, read as two float4 broadcasts).  Thread = 4 pixels
// (linear tile indices t, t + 256, ...), each with kCkStamps accumulators.
constexpr int kCkThreads = 256, kCkPix = 4, kCkStamps = 7;

int ck_tile_rows(int S) { return S >= kCkThreads * kCkPix ? 1 : (kCkThreads * kCkPix) / S; }

size_t ck_smem_bytes(int S, int L, int ty) {
  return ((size_t)(S + L - 1) * (ty + L - 1) + 3) / 4 * 16 + (size_t)L * L * 8 * sizeof(float);
}

__global__ void __launch_bounds__(kCkThreads) fit_ck_kernel(const float *__restrict__ R, const float *__restrict__ basis,
                                                            const int *stamp_xy, FitDims f, int ty, float *__restrict__ C) {
  extern __shared__ float4 ck_smem[];
  const int st = blockIdx.x, ty0 = blockIdx.y * ty, S = f.S, L = f.L, h = (L - 1) / 2, hs = (S - 1) / 2;
  const int rows = min(ty, S - ty0);
  if (rows <= 0) return;
  const int PW = S + L - 1, PH = rows + L - 1, LL = L * L;
  float *Rp = reinterpret_cast<float *>(ck_smem);
  float4 *Bs = ck_smem + (PW * PH + 3) / 4;  // [tap][2] float4 = 8 stamps (7 used)
  const int xs = stamp_xy[2 * st], ys = stamp_xy[2 * st + 1];
  const int ox = xs - hs - h, oy = ys - hs + ty0 - h;  // frame position of Rp[0][0]
  for (int e = threadIdx.x; e < PW * PH; e += blockDim.x) {
    const int gx = ox + e % PW, gy = oy + e / PW;
    Rp[e] = (gx >= 0 && gx < f.W && gy >= f.r0 && gy < f.r1) ? __ldg(R + (size_t)(gy - f.r0) * f.pitch + gx) : 0.0f;
  }
  int off[kCkPix];      // Rp index of tap (0, 0) for the pixel: (qy + 2h) * PW + qx + 2h
  int pglob[kCkPix];    // global stamp-pixel index, or -1
  bool inside[kCkPix];
#pragma unroll
  for (int m = 0; m < kCkPix; ++m) {
    const int q = threadIdx.x + kCkThreads * m;
    const int qy = q / S, qx = q % S;
    const bool valid = q < rows * S;
    off[m] = valid ? (qy + 2 * h) * PW + qx + 2 * h : 2 * h * PW + 2 * h;
    pglob[m] = valid ? st * S * S + (ty0 + qy) * S + qx : -1;
    const int x = xs - hs + qx, y = ys - hs + ty0 + qy;
    inside[m] = valid && x >= 0 && x < f.W && y >= 0 && y < f.H;
  }
  for (int k0 = 0; k0 < f.N; k0 += kCkStamps) {
    __syncthreads();  // the previous chunk is consumed (first time: the patch is staged)
    for (int e = threadIdx.x; e < LL * 8; e += blockDim.x) {
      const int tap = e >> 3, j = e & 7;
      reinterpret_cast<float *>(Bs)[e] = (j < kCkStamps && k0 + j < f.N) ? basis[(size_t)(k0 + j) * LL + tap] : 0.0f;
    }
    __syncthreads();
    float acc[kCkPix][kCkStamps];
#pragma unroll
    for (int m = 0; m < kCkPix; ++m)
#pragma unroll
      for (int j = 0; j < kCkStamps; ++j) acc[m][j] = 0.0f;
    for (int vi = 0; vi < L; ++vi) {
      const float4 *brow = Bs + vi * L * 2;
      const int rbase = -vi * PW;
#pragma unroll 2
      for (int ui = 0; ui < L; ++ui) {
        const float4 b0 = brow[2 * ui], b1 = brow[2 * ui + 1];
        const float bv[kCkStamps] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z};
#pragma unroll
        for (int m = 0; m < kCkPix; ++m) {
          const float r = Rp[off[m] + rbase - ui];
#pragma unroll
          for (int j = 0; j < kCkStamps; ++j) acc[m][j] = fmaf(bv[j], r, acc[m][j]);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < kCkPix; ++m)
      if (pglob[m] >= 0)
#pragma unroll
        for (int j = 0; j < kCkStamps; ++j)
          if (k0 + j < f.N) C[(size_t)pglob[m] * f.N + k0 + j] = inside[m] ? acc[m][j] : 0.0f;
  }
}

// S[(e1 * NE + e2) * n_mu + mu] += sum over this CTA's pixels of w E_e1 E_e2 mu(p)
// (e1 <= e2).  Thread = one column pair; CTA = one pixel range x one pair tile.  Pixels
// outside the frame, or outside the rows [r0, r1) the buffers hold, add nothing.
// The monomials mu = xt^i yt^j factor by rows: consecutive stamp pixels of one frame row
// share yt, so each thread sums R_i = sum w E xt^i over the pixels of the current row and
// adds R_i yt^j into the (i, j) moments when the row changes (once per run of at most a
// stamp width of pixels).  Everything runs on the FP32 pipe in double-float arithmetic
// (value = hi + lo, about 48 significant bits; GB300's FP64 rate is about 1/60 of its
// FP32 rate): E_e1 E_e2 is a product of two float32 values, exact as hi + lo with one FMA
// (Dekker/Knuth two-product); w xt^i and yt are split into hi + lo once per pixel; every
// addition is an error-free two-sum (Knuth), the rounding errors gathered in the lo part.
// Each CTA's moments (sums over a few dozen rows) are converted to FP64 for the atomic
// additions across CTAs.  The row sums are indexed for the largest degree (kMaxDeg) so
// that they stay in registers; the moments, touched once per row, sit in shared memory.
constexpr int kMaxDeg = 6;  // moment degree 2 max(d, bd)
constexpr int kGramThreads = 224;  // column pairs per CTA at most (1326 pairs = 6 x 221)
__host__ __device__ constexpr int idx6(int i, int j) { return i * (kMaxDeg + 1) - i * (i - 1) / 2 + j; }

// (h, l) += (eh + el) (wh + wl), the el wl term (about 2^-48 of the product) dropped
__device__ __forceinline__ void df_madd(float &h, float &l, float eh, float el, float wh, float wl) {
  const float th = eh * wh;
  float tl = fmaf(eh, wh, -th);
  tl = fmaf(eh, wl, tl);
  tl = fmaf(el, wh, tl);
  const float sum = h + th;           // two-sum of h and th
  const float bv = sum - h;
  const float err = (h - (sum - bv)) + (th - bv);
  l += err + tl;
  h = sum;
}

__global__ void __launch_bounds__(kGramThreads) fit_gram_kernel(const float *__restrict__ C, const float *__restrict__ I,
                                                       const float *__restrict__ weight, const int *stamp_xy, FitDims f,
                                                       int px_per_cta, double *__restrict__ S) {
  __shared__ float Es[kChunk][66];            // extended columns of the staged pixels (NE <= 66)
  // w xt^i = hi + lo (zero for i > D), as (hi_i, lo_i, hi_i+1, lo_i+1) quadruples: four
  // 16-byte loads per pixel instead of fourteen 4-byte ones (the loop is issue-bound)
  __shared__ float4 WX4[kChunk][(kMaxDeg + 2) / 2];
  __shared__ float Yth[kChunk], Ytl[kChunk];  // yt of the pixel's row, hi + lo
  __shared__ int Yv[kChunk];                  // its frame row, -1 for a pixel that adds nothing
  __shared__ int Ix[kChunk];                  // offset of its I value, -1 outside
  // the thread's moments, double-float (touched once per row): [moment][thread], so a
  // warp's accesses are consecutive
  __shared__ float accH[kMaxMu][kGramThreads], accL[kMaxMu][kGramThreads];
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
  float *aH = &accH[0][threadIdx.x], *aL = &accL[0][threadIdx.x];  // moment m at [m * kGramThreads]
#pragma unroll
  for (int m = 0; m < kMaxMu; ++m) aH[m * kGramThreads] = aL[m * kGramThreads] = 0.0f;
  // the current row's sums, double-float, in two independent sets (alternate pixels of a
  // row), so consecutive pixels' additions do not wait for each other
  float rh0[kMaxDeg + 1], rl0[kMaxDeg + 1], rh1[kMaxDeg + 1], rl1[kMaxDeg + 1];
#pragma unroll
  for (int i = 0; i <= kMaxDeg; ++i) rh0[i] = rl0[i] = rh1[i] = rl1[i] = 0.0f;
  int cur_y = -1;
  float cur_yh = 0.0f, cur_yl = 0.0f;
  auto flush = [&]() {  // the current row's sums R_i into the moments: M_ij += R_i yt^j
    float rh[kMaxDeg + 1], rl[kMaxDeg + 1];
#pragma unroll
    for (int i = 0; i <= kMaxDeg; ++i) {  // the two sets added (two-sum), renormalised
      const float sum = rh0[i] + rh1[i], bv = sum - rh0[i];
      const float lo = ((rh0[i] - (sum - bv)) + (rh1[i] - bv)) + (rl0[i] + rl1[i]);
      rh[i] = sum + lo;
      rl[i] = lo - (rh[i] - sum);
      rh0[i] = rl0[i] = rh1[i] = rl1[i] = 0.0f;
    }
    float yh = 1.0f, yl = 0.0f;  // yt^j, double-float
#pragma unroll
    for (int j = 0; j <= kMaxDeg; ++j) {
#pragma unroll
      for (int i = 0; i + j <= kMaxDeg; ++i) {
        const int m = idx6(i, j) * kGramThreads;
        float h = aH[m], l = aL[m];
        df_madd(h, l, rh[i], rl[i], yh, yl);
        aH[m] = h;
        aL[m] = l;
      }
      const float ph = yh * cur_yh;  // yt^(j+1) = yt^j yt
      const float pl = fmaf(yh, cur_yl, fmaf(yl, cur_yh, fmaf(yh, cur_yh, -ph)));
      yh = ph + pl;
      yl = pl - (yh - ph);
    }
  };
  const int p0 = blockIdx.x * px_per_cta, p1 = min(f.P, p0 + px_per_cta);
  for (int pc = p0; pc < p1; pc += kChunk) {
    __syncthreads();
    // per pixel once: position, weight and monomial factors; then the columns
    for (int q = threadIdx.x; q < kChunk; q += blockDim.x) {
      const int p = pc + q;
      double w = 0.0, xt = 0.0, yt = 0.0;
      int yv = -1, ix = -1;
      if (p < p1) {
        int x, y;
        stamp_pixel(f, stamp_xy, p, x, y);
        if (x >= 0 && x < f.W && y >= f.r0 && y < f.r1) {
          ix = (y - f.r0) * f.pitch + x;
          w = weight ? (double)weight[ix] : 1.0;
          xt = norm_coord(x, f.W);
          yt = norm_coord(y, f.H);
          yv = y;
        }
      }
      double v = w;
      float wx_h[kMaxDeg + 2], wx_l[kMaxDeg + 2];
#pragma unroll
      for (int i = 0; i <= kMaxDeg + 1; ++i) {
        const double wx = i <= f.D ? v : 0.0;
        wx_h[i] = (float)wx;
        wx_l[i] = (float)(wx - (double)wx_h[i]);
        v *= xt;
      }
#pragma unroll
      for (int i2 = 0; i2 < (kMaxDeg + 2) / 2; ++i2)
        WX4[q][i2] = make_float4(wx_h[2 * i2], wx_l[2 * i2], wx_h[2 * i2 + 1], wx_l[2 * i2 + 1]);
      Yth[q] = (float)yt;
      Ytl[q] = (float)(yt - (double)(float)yt);
      Yv[q] = yv;
      Ix[q] = ix;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kChunk * f.NE; i += blockDim.x) {
      const int q = i / f.NE, e = i % f.NE, ix = Ix[q];
      float v = 0.0f;
      if (ix >= 0) {
        if (e < f.N) v = C[(size_t)(pc + q) * f.N + e];
        else if (e == f.N) v = I[ix];
        else v = 1.0f;
      }
      Es[q][e] = v;
    }
    __syncthreads();
    if (pair < npairs) {
      const int nq = min(kChunk, p1 - pc);
      for (int q = 0; q < nq;) {
        const int yv = Yv[q];  // the same for every thread: uniform branches
        if (yv < 0) {
          ++q;
          continue;
        }
        if (yv != cur_y) {
          flush();
          cur_y = yv;
          cur_yh = Yth[q];
          cur_yl = Ytl[q];
        }
        const float a = Es[q][e1], c = Es[q][e2];
        const float eh = a * c, el = fmaf(a, c, -eh);  // E_e1 E_e2 = eh + el exactly
        if (q + 1 < nq && Yv[q + 1] == yv) {  // two pixels of the row, one per set
          const float a1 = Es[q + 1][e1], c1 = Es[q + 1][e2];
          const float eh1 = a1 * c1, el1 = fmaf(a1, c1, -eh1);
#pragma unroll
          for (int i2 = 0; i2 < (kMaxDeg + 2) / 2; ++i2) {
            if (2 * i2 > f.D) break;
            const float4 w0 = WX4[q][i2], w1 = WX4[q + 1][i2];
            df_madd(rh0[2 * i2], rl0[2 * i2], eh, el, w0.x, w0.y);
            df_madd(rh1[2 * i2], rl1[2 * i2], eh1, el1, w1.x, w1.y);
            if (2 * i2 + 1 <= f.D && 2 * i2 + 1 <= kMaxDeg) {
              df_madd(rh0[2 * i2 + 1], rl0[2 * i2 + 1], eh, el, w0.z, w0.w);
              df_madd(rh1[2 * i2 + 1], rl1[2 * i2 + 1], eh1, el1, w1.z, w1.w);
            }
          }
          q += 2;
        } else {
#pragma unroll
          for (int i2 = 0; i2 < (kMaxDeg + 2) / 2; ++i2) {
            if (2 * i2 > f.D) break;
            const float4 w0 = WX4[q][i2];
            df_madd(rh0[2 * i2], rl0[2 * i2], eh, el, w0.x, w0.y);
            if (2 * i2 + 1 <= f.D && 2 * i2 + 1 <= kMaxDeg) df_madd(rh0[2 * i2 + 1], rl0[2 * i2 + 1], eh, el, w0.z, w0.w);
          }
          ++q;
        }
      }
    }
  }
  if (pair < npairs) {
    flush();
    double *dst = S + ((size_t)e1 * f.NE + e2) * f.n_mu;
#pragma unroll
    for (int i = 0; i <= kMaxDeg; ++i)
#pragma unroll
      for (int j = 0; i + j <= kMaxDeg; ++j)
        if (i + j <= f.D)
          atomicAdd(dst + mono_index(i, j, f.D),
                    (double)aH[idx6(i, j) * kGramThreads] + (double)aL[idx6(i, j) * kGramThreads]);
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

// Blocked right-looking Cholesky in place (lower triangle of row-major A, M x M), panels
// of kPanel columns.  FP64 runs at a small fraction of the FP32 rate on this part, so the
// O(M^3) work is spread over the whole GPU: per panel p,
//   chol_diag_kernel    factors the kPanel x kPanel diagonal block in shared memory (one
//                       CTA) and reports the first non-positive pivot in *info;
//   chol_trsm_kernel    A[i][panel] <- A[i][panel] L_pp^-T for the rows below (one row per
//                       warp);
//   chol_update_kernel  A[i][j] -= sum_{k in panel} A[i][k] A[j][k] for the trailing lower
//                       triangle (32 x 32 tiles).
// Every kernel returns at once when *info >= 0 (an earlier pivot failed).
constexpr int kPanel = 64;

__global__ void __launch_bounds__(256) chol_diag_kernel(double *A, int M, int p, int *info) {
  // Right-looking, one column per step: thread 0 takes the pivot's square root and its
  // reciprocal (one FP64 division per column, not one per thread), the threads scale the
  // column, then update the trailing lower triangle on a 16 x 16 thread grid (rows ty + 16a,
  // columns tx + 16c: no index divisions).
  __shared__ double Ls[kPanel][kPanel + 1];
  __shared__ double pinv;
  __shared__ int fail;
  if (*info >= 0) return;
  const int b = min(kPanel, M - p);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int r = ty; r < b; r += 16)
    for (int c = tx; c < b; c += 16) Ls[r][c] = c <= r ? A[(size_t)(p + r) * M + p + c] : 0.0;
  if (threadIdx.x == 0) fail = -1;
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (threadIdx.x == 0) {
      const double d = Ls[j][j];
      if (!(d > 0.0)) {
        fail = p + j;
      } else {
        const double sd = sqrt(d);
        Ls[j][j] = sd;
        pinv = 1.0 / sd;
      }
    }
    __syncthreads();
    if (fail >= 0) break;
    const double inv = pinv;
    for (int i = j + 1 + threadIdx.x; i < b; i += blockDim.x) Ls[i][j] *= inv;
    __syncthreads();
    // rows r > j, columns j < c <= r
    const int r0 = j + 1 + ty, c0 = j + 1 + tx;
    for (int r = r0; r < b; r += 16) {
      const double lr = Ls[r][j];
      for (int c = c0; c <= r; c += 16) Ls[r][c] = fma(-lr, Ls[c][j], Ls[r][c]);
    }
    __syncthreads();
  }
  for (int r = ty; r < b; r += 16)
    for (int c = tx; c <= r; c += 16) A[(size_t)(p + r) * M + p + c] = Ls[r][c];
  if (threadIdx.x == 0 && fail >= 0) *info = fail;
}

__global__ void __launch_bounds__(256) chol_trsm_kernel(double *A, int M, int p, const int *info) {
  // One warp per row below the panel: x L_pp^T = a, column by column; lane l holds x[l] and
  // x[l + 32].  Step c: the owner's entry times 1 / L_cc is x_c (broadcast by a shuffle),
  // then every later entry k takes its -x_c L_kc (a multiply-add per lane, no reduction).
  __shared__ double Ls[kPanel][kPanel + 1];
  __shared__ double inv[kPanel];
  if (*info >= 0) return;
  const int b = min(kPanel, M - p);
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int r = e / b, c = e % b;
    Ls[r][c] = c <= r ? A[(size_t)(p + r) * M + p + c] : 0.0;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < b; c += blockDim.x) inv[c] = 1.0 / Ls[c][c];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = p + b + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= M) return;
  double *row = A + (size_t)i * M + p;
  double v0 = lane < b ? row[lane] : 0.0, v1 = lane + 32 < b ? row[lane + 32] : 0.0;
  for (int c = 0; c < b; ++c) {
    const double xc = __shfl_sync(0xffffffffu, c < 32 ? v0 : v1, c & 31) * inv[c];
    if (lane == (c & 31)) {
      if (c < 32) v0 = xc;
      else v1 = xc;
    }
    if (lane > c && lane < b) v0 = fma(-xc, Ls[lane][c], v0);
    if (lane + 32 > c && lane + 32 < b) v1 = fma(-xc, Ls[lane + 32][c], v1);
  }
  if (lane < b) row[lane] = v0;
  if (lane + 32 < b) row[lane + 32] = v1;
}

__global__ void __launch_bounds__(256) chol_update_kernel(double *A, int M, int p, const int *info) {
  __shared__ double Pi[32][kPanel + 1], Pj[32][kPanel + 1];
  if (*info >= 0) return;
  const int b = min(kPanel, M - p), q = p + b;
  // lower-triangular tile (ti >= tj) of the trailing matrix from the linear block index
  int t = blockIdx.x, ti = 0;
  while (t > ti) {
    t -= ti + 1;
    ++ti;
  }
  const int tj = t, i0 = q + 32 * ti, j0 = q + 32 * tj;
  for (int e = threadIdx.x; e < 32 * b; e += blockDim.x) {
    const int r = e / b, c = e % b;
    Pi[r][c] = i0 + r < M ? A[(size_t)(i0 + r) * M + p + c] : 0.0;
    Pj[r][c] = j0 + r < M ? A[(size_t)(j0 + r) * M + p + c] : 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x & 31, r0 = threadIdx.x >> 5;  // column j0 + c, rows i0 + r0 + 8 m
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < b; ++k) {
    const double pj = Pj[c][k];
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[m] = fma(Pi[r0 + 8 * m][k], pj, acc[m]);
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int i = i0 + r0 + 8 * m, j = j0 + c;
    if (i < M && j <= i) A[(size_t)i * M + j] -= acc[m];
  }
}

// G G^T x = b (G from the Cholesky kernels); skipped, leaving x = 0, when info >= 0.  One
// CTA: row i's dot product is split over the threads, reduced per warp and across warps.
__global__ void __launch_bounds__(256) fit_solve_kernel(const double *G, const double *b, int M, const int *info,
                                                        double *x) {
  // Column-oriented substitutions: thread t owns the entries k = t + 256 q (q < 4, M <=
  // 1024), kept in registers; each step is one multiply by the owner of entry i (the
  // diagonal's reciprocals formed in parallel first: FP64 division is slow on this part),
  // its value passed through shared memory with one barrier, and one multiply-add per owned
  // entry.  The entries of G a step needs do not depend on the solution, so each thread
  // loads the next step's while this one runs (an L2 read is not on the step's path).
  constexpr int kOwn = 4;
  __shared__ double inv[1024], val[2];
  if (*info >= 0) {
    for (int i = threadIdx.x; i < M; i += blockDim.x) x[i] = 0.0;
    return;
  }
  const int t = threadIdx.x;
  double v[kOwn], g[kOwn], gn[kOwn];
#pragma unroll
  for (int q = 0; q < kOwn; ++q) {
    const int k = t + 256 * q;
    v[q] = k < M ? b[k] : 0.0;
  }
  for (int k = t; k < M; k += blockDim.x) inv[k] = 1.0 / G[(size_t)k * M + k];
  // forward: G y = b; v_k <- v_k - G_ki y_i for k > i (column i of G).  Steps i in
  // [256 qo, 256 qo + 256) are owned through v[qo] (qo unrolled: no indexed register array)
#pragma unroll
  for (int q = 0; q < kOwn; ++q) {
    const int k = t + 256 * q;
    g[q] = (k > 0 && k < M) ? G[(size_t)k * M] : 0.0;
  }
  __syncthreads();
#pragma unroll
  for (int qo = 0; qo < kOwn; ++qo) {
    const int i_end = min(M, 256 * (qo + 1));
    for (int i = 256 * qo; i < i_end; ++i) {
#pragma unroll
      for (int q = 0; q < kOwn; ++q) {
        const int k = t + 256 * q;
        gn[q] = (i + 1 < M && k > i + 1 && k < M) ? G[(size_t)k * M + i + 1] : 0.0;
      }
      if ((i & 255) == t) {
        v[qo] *= inv[i];  // y_i
        val[i & 1] = v[qo];
      }
      __syncthreads();
      const double yi = val[i & 1];
#pragma unroll
      for (int q = 0; q < kOwn; ++q) {
        const int k = t + 256 * q;
        if (k > i && k < M) v[q] = fma(-g[q], yi, v[q]);
        g[q] = gn[q];
      }
    }
  }
  // backward: G^T x = y; v_k <- v_k - G_ik x_i for k < i (row i of G)
#pragma unroll
  for (int q = 0; q < kOwn; ++q) {
    const int k = t + 256 * q;
    g[q] = (k < M - 1) ? G[(size_t)(M - 1) * M + k] : 0.0;
  }
  __syncthreads();
#pragma unroll
  for (int qo = kOwn - 1; qo >= 0; --qo) {
    for (int i = min(M, 256 * (qo + 1)) - 1; i >= 256 * qo; --i) {
#pragma unroll
      for (int q = 0; q < kOwn; ++q) {
        const int k = t + 256 * q;
        gn[q] = (i >= 1 && k < i - 1) ? G[(size_t)(i - 1) * M + k] : 0.0;
      }
      if ((i & 255) == t) {
        v[qo] *= inv[i];  // x_i
        val[i & 1] = v[qo];
      }
      __syncthreads();
      const double xi = val[i & 1];
#pragma unroll
      for (int q = 0; q < kOwn; ++q) {
        const int k = t + 256 * q;
        if (k < i) v[q] = fma(-g[q], xi, v[q]);
        g[q] = gn[q];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kOwn; ++q) {
    const int k = t + 256 * q;
    if (k < M) x[k] = v[q];
  }
}

// (h, l) += e (wh + wl) for a float e: the double-float multiply-add above with el = 0
__device__ __forceinline__ void df_madd1(float &h, float &l, float e, float wh, float wl) {
  const float th = e * wh;
  float tl = fmaf(e, wh, -th);
  tl = fmaf(e, wl, tl);
  const float sum = h + th;
  const float bv = sum - h;
  const float err = (h - (sum - bv)) + (th - bv);
  l += err + tl;
  h = sum;
}

// (ah + al)(bh + bl) as a normalised double-float (the al bl term dropped)
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &h, float &l) {
  const float ph = ah * bh;
  float pl = fmaf(ah, bh, -ph);
  pl = fmaf(ah, bl, pl);
  pl = fmaf(al, bh, pl);
  h = ph + pl;
  l = pl - (h - ph);
}

// (2 x - (n - 1)) / (n - 1) as hi + lo floats (Dekker: the float quotient, then the exact
// remainder divided once more); 0 for n = 1.  Integer frame sizes < 2^24 are exact floats.
__device__ __forceinline__ void df_norm_coord(int x, int n, float &h, float &l) {
  if (n <= 1) {
    h = 0.0f;
    l = 0.0f;
    return;
  }
  const float a = (float)(2 * x - (n - 1)), den = (float)(n - 1);
  const float q1 = a / den;
  const float r = fmaf(-q1, den, a);  // exact: a - q1 den
  const float q2 = r / den;
  h = q1 + q2;
  l = q2 - (h - q1);
}

// chi^2 = sum w (model - I)^2 at the solution, a direct second pass.  Double-float
// arithmetic on the FP32 pipe (FP64 runs at about 1/60 of its rate here): per pixel
// G_t = sum_k c[k][t] C_k (C_k is a float, c[k][t] split into hi + lo once per CTA), then
// model = sum_t m_t G_t + the background polynomial, the monomials xt^i yt^j in double-float;
// the residual and w r^2 in FP64.  CTA = kChiPix stamp pixels, their C rows staged in
// shared memory by coalesced loads.
constexpr int kChiPix = 128;

__global__ void __launch_bounds__(kChiPix) fit_chi2_kernel(const float *__restrict__ C, const float *__restrict__ I,
                                                           const float *__restrict__ weight, const int *stamp_xy,
                                                           FitDims f, const double *coef, const int *info,
                                                           double *chi2) {
  __shared__ float Cs[kChiPix * 64];                // N <= 64
  __shared__ float ch[64 * 10 + 10], cl[64 * 10 + 10];  // M = N T + Tb <= 650
  __shared__ double red[32];
  if (*info >= 0) return;  // no solution: chi^2 stays 0
  const int p0 = blockIdx.x * kChiPix, np = min(kChiPix, f.P - p0);
  for (int i = threadIdx.x; i < f.M; i += kChiPix) {
    const double c = coef[i];
    const float hi = (float)c;
    ch[i] = hi;
    cl[i] = (float)(c - (double)hi);
  }
  {
    const float *src = C + (size_t)p0 * f.N;
    const int n = np * f.N;
    for (int i = threadIdx.x; i < n; i += kChiPix) Cs[i] = __ldg(src + i);
  }
  __syncthreads();
  double r2 = 0.0;
  const int t = threadIdx.x;
  if (t < np) {
    int x, y;
    stamp_pixel(f, stamp_xy, p0 + t, x, y);
    if (x >= 0 && x < f.W && y >= 0 && y < f.H) {
      // monomials xt^i yt^j of degree <= D = max(d, bd), index mono_index(i, j, D)
      const int D = f.d > f.bd ? f.d : f.bd;
      float xh, xl, yh, yl;
      df_norm_coord(x, f.W, xh, xl);
      df_norm_coord(y, f.H, yh, yl);
      float mh[10], ml[10];
      {
        float pih = 1.0f, pil = 0.0f;  // xt^i
        int u = 0;
#pragma unroll
        for (int i = 0; i <= 3; ++i) {
          float qh = pih, ql = pil;  // xt^i yt^j
#pragma unroll
          for (int j = 0; j <= 3 - i; ++j) {
            if (i + j <= D) {
#pragma unroll
              for (int v = 0; v < 10; ++v)
                if (v == u) {
                  mh[v] = qh;
                  ml[v] = ql;
                }
              ++u;
            }
            df_mul(qh, ql, yh, yl, qh, ql);
          }
          df_mul(pih, pil, xh, xl, pih, pil);
        }
      }
      // G_t = sum_k c[k][t] C_k
      float gh[10], gl[10];
#pragma unroll
      for (int u = 0; u < 10; ++u) gh[u] = gl[u] = 0.0f;
      const float *crow = Cs + t * f.N;
      for (int k = 0; k < f.N; ++k) {
        const float ck = crow[k];
        const float *h = ch + k * f.T, *l = cl + k * f.T;
#pragma unroll
        for (int u = 0; u < 10; ++u)
          if (u < f.T) df_madd1(gh[u], gl[u], ck, h[u], l[u]);
      }
      // model = sum_t m_t G_t (t = (i, j), i + j <= d) + sum over the background terms
      float mdh = 0.0f, mdl = 0.0f;
      {
        int u = 0;
        for (int i = 0; i <= f.d; ++i)
          for (int j = 0; j <= f.d - i; ++j, ++u) {
            const int mi = mono_index(i, j, D);
            float a_h = 0.f, a_l = 0.f, b_h = 0.f, b_l = 0.f;
#pragma unroll
            for (int v = 0; v < 10; ++v) {
              if (v == u) {
                a_h = gh[v];
                a_l = gl[v];
              }
              if (v == mi) {
                b_h = mh[v];
                b_l = ml[v];
              }
            }
            df_madd(mdh, mdl, a_h, a_l, b_h, b_l);
          }
        int q = f.N * f.T;
        for (int i = 0; i <= f.bd; ++i)
          for (int j = 0; j <= f.bd - i; ++j, ++q) {
            const int mi = mono_index(i, j, D);
            float b_h = 0.f, b_l = 0.f;
#pragma unroll
            for (int v = 0; v < 10; ++v)
              if (v == mi) {
                b_h = mh[v];
                b_l = ml[v];
              }
            df_madd(mdh, mdl, b_h, b_l, ch[q], cl[q]);
          }
      }
      const double r = ((double)mdh + (double)mdl) - (double)I[(size_t)y * f.pitch + x];
      r2 = (weight ? (double)weight[(size_t)y * f.pitch + x] : 1.0) * r * r;
    }
  }
  const double sum = block_sum_d(r2, red);
  if (threadIdx.x == 0) atomicAdd(chi2, sum);
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
  f.r0 = 0;
  f.r1 = H;
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

namespace {

// C_k at the stamp pixels and their moments added into S (which the caller zeroed).
int queue_moments(const float *R, const float *I, const float *weight, const FitDims &f, const int *stamp_xy,
                  const float *basis, float *C, double *S, cudaStream_t s) {
  cudaError_t e;
  const int ty = ck_tile_rows(f.S);
  const size_t ck_smem = ck_smem_bytes(f.S, f.L, ty);
  if ((e = cudaFuncSetAttribute(fit_ck_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ck_smem)) != cudaSuccess)
    return cuda_status(e, "fit_ck_kernel smem attribute");
  fit_ck_kernel<<<dim3(f.n_stamps, (f.S + ty - 1) / ty), kCkThreads, ck_smem, s>>>(R, basis, stamp_xy, f, ty, C);
  // Tiles of column pairs as even as whole warps allow (1326 pairs: 6 tiles of 224), and
  // pixel ranges in a multiple of the SM count, so the CTAs fill whole waves.
  const int npairs = f.NE * (f.NE + 1) / 2;
  const int ytiles = (npairs + kGramThreads - 1) / kGramThreads;
  const int tpb = ((npairs + ytiles - 1) / ytiles + 31) / 32 * 32;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int xtiles = (int)(((long long)f.P + (long long)nsm * 4096 - 1) / ((long long)nsm * 4096)) * nsm;
  xtiles = std::min(xtiles, (f.P + kChunk - 1) / kChunk);
  const int px_per_cta = (f.P + xtiles - 1) / xtiles;
  dim3 ggrid((f.P + px_per_cta - 1) / px_per_cta, ytiles);
  fit_gram_kernel<<<ggrid, tpb, 0, s>>>(C, I, weight, stamp_xy, f, px_per_cta, S);
  return cuda_status(cudaGetLastError(), "fit moment kernels launch");
}

// A, b from S, the blocked Cholesky and the substitution into x (x = 0 and info = the
// failing pivot when A is not positive definite).
int queue_solve(const double *S, const FitDims &f, double *A, double *b, double *x, int *info, cudaStream_t s) {
  fit_assemble_kernel<<<(f.M * f.M + 255) / 256, 256, 0, s>>>(S, f, A, b);
  cudaError_t e;
  if ((e = cudaMemsetAsync(info, 0xFF, sizeof(int), s)) != cudaSuccess) return cuda_status(e, "info reset");
  for (int p = 0; p < f.M; p += kPanel) {
    chol_diag_kernel<<<1, 256, 0, s>>>(A, f.M, p, info);
    const int rest = f.M - p - kPanel;
    if (rest > 0) {
      chol_trsm_kernel<<<(rest + 7) / 8, 256, 0, s>>>(A, f.M, p, info);
      const int nt = (rest + 31) / 32;
      chol_update_kernel<<<nt * (nt + 1) / 2, 256, 0, s>>>(A, f.M, p, info);
    }
  }
  fit_solve_kernel<<<1, 256, 0, s>>>(A, b, f.M, info, x);
  return cuda_status(cudaGetLastError(), "fit solve kernels launch");
}

// chi^2 at the solution from the moments alone: sum w (v.c - I)^2 = sum w I^2 - 2 b.c + c.A c,
// and A c = b at the solution, so chi^2 = sum w I^2 - b.c (0 when the solve failed).
__global__ void __launch_bounds__(256) fit_chi2_moments_kernel(const double *S, FitDims f, const double *b,
                                                               const double *x, const int *info, double *chi2) {
  __shared__ double red[32];
  double v = 0.0;
  for (int u = threadIdx.x; u < f.M; u += blockDim.x) v = fma(b[u], x[u], v);
  const double bx = block_sum_d(v, red);
  if (threadIdx.x == 0) *chi2 = *info < 0 ? moment(S, f, f.N, f.N, 0) - bx : 0.0;
}

}  // namespace

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
  int st = queue_moments(R, I, weight, f, stamp_xy, basis, C, S, s);
  if (st == SVK_OK) st = queue_solve(S, f, A, b, coeffs_out, info_out, s);
  if (st != SVK_OK) return st;
  if (chi2_out)
    fit_chi2_kernel<<<(f.P + kChiPix - 1) / kChiPix, kChiPix, 0, s>>>(C, I, weight, stamp_xy, f, coeffs_out, info_out,
                                                                    chi2_out);
  return cuda_status(cudaGetLastError(), "fit kernels launch");
}

size_t fit_moments_count(int N, int degree, int bg_degree) {
  const FitDims f = dims(1, 1, 1, 1, 1, N, 1, degree, bg_degree);
  return (size_t)f.NE * f.NE * f.n_mu;
}

size_t fit_moments_workspace_size(int n_stamps, int stamp_size, int N) {
  return ((size_t)n_stamps * stamp_size * stamp_size * N * sizeof(float) + 255) & ~size_t(255);
}

int launch_fit_moments(const float *R, const float *I, const float *weight, int W, int H, int pitch, int row_begin,
                       int row_end, const int *stamp_xy, int n_stamps, int stamp_size, const float *basis, int N, int L,
                       int degree, int bg_degree, double *moments, bool accumulate, void *ws, size_t ws_bytes,
                       cudaStream_t s) {
  FitDims f = dims(W, H, pitch, n_stamps, stamp_size, N, L, degree, bg_degree);
  if (f.NE > 66) return set_error(SVK_ERR_UNSUPPORTED, "fit supports N <= 64 basis stamps (got %d)", N);
  f.r0 = row_begin;
  f.r1 = row_end;
  if (!ws || ws_bytes < fit_moments_workspace_size(n_stamps, stamp_size, N))
    return set_error(SVK_ERR_WORKSPACE, "fit moments workspace too small");
  if (!accumulate) {
    const cudaError_t e = cudaMemsetAsync(moments, 0, fit_moments_count(N, degree, bg_degree) * sizeof(double), s);
    if (e != cudaSuccess) return cuda_status(e, "moments reset");
  }
  return queue_moments(R, I, weight, f, stamp_xy, basis, static_cast<float *>(ws), moments, s);
}

size_t fit_solve_workspace_size(int N, int degree, int bg_degree) {
  const FitDims f = dims(1, 1, 1, 1, 1, N, 1, degree, bg_degree);
  return (((size_t)f.M * f.M * sizeof(double) + 255) & ~size_t(255)) + (((size_t)f.M * sizeof(double) + 255) & ~size_t(255));
}

int launch_fit_solve(const double *moments, int N, int degree, int bg_degree, double *coeffs_out, double *chi2_out,
                     int *info_out, void *ws, size_t ws_bytes, cudaStream_t s) {
  const FitDims f = dims(1, 1, 1, 1, 1, N, 1, degree, bg_degree);
  if (!ws || ws_bytes < fit_solve_workspace_size(N, degree, bg_degree))
    return set_error(SVK_ERR_WORKSPACE, "fit solve workspace too small");
  double *A = static_cast<double *>(ws);
  double *b = reinterpret_cast<double *>(static_cast<unsigned char *>(ws) +
                                         (((size_t)f.M * f.M * sizeof(double) + 255) & ~size_t(255)));
  int st = queue_solve(moments, f, A, b, coeffs_out, info_out, s);
  if (st != SVK_OK) return st;
  if (chi2_out) fit_chi2_moments_kernel<<<1, 256, 0, s>>>(moments, f, b, coeffs_out, info_out, chi2_out);
  return cuda_status(cudaGetLastError(), "fit chi2 launch");
}

}  // namespace svk
