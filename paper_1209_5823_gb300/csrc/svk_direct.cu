// svk_direct.cu -- direct form of the spatially-varying convolution (Eq. 1-3) on the
// CUDA cores: the kernel K_{x,y} = sum_k a_k(x,y) B_k is formed at every output pixel
// (Sec. 3: the best kernel at every pixel; Sec. 4: one kernel per output pixel) and
// applied to the reference image, FP32 FFMA.
//
// Layout of one CTA (32 x TY threads, TY = 12 rows: three warps per scheduler at 168
// registers, measured faster than 8 or 16 rows for L = 7 .. 31):
//   * output tile 128 x TY pixels; thread (tx, ty) owns pixels x0 + tx + 32 p (p < 4) of
//     row y0 + ty, so every shared-memory read of R is conflict-free and every global
//     store is coalesced;
//   * the R tile plus an h-pixel halo is staged in shared memory by one 2-D TMA load
//     (out-of-frame pixels arrive as zeros -- the zero-padding edge convention);
//     the box starts on a 16-byte boundary, so its x origin is rounded down by xoff;
//   * the basis is consumed NC stamps at a time from a [tap][NC] table in shared
//     memory (uniform broadcast reads), together with the chunk's coefficients;
//   * per tap: K_p = sum_j a_j(p) B_j(tap) for the chunk, acc_p += K_p * R(x_p - u, y - v).
#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
namespace {

constexpr int kTX = 32, kP = 4, kTileW = kTX * kP;

__host__ __device__ inline int round_up4(int v) { return (v + 3) & ~3; }
__host__ __device__ inline int box_w(int h) { return round_up4(kTileW + 2 * h + 3); }
__host__ __device__ inline int box_h(int h, int ty) { return ty + 2 * h; }

template <int NC>
struct Cfg {
  static constexpr int NCP = (NC + 3) & ~3;  // table row stride (16-byte rows)
};

template <int NC, int TY>
size_t direct_smem_bytes(int L) {
  const int h = (L - 1) / 2;
  size_t b = (size_t)box_w(h) * box_h(h, TY) * 4;             // R tile
  b += (size_t)L * L * Cfg<NC>::NCP * 4;                      // basis chunk [tap][NCP]
  b += (size_t)NC * 10 * 4;                                   // coefficient chunk
  b += 16;                                                    // mbarrier
  return b + 128;                                             // alignment slack
}

template <int NC, int TY>
__global__ void __launch_bounds__(kTX * TY, 1)
    direct_kernel(const __grid_constant__ CUtensorMap tmR, int use_tma, const float *__restrict__ R,
                  int pitch_R, const float *__restrict__ I, int pitch_I, int W, int H,
                  const float *__restrict__ basis, int N, int L, const float *__restrict__ coeffs,
                  int degree, float *__restrict__ out, int pitch_out, int y_begin, int y_end, int r0, int r1,
                  uint32_t *status) {
  constexpr int NCP = Cfg<NC>::NCP;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int h = (L - 1) / 2, LL = L * L, T = (degree + 1) * (degree + 2) / 2;
  const int BW = box_w(h), BH = box_h(h, TY);
  float *Rs = reinterpret_cast<float *>(smem);
  float *Bs = Rs + BW * BH;
  float *Cs = Bs + LL * NCP;
  uint64_t *bar = reinterpret_cast<uint64_t *>(reinterpret_cast<uintptr_t>(Cs + NC * 10 + 1) & ~uintptr_t(7));

  const int tid = threadIdx.y * kTX + threadIdx.x;
  constexpr int kThreads = kTX * TY;
  const int x0 = blockIdx.x * kTileW, y0 = y_begin + blockIdx.y * TY;
  const int xs = ((x0 - h) >> 2) << 2;  // floor to a multiple of 4 (16-byte TMA origin)
  const int xoff = (x0 - h) - xs;

  // ---- stage the R tile + halo
  if (use_tma) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
      mbar_arrive_expect_tx(bar, (uint32_t)(BW * BH * 4));
      tma_load_2d(Rs, &tmR, bar, xs, y0 - h - r0);  // the map covers the held rows
    }
  } else {
    for (int i = tid; i < BW * BH; i += kThreads) {
      const int r = i / BW, c = i % BW, gy = y0 - h + r, gx = xs + c;
      Rs[i] = (gx >= 0 && gx < W && gy >= r0 && gy < r1) ? R[(size_t)(gy - r0) * pitch_R + gx] : 0.0f;
    }
  }

  // ---- normalised coordinates of the thread's pixels
  const int tx = threadIdx.x, ty = threadIdx.y, y = y0 + ty;
  const float yt = H > 1 ? (2.0f * (float)y - (float)(H - 1)) / (float)(H - 1) : 0.0f;
  float xt[kP];
#pragma unroll
  for (int p = 0; p < kP; ++p) {
    const int x = x0 + tx + 32 * p;
    xt[p] = W > 1 ? (2.0f * (float)x - (float)(W - 1)) / (float)(W - 1) : 0.0f;
  }

  float acc[kP];
#pragma unroll
  for (int p = 0; p < kP; ++p) acc[p] = 0.0f;

  bool tile_ready = !use_tma;
  for (int k0 = 0; k0 < N; k0 += NC) {
    __syncthreads();  // previous chunk consumed (and, first time, mbarrier initialised)
    for (int i = tid; i < LL * NCP; i += kThreads) {
      const int tap = i / NCP, j = i % NCP;
      Bs[i] = (j < NC && k0 + j < N) ? basis[(size_t)(k0 + j) * LL + tap] : 0.0f;
    }
    for (int i = tid; i < NC * 10; i += kThreads) {
      const int j = i / 10, t = i % 10;
      Cs[i] = (k0 + j < N && t < T) ? coeffs[(size_t)(k0 + j) * T + t] : 0.0f;
    }
    __syncthreads();
    if (!tile_ready) {
      // Every thread waits for the tile with the same limit, started at the same barrier,
      // so they give up together unless the copy lands within the microseconds between
      // their deadlines after 2 s; a thread that gives up leaves, and the hardware counts
      // exited threads as arrived at the block's later barriers.  A block-wide vote here
      // (or a thread-0 decision broadcast through shared memory) makes the compiler spill
      // in the main loop at the 168-register budget: measured 6 % slower.
      if (!mbar_wait_bounded(bar, 0, status)) return;
      tile_ready = true;
    }
    // a_j(x_p, y) = sum_t c[k0+j][t] xt^i yt^j for the chunk (Eq. 3, order <= 3): per stamp
    // alpha_i = sum_jj c[(i, jj)] yt^jj (the same for the thread's pixels, which share a
    // row), then Horner in xt.  Coefficient slots are packed (i outer, jj inner), skipping
    // terms above `degree`.
    float a[NC][kP];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      float al[4];
      int tt = 0;
#pragma unroll
      for (int i = 0; i <= 3; ++i) {
        float sacc = 0.0f, yj = 1.0f;
#pragma unroll
        for (int jj = 0; jj <= 3 - i; ++jj) {
          if (i + jj <= degree) sacc = fmaf(Cs[j * 10 + tt++], yj, sacc);
          yj *= yt;
        }
        al[i] = sacc;
      }
#pragma unroll
      for (int p = 0; p < kP; ++p) a[j][p] = fmaf(fmaf(fmaf(al[3], xt[p], al[2]), xt[p], al[1]), xt[p], al[0]);
    }
    for (int vi = 0; vi < L; ++vi) {
      // smem row of image row y - v with v = vi - h; smem column of x - u with u = ui - h
      const float *rrow = Rs + (ty + 2 * h - vi) * BW + tx + 2 * h + xoff;
      const float4 *brow = reinterpret_cast<const float4 *>(Bs + vi * L * NCP);
#pragma unroll 1
      for (int ui = 0; ui < L; ++ui) {
        float r[kP];
#pragma unroll
        for (int p = 0; p < kP; ++p) {
          const long long ri = (rrow - Rs) + 32 * p - ui;  // the staged tile holds BW x BH values
          r[p] = SVK_CHECK(ri >= 0 && ri < (long long)BW * BH, status, 6) ? rrow[32 * p - ui] : 0.0f;
        }
        float k0s[kP], k1s[kP];
#pragma unroll
        for (int p = 0; p < kP; ++p) k0s[p] = k1s[p] = 0.0f;
        const float4 *bt = brow + ui * (NCP / 4);
#pragma unroll
        for (int q = 0; q < NCP / 4; ++q) {
          const float4 b = bt[q];
          const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int j = 4 * q + e;
            if (j < NC) {
#pragma unroll
              for (int p = 0; p < kP; ++p) {
                if (j & 1) k1s[p] = fmaf(a[j][p], bv[e], k1s[p]);
                else k0s[p] = fmaf(a[j][p], bv[e], k0s[p]);
              }
            }
          }
        }
#pragma unroll
        for (int p = 0; p < kP; ++p) acc[p] = fmaf(k0s[p] + k1s[p], r[p], acc[p]);
      }
    }
  }

  if (y < y_end) {
#pragma unroll
    for (int p = 0; p < kP; ++p) {
      const int x = x0 + tx + 32 * p;
      if (x < W) {
        float v = acc[p];
        if (I) v -= I[(size_t)y * pitch_I + x];
        out[(size_t)y * pitch_out + x] = v;
      }
    }
  }
}

template <int NC, int TY>
int launch_nc(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H, const float *basis,
              int N, int L, const float *coeffs, int degree, float *out, int pitch_out, int y_begin, int y_end,
              int r0, int r1, cudaStream_t s) {
  const int h = (L - 1) / 2;
  const size_t smem = direct_smem_bytes<NC, TY>(L);
  cudaError_t e = cudaFuncSetAttribute(direct_kernel<NC, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e, "direct_kernel smem attribute");
  CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  const int use_tma = encode_tmap_2d_f32(&tm, R, W, r1 - r0, pitch_R, box_w(h), box_h(h, TY)) ? 1 : 0;
  dim3 grid((W + kTileW - 1) / kTileW, (y_end - y_begin + TY - 1) / TY), block(kTX, TY);
  if (grid.y == 0) return SVK_OK;
  direct_kernel<NC, TY><<<grid, block, smem, s>>>(tm, use_tma, R, pitch_R, I, pitch_I, W, H, basis, N, L, coeffs,
                                             degree, out, pitch_out, y_begin, y_end, r0, r1, device_status_word());
  return cuda_status(cudaGetLastError(), "direct_kernel launch");
}

}  // namespace

int direct_rows(int) { return 12; }

namespace {
template <int TY>
int launch_ty(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H, const float *basis, int N,
              int L, const float *coeffs, int degree, float *out, int pitch_out, int y_begin, int y_end,
              int r0, int r1, cudaStream_t s) {
  if (N <= 4)
    return launch_nc<4, TY>(R, pitch_R, I, pitch_I, W, H, basis, N, L, coeffs, degree, out, pitch_out, y_begin, y_end, r0, r1, s);
  if (N <= 6)  // the T-form's six stamps at degree 2
    return launch_nc<6, TY>(R, pitch_R, I, pitch_I, W, H, basis, N, L, coeffs, degree, out, pitch_out, y_begin, y_end, r0, r1, s);
  if (N <= 8)
    return launch_nc<8, TY>(R, pitch_R, I, pitch_I, W, H, basis, N, L, coeffs, degree, out, pitch_out, y_begin, y_end, r0, r1, s);
  if (N <= 10)  // the T-form's ten stamps at degree 3
    return launch_nc<10, TY>(R, pitch_R, I, pitch_I, W, H, basis, N, L, coeffs, degree, out, pitch_out, y_begin, y_end,
                             r0, r1, s);
  if (N <= 16)
    return launch_nc<16, TY>(R, pitch_R, I, pitch_I, W, H, basis, N, L, coeffs, degree, out, pitch_out, y_begin, y_end,
                             r0, r1, s);
  return launch_nc<25, TY>(R, pitch_R, I, pitch_I, W, H, basis, N, L, coeffs, degree, out, pitch_out, y_begin, y_end, r0, r1, s);
}
}  // namespace

int launch_direct(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H, const float *basis,
                  int N, int L, const float *coeffs, int degree, float *out, int pitch_out, cudaStream_t s,
                  int y_begin, int y_end, int r_begin, int r_end) {
  if (y_end < 0) y_end = H;
  if (r_end < 0) r_end = H;
  return launch_ty<12>(R, pitch_R, I, pitch_I, W, H, basis, N, L, coeffs, degree, out, pitch_out, y_begin, y_end,
                       r_begin, r_end, s);
}


// ---------------------------------------------------------------------------------
// T-factored form on the CUDA cores.  The kernel field is linear in the coefficients,
// so (R (x) K_{x,y})(x,y) = sum_t m_t(x~,y~) (R (x) K_t)(x,y) with K_t = sum_k c[k][t] B_k
// (Eq. 2 with the polynomial of Eq. 3 expanded): every pixel accumulates the T ordinary
// convolutions C_t = R (x) K_t -- T FFMAs per tap, no per-pixel kernel -- and combines
// them with its monomials once, in the epilogue.
//
// Layout of one CTA (32 x 8 threads, 128 x 16 output pixels): thread (tx, ty) owns the
// four consecutive pixels x0 + 4 tx + p (p < 4) of rows y0 + ty and y0 + ty + 8.  Taps
// go in groups of four (the K_t table is zero beyond L): for one kernel row v and tap
// group g the 16 (pixel, tap) pairs of a row read only 7 consecutive R values, fetched
// as 16-byte loads of the R tile, and one 16-byte load of the table gives K_t for the
// group's four taps.  Where those 7 values sit against the 16-byte grid depends only on
// h mod 4 (the template parameter S), so every register index is a constant.  The R
// tile (plus halo, plus 4 columns on each side for the 16-byte grid) is staged by one
// 2-D TMA load with zero fill outside the frame.
namespace {
constexpr int kTfTY = 8, kTfRows = 2 * kTfTY, kTfTileW = 4 * kTX;

__host__ __device__ inline int tf_box_w(int h) { return round_up4(2 * h + kTfTileW + 12); }
__host__ __device__ inline int tf_groups(int L) { return (L + 3) / 4; }

template <int T>
size_t tform_fp32_smem_bytes(int L) {
  const int h = (L - 1) / 2;
  return (size_t)tf_box_w(h) * box_h(h, kTfRows) * 4 + (size_t)L * tf_groups(L) * T * 16 + 16 + 128;
}

template <int T, int S>
__global__ void __launch_bounds__(kTX * kTfTY, 2)
    tform_fp32_kernel(const __grid_constant__ CUtensorMap tmR, int use_tma, const float *__restrict__ R,
                      int pitch_R, const float *__restrict__ I, int pitch_I, int W, int H,
                      const float *__restrict__ Kt, int L, float *__restrict__ out, int pitch_out, int y_begin,
                      int y_end, int r0, int r1, uint32_t *status) {
  constexpr int D = T == 1 ? 0 : (T == 3 ? 1 : (T == 6 ? 2 : 3));  // spatial degree
  constexpr int kThreads = kTX * kTfTY;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int h = (L - 1) / 2, LL = L * L, G = tf_groups(L);
  const int BW = tf_box_w(h), BH = box_h(h, kTfRows);
  float *Rs = reinterpret_cast<float *>(smem);
  float4 *Ks = reinterpret_cast<float4 *>(Rs + BW * BH);  // [v][g][t] -> taps 4g..4g+3
  uint64_t *bar = reinterpret_cast<uint64_t *>(Ks + L * G * T);

  const int tid = threadIdx.y * kTX + threadIdx.x;
  const int x0 = blockIdx.x * kTfTileW, y0 = y_begin + blockIdx.y * kTfRows;
  const int xs = (((x0 - h) >> 2) << 2) - 4;  // 16-byte grid, 4 spare columns on the left
  // column of R(x0 + 4 tx + p - u) in the tile for tap u = 4 g + k - h:
  //   4 tx + p + A - 4 g - k + 4 with A = x0 + h - xs - 4 = 4 a + S
  const int a = (x0 + h - xs - 4 - S) >> 2;

  if (use_tma) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
      mbar_arrive_expect_tx(bar, (uint32_t)(BW * BH * 4));
      tma_load_2d(Rs, &tmR, bar, xs, y0 - h - r0);  // the map covers the held rows
    }
  } else {
    for (int i = tid; i < BW * BH; i += kThreads) {
      const int r = i / BW, c = i % BW, gy = y0 - h + r, gx = xs + c;
      Rs[i] = (gx >= 0 && gx < W && gy >= r0 && gy < r1) ? R[(size_t)(gy - r0) * pitch_R + gx] : 0.0f;
    }
  }
  float *Kf = reinterpret_cast<float *>(Ks);
  for (int i = tid; i < L * G * T * 4; i += kThreads) {
    const int k = i & 3, t = (i >> 2) % T, vg = (i >> 2) / T, g = vg % G, v = vg / G, u = 4 * g + k;
    Kf[i] = u < L ? Kt[(size_t)t * LL + v * L + u] : 0.0f;
  }
  __syncthreads();
  if (use_tma && !mbar_wait_bounded(bar, 0, status)) return;  // TMA never landed: give up cleanly

  const int tx = threadIdx.x, ty = threadIdx.y;
  float acc[T][8];
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int p = 0; p < 8; ++p) acc[t][p] = 0.0f;

  for (int vi = 0; vi < L; ++vi) {
    // tile rows of image rows y - v (v = vi - h) for the thread's two output rows
    const float *row0 = Rs + (ty + 2 * h - vi) * BW + 4 * tx + 4 * a;
    const float *row1 = row0 + kTfTY * BW;
    const float4 *kv = Ks + vi * G * T;
#pragma unroll 1
    for (int g = 0; g < G; ++g) {
      // w[i] = R at tile column 4 tx + 4 (a - g) + i; the group needs i in [S + 1, S + 7]
      float w0[12], w1[12];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if ((c == 0 && S <= 2) || c == 1 || (c == 2 && S >= 1)) {
          const long long i0 = (row0 - Rs) - 4 * g + 4 * c, i1 = i0 + (long long)kTfTY * BW;  // tile: BW x BH
          const bool in = SVK_CHECK(i0 >= 0 && i1 + 4 <= (long long)BW * BH, status, 7);
          const float4 q0 = in ? *reinterpret_cast<const float4 *>(row0 - 4 * g + 4 * c) : make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 q1 = in ? *reinterpret_cast<const float4 *>(row1 - 4 * g + 4 * c) : make_float4(0.f, 0.f, 0.f, 0.f);
          w0[4 * c] = q0.x, w0[4 * c + 1] = q0.y, w0[4 * c + 2] = q0.z, w0[4 * c + 3] = q0.w;
          w1[4 * c] = q1.x, w1[4 * c + 1] = q1.y, w1[4 * c + 2] = q1.z, w1[4 * c + 3] = q1.w;
        }
      }
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const float4 k4 = kv[g * T + t];
        const float kk[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            acc[t][p] = fmaf(kk[k], w0[S + 4 + p - k], acc[t][p]);
            acc[t][4 + p] = fmaf(kk[k], w1[S + 4 + p - k], acc[t][4 + p]);
          }
      }
    }
  }

  // D = sum_t m_t C_t - I, monomials x~^i y~^j in the coefficient order (i outer, j inner)
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    const int y = y0 + ty + kTfTY * rr;
    if (y >= y_end) continue;
    const float yt = H > 1 ? (2.0f * (float)y - (float)(H - 1)) / (float)(H - 1) : 0.0f;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int x = x0 + 4 * tx + p;
      if (x >= W) continue;
      const float xt = W > 1 ? (2.0f * (float)x - (float)(W - 1)) / (float)(W - 1) : 0.0f;
      float v = 0.0f, xp = 1.0f;
      int t = 0;
#pragma unroll
      for (int i = 0; i <= D; ++i) {
        float inner = 0.0f, yp = 1.0f;
#pragma unroll
        for (int j = 0; j <= D - i; ++j) {
          inner = fmaf(acc[t++][4 * rr + p], yp, inner);
          yp *= yt;
        }
        v = fmaf(inner, xp, v);
        xp *= xt;
      }
      if (I) v -= I[(size_t)y * pitch_I + x];
      out[(size_t)y * pitch_out + x] = v;
    }
  }
}

template <int T, int S>
int launch_tf(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H, const float *Kt, int L,
              float *out, int pitch_out, int y_begin, int y_end, int r0, int r1, cudaStream_t s) {
  const int h = (L - 1) / 2;
  const size_t smem = tform_fp32_smem_bytes<T>(L);
  cudaError_t e =
      cudaFuncSetAttribute(tform_fp32_kernel<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e, "tform_fp32_kernel smem attribute");
  CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  const int use_tma = encode_tmap_2d_f32(&tm, R, W, r1 - r0, pitch_R, tf_box_w(h), box_h(h, kTfRows)) ? 1 : 0;
  dim3 grid((W + kTfTileW - 1) / kTfTileW, (y_end - y_begin + kTfRows - 1) / kTfRows), block(kTX, kTfTY);
  if (grid.y == 0) return SVK_OK;
  tform_fp32_kernel<T, S><<<grid, block, smem, s>>>(tm, use_tma, R, pitch_R, I, pitch_I, W, H, Kt, L, out,
                                                    pitch_out, y_begin, y_end, r0, r1, device_status_word());
  return cuda_status(cudaGetLastError(), "tform_fp32_kernel launch");
}

template <int T>
int launch_tf_s(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H, const float *Kt, int L,
                float *out, int pitch_out, int y_begin, int y_end, int r0, int r1, cudaStream_t s) {
  switch (((L - 1) / 2) & 3) {
    case 0: return launch_tf<T, 0>(R, pitch_R, I, pitch_I, W, H, Kt, L, out, pitch_out, y_begin, y_end, r0, r1, s);
    case 1: return launch_tf<T, 1>(R, pitch_R, I, pitch_I, W, H, Kt, L, out, pitch_out, y_begin, y_end, r0, r1, s);
    case 2: return launch_tf<T, 2>(R, pitch_R, I, pitch_I, W, H, Kt, L, out, pitch_out, y_begin, y_end, r0, r1, s);
    default: return launch_tf<T, 3>(R, pitch_R, I, pitch_I, W, H, Kt, L, out, pitch_out, y_begin, y_end, r0, r1, s);
  }
}
}  // namespace

int tform_fp32_rows(int) { return kTfRows; }

int launch_tform_fp32(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H, const float *Kt, int T,
                      int L, float *out, int pitch_out, cudaStream_t s, int y_begin, int y_end, int r_begin,
                      int r_end) {
  if (y_end < 0) y_end = H;
  const int r0 = r_begin, r1 = r_end < 0 ? H : r_end;
  switch (T) {
    case 1: return launch_tf_s<1>(R, pitch_R, I, pitch_I, W, H, Kt, L, out, pitch_out, y_begin, y_end, r0, r1, s);
    case 3: return launch_tf_s<3>(R, pitch_R, I, pitch_I, W, H, Kt, L, out, pitch_out, y_begin, y_end, r0, r1, s);
    case 6: return launch_tf_s<6>(R, pitch_R, I, pitch_I, W, H, Kt, L, out, pitch_out, y_begin, y_end, r0, r1, s);
    case 10: return launch_tf_s<10>(R, pitch_R, I, pitch_I, W, H, Kt, L, out, pitch_out, y_begin, y_end, r0, r1, s);
    default: return set_error(SVK_ERR_ARG, "T-form: T=%d is not a number of monomials of degree <= 3", T);
  }
}

}  // namespace svk
