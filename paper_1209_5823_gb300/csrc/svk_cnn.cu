// svk_cnn.cu -- the coefficient network: a small CNN that maps a (R, I) star-stamp pair
// [2][64][64] to the local kernel coefficients a_k of Eq. 2 / Eq. 3 at the stamp, trained
// and run on the device by the kernels below.
//
//   conv 3x3 (2 -> 32, stride 2, pad 1) -> ReLU      64x64 -> 32x32
//   conv 3x3 (32 -> 32, stride 2, pad 1) -> ReLU     32x32 -> 16x16
//   conv 3x3 (32 -> 32, stride 2, pad 1) -> ReLU     16x16 -> 8x8
//   conv 3x3 (32 -> 32, stride 1, pad 1) -> ReLU     8x8
//   global average pool -> linear (32 -> n_out)
//
// Precision: weights are used rounded to BF16 (the FP32 master copy is what Adam
// updates); the input, every stored activation and every stored pre-activation gradient
// are BF16; all sums accumulate in FP32.  Convolution is cross-correlation.
// Parameter order (flat FP32): per conv layer w[Cout][Cin][3][3], b[Cout]; then the
// linear layer w[n_out][32], b[n_out].
//
// The three 32-channel layers run on the tensor cores (tcgen05.mma, BF16 operands, FP32
// accumulators in TMEM) as implicit GEMMs over NHWC activations:
//   forward      rows = output pixels, K = 9 taps x 32 input channels, N = 32 outputs;
//   data grad    rows = input pixels,  K = 9 taps x 32 output channels (the transposed
//                convolution: a tap contributes where the strided position is hit);
//   weight grad  rows = 9 taps x 32 input channels (+ a row of ones for the bias),
//                K = output pixels (split over CTAs, partial sums reduced in a fixed
//                order, so the gradient is deterministic), N = 32 outputs.
// The 2-channel first layer runs forward on the FP32 pipe (18 products per output) and
// its weight gradient on the tensor cores like the others.
#include <cuda_bf16.h>

#include "svk_common.cuh"
#include "svk_internal.h"
#include "svk_umma.cuh"

namespace svk {
namespace {

constexpr int kIn = 64, kCh = 32, kLayers = 4, kTaps = 9;
constexpr int kCin[kLayers] = {2, kCh, kCh, kCh};
constexpr int kStride[kLayers] = {2, 2, 2, 1};
constexpr int kHout[kLayers] = {32, 16, 8, 8};
constexpr int kLgIn[kLayers] = {6, 5, 4, 3};   // log2 kHin
constexpr int kLgOut[kLayers] = {5, 4, 3, 3};  // log2 kHout

// Packed UMMA B operand of a 32-channel layer: K = tap * 32 + channel (288), 32 rows, in
// the K-major no-swizzle layout: 36 core-matrix columns of [32 rows][8 BF16].
constexpr int kK = kTaps * kCh;            // 288
constexpr int kKChunks = kK / 8;           // 36
constexpr int kPack = kK * kCh;            // 9216 BF16 per packed operand
constexpr uint32_t kPackBytes = kPack * 2; // 18,432
constexpr uint32_t kIdesc = idesc_f16(1, 128, 32);  // BF16 x BF16 -> FP32, M = 128, N = 32

typedef __nv_bfloat16 bf16;

struct Layout {
  size_t w[kLayers], b[kLayers], fcw, fcb, total;  // parameter offsets (floats)
};

Layout param_layout(int n_out) {
  Layout l;
  size_t o = 0;
  for (int i = 0; i < kLayers; ++i) {
    l.w[i] = o;
    o += (size_t)kCh * kCin[i] * 9;
    l.b[i] = o;
    o += kCh;
  }
  l.fcw = o;
  o += (size_t)n_out * kCh;
  l.fcb = o;
  o += n_out;
  l.total = o;
  return l;
}

// Weight-gradient split: K (the output pixels of a layer) in chunks of a multiple of 64
// pixels, about kWgChunks chunks per layer.  Depends on the batch only (deterministic).
constexpr int kWgChunks = 128;
constexpr int kWgStage = 64;  // pixels per pipeline stage (4 MMAs of K = 16)

int wg_per_chunk(int P) {
  const int stages = (P + kWgStage - 1) / kWgStage;
  return kWgStage * ((stages + kWgChunks - 1) / kWgChunks);
}
int wg_nchunks(int P) { return (P + wg_per_chunk(P) - 1) / wg_per_chunk(P); }
int wg_rows(int cin) { return cin * kTaps + 1; }  // taps x channels, then the bias row

struct Work {  // byte offsets into the workspace
  size_t wq;                     // float[param total]: parameters rounded to BF16
  size_t wf[kLayers], wd[kLayers];  // packed BF16 operands (forward, data grad), layers 1..3
  size_t act[kLayers], dz[kLayers];  // BF16 NHWC [B][H][H][32]: post-ReLU, pre-activation grad
  size_t pooled, dpooled, out, dout, part, total;
};

Work work_layout(int B, int n_out) {
  Work w{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 255) & ~size_t(255);
    return at;
  };
  w.wq = take(param_layout(n_out).total * sizeof(float));
  for (int i = 1; i < kLayers; ++i) {
    w.wf[i] = take(kPackBytes);
    w.wd[i] = take(kPackBytes);
  }
  size_t part = 0;
  for (int i = 0; i < kLayers; ++i) {
    const size_t n = (size_t)B * kCh * kHout[i] * kHout[i];
    w.act[i] = take(n * sizeof(bf16));
    w.dz[i] = take(n * sizeof(bf16));
    const int P = B * kHout[i] * kHout[i];
    const size_t pb = (size_t)wg_nchunks(P) * wg_rows(kCin[i]) * kCh * sizeof(float);
    part = pb > part ? pb : part;
  }
  w.pooled = take((size_t)B * kCh * sizeof(float));
  w.dpooled = take((size_t)B * kCh * sizeof(float));
  w.out = take((size_t)B * n_out * sizeof(float));
  w.dout = take((size_t)B * n_out * sizeof(float));
  w.part = take(part);
  w.total = o;
  return w;
}

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

__device__ __forceinline__ float lo_f(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float hi_f(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// Rounded parameters (FP32 values of the BF16 weights) and the packed tensor-core
// operands of layers 1..3:  wf[j][o][t] = W[o][c][tap],  wd[j][c][t] = W[o][c][tap]  with
// k = 8 j + t = 32 tap + (c for wf, o for wd).
__global__ void pack_kernel(const float *__restrict__ p, float *__restrict__ wq, int n_params, bf16 *wf1, bf16 *wd1,
                            bf16 *wf2, bf16 *wd2, bf16 *wf3, bf16 *wd3, size_t w1, size_t w2, size_t w3) {
  const int n = n_params + 3 * kPack;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < n_params) {
      wq[i] = bf16r(p[i]);
      continue;
    }
    const int l = (i - n_params) / kPack, e = (i - n_params) % kPack;
    const int j = e >> 8, r = (e >> 3) & 31, t = e & 7;
    const int k = 8 * j + t, tap = k >> 5, ch = k & 31;
    const float *w = p + (l == 0 ? w1 : l == 1 ? w2 : w3);
    bf16 *f = l == 0 ? wf1 : l == 1 ? wf2 : wf3;
    bf16 *d = l == 0 ? wd1 : l == 1 ? wd2 : wd3;
    f[e] = __float2bfloat16_rn(w[(r * kCh + ch) * 9 + tap]);  // o = r, c = ch
    d[e] = __float2bfloat16_rn(w[(ch * kCh + r) * 9 + tap]);  // c = r, o = ch
  }
}

// First layer, forward: out[b][y][x][o] = relu(b[o] + sum_{c,dy,dx} w[o][c][dy][dx]
// x[b][c][2y+dy-1][2x+dx-1]) with x rounded to BF16; one thread per output pixel, all 32
// channels, stored as BF16 NHWC.
__global__ void __launch_bounds__(256) conv1_fwd_kernel(const float *__restrict__ x, const float *__restrict__ w,
                                                        const float *__restrict__ bias, bf16 *__restrict__ out,
                                                        int B) {
  __shared__ float ws[kCh * 2 * 9], bs[kCh];
  for (int i = threadIdx.x; i < kCh * 2 * 9; i += blockDim.x) ws[i] = w[i];
  if (threadIdx.x < kCh) bs[threadIdx.x] = bias[threadIdx.x];
  __syncthreads();
  const int n = B * 32 * 32;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const int xo = idx & 31, yo = (idx >> 5) & 31, b = idx >> 10;
    float v[2][9];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const int yy = 2 * yo + t / 3 - 1, xx = 2 * xo + t % 3 - 1;
        v[c][t] = (yy >= 0 && yy < kIn && xx >= 0 && xx < kIn)
                      ? bf16r(__ldg(x + (((size_t)b * 2 + c) * kIn + yy) * kIn + xx))
                      : 0.0f;
      }
    uint32_t o32[16];
#pragma unroll
    for (int o = 0; o < kCh; o += 2) {
      float a0 = bs[o], a1 = bs[o + 1];
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          a0 = fmaf(ws[(o * 2 + c) * 9 + t], v[c][t], a0);
          a1 = fmaf(ws[((o + 1) * 2 + c) * 9 + t], v[c][t], a1);
        }
      o32[o >> 1] = pack2(fmaxf(a0, 0.0f), fmaxf(a1, 0.0f));
    }
    uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)idx * kCh);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = make_uint4(o32[4 * q], o32[4 * q + 1], o32[4 * q + 2], o32[4 * q + 3]);
  }
}

// ------------------------------------------------------ 32-channel layers on tcgen05
enum ConvMode { kFwd = 0, kDgrad = 1 };
constexpr int kConvThreads = 256;
constexpr uint32_t kConvABytes = kKChunks * 128 * 16;  // 73,728: [36][128 rows][16 B]
constexpr uint32_t kConvSmem = kConvABytes + kPackBytes + 64;

// One 128-row tile per iteration of a persistent loop.  Rows are pixels of the grid G
// (side 2^lg_g); source pixels lie on the grid S (side 2^lg_s), NHWC BF16 with 32
// channels.  A row's K chunk (tap, 8 channels) is 16 contiguous bytes of the source:
//   forward  (grid G = output): source pixel (s y + dy - 1, s x + dx - 1);
//   data grad (grid G = layer input): source pixel ((y + 1 - dy) / s, (x + 1 - dx) / s)
//            where both divisions are exact, else zero.
// Epilogue: forward adds the bias and applies the ReLU; data grad multiplies by the
// ReLU mask of the layer below (act > 0).  Both store BF16 NHWC rows.
template <int MODE>
__global__ void __launch_bounds__(kConvThreads, 2)
    conv_mma_kernel(const bf16 *__restrict__ src, const bf16 *__restrict__ wpack, const float *__restrict__ bias,
                    const bf16 *__restrict__ mask, bf16 *__restrict__ out, int B, int lg_s, int lg_g, int stride,
                    uint32_t *status) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t *sA = smem;
  uint8_t *sB = smem + kConvABytes;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kConvABytes + kPackBytes);
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = 1 << lg_s, G = 1 << lg_g;
  const int P = B << (2 * lg_g);
  const int ntiles = (P + 127) >> 7;

  {  // the packed weights, once
    const uint4 *g = reinterpret_cast<const uint4 *>(wpack);
    uint4 *d = reinterpret_cast<uint4 *>(sB);
    for (int i = tid; i < (int)(kPackBytes / 16); i += kConvThreads) d[i] = __ldg(g + i);
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(slot, 32);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const uint32_t aBase = smem_u32(sA), bBase = smem_u32(sB);

  const int m = tid & 127, half = tid >> 7;
  uint32_t it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    // ---- A tile: row m, chunks (tap, c8) with c8 in {2 half, 2 half + 1}
    const int p = (tile << 7) + m;
    const bool valid = p < P;
    const int b = p >> (2 * lg_g), y = (p >> lg_g) & (G - 1), x = p & (G - 1);
    uint4 v[kTaps][2];
#pragma unroll
    for (int t = 0; t < kTaps; ++t) {
      const int dy = t / 3, dx = t % 3;
      int yy, xx;
      bool ok;
      if (MODE == kFwd) {
        yy = stride * y + dy - 1;
        xx = stride * x + dx - 1;
        ok = valid && yy >= 0 && yy < S && xx >= 0 && xx < S;
      } else {
        const int ty = y + 1 - dy, tx = x + 1 - dx;
        ok = valid && ty >= 0 && tx >= 0 && (ty % stride) == 0 && (tx % stride) == 0;
        yy = ty / stride;
        xx = tx / stride;
        ok = ok && yy < S && xx < S;
      }
      const size_t pix = ((((size_t)b << lg_s) + (ok ? yy : 0)) << lg_s) + (ok ? xx : 0);
      const uint4 *s4 = reinterpret_cast<const uint4 *>(src + pix * kCh) + 2 * half;
      v[t][0] = ok ? __ldg(s4) : make_uint4(0, 0, 0, 0);
      v[t][1] = ok ? __ldg(s4 + 1) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int t = 0; t < kTaps; ++t) {
      const int j0 = t * 4 + 2 * half;
      *reinterpret_cast<uint4 *>(sA + (uint32_t)j0 * 2048u + (uint32_t)m * 16u) = v[t][0];
      *reinterpret_cast<uint4 *>(sA + (uint32_t)(j0 + 1) * 2048u + (uint32_t)m * 16u) = v[t][1];
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int k = 0; k < kKChunks / 2; ++k) {
        const uint64_t a = sdesc(aBase + (uint32_t)k * 2u * 2048u, 2048u, 128u);
        const uint64_t bd = sdesc(bBase + (uint32_t)k * 2u * 512u, 512u, 128u);
        umma_f16(tmem, a, bd, kIdesc, k > 0 ? 1u : 0u);
      }
      umma_commit(bar);
    }
    const bool ok = mbar_wait_bounded(bar, it & 1u, status);
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    // ---- epilogue: warp -> TMEM lane quadrant (warp & 3), column half (warp >> 2)
    {
      const int q = warp & 3, h = warp >> 2;
      const int row = 32 * q + lane;
      const int pr = (tile << 7) + row;
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * h), r);
      tmem_ld_wait();
      if (pr < P) {
        uint32_t o32[8];
        if (MODE == kFwd) {
#pragma unroll
          for (int i = 0; i < 8; ++i)
            o32[i] = pack2(fmaxf(__uint_as_float(r[2 * i]) + __ldg(bias + 16 * h + 2 * i), 0.0f),
                           fmaxf(__uint_as_float(r[2 * i + 1]) + __ldg(bias + 16 * h + 2 * i + 1), 0.0f));
        } else {
          const uint4 *mk = reinterpret_cast<const uint4 *>(mask + (size_t)pr * kCh + 16 * h);
          const uint4 m0 = __ldg(mk), m1 = __ldg(mk + 1);
          const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
          for (int i = 0; i < 8; ++i)
            o32[i] = pack2(lo_f(mw[i]) > 0.0f ? __uint_as_float(r[2 * i]) : 0.0f,
                           hi_f(mw[i]) > 0.0f ? __uint_as_float(r[2 * i + 1]) : 0.0f);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)pr * kCh + 16 * h);
        dst[0] = make_uint4(o32[0], o32[1], o32[2], o32[3]);
        dst[1] = make_uint4(o32[4], o32[5], o32[6], o32[7]);
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

// ---------------------------------------------------- weight gradient on tcgen05
// dW^T[(tap, c)][o] = sum_p col[p][(tap, c)] dz[p][o], db[o] = sum_p dz[p][o]: rows are
// (tap, input channel) plus one row of ones (the bias), K runs over the output pixels of
// one chunk, N = 32 output channels.  Both operands are stored p-major in memory, so each
// 8 x 8 block is transposed in registers on its way to shared memory (K-major UMMA
// layout).  Two pipeline stages of 64 pixels; each CTA writes its chunk's partial sums.
constexpr int kWgThreads = 256;

template <int CIN>
struct WgShape {
  static constexpr int MT = CIN == kCh ? 3 : 1;  // 128-row M tiles
  static constexpr int ROWS = MT * 128;
  static constexpr int NDATA = CIN * kTaps;       // data rows; row NDATA holds ones
  static constexpr uint32_t LBO_A = ROWS * 16 + 16;  // +16 B: the 8 K chunks on distinct banks
  static constexpr uint32_t A_STAGE = 8 * LBO_A;
  static constexpr uint32_t LBO_B = kCh * 16 + 16;
  static constexpr uint32_t B_STAGE = 8 * LBO_B;
  static constexpr uint32_t SMEM = 2 * (A_STAGE + B_STAGE) + 64;
  static constexpr uint32_t TMEM_COLS = MT == 3 ? 128 : 32;
};

// r[i] = row i (8 BF16); t[j] = column j (element i = r[i][j]).
__device__ __forceinline__ void transpose8(const uint4 (&r)[8], uint4 (&t)[8]) {
  uint32_t w[8][4], o[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    w[i][0] = r[i].x;
    w[i][1] = r[i].y;
    w[i][2] = r[i].z;
    w[i][3] = r[i].w;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const uint32_t a = w[2 * rr][q], b = w[2 * rr + 1][q];
      o[2 * q][rr] = __byte_perm(a, b, 0x5410);      // element 2q of rows 2rr, 2rr+1
      o[2 * q + 1][rr] = __byte_perm(a, b, 0x7632);  // element 2q+1
    }
#pragma unroll
  for (int j = 0; j < 8; ++j) t[j] = make_uint4(o[j][0], o[j][1], o[j][2], o[j][3]);
}

// Source of the weight gradient: CIN == 32, the layer input as BF16 NHWC [B][S][S][32];
// CIN == 2, the network input as float32 NCHW [B][2][64][64], rounded to BF16 here.
template <int CIN>
__global__ void __launch_bounds__(kWgThreads, 1)
    wgrad_kernel(const void *__restrict__ src_v, const bf16 *__restrict__ dz, float *__restrict__ part, int B,
                 int lg_s, int lg_g, int stride, int per_chunk, uint32_t *status) {
  using Sh = WgShape<CIN>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * (Sh::A_STAGE + Sh::B_STAGE));
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = 1 << lg_s, G = 1 << lg_g;
  const int P = B << (2 * lg_g);
  const int p_begin = blockIdx.x * per_chunk;
  const int p_end = min(P, p_begin + per_chunk);
  const int nst = (p_end - p_begin + kWgStage - 1) / kWgStage;
  constexpr int NC = Sh::ROWS - Sh::NDATA;  // constant rows per K chunk

  for (int i = tid; i < 2 * 8 * NC; i += kWgThreads) {  // the ones row and the zero rows
    const int st = i / (8 * NC), kc = (i / NC) % 8, row = Sh::NDATA + i % NC;
    const uint32_t v = row == Sh::NDATA ? 0x3F803F80u : 0u;  // BF16 1.0 pairs
    *reinterpret_cast<uint4 *>(smem + st * Sh::A_STAGE + kc * Sh::LBO_A + row * 16) = make_uint4(v, v, v, v);
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(slot, Sh::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const uint4 zero = make_uint4(0, 0, 0, 0);

  bool failed = false;
  for (int s = 0; s < nst; ++s) {
    const int buf = s & 1;
    if (s >= 2) {  // the MMAs of stage s - 2 have read this buffer
      const bool ok = mbar_wait_bounded(&bar[buf], (uint32_t)(((s - 2) >> 1) & 1), status);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    uint8_t *sA = smem + buf * Sh::A_STAGE;
    uint8_t *sB = smem + 2 * Sh::A_STAGE + buf * Sh::B_STAGE;
    const int p0 = p_begin + s * kWgStage;
    constexpr int NG = CIN == kCh ? kTaps * 4 : Sh::NDATA;  // A units per K chunk
    for (int u = tid; u < (NG + 4) * 8; u += kWgThreads) {
      const int kc = u & 7, g = u >> 3;
      if (g >= NG) {  // dz: 8 pixels x 8 output channels -> rows o, K = pixels
        const int o8 = g - NG;
        uint4 r[8], t[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int p = p0 + kc * 8 + e;
          r[e] = p < p_end ? __ldg(reinterpret_cast<const uint4 *>(dz + (size_t)p * kCh) + o8) : zero;
        }
        transpose8(r, t);
        uint8_t *dst = sB + kc * Sh::LBO_B + o8 * 128;
#pragma unroll
        for (int j = 0; j < 8; ++j) *reinterpret_cast<uint4 *>(dst + j * 16) = t[j];
      } else if (CIN == kCh) {  // 8 pixels x 8 input channels of one tap -> rows (tap, c)
        const int tap = g >> 2, c8 = g & 3, dy = tap / 3, dx = tap % 3;
        const bf16 *src = static_cast<const bf16 *>(src_v);
        uint4 r[8], t[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int p = p0 + kc * 8 + e;
          const int b = p >> (2 * lg_g), y = (p >> lg_g) & (G - 1), x = p & (G - 1);
          const int yy = stride * y + dy - 1, xx = stride * x + dx - 1;
          const bool ok = p < p_end && yy >= 0 && yy < S && xx >= 0 && xx < S;
          const size_t pix = ((((size_t)b << lg_s) + (ok ? yy : 0)) << lg_s) + (ok ? xx : 0);
          r[e] = ok ? __ldg(reinterpret_cast<const uint4 *>(src + pix * kCh) + c8) : zero;
        }
        transpose8(r, t);
        uint8_t *dst = sA + kc * Sh::LBO_A + (tap * kCh + c8 * 8) * 16;
#pragma unroll
        for (int j = 0; j < 8; ++j) *reinterpret_cast<uint4 *>(dst + j * 16) = t[j];
      } else {  // first layer: row (tap, c) of 8 pixels straight from the float input
        const int tap = g / CIN, c = g % CIN, dy = tap / 3, dx = tap % 3;
        const float *src = static_cast<const float *>(src_v);
        float f[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int p = p0 + kc * 8 + e;
          const int b = p >> (2 * lg_g), y = (p >> lg_g) & (G - 1), x = p & (G - 1);
          const int yy = stride * y + dy - 1, xx = stride * x + dx - 1;
          const bool ok = p < p_end && yy >= 0 && yy < S && xx >= 0 && xx < S;
          f[e] = ok ? __ldg(src + (((((size_t)b * CIN + c) << lg_s) + yy) << lg_s) + xx) : 0.0f;
        }
        *reinterpret_cast<uint4 *>(sA + kc * Sh::LBO_A + g * 16) =
            make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int k = 0; k < kWgStage / 16; ++k)
#pragma unroll
        for (int i = 0; i < Sh::MT; ++i)
          umma_f16(tmem + 32u * i, sdesc(a0 + k * 2u * Sh::LBO_A + i * 2048u, Sh::LBO_A, 128u),
                   sdesc(b0 + k * 2u * Sh::LBO_B, Sh::LBO_B, 128u), kIdesc, (s > 0 || k > 0) ? 1u : 0u);
      umma_commit(&bar[buf]);
    }
  }
  if (!failed && nst > 0) {  // the last commit covers every MMA before it
    const int sl = nst - 1;
    const bool ok = mbar_wait_bounded(&bar[sl & 1], (uint32_t)((sl >> 1) & 1), status);
    failed = __syncthreads_or(!ok);
  }
  if (!failed && nst > 0) {
    tc_fence_after();
    const int q = warp & 3, h = warp >> 2;
#pragma unroll
    for (int i = 0; i < Sh::MT; ++i) {
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + 32u * i + 16u * h, r);
      tmem_ld_wait();
      const int row = 128 * i + 32 * q + lane;
      if (row <= Sh::NDATA) {
        float4 *dst = reinterpret_cast<float4 *>(part + ((size_t)blockIdx.x * (Sh::NDATA + 1) + row) * kCh + 16 * h);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]), __uint_as_float(r[4 * j + 2]),
                               __uint_as_float(r[4 * j + 3]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, Sh::TMEM_COLS);
}

// Partial sums of the chunks, added in chunk order: dw[o][c][tap], db[o].
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int nchunks, int cin, float *__restrict__ gw,
                                    float *__restrict__ gb) {
  const int rows = cin * kTaps + 1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * kCh) return;
  const int row = i / kCh, o = i % kCh;
  float s = 0.0f;
  for (int c = 0; c < nchunks; ++c) s += part[((size_t)c * rows + row) * kCh + o];
  if (row < cin * kTaps) gw[((size_t)o * cin + row % cin) * 9 + row / cin] = s;
  else gb[o] = s;
}

// pooled[b][c] = mean over the 8x8 positions; out[b][j] = fcb[j] + sum_c fcw[j][c] pooled[b][c]
__global__ void pool_fc_kernel(const bf16 *__restrict__ act, const float *__restrict__ fcw,
                               const float *__restrict__ fcb, float *__restrict__ pooled, float *__restrict__ out,
                               int n_out) {
  __shared__ float pl[kCh];
  const int b = blockIdx.x;
  if (threadIdx.x < kCh) {
    const bf16 *a = act + (size_t)b * 64 * kCh + threadIdx.x;
    float s = 0.0f;
    for (int i = 0; i < 64; ++i) s += __bfloat162float(a[i * kCh]);
    pl[threadIdx.x] = s * (1.0f / 64.0f);
    pooled[b * kCh + threadIdx.x] = pl[threadIdx.x];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n_out; j += blockDim.x) {
    float s = fcb[j];
    for (int c = 0; c < kCh; ++c) s = fmaf(fcw[j * kCh + c], pl[c], s);
    out[(size_t)b * n_out + j] = s;
  }
}

// loss = mean (out - target)^2 (accumulated into *loss); dout = 2 (out - target) / (B n_out)
__global__ void mse_kernel(const float *__restrict__ out, const float *__restrict__ target, float *__restrict__ dout,
                           float *loss, int n) {
  __shared__ float red[32];
  float s = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float d = out[i] - target[i];
    dout[i] = 2.0f * d / (float)n;
    s = fmaf(d, d, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    atomicAdd(loss, t / (float)n);
  }
}

// linear layer gradients and dL/dpooled
__global__ void fc_bwd_kernel(const float *__restrict__ dout, const float *__restrict__ pooled,
                              const float *__restrict__ fcw, float *__restrict__ dfcw, float *__restrict__ dfcb,
                              float *__restrict__ dpooled, int B, int n_out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_out * kCh) {  // dfcw[j][c] = sum_b dout[b][j] pooled[b][c]
    const int j = t / kCh, c = t % kCh;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s = fmaf(dout[(size_t)b * n_out + j], pooled[b * kCh + c], s);
    dfcw[t] = s;
  }
  if (t < n_out) {
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += dout[(size_t)b * n_out + t];
    dfcb[t] = s;
  }
  if (t < B * kCh) {  // dpooled[b][c] = sum_j dout[b][j] fcw[j][c]
    const int b = t / kCh, c = t % kCh;
    float s = 0.0f;
    for (int j = 0; j < n_out; ++j) s = fmaf(dout[(size_t)b * n_out + j], fcw[j * kCh + c], s);
    dpooled[t] = s;
  }
}

// Gradient at the last layer's pre-activation: dpooled / 64 at every position, masked by
// the ReLU (act > 0), stored BF16 NHWC.
__global__ void unpool_mask_kernel(const float *__restrict__ dpooled, const bf16 *__restrict__ act,
                                   bf16 *__restrict__ dz, int B) {
  const int n = B * 64 * kCh;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g = dpooled[(i >> 11) * kCh + (i & 31)] * (1.0f / 64.0f);
    dz[i] = __float2bfloat16_rn(__bfloat162float(act[i]) > 0.0f ? g : 0.0f);
  }
}

__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

int grid_for(size_t n, int threads = 256) {
  const size_t g = (n + threads - 1) / threads;
  return (int)(g < 8192 ? (g > 0 ? g : 1) : 8192);
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <int MODE>
int conv_mma(const bf16 *src, const bf16 *wpack, const float *bias, const bf16 *mask, bf16 *out, int B, int lg_s,
             int lg_g, int stride, int nsm, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(conv_mma_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kConvSmem);
  if (e != cudaSuccess) return cuda_status(e, "network convolution attributes");
  const int ntiles = ((B << (2 * lg_g)) + 127) >> 7;
  const int grid = ntiles < 2 * nsm ? ntiles : 2 * nsm;
  conv_mma_kernel<MODE><<<grid, kConvThreads, kConvSmem, s>>>(src, wpack, bias, mask, out, B, lg_s, lg_g, stride,
                                                              device_status_word());
  return cuda_status(cudaGetLastError(), "network convolution");
}

template <int CIN>
int wgrad(const void *src, const bf16 *dz, float *part, float *gw, float *gb, int B, int lg_s, int lg_g, int stride,
          cudaStream_t s) {
  using Sh = WgShape<CIN>;
  cudaError_t e = cudaFuncSetAttribute(wgrad_kernel<CIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
  if (e != cudaSuccess) return cuda_status(e, "network weight-gradient attributes");
  const int P = B << (2 * lg_g);
  const int per = wg_per_chunk(P), nch = wg_nchunks(P);
  wgrad_kernel<CIN><<<nch, kWgThreads, Sh::SMEM, s>>>(src, dz, part, B, lg_s, lg_g, stride, per, device_status_word());
  const int rows = wg_rows(CIN);
  wgrad_reduce_kernel<<<(rows * kCh + 255) / 256, 256, 0, s>>>(part, nch, CIN, gw, gb);
  return cuda_status(cudaGetLastError(), "network weight gradient");
}

struct Bufs {
  float *wq;
  bf16 *wf[kLayers], *wd[kLayers], *act[kLayers], *dz[kLayers];
  float *pooled, *dpooled, *out, *dout, *part;
};

Bufs bufs(void *ws_v, const Work &Wk) {
  uint8_t *ws = static_cast<uint8_t *>(ws_v);
  Bufs b{};
  b.wq = reinterpret_cast<float *>(ws + Wk.wq);
  for (int i = 0; i < kLayers; ++i) {
    b.wf[i] = i > 0 ? reinterpret_cast<bf16 *>(ws + Wk.wf[i]) : nullptr;
    b.wd[i] = i > 0 ? reinterpret_cast<bf16 *>(ws + Wk.wd[i]) : nullptr;
    b.act[i] = reinterpret_cast<bf16 *>(ws + Wk.act[i]);
    b.dz[i] = reinterpret_cast<bf16 *>(ws + Wk.dz[i]);
  }
  b.pooled = reinterpret_cast<float *>(ws + Wk.pooled);
  b.dpooled = reinterpret_cast<float *>(ws + Wk.dpooled);
  b.out = reinterpret_cast<float *>(ws + Wk.out);
  b.dout = reinterpret_cast<float *>(ws + Wk.dout);
  b.part = reinterpret_cast<float *>(ws + Wk.part);
  return b;
}

int pack(const float *params, const Layout &L, const Bufs &b, cudaStream_t s) {
  pack_kernel<<<grid_for(L.total + 3 * kPack), 256, 0, s>>>(params, b.wq, (int)L.total, b.wf[1], b.wd[1], b.wf[2],
                                                           b.wd[2], b.wf[3], b.wd[3], L.w[1], L.w[2], L.w[3]);
  return cuda_status(cudaGetLastError(), "network weight packing");
}

// x -> act[0..3] -> pooled -> out (parameters already packed)
int forward(const float *x, const Layout &L, const Bufs &b, int B, int n_out, float *out, int nsm, cudaStream_t s) {
  conv1_fwd_kernel<<<grid_for((size_t)B * 1024), 256, 0, s>>>(x, b.wq + L.w[0], b.wq + L.b[0], b.act[0], B);
  int st = cuda_status(cudaGetLastError(), "network first layer");
  for (int li = 1; li < kLayers && st == SVK_OK; ++li)
    st = conv_mma<kFwd>(b.act[li - 1], b.wf[li], b.wq + L.b[li], nullptr, b.act[li], B, kLgIn[li], kLgOut[li],
                        kStride[li], nsm, s);
  if (st != SVK_OK) return st;
  pool_fc_kernel<<<B, 64, 0, s>>>(b.act[kLayers - 1], b.wq + L.fcw, b.wq + L.fcb, b.pooled, out, n_out);
  return cuda_status(cudaGetLastError(), "network pooling");
}

int check_ws(void *ws, size_t ws_bytes, int B, int n_out) {
  if (!ws || ws_bytes < work_layout(B, n_out).total)
    return set_error(SVK_ERR_WORKSPACE, "network workspace too small");
  if (reinterpret_cast<uintptr_t>(ws) % 256)
    return set_error(SVK_ERR_ARG, "network workspace must be 256-byte aligned");
  return SVK_OK;
}

// Field fit of local coefficient predictions: for each stamp k-vector a_s at position
// (x_s, y_s), least squares for c[k][t] in a_k(x_s, y_s) = sum_t c[k][t] m_t(xt_s, yt_s):
// one T x T FP64 normal matrix shared by every k, Cholesky in shared memory, then N solves.
__global__ void field_fit_kernel(const float *__restrict__ local, const int *__restrict__ xy, const float *__restrict__ wts,
                                 int S, int N, int W, int H, int degree, double *__restrict__ coeffs, int *info) {
  __shared__ double A[10][10];
  __shared__ double Gc[10][10];
  __shared__ int bad;
  const int T = (degree + 1) * (degree + 2) / 2;
  auto mono = [&](int s, double *m) {
    const double xt = W > 1 ? (2.0 * xy[2 * s] - (W - 1)) / (double)(W - 1) : 0.0;
    const double yt = H > 1 ? (2.0 * xy[2 * s + 1] - (H - 1)) / (double)(H - 1) : 0.0;
    int t = 0;
    double xi = 1.0;
    for (int i = 0; i <= degree; ++i) {
      double yj = 1.0;
      for (int j = 0; j <= degree - i; ++j) {
        m[t++] = xi * yj;
        yj *= yt;
      }
      xi *= xt;
    }
  };
  if (threadIdx.x < T * T) {
    const int r = threadIdx.x / T, c = threadIdx.x % T;
    double acc = 0.0, m[10];
    for (int s = 0; s < S; ++s) {
      mono(s, m);
      acc += (wts ? (double)wts[s] : 1.0) * m[r] * m[c];
    }
    A[r][c] = acc;
  }
  if (threadIdx.x == 0) bad = -1;
  __syncthreads();
  if (threadIdx.x == 0) {  // T <= 10: serial textbook Cholesky
    for (int j = 0; j < T && bad < 0; ++j) {
      double d = A[j][j];
      for (int k = 0; k < j; ++k) d -= Gc[j][k] * Gc[j][k];
      if (!(d > 0.0)) {
        bad = j;
        break;
      }
      Gc[j][j] = sqrt(d);
      for (int i = j + 1; i < T; ++i) {
        double v = A[i][j];
        for (int k = 0; k < j; ++k) v -= Gc[i][k] * Gc[j][k];
        Gc[i][j] = v / Gc[j][j];
      }
    }
    *info = bad;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    double b[10], y[10], m[10];
    for (int t = 0; t < T; ++t) b[t] = 0.0;
    for (int s = 0; s < S; ++s) {
      mono(s, m);
      const double a = (wts ? (double)wts[s] : 1.0) * (double)local[(size_t)s * N + k];
      for (int t = 0; t < T; ++t) b[t] += m[t] * a;
    }
    if (bad >= 0) {
      for (int t = 0; t < T; ++t) coeffs[(size_t)k * T + t] = 0.0;
      continue;
    }
    for (int i = 0; i < T; ++i) {
      double v = b[i];
      for (int q = 0; q < i; ++q) v -= Gc[i][q] * y[q];
      y[i] = v / Gc[i][i];
    }
    for (int i = T - 1; i >= 0; --i) {
      double v = y[i];
      for (int q = i + 1; q < T; ++q) v -= Gc[q][i] * b[q];
      b[i] = v / Gc[i][i];
    }
    for (int t = 0; t < T; ++t) coeffs[(size_t)k * T + t] = b[t];
  }
}

}  // namespace

int cnn_field_fit(const float *local, const int *xy, const float *wts, int S, int N, int W, int H, int degree,
                  double *coeffs, int *info, cudaStream_t s) {
  field_fit_kernel<<<1, 128, 0, s>>>(local, xy, wts, S, N, W, H, degree, coeffs, info);
  return cuda_status(cudaGetLastError(), "field fit");
}

int cnn_param_count(int n_out) { return (int)param_layout(n_out).total; }
size_t cnn_workspace_size(int B, int n_out) { return work_layout(B, n_out).total; }

int cnn_forward(const float *params, const float *x, int B, int n_out, float *out, void *ws, size_t ws_bytes,
                cudaStream_t s) {
  int st = check_ws(ws, ws_bytes, B, n_out);
  if (st != SVK_OK) return st;
  const Layout L = param_layout(n_out);
  const Bufs b = bufs(ws, work_layout(B, n_out));
  if ((st = pack(params, L, b, s)) != SVK_OK) return st;
  return forward(x, L, b, B, n_out, out, sm_count(), s);
}

int cnn_gradient(const float *params, const float *x, const float *target, int B, int n_out, float *grad, float *loss,
                 void *ws, size_t ws_bytes, cudaStream_t s) {
  int st = check_ws(ws, ws_bytes, B, n_out);
  if (st != SVK_OK) return st;
  const Layout L = param_layout(n_out);
  const Bufs b = bufs(ws, work_layout(B, n_out));
  const int nsm = sm_count();
  if ((st = pack(params, L, b, s)) != SVK_OK) return st;
  if ((st = forward(x, L, b, B, n_out, b.out, nsm, s)) != SVK_OK) return st;
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), s);
  if (e != cudaSuccess) return cuda_status(e, "loss reset");
  const int n = B * n_out;
  mse_kernel<<<grid_for(n), 256, 0, s>>>(b.out, target, b.dout, loss, n);
  fc_bwd_kernel<<<grid_for((size_t)(n_out * kCh > B * kCh ? n_out * kCh : B * kCh)), 256, 0, s>>>(
      b.dout, b.pooled, b.wq + L.fcw, grad + L.fcw, grad + L.fcb, b.dpooled, B, n_out);
  unpool_mask_kernel<<<grid_for((size_t)B * 64 * kCh), 256, 0, s>>>(b.dpooled, b.act[kLayers - 1],
                                                                    b.dz[kLayers - 1], B);
  if ((st = cuda_status(cudaGetLastError(), "network output gradient")) != SVK_OK) return st;
  for (int li = kLayers - 1; li >= 1; --li) {
    st = wgrad<kCh>(b.act[li - 1], b.dz[li], b.part, grad + L.w[li], grad + L.b[li], B, kLgIn[li], kLgOut[li],
                    kStride[li], s);
    if (st == SVK_OK)
      st = conv_mma<kDgrad>(b.dz[li], b.wd[li], nullptr, b.act[li - 1], b.dz[li - 1], B, kLgOut[li], kLgIn[li],
                            kStride[li], nsm, s);
    if (st != SVK_OK) return st;
  }
  return wgrad<2>(x, b.dz[0], b.part, grad + L.w[0], grad + L.b[0], B, kLgIn[0], kLgOut[0], kStride[0], s);
}

int cnn_adam(float *params, float *m, float *v, const float *grad, int n, int step, float lr, float b1, float b2,
             float eps, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  adam_kernel<<<grid_for(n), 256, 0, s>>>(params, m, v, grad, n, lr, b1, b2, eps, c1, c2);
  return cuda_status(cudaGetLastError(), "adam");
}

}  // namespace svk
