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
// Every convolution runs on the tensor cores (tcgen05.mma, BF16 operands, FP32
// accumulators in TMEM) as an implicit GEMM over NHWC activations:
//   forward      rows = output pixels, K = 9 taps x input channels (18, padded to 32,
//                for the 2-channel first layer), N = 32 outputs;
//   data grad    rows = input pixels,  K = the taps that hit the strided grid x 32 output
//                channels (the transposed convolution; for stride 2 the rows are split
//                into the four parity classes, which have 1, 2 or 4 such taps);
//   weight grad  rows = 9 taps x input channels (+ a row of ones for the bias),
//                K = output pixels (split over CTAs, partial sums reduced in a fixed
//                order, so the gradient is deterministic), N = 32 outputs.
// Every kernel is launched as a programmatic dependent of the one before; the weight
// gradients of the 32-channel layers run on a second stream beside the data gradients
// (cnn_gradient).
#include <cuda_bf16.h>

#include <mutex>

#include "svk_common.cuh"
#include "svk_internal.h"
#include "svk_umma.cuh"

namespace svk {
namespace {

constexpr int kCh = 32, kLayers = 4, kTaps = 9;
constexpr int kCin[kLayers] = {2, kCh, kCh, kCh};
constexpr int kStride[kLayers] = {2, 2, 2, 1};
constexpr int kHout[kLayers] = {32, 16, 8, 8};
constexpr int kLgIn[kLayers] = {6, 5, 4, 3};   // log2 kHin
constexpr int kLgOut[kLayers] = {5, 4, 3, 3};  // log2 kHout

// Packed UMMA B operand of a 32-channel layer: K = tap * 32 + channel (288), 32 rows, in
// the K-major no-swizzle layout: 36 core-matrix columns of [32 rows][8 BF16].
constexpr int kK = kTaps * kCh;            // 288
constexpr int kPack = kK * kCh;            // 9216 BF16 per packed operand
constexpr uint32_t kPackBytes = kPack * 2; // 18,432
constexpr int kPack0 = 4 * kCh * 8;         // first layer: K = 18 padded to 32, 1024 BF16
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

// Weight-gradient split: K (the output pixels of a layer, a multiple of 64) in chunks of
// whole pipeline stages (64 pixels for a 32-channel layer, 128 for the first layer):
// about 152 chunks of at least two stages for a 32-channel layer (one CTA on each of 152
// SMs), about 304 for the first layer (two per SM).  Depends on the batch only, so the
// gradient is deterministic.
int wg_stage_px(int cin) { return cin == kCh ? 64 : 128; }
int wg_target(int cin) { return cin == kCh ? 152 : 304; }
int wg_per_chunk(int P, int cin) {
  const int px = wg_stage_px(cin), stages = (P + px - 1) / px;
  const int per = (stages + wg_target(cin) - 1) / wg_target(cin);
  return px * (cin == kCh && per < 2 ? 2 : per);
}
int wg_nchunks(int P, int cin) { return (P + wg_per_chunk(P, cin) - 1) / wg_per_chunk(P, cin); }
int wg_rows(int cin) { return cin * kTaps + 1; }  // taps x channels, then the bias row

struct Work {  // byte offsets into the workspace
  size_t wq;                     // float[param total]: parameters rounded to BF16
  size_t wf[kLayers], wd[kLayers];  // packed BF16 operands (forward, data grad), layers 1..3
  size_t act[kLayers], dz[kLayers];  // BF16 NHWC [B][H][H][32]: post-ReLU, pre-activation grad
  size_t pooled, out, dout, part[kLayers], total;
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
  w.wf[0] = take(kPack0 * sizeof(bf16));
  for (int i = 1; i < kLayers; ++i) {
    w.wf[i] = take(kPackBytes);
    w.wd[i] = take(kPackBytes);
  }
  for (int i = 0; i < kLayers; ++i) {
    const size_t n = (size_t)B * kCh * kHout[i] * kHout[i];
    w.act[i] = take(n * sizeof(bf16));
    w.dz[i] = take(n * sizeof(bf16));
    const int P = B * kHout[i] * kHout[i];
    w.part[i] = take((size_t)wg_nchunks(P, kCin[i]) * wg_rows(kCin[i]) * kCh * sizeof(float));
  }
  w.pooled = take((size_t)B * kCh * sizeof(float));
  w.out = take((size_t)B * n_out * sizeof(float));
  w.dout = take((size_t)B * n_out * sizeof(float));
  w.total = o;
  return w;
}

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

// 32-byte global accesses (one sector per lane and instruction); addresses 32-byte aligned.
__device__ __forceinline__ void ld_nc_v8(const void *p, uint32_t (&r)[8]) {
  asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "l"(p));
}

__device__ __forceinline__ void st_v8(void *p, const uint32_t (&r)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(r[0]), "r"(r[1]), "r"(r[2]),
               "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

__device__ __forceinline__ float lo_f(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float hi_f(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// Rounded parameters (FP32 values of the BF16 weights) and the packed tensor-core
// operands.  Layers 1..3 (K = 8 j + t = 32 tap + channel):  wf[j][o][t] = W[o][c][tap]
// with c the K channel, wd[j][c][t] = W[o][c][tap] with o the K channel.  Layer 0
// (K = 2 tap + c < 18, zero above): wf0[j][o][t] = W0[o][c][tap].
__global__ void pack_kernel(const float *__restrict__ p, float *__restrict__ wq, int n_params, bf16 *wf0, bf16 *wf1,
                            bf16 *wd1, bf16 *wf2, bf16 *wd2, bf16 *wf3, bf16 *wd3, size_t w0, size_t w1, size_t w2,
                            size_t w3, float *loss) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  if (loss && blockIdx.x == 0 && threadIdx.x == 0) *loss = 0.0f;  // the gradient call's loss sum starts here
  const int n = n_params + kPack0 + 3 * kPack;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < n_params) {
      wq[i] = bf16r(p[i]);
      continue;
    }
    if (i < n_params + kPack0) {
      const int e = i - n_params, j = e >> 8, r = (e >> 3) & 31, k = 8 * j + (e & 7);
      wf0[e] = __float2bfloat16_rn(k < 2 * kTaps ? p[w0 + (r * 2 + (k & 1)) * 9 + (k >> 1)] : 0.0f);
      continue;
    }
    const int l = (i - n_params - kPack0) / kPack, e = (i - n_params - kPack0) % kPack;
    const int j = e >> 8, r = (e >> 3) & 31, t = e & 7;
    const int k = 8 * j + t, tap = k >> 5, ch = k & 31;
    const float *w = p + (l == 0 ? w1 : l == 1 ? w2 : w3);
    bf16 *f = l == 0 ? wf1 : l == 1 ? wf2 : wf3;
    bf16 *d = l == 0 ? wd1 : l == 1 ? wd2 : wd3;
    f[e] = __float2bfloat16_rn(w[(r * kCh + ch) * 9 + tap]);  // o = r, c = ch
    d[e] = __float2bfloat16_rn(w[(ch * kCh + r) * 9 + tap]);  // c = r, o = ch
  }
}

// ------------------------------------------------ first layer forward on tcgen05
// K = 9 taps x 2 channels = 18 (k = 2 tap + c), zero-padded to 32 (4 chunks of 8).  A
// tile is 128 output pixels = 4 rows of the 32 x 32 grid; one TMA load (issued a tile
// ahead, double-buffered) stages the 9 input rows those rows read, 2 channels of 64
// floats (zero fill above the stamp), and each thread builds its pixel's A row from them
// (rounded to BF16).  128 threads: the epilogue warp q drains TMEM lanes 32 q .. 32 q + 31
// (bias, ReLU, BF16 NHWC rows of 64 bytes).
constexpr int kC1Threads = 128;
constexpr int kC1Chunks = 4;
constexpr int kC1Rows = 9;                                // input rows of 4 output rows
constexpr uint32_t kC1XBytes = 2 * kC1Rows * 64 * 4;      // [c][9 rows][64 floats] = 4608
constexpr uint32_t kC1XStage = 5120;                      // rounded to 1 KB
constexpr uint32_t kC1ABytes = kC1Chunks * 128 * 16;      // [4][128 rows][16 B]
constexpr uint32_t kC1BBytes = kC1Chunks * kCh * 16;      // [4][32 rows][16 B]
constexpr uint32_t kC1Smem = 2 * kC1XStage + kC1ABytes + kC1BBytes + 64 + 1024;

__global__ void __launch_bounds__(kC1Threads, 6)
    conv1_mma_kernel(const __grid_constant__ CUtensorMap xm, const bf16 *__restrict__ wpack,
                     const float *__restrict__ bias, bf16 *__restrict__ out, int B, uint32_t *status) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sx = sm;                          // two staged input blocks
  uint8_t *sA = sm + 2 * kC1XStage;
  uint8_t *sB = sA + kC1ABytes;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sB + kC1BBytes);
  uint64_t *tbar = bar + 1;  // two: the staged input of each buffer landed
  uint32_t *slot = reinterpret_cast<uint32_t *>(tbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int S = 64, lg_g = 5, G = 32;  // 64 x 64 inputs, 32 x 32 outputs, stride 2
  const int P = B << (2 * lg_g);
  const int ntiles = (P + 127) >> 7;

  {  // the packed weights, once
    const uint4 *g = reinterpret_cast<const uint4 *>(wpack);
    uint4 *d = reinterpret_cast<uint4 *>(sB);
    for (int i = tid; i < (int)(kC1BBytes / 16); i += kC1Threads) d[i] = __ldg(g + i);
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(&tbar[0], 1);
    mbar_init(&tbar[1], 1);
    fence_mbar_init();
    prefetch_tmap(&xm);
  }
  if (warp == 0) tmem_alloc(slot, 32);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const uint32_t aBase = smem_u32(sA), bBase = smem_u32(sB);
  float bv[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) bv[i] = __ldg(bias + i);

  uint32_t issued = 0;  // loads issued (thread 0)
  auto issue = [&](int tile, int sb) {  // rows 2 y0 - 1 .. 2 y0 + 7 of the tile's stamp
    const int p = tile << 7, b = p >> (2 * lg_g), y0 = (p >> lg_g) & (G - 1);
    mbar_arrive_expect_tx(&tbar[sb], kC1XBytes);
    tma_load_4d(sx + sb * kC1XStage, &xm, &tbar[sb], 0, 2 * y0 - 1, 0, b);
    ++issued;
  };
  if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  uint32_t it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int buf = it & 1;
    const bool okx = mbar_wait_bounded(&tbar[buf], (it >> 1) & 1u, status);
    if (__syncthreads_or(!okx)) break;
    {  // row tid: output pixel (y, xo); input row 2 y + dy - 1 is staged row 2 (y - y0) + dy
      const float *xs = reinterpret_cast<const float *>(sx + buf * kC1XStage);  // [c][9][64]
      const int p = (tile << 7) + tid;
      const bool valid = p < P;
      const int y = (p >> lg_g) & (G - 1), xo = p & (G - 1), yl = y - (((tile << 7) >> lg_g) & (G - 1));
      float f[2 * kTaps];
#pragma unroll
      for (int t = 0; t < kTaps; ++t) {
        const int xx = 2 * xo + t % 3 - 1;
        const bool ok = valid && xx >= 0 && xx < S;
#pragma unroll
        for (int c = 0; c < 2; ++c) f[2 * t + c] = ok ? xs[(c * kC1Rows + 2 * yl + t / 3) * S + xx] : 0.0f;
      }
      uint8_t *row = sA + (uint32_t)tid * 16u;  // the MMAs of the previous tile have completed
      *reinterpret_cast<uint4 *>(row) =
          make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
      *reinterpret_cast<uint4 *>(row + 2048) =
          make_uint4(pack2(f[8], f[9]), pack2(f[10], f[11]), pack2(f[12], f[13]), pack2(f[14], f[15]));
      *reinterpret_cast<uint4 *>(row + 4096) = make_uint4(pack2(f[16], f[17]), 0u, 0u, 0u);
      *reinterpret_cast<uint4 *>(row + 6144) = make_uint4(0u, 0u, 0u, 0u);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int k = 0; k < kC1Chunks / 2; ++k)
        umma_f16(tmem, sdesc(aBase + (uint32_t)k * 2u * 2048u, 2048u, 128u),
                 sdesc(bBase + (uint32_t)k * 2u * 512u, 512u, 128u), kIdesc, k > 0 ? 1u : 0u);
      umma_commit(bar);
      // the other staged block was read before the barrier above: the next tile's rows
      if (tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x, buf ^ 1);
    }
    const bool ok = mbar_wait_bounded(bar, it & 1u, status);
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    const int pr = (tile << 7) + 32 * warp + lane;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * hh), r);
      tmem_ld_wait();
      if (pr < P) {
        uint32_t o32[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
          o32[i] = pack2(fmaxf(__uint_as_float(r[2 * i]) + bv[16 * hh + 2 * i], 0.0f),
                         fmaxf(__uint_as_float(r[2 * i + 1]) + bv[16 * hh + 2 * i + 1], 0.0f));
        st_v8(out + (size_t)pr * kCh + 16 * hh, o32);
      }
    }
    tc_fence_before();
  }
  // after a wait gave up, a load issued ahead may still be in flight: wait for it (bounded)
  if (tid == 0 && issued > it)
    mbar_wait_bounded(&tbar[(issued - 1) & 1], ((issued - 1) >> 1) & 1u, status);
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

enum ConvMode { kFwd = 0, kDgrad = 1 };

// --------------------------------- 32-channel layers, TMA-fed: forward and data grad
// A 128-row tile covers whole rows of one image (grid side 16: 8 rows) or two whole
// images (side 8); for the stride-2 data gradient the grid is a parity class of the
// layer input (side G / 2), rows in class order.  For each tap one 4-D TMA load brings
// the tile's source pixels, 32 channels each, with zero fill outside the image, into an
// 8 KB stage in the 64-byte-swizzled K-major UMMA layout (128 rows of 64 bytes, 8-row
// groups 512 bytes apart); two MMAs of K = 16 take the tap's channels 0-15 and 16-31
// (start address + 32 bytes).  Sources:
//   forward      pixel (s x + dx - 1, s y + dy - 1): traversal stride s, 9 taps;
//   data grad    stride 1: pixel (x + 1 - dx, y + 1 - dy), 9 taps; stride 2, class
//                (py, px): pixel (xc + (px && ix == 0), yc + (py && iy == 0)) for the
//                class's taps dy = ty0 + 2 iy, dx = tx0 + 2 ix (1, 2 or 4 of them).
// Warp 0 issues the loads, warp 1 the MMAs into one of two TMEM accumulators, warps 2-5
// drain the other: forward adds the bias and applies the ReLU, data grad multiplies by
// the ReLU mask of the layer below; both store BF16 rows of 64 bytes.
constexpr int kTfStages = 6;
constexpr uint32_t kTfStageBytes = 128 * 64;  // one tap's A operand
constexpr int kTfThreads = 192;
constexpr uint32_t kTfSmem = kTfStages * kTfStageBytes + kPackBytes + 256 + 1024;  // + barriers, alignment

// K-major, 64-byte swizzle: start >> 4 | (LBO 16 B, unused) | SBO 512 B >> 4 | version 1 |
// layout 4 (SWIZZLE_64B) at bits 61-63.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(512u >> 4) << 32) | (1ull << 46) |
         (4ull << 61);
}

struct TfGeom {
  int lg_c;       // log2 of the row grid side (the class grid for the stride-2 data grad)
  int lg_g;       // log2 of the output grid side
  int TH, NB;     // rows per tile, images per tile
  int tpi;        // tiles per image (NB == 1)
  int tiles_c;    // tiles per class
  int stride;     // the layer's stride
  int split;      // data grad with stride 2: four parity classes
};

// Tap i of a tile (in registers: the producer and MMA threads call this per tap): the
// source offsets (ox, oy) added to (f x0, f y0), f the forward stride (1 for the data
// grad), and the weight tap it reads.  ntaps: 9, or the class's 1, 2 or 4.
__device__ __forceinline__ int tf_ntaps(bool split, int cls) {
  return split ? ((cls >> 1) ? 2 : 1) * ((cls & 1) ? 2 : 1) : kTaps;
}

template <int MODE>
__device__ __forceinline__ void tf_tap(bool split, int cls, int i, int &ox, int &oy, int &wtap) {
  if (MODE == kFwd || !split) {
    const int dy = i / 3, dx = i - 3 * dy;
    ox = MODE == kFwd ? dx - 1 : 1 - dx;
    oy = MODE == kFwd ? dy - 1 : 1 - dy;
    wtap = i;
  } else {
    const int py = cls >> 1, px = cls & 1;
    const int iy = px ? i >> 1 : i, ix = px ? i & 1 : 0;  // ndx = 2 when px
    ox = px & (ix == 0);
    oy = py & (iy == 0);
    wtap = ((py ? 0 : 1) + 2 * iy) * 3 + (px ? 0 : 1) + 2 * ix;
  }
}

template <int MODE>
__global__ void __launch_bounds__(kTfThreads, 2)
    conv_tma_kernel(const __grid_constant__ CUtensorMap src, const bf16 *__restrict__ wpack,
                    const float *__restrict__ bias, const bf16 *__restrict__ mask, bf16 *__restrict__ out, int B,
                    const TfGeom geo, uint32_t *status) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = sm;                                  // kTfStages x 8 KB, 1024-byte aligned
  uint8_t *sB = sm + kTfStages * kTfStageBytes;      // packed weights [36][32][16 B]
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + kPackBytes);
  uint64_t *empty = full + kTfStages, *tfull = empty + kTfStages, *tempty = tfull + 2, *drain = tempty + 2;
  uint32_t *slot = reinterpret_cast<uint32_t *>(drain + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Pc = B << (2 * geo.lg_c);  // rows of one class (of the grid when not split)
  const int ntiles = geo.split ? 4 * geo.tiles_c : geo.tiles_c;
  const int f = MODE == kFwd ? geo.stride : 1;
  // tile -> class, first image and first row of the class grid
  auto tile_origin = [&](int tile, int &cls, int &b0, int &y0) {
    cls = geo.split ? tile / geo.tiles_c : 0;
    const int t = tile - cls * geo.tiles_c;
    b0 = geo.NB == 1 ? t / geo.tpi : t * geo.NB;
    y0 = geo.NB == 1 ? (t % geo.tpi) * geo.TH : 0;
  };

  {  // the packed weights (generic-proxy stores, fenced for the tensor cores below)
    const uint4 *g = reinterpret_cast<const uint4 *>(wpack);
    uint4 *d = reinterpret_cast<uint4 *>(sB);
    for (int i = tid; i < (int)(kPackBytes / 16); i += kTfThreads) d[i] = __ldg(g + i);
  }
  if (warp == 1) {
    tmem_alloc(slot, 64);
    if (lane == 0) {
      for (int i = 0; i < kTfStages; ++i) {
        mbar_init(&full[i], 1);
        mbar_init(&empty[i], 1);
      }
      for (int i = 0; i < 2; ++i) {
        mbar_init(&tfull[i], 1);
        mbar_init(&tempty[i], 128);
      }
      mbar_init(drain, 1);
      fence_mbar_init();
    }
  }
  if (warp == 0 && lane == 0) prefetch_tmap(&src);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  if (warp == 0) {
    // ============================================================= TMA producer
    if (lane == 0) {
      uint32_t seq = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int cls, b0, y0;
        tile_origin(tile, cls, b0, y0);
        const int n = tf_ntaps(geo.split, cls);
        for (int i = 0; i < n; ++i, ++seq) {
          int ox, oy, wt;
          tf_tap<MODE>(geo.split, cls, i, ox, oy, wt);
          const int stage = seq % kTfStages;
          if (!mbar_wait_bounded(&empty[stage], ((seq / kTfStages) & 1) ^ 1, status)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[stage], kTfStageBytes);
          tma_load_4d(sA + stage * kTfStageBytes, &src, &full[stage], 0, ox, f * y0 + oy, b0);
        }
      }
      // on the normal path the MMAs consumed every load (they waited for each); after a
      // timeout, wait (bounded) for the last load issued before leaving
      if (!ok && seq > 0) mbar_wait_bounded(&full[(seq - 1) % kTfStages], ((seq - 1) / kTfStages) & 1, status);
    }
  } else if (warp == 1) {
    // ============================================================= MMA issuer
    if (lane == 0) {
      uint32_t seq = 0, tcount = 0;
      const uint32_t a0 = smem_u32(sA), b0s = smem_u32(sB);
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tcount) {
        int cls, b0, y0;
        tile_origin(tile, cls, b0, y0);
        const int n = tf_ntaps(geo.split, cls);
        const int buf = tcount & 1;
        if (!mbar_wait_bounded(&tempty[buf], ((tcount >> 1) & 1) ^ 1, status)) break;
        tc_fence_after();
        const uint32_t d = tmem + 32u * buf;
        bool ok = true;
        for (int i = 0; i < n; ++i, ++seq) {
          int ox, oy, wt;
          tf_tap<MODE>(geo.split, cls, i, ox, oy, wt);
          const int stage = seq % kTfStages;
          if (!mbar_wait_bounded(&full[stage], (seq / kTfStages) & 1, status)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int k = 0; k < 2; ++k)
            umma_f16(d, sdesc_sw64(a0 + stage * kTfStageBytes + 32u * k),
                     sdesc(b0s + (uint32_t)(4 * wt + 2 * k) * 512u, 512u, 128u), kIdesc, (i > 0 || k > 0) ? 1u : 0u);
          umma_commit(&empty[stage]);
        }
        if (!ok) break;
        umma_commit(&tfull[buf]);
      }
      umma_commit(drain);
      mbar_wait_bounded(drain, 0, status);
    }
    __syncwarp();
  } else {
    // ============================================================= epilogue (warps 2-5)
    const int q = warp & 3;  // TMEM lanes 32 q .. 32 q + 31 = tile rows
    float bv[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) bv[i] = MODE == kFwd ? __ldg(bias + i) : 0.0f;
    uint32_t tcount = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tcount) {
      int cls, b0, y0;
      tile_origin(tile, cls, b0, y0);
      // output pixel of this lane's row: tiles are contiguous 128-row ranges of their class
      const int r = ((tile - cls * geo.tiles_c) << 7) + 32 * q + lane;
      int p = r < Pc ? r : -1;
      if (geo.split && p >= 0) {
        const int gc = 1 << geo.lg_c, b = r >> (2 * geo.lg_c), yc = (r >> geo.lg_c) & (gc - 1), xc = r & (gc - 1);
        p = (((b << geo.lg_g) + 2 * yc + (cls >> 1)) << geo.lg_g) + 2 * xc + (cls & 1);
      }
      uint32_t mw[2][8];
      if (MODE == kDgrad && p >= 0) {  // the ReLU mask, read while the MMAs run
        ld_nc_v8(mask + (size_t)p * kCh, mw[0]);
        ld_nc_v8(mask + (size_t)p * kCh + 16, mw[1]);
      }
      const int buf = tcount & 1;
      // the warp leaves together if any lane's wait ran out (the TMEM loads below are
      // warp-aligned)
      const bool okw = mbar_wait_bounded(&tfull[buf], (tcount >> 1) & 1, status);
      if (__any_sync(0xffffffffu, !okw)) break;
      tc_fence_after();
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        uint32_t rr[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + 32u * buf + 16u * hh, rr);
        tmem_ld_wait();
        if (p >= 0) {
          uint32_t o32[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (MODE == kFwd)
              o32[i] = pack2(fmaxf(__uint_as_float(rr[2 * i]) + bv[16 * hh + 2 * i], 0.0f),
                             fmaxf(__uint_as_float(rr[2 * i + 1]) + bv[16 * hh + 2 * i + 1], 0.0f));
            else
              o32[i] = pack2(lo_f(mw[hh][i]) > 0.0f ? __uint_as_float(rr[2 * i]) : 0.0f,
                             hi_f(mw[hh][i]) > 0.0f ? __uint_as_float(rr[2 * i + 1]) : 0.0f);
          }
          st_v8(out + (size_t)p * kCh + 16 * hh, o32);
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[buf]);
    }
  }
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 64);
}

// ------------------------------ weight gradient of the 32-channel layers, TMA-fed
// dW^T[(tap, c)][o] = sum_p col[p][(tap, c)] dz[p][o] with both operands MN-major: a stage
// of 64 output pixels holds, per tap, the 64 source pixels' 32 channels (one 4-D TMA
// load, traversal stride s, zero fill) as a [64 pixels][64 B] tile in the 64-byte swizzle,
// i.e. 8 atoms of 8 K rows (pixels) x 32 M elements; taps follow each other 4 KB apart
// (the LBO between M atoms), 8-pixel groups are 512 B apart (the SBO).  Tiles 9-11 are
// constant: the bias row (element 0 of every pixel = 1) and zeros, so M-tile 2 (rows
// 256-383) is tap 8, the bias row and padding.  The dz tile [64 pixels][32 o] is the B
// operand in the same layout.  Warp 0 loads, warp 1 issues 3 M-tiles x 4 K-steps per
// stage, warps 2-5 write the chunk's partial sums from TMEM.
constexpr int kWtStages = 3;
constexpr uint32_t kWtTile = 64 * 64;           // [64 pixels][64 B]
constexpr uint32_t kWtStage = 13 * kWtTile;     // taps 0-8, bias tile, two zero tiles, dz tile
constexpr int kWtThreads = 192;
constexpr uint32_t kWtSmem = kWtStages * kWtStage + 256 + 1024;
constexpr uint32_t kIdescMN = kIdesc | (1u << 15) | (1u << 16);  // A and B MN-major

// MN-major, 64-byte swizzle: start >> 4 | LBO (between 32-element MN atoms) | SBO 512 B
// (between 8-row K groups) | version 1 | layout 4 (SWIZZLE_64B).
__device__ __forceinline__ uint64_t sdesc_mn_sw64(uint32_t saddr, uint32_t lbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)(512u >> 4) << 32) | (1ull << 46) | (4ull << 61);
}

struct WtGeom {
  int lg_g, TH, stride, per;  // dz grid side 2^lg_g (rows of 64 / side pixels per stage), stages per chunk
};

__global__ void __launch_bounds__(kWtThreads, 1)
    wgrad_tma_kernel(const __grid_constant__ CUtensorMap act, const __grid_constant__ CUtensorMap dzm,
                     float *__restrict__ part, int B, const WtGeom geo, uint32_t *status) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(sm + kWtStages * kWtStage);
  uint64_t *empty = full + kWtStages, *tdone = empty + kWtStages;
  uint32_t *slot = reinterpret_cast<uint32_t *>(tdone + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int total = B << (2 * geo.lg_g - 6);  // stages of 64 pixels in the layer
  const int s_begin = blockIdx.x * geo.per, s_end = min(total, s_begin + geo.per);
  const int nst = s_end - s_begin;

  // constant tiles 9-11 of every stage: element 0 of each pixel row = 1 (BF16), rest 0; in
  // the 64-byte swizzle a row's 16-byte chunk c sits at chunk c ^ ((row >> 1) & 3)
  for (int i = tid; i < kWtStages * 3 * (int)(kWtTile / 16); i += kWtThreads) {
    const int st = i / (3 * (kWtTile / 16)), rem = i % (3 * (kWtTile / 16));
    const int tile = 9 + rem / (kWtTile / 16), q16 = rem % (kWtTile / 16), row = q16 >> 2, chunk = q16 & 3;
    const bool one = tile == 9 && chunk == ((row >> 1) & 3);  // logical chunk 0 of the row
    *reinterpret_cast<uint4 *>(sm + st * kWtStage + tile * kWtTile + q16 * 16) =
        make_uint4(one ? 0x3F80u : 0u, 0u, 0u, 0u);
  }
  if (warp == 1) {
    tmem_alloc(slot, 128);
    if (lane == 0) {
      for (int i = 0; i < kWtStages; ++i) {
        mbar_init(&full[i], 1);
        mbar_init(&empty[i], 1);
      }
      mbar_init(tdone, 1);
      fence_mbar_init();
    }
  }
  if (warp == 0 && lane == 0) {
    prefetch_tmap(&act);
    prefetch_tmap(&dzm);
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const int G = 1 << geo.lg_g;

  if (warp == 0) {
    // ============================================================= TMA producer
    if (lane == 0) {
      bool ok = true;
      int k = 0;
      for (; k < nst; ++k) {
        const int stage = k % kWtStages;
        if (!mbar_wait_bounded(&empty[stage], ((k / kWtStages) & 1) ^ 1, status)) {
          ok = false;
          break;
        }
        const int p0 = (s_begin + k) << 6, b = p0 >> (2 * geo.lg_g), y0 = (p0 >> geo.lg_g) & (G - 1);
        uint8_t *base = sm + stage * kWtStage;
        mbar_arrive_expect_tx(&full[stage], 10 * kWtTile);
        for (int t = 0; t < kTaps; ++t)
          tma_load_4d(base + t * kWtTile, &act, &full[stage], 0, t % 3 - 1, geo.stride * y0 + t / 3 - 1, b);
        tma_load_4d(base + 12 * kWtTile, &dzm, &full[stage], 0, 0, y0, b);
      }
      if (!ok && k > 0) mbar_wait_bounded(&full[(k - 1) % kWtStages], ((k - 1) / kWtStages) & 1, status);
    }
  } else if (warp == 1) {
    // ============================================================= MMA issuer
    if (lane == 0) {
      bool ok = true;
      const uint32_t a0 = smem_u32(sm);
      for (int k = 0; k < nst && ok; ++k) {
        const int stage = k % kWtStages;
        if (!mbar_wait_bounded(&full[stage], (k / kWtStages) & 1, status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = a0 + stage * kWtStage;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)  // 16 pixels = two 8-row K groups per MMA
#pragma unroll
          for (int i = 0; i < 3; ++i)
            umma_f16(tmem + 32u * i, sdesc_mn_sw64(base + (uint32_t)(4 * i) * kWtTile + 1024u * ks, kWtTile),
                     sdesc_mn_sw64(base + 12u * kWtTile + 1024u * ks, kWtTile), kIdescMN,
                     (k > 0 || ks > 0) ? 1u : 0u);
        umma_commit(&empty[stage]);
      }
      umma_commit(tdone);  // covers every MMA issued
      mbar_wait_bounded(tdone, 0, status);
    }
    __syncwarp();
  } else {
    // ============================================================= epilogue (warps 2-5)
    const int q = warp & 3;
    // one decision per warp: the TMEM loads below are warp-aligned
    const bool ok = __all_sync(0xffffffffu, nst > 0 && mbar_wait_bounded(tdone, 0, status));
    if (ok) {
      tc_fence_after();
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int row = 128 * i + 32 * q + lane;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t r[16];
          tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + 32u * i + 16u * hh, r);
          tmem_ld_wait();
          if (row <= kTaps * kCh) {
            float *dst = part + ((size_t)blockIdx.x * (kTaps * kCh + 1) + row) * kCh + 16 * hh;
            const uint32_t lo[8] = {r[0], r[1], r[2], r[3], r[4], r[5], r[6], r[7]};
            const uint32_t hi[8] = {r[8], r[9], r[10], r[11], r[12], r[13], r[14], r[15]};
            st_v8(dst, lo);
            st_v8(dst + 8, hi);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 128);
}

// ------------------------------------- weight gradient of the first layer on tcgen05
// dW^T[(tap, c)][o] = sum_p col[p][(tap, c)] dz[p][o], db[o] = sum_p dz[p][o]: 18 rows
// (tap, input channel) plus one row of ones (the bias), padded to 128; K runs over the
// output pixels of one chunk, N = 32 output channels.  A stage is 128 output pixels = 4
// rows of the 32 x 32 grid; its TMA loads, issued one stage ahead, bring the 9 input rows
// (2 channels, float32) those rows read and the dz tile (64-byte swizzle: the MN-major B
// operand).  The threads build the A rows from the staged input (8 pixels of one channel
// per 16-byte core-matrix row, rounded to BF16; K-major).  Two stage buffers; each CTA
// writes its chunk's partial sums.
struct Wg1 {
  static constexpr int CIN = 2;
  static constexpr int ROWS = 128;
  static constexpr int NDATA = CIN * kTaps;        // data rows; row NDATA holds ones
  static constexpr int KCS = 16;                   // K chunks (8 pixels each) per stage
  static constexpr int STAGE_PX = 8 * KCS;
  static constexpr uint32_t LBO_A = ROWS * 16 + 16;  // +16 B: 8 consecutive K chunks on distinct banks
  static constexpr uint32_t A_STAGE = KCS * LBO_A;
  static constexpr uint32_t B_STAGE = STAGE_PX * 64;  // [128 pixels][64 B], 64-byte swizzle
  static constexpr int XROWS = 9;                      // input rows of 4 output rows
  static constexpr uint32_t X_BYTES = CIN * XROWS * 64 * 4;  // [c][row][64 floats]
  static constexpr uint32_t X_STAGE = 5120;                  // X_BYTES rounded to 1 KB
  static constexpr uint32_t SMEM = 2 * (B_STAGE + X_STAGE + A_STAGE) + 64 + 1024;
  static constexpr uint32_t TMEM_COLS = 32;
  static constexpr int THREADS = NDATA * KCS;  // one A unit per thread per stage: 288
};

// Source: the network input as float32 NCHW [B][2][64][64].  A unit is 8 consecutive
// pixels of one K chunk: since the grid side is a multiple of 8 and chunks start at
// multiples of 128 pixels, they lie in one image row.
__global__ void __launch_bounds__(Wg1::THREADS, 2)
    wgrad1_kernel(const __grid_constant__ CUtensorMap xm, const __grid_constant__ CUtensorMap dzm,
                  float *__restrict__ part, int B, int lg_s, int lg_g, int stride, int per_chunk, uint32_t *status) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  using Sh = Wg1;
  constexpr int CIN = Sh::CIN;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sx = sm + 2 * Sh::B_STAGE;    // staged input rows, after the B stages (1024-aligned)
  uint8_t *smem = sx + 2 * Sh::X_STAGE;  // the A stages
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * Sh::A_STAGE);
  uint64_t *tbar = bar + 2;  // the dz tile of each stage landed
  uint32_t *slot = reinterpret_cast<uint32_t *>(tbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = 1 << lg_s, G = 1 << lg_g;
  const int P = B << (2 * lg_g);
  const int p_begin = blockIdx.x * per_chunk;
  const int p_end = min(P, p_begin + per_chunk);
  const int nst = (p_end - p_begin + Sh::STAGE_PX - 1) / Sh::STAGE_PX;
  constexpr int NC = Sh::ROWS - Sh::NDATA;  // constant rows per K chunk

  for (int i = tid; i < 2 * Sh::KCS * NC; i += Sh::THREADS) {  // the ones row and the zero rows
    const int st = i / (Sh::KCS * NC), kc = (i / NC) % Sh::KCS, row = Sh::NDATA + i % NC;
    const uint32_t v = row == Sh::NDATA ? 0x3F803F80u : 0u;  // BF16 1.0 pairs
    *reinterpret_cast<uint4 *>(smem + st * Sh::A_STAGE + kc * Sh::LBO_A + row * 16) = make_uint4(v, v, v, v);
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar[i], 1);
      mbar_init(&tbar[i], 1);
    }
    fence_mbar_init();
    prefetch_tmap(&dzm);
    prefetch_tmap(&xm);
  }
  if (warp == 0) tmem_alloc(slot, Sh::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  // the stage's TMA loads into buffer sb: its dz tile and the 9 input rows of its 4
  // output rows (row 2 y0 - 1 may lie above the stamp: zero fill)
  int issued = 0, landed = 0;  // stage loads issued (thread 0), stages whose loads were waited for
  auto issue = [&](int st, int sb) {
    const int p0 = p_begin + st * Sh::STAGE_PX, b = p0 >> (2 * lg_g), y0 = (p0 >> lg_g) & (G - 1);
    mbar_arrive_expect_tx(&tbar[sb], Sh::B_STAGE + Sh::X_BYTES);
    tma_load_4d(sm + sb * Sh::B_STAGE, &dzm, &tbar[sb], 0, 0, y0, b);
    tma_load_4d(sx + sb * Sh::X_STAGE, &xm, &tbar[sb], 0, stride * y0 - 1, 0, b);
    ++issued;
  };
  if (tid == 0 && nst > 0) issue(0, 0);

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
    // one stage ahead: buffer buf ^ 1 is free once the MMAs of stage s - 1 are done (a
    // wait that gives up leaves the load unissued, and the wait for it below gives up too)
    if (tid == 0 && s + 1 < nst &&
        (s == 0 || mbar_wait_bounded(&bar[buf ^ 1], (uint32_t)(((s - 1) >> 1) & 1), status)))
      issue(s + 1, buf ^ 1);
    const bool okt = mbar_wait_bounded(&tbar[buf], (uint32_t)((s >> 1) & 1), status);
    if (__syncthreads_or(!okt)) {
      failed = true;
      break;
    }
    landed = s + 1;
    uint8_t *sA = smem + buf * Sh::A_STAGE;
    uint8_t *sB = sm + buf * Sh::B_STAGE;
    const float *xs = reinterpret_cast<const float *>(sx + buf * Sh::X_STAGE);  // [c][9 rows][64]
    const int p0 = p_begin + s * Sh::STAGE_PX, y0 = (p0 >> lg_g) & (G - 1);
    for (int u = tid; u < Sh::NDATA * Sh::KCS; u += Sh::THREADS) {
      // row (tap, c), pixels pq .. pq + 7 (output row y, columns x0 ..): input row
      // 2 y + dy - 1 is staged row 2 (y - y0) + dy, column 2 x + dx - 1
      const int kc = u % Sh::KCS, g = u / Sh::KCS;
      const int pq = p0 + kc * 8;
      const bool in = pq < p_end;
      const int y = (pq >> lg_g) & (G - 1), x0 = pq & (G - 1);
      const int tap = g / CIN, c = g % CIN, dy = tap / 3, dx = tap % 3;
      const float *row = xs + (c * Sh::XROWS + stride * (y - y0) + dy) * S;
      float f[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int xx = stride * (x0 + e) + dx - 1;
        f[e] = (in && xx >= 0 && xx < S) ? row[xx] : 0.0f;
      }
      *reinterpret_cast<uint4 *>(sA + kc * Sh::LBO_A + g * 16) =
          make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int k = 0; k < Sh::STAGE_PX / 16; ++k)
        umma_f16(tmem, sdesc(a0 + k * 2u * Sh::LBO_A, Sh::LBO_A, 128u), sdesc_mn_sw64(b0 + 1024u * k, Sh::B_STAGE),
                 kIdesc | (1u << 16), (s > 0 || k > 0) ? 1u : 0u);  // B MN-major
      umma_commit(&bar[buf]);
    }
  }
  // after a wait gave up, a load issued ahead may still be in flight: wait for it (bounded)
  if (tid == 0 && issued > landed) mbar_wait_bounded(&tbar[(issued - 1) & 1], ((issued - 1) >> 1) & 1, status);
  if (!failed && nst > 0) {  // the last commit covers every MMA before it
    const int sl = nst - 1;
    const bool ok = mbar_wait_bounded(&bar[sl & 1], (uint32_t)((sl >> 1) & 1), status);
    failed = __syncthreads_or(!ok);
  }
  if (!failed && nst > 0 && warp < 8) {  // warps 0-7: TMEM lane quadrant warp & 3, column half warp / 4
    tc_fence_after();
    const int q = warp & 3, h = warp >> 2;
    {
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + 16u * h, r);
      tmem_ld_wait();
      const int row = 32 * q + lane;
      if (row <= Sh::NDATA) {
        float *dst = part + ((size_t)blockIdx.x * (Sh::NDATA + 1) + row) * kCh + 16 * h;
        const uint32_t lo[8] = {r[0], r[1], r[2], r[3], r[4], r[5], r[6], r[7]};
        const uint32_t hi[8] = {r[8], r[9], r[10], r[11], r[12], r[13], r[14], r[15]};
        st_v8(dst, lo);
        st_v8(dst + 8, hi);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, Sh::TMEM_COLS);
}

// Partial sums of the chunks: dw[o][c][tap], db[o], every layer in one launch.  One
// block of 1024 threads per row (tap, c) or bias row of a layer: 32 chunk slices, each
// summed in chunk order, then added in slice order.
constexpr int kRedSlices = 32;

struct WgradSet {
  const float *part[kLayers];
  float *gw[kLayers], *gb[kLayers];
  int cin[kLayers], nchunks[kLayers], row0[kLayers + 1];  // row0: first block of each layer
};

__global__ void __launch_bounds__(kRedSlices * kCh) wgrad_reduce_kernel(const __grid_constant__ WgradSet ws) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  __shared__ float red[kRedSlices][kCh];
  int l = 0;
  while (l + 1 < kLayers && (int)blockIdx.x >= ws.row0[l + 1]) ++l;
  const int cin = ws.cin[l], rows = cin * kTaps + 1, row = blockIdx.x - ws.row0[l];
  const int o = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const float *part = ws.part[l];
  float s = 0.0f;
#pragma unroll 4
  for (int c = sl; c < ws.nchunks[l]; c += kRedSlices) s += part[((size_t)c * rows + row) * kCh + o];
  red[sl][o] = s;
  __syncthreads();
  if (threadIdx.x < kCh) {
    float t = 0.0f;
    for (int i = 0; i < kRedSlices; ++i) t += red[i][o];
    if (row < cin * kTaps) ws.gw[l][((size_t)o * cin + row % cin) * 9 + row / cin] = t;
    else ws.gb[l][o] = t;
  }
}

// pooled[b][c] = mean over the 8x8 positions; out[b][j] = fcb[j] + sum_c fcw[j][c] pooled[b][c].
// With a target (training): dout = 2 (out - target) / (B n_out) and the block's share of
// the mean squared error added to *loss.  One block of 64 threads per sample.
__global__ void pool_fc_kernel(const bf16 *__restrict__ act, const float *__restrict__ fcw,
                               const float *__restrict__ fcb, float *__restrict__ pooled, float *__restrict__ out,
                               int n_out, const float *__restrict__ target, float *__restrict__ dout, float *loss,
                               int B) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  __shared__ float pl[kCh];
  __shared__ float red[2];
  const int b = blockIdx.x;
  if (threadIdx.x < kCh) {
    const bf16 *a = act + (size_t)b * 64 * kCh + threadIdx.x;
    float s = 0.0f;
    for (int i = 0; i < 64; ++i) s += __bfloat162float(a[i * kCh]);
    pl[threadIdx.x] = s * (1.0f / 64.0f);
    pooled[b * kCh + threadIdx.x] = pl[threadIdx.x];
  }
  __syncthreads();
  const float inv_n = 1.0f / (float)B / (float)n_out;
  float sq = 0.0f;
  for (int j = threadIdx.x; j < n_out; j += blockDim.x) {
    float s = fcb[j];
    for (int c = 0; c < kCh; ++c) s = fmaf(fcw[j * kCh + c], pl[c], s);
    out[(size_t)b * n_out + j] = s;
    if (target) {
      const float d = s - target[(size_t)b * n_out + j];
      dout[(size_t)b * n_out + j] = 2.0f * d * inv_n;
      sq = fmaf(d, d, sq);
    }
  }
  if (!target) return;
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(loss, (red[0] + red[1]) * inv_n);
}

// Output-layer gradients in one launch.  Blocks 0 .. n_out - 1: the linear layer's
// weight gradients dfcw[j][c] = sum_b dout[b][j] pooled[b][c] and dfcb[j] = sum_b dout[b][j]
// (8 batch slices added in order).  The other blocks, one thread per (b, c):
// dpooled[b][c] = sum_j dout[b][j] fcw[j][c], spread as dpooled / 64 over the 8x8
// positions, masked by the ReLU (act > 0), stored BF16 NHWC as the last layer's dz.
__global__ void __launch_bounds__(256) fc_grad_kernel(const float *__restrict__ dout, const float *__restrict__ pooled,
                                                      const float *__restrict__ fcw, const bf16 *__restrict__ act,
                                                      float *__restrict__ dfcw, float *__restrict__ dfcb,
                                                      bf16 *__restrict__ dz, int B, int n_out) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  if ((int)blockIdx.x < n_out) {
    __shared__ float red[8][kCh + 1];
    const int j = blockIdx.x, c = threadIdx.x & 31, part = threadIdx.x >> 5;
    float s = 0.0f, sb = 0.0f;
#pragma unroll 8
    for (int b = part; b < B; b += 8) {
      const float d = dout[(size_t)b * n_out + j];
      s = fmaf(d, pooled[b * kCh + c], s);
      sb += d;
    }
    red[part][c] = s;
    if (c == 0) red[part][kCh] = sb;
    __syncthreads();
    if (threadIdx.x <= kCh) {
      float t = 0.0f;
      for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x];
      if (threadIdx.x < kCh) dfcw[j * kCh + threadIdx.x] = t;
      else dfcb[j] = t;
    }
    return;
  }
  const int t = (blockIdx.x - n_out) * blockDim.x + threadIdx.x;
  if (t >= B * kCh) return;
  const int b = t / kCh, c = t % kCh;
  float s = 0.0f;
#pragma unroll 8
  for (int j = 0; j < n_out; ++j) s = fmaf(dout[(size_t)b * n_out + j], fcw[j * kCh + c], s);
  const bf16 g = __float2bfloat16_rn(s * (1.0f / 64.0f));
  const bf16 z = __float2bfloat16_rn(0.0f);
  for (int i = 0; i < 64; ++i) {
    const size_t at = ((size_t)b * 64 + i) * kCh + c;
    dz[at] = __bfloat162float(act[at]) > 0.0f ? g : z;
  }
}

__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Adam with the step count in device memory (bias corrections formed here).
__global__ void adam_dstep_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                                  const float *__restrict__ g, int n, const int *__restrict__ step, float lr, float b1,
                                  float b2, float eps) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  const float t = (float)*step;
  const float c1 = 1.0f - powf(b1, t), c2 = 1.0f - powf(b2, t);
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

int conv1(const float *x, const bf16 *wpack, const float *bias, bf16 *out, int B, int nsm, cudaStream_t s) {
  CUtensorMap tx;  // the stamps, 9 input rows per box
  if (!encode_tmap_stamps_f32(&tx, x, 64, 2, B, kC1Rows)) return set_error(SVK_ERR_CUDA, "network tensor map refused");
  cudaError_t e = cudaFuncSetAttribute(conv1_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kC1Smem);
  if (e != cudaSuccess) return cuda_status(e, "network first-layer attributes");
  const int ntiles = ((B << 10) + 127) >> 7;
  const int grid = ntiles < 6 * nsm ? ntiles : 6 * nsm;
  return cuda_status(launch_dependent(conv1_mma_kernel, grid, kC1Threads, kC1Smem, s, tx, wpack, bias, out, B,
                                      device_status_word()),
                     "network first layer");
}

// A 32-channel layer through the TMA-fed kernel.  Forward: source NHWC [B][S][S][32]
// (the layer input), output side 2^lg_g.  Data grad: source = the layer's dz (side S),
// output = dz of the layer below (side 2^lg_g), mask = that layer's activations.
template <int MODE>
int conv_tma(const bf16 *src, int S, const bf16 *wpack, const float *bias, const bf16 *mask, bf16 *out, int B,
             int lg_g, int stride, int nsm, cudaStream_t s) {
  TfGeom geo;
  geo.lg_g = lg_g;
  geo.stride = stride;
  geo.split = MODE == kDgrad && stride == 2;
  geo.lg_c = geo.split ? lg_g - 1 : lg_g;
  const int gc = 1 << geo.lg_c;
  if (gc >= 16) {  // whole rows: 128 / gc of them per tile
    geo.TH = 128 / gc;
    geo.NB = 1;
    geo.tpi = gc / geo.TH;
  } else {  // whole images: 128 / gc^2 of them per tile
    geo.TH = gc;
    geo.NB = 128 / (gc * gc);
    geo.tpi = 1;
  }
  geo.tiles_c = ((B << (2 * geo.lg_c)) + 127) >> 7;
  const int f = MODE == kFwd ? stride : 1;  // traversal stride of the source
  CUtensorMap tm;
  if (!encode_tmap_nhwc32_bf16(&tm, src, S, B, f * gc, f * geo.TH, geo.NB, f))
    return set_error(SVK_ERR_CUDA, "network tensor map refused");
  cudaError_t e = cudaFuncSetAttribute(conv_tma_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kTfSmem);
  if (e != cudaSuccess) return cuda_status(e, "network convolution attributes");
  const int ntiles = geo.split ? 4 * geo.tiles_c : geo.tiles_c;
  const int grid = ntiles < 2 * nsm ? ntiles : 2 * nsm;  // two CTAs per SM
  return cuda_status(launch_dependent(conv_tma_kernel<MODE>, grid, kTfThreads, kTfSmem, s, tm, wpack, bias, mask, out,
                                      B, geo, device_status_word()),
                     "network convolution");
}

// A 32-channel layer's partial weight-gradient sums through the TMA-fed kernel: source
// = the layer input (side S), dz = the layer's output gradient (side 2^lg_g).
int wgrad_tma(const bf16 *src, int S, const bf16 *dz, float *part, int B, int lg_g, int stride, cudaStream_t s) {
  const int G = 1 << lg_g, P = B << (2 * lg_g);
  WtGeom geo;
  geo.lg_g = lg_g;
  geo.TH = 64 / G;
  geo.stride = stride;
  geo.per = wg_per_chunk(P, kCh) / 64;
  const int nch = wg_nchunks(P, kCh);
  CUtensorMap ta, td;
  if (!encode_tmap_nhwc32_bf16(&ta, src, S, B, stride * G, stride * geo.TH, 1, stride) ||
      !encode_tmap_nhwc32_bf16(&td, dz, G, B, G, geo.TH, 1, 1))
    return set_error(SVK_ERR_CUDA, "network tensor map refused");
  cudaError_t e = cudaFuncSetAttribute(wgrad_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWtSmem);
  if (e != cudaSuccess) return cuda_status(e, "network weight-gradient attributes");
  return cuda_status(launch_dependent(wgrad_tma_kernel, nch, kWtThreads, kWtSmem, s, ta, td, part, B, geo,
                                      device_status_word()),
                     "network weight gradient");
}

// The first layer's partial weight-gradient sums (reduced for all layers by
// wgrad_reduce_kernel).
int wgrad1(const float *x, const bf16 *dz, float *part, int B, cudaStream_t s) {
  CUtensorMap td, tx;  // dz of the first layer: 32 x 32 grid, boxes of 4 rows; its input: 9 rows
  if (!encode_tmap_nhwc32_bf16(&td, dz, 32, B, 32, Wg1::STAGE_PX / 32, 1, 1) ||
      !encode_tmap_stamps_f32(&tx, x, 64, 2, B, Wg1::XROWS))
    return set_error(SVK_ERR_CUDA, "network tensor map refused");
  cudaError_t e = cudaFuncSetAttribute(wgrad1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Wg1::SMEM);
  if (e != cudaSuccess) return cuda_status(e, "network weight-gradient attributes");
  const int P = B << (2 * kLgOut[0]);
  const int per = wg_per_chunk(P, 2), nch = wg_nchunks(P, 2);
  return cuda_status(launch_dependent(wgrad1_kernel, nch, Wg1::THREADS, Wg1::SMEM, s, tx, td, part, B, kLgIn[0],
                                      kLgOut[0], kStride[0], per, device_status_word()),
                     "network weight gradient");
}

struct Bufs {
  float *wq;
  bf16 *wf[kLayers], *wd[kLayers], *act[kLayers], *dz[kLayers];
  float *pooled, *out, *dout, *part[kLayers];
};

Bufs bufs(void *ws_v, const Work &Wk) {
  uint8_t *ws = static_cast<uint8_t *>(ws_v);
  Bufs b{};
  b.wq = reinterpret_cast<float *>(ws + Wk.wq);
  for (int i = 0; i < kLayers; ++i) {
    b.wf[i] = reinterpret_cast<bf16 *>(ws + Wk.wf[i]);
    b.wd[i] = i > 0 ? reinterpret_cast<bf16 *>(ws + Wk.wd[i]) : nullptr;
    b.act[i] = reinterpret_cast<bf16 *>(ws + Wk.act[i]);
    b.dz[i] = reinterpret_cast<bf16 *>(ws + Wk.dz[i]);
    b.part[i] = reinterpret_cast<float *>(ws + Wk.part[i]);
  }
  b.pooled = reinterpret_cast<float *>(ws + Wk.pooled);
  b.out = reinterpret_cast<float *>(ws + Wk.out);
  b.dout = reinterpret_cast<float *>(ws + Wk.dout);
  return b;
}

int pack(const float *params, const Layout &L, const Bufs &b, cudaStream_t s, float *loss = nullptr) {
  return cuda_status(launch_dependent(pack_kernel, grid_for(L.total + kPack0 + 3 * kPack), 256, 0, s, params, b.wq,
                                      (int)L.total, b.wf[0], b.wf[1], b.wd[1], b.wf[2], b.wd[2], b.wf[3], b.wd[3],
                                      L.w[0], L.w[1], L.w[2], L.w[3], loss),
                     "network weight packing");
}

// x -> act[0..3] -> pooled -> out (parameters already packed)
int forward(const float *x, const Layout &L, const Bufs &b, int B, int n_out, float *out, int nsm, cudaStream_t s,
            const float *target = nullptr, float *loss = nullptr) {
  int st = conv1(x, b.wf[0], b.wq + L.b[0], b.act[0], B, nsm, s);
  for (int li = 1; li < kLayers && st == SVK_OK; ++li)
    st = conv_tma<kFwd>(b.act[li - 1], 1 << kLgIn[li], b.wf[li], b.wq + L.b[li], nullptr, b.act[li], B, kLgOut[li],
                        kStride[li], nsm, s);
  if (st != SVK_OK) return st;
  return cuda_status(launch_dependent(pool_fc_kernel, B, 64, 0, s, b.act[kLayers - 1], b.wq + L.fcw, b.wq + L.fcb,
                                      b.pooled, out, n_out, target, b.dout, loss, B),
                     "network pooling");
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
// one T x T FP64 normal matrix shared by every k, Cholesky, then N solves.  Block j solves
// stamps' coefficient sets k = kFfPerBlock j .. + kFfPerBlock - 1; every block forms the
// normal matrix itself (it is small) so no block waits for another.  The stamps pass in
// chunks: their monomials and weights go to shared memory once, and each sum (a normal-
// matrix entry, or a right-hand side entry (k, t)) is taken by one warp, lanes striding
// over the chunk's stamps, then a shuffle tree, then added to its running total in chunk
// order (deterministic).
constexpr int kFfThreads = 256, kFfChunk = 256, kFfPerBlock = 4;

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kFfThreads) field_fit_kernel(const float *__restrict__ local, const int *__restrict__ xy,
                                                              const float *__restrict__ wts, int S, int N, int W, int H,
                                                              int degree, double *__restrict__ coeffs, int *info) {
  __shared__ double mono[kFfChunk][10];
  __shared__ double wt[kFfChunk];
  __shared__ double Asum[55], bsum[kFfPerBlock * 10];
  __shared__ double Gc[10][10];
  __shared__ int bad;
  const int T = (degree + 1) * (degree + 2) / 2, P = T * (T + 1) / 2;
  const int k0 = blockIdx.x * kFfPerBlock, nk = min(kFfPerBlock, N - k0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = kFfThreads / 32;
  for (int i = threadIdx.x; i < P; i += kFfThreads) Asum[i] = 0.0;
  for (int i = threadIdx.x; i < nk * T; i += kFfThreads) bsum[i] = 0.0;
  if (threadIdx.x == 0) bad = -1;
  for (int s0 = 0; s0 < S; s0 += kFfChunk) {
    const int cs = min(kFfChunk, S - s0);
    __syncthreads();  // the previous chunk's sums are done with mono and wt
    for (int i = threadIdx.x; i < cs; i += kFfThreads) {
      const int s = s0 + i;
      const double xt = W > 1 ? (2.0 * xy[2 * s] - (W - 1)) / (double)(W - 1) : 0.0;
      const double yt = H > 1 ? (2.0 * xy[2 * s + 1] - (H - 1)) / (double)(H - 1) : 0.0;
      int t = 0;
      double xi = 1.0;
      for (int p = 0; p <= degree; ++p) {
        double yj = 1.0;
        for (int q = 0; q <= degree - p; ++q) {
          mono[i][t++] = xi * yj;
          yj *= yt;
        }
        xi *= xt;
      }
      wt[i] = wts ? (double)wts[s] : 1.0;
    }
    __syncthreads();
    // normal-matrix entries r <= c (pair e = c (c + 1) / 2 + r), then right-hand sides
    for (int e = warp; e < P + nk * T; e += nw) {
      double acc = 0.0;
      if (e < P) {
        int c = 0;
        while ((c + 1) * (c + 2) / 2 <= e) ++c;
        const int r = e - c * (c + 1) / 2;
        for (int i = lane; i < cs; i += 32) acc += wt[i] * mono[i][r] * mono[i][c];
      } else {
        const int kk = (e - P) / T, t = (e - P) % T;
        for (int i = lane; i < cs; i += 32) acc += mono[i][t] * wt[i] * (double)local[(size_t)(s0 + i) * N + k0 + kk];
      }
      acc = warp_sum_d(acc);
      if (lane == 0) {
        if (e < P) Asum[e] += acc;
        else bsum[e - P] += acc;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // T <= 10: serial textbook Cholesky
    for (int j = 0; j < T && bad < 0; ++j) {
      double d = Asum[j * (j + 1) / 2 + j];
      for (int k = 0; k < j; ++k) d -= Gc[j][k] * Gc[j][k];
      if (!(d > 0.0)) {
        bad = j;
        break;
      }
      Gc[j][j] = sqrt(d);
      for (int i = j + 1; i < T; ++i) {
        double v = Asum[i * (i + 1) / 2 + j];
        for (int k = 0; k < j; ++k) v -= Gc[i][k] * Gc[j][k];
        Gc[i][j] = v / Gc[j][j];
      }
    }
    if (blockIdx.x == 0) *info = bad;
  }
  __syncthreads();
  if ((int)threadIdx.x < nk) {
    const int kk = threadIdx.x, k = k0 + kk;
    double b[10], y[10];
    for (int t = 0; t < T; ++t) b[t] = bsum[kk * T + t];
    if (bad >= 0) {
      for (int t = 0; t < T; ++t) coeffs[(size_t)k * T + t] = 0.0;
    } else {
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
}

}  // namespace

int cnn_field_fit(const float *local, const int *xy, const float *wts, int S, int N, int W, int H, int degree,
                  double *coeffs, int *info, cudaStream_t s) {
  field_fit_kernel<<<(N + kFfPerBlock - 1) / kFfPerBlock, kFfThreads, 0, s>>>(local, xy, wts, S, N, W, H, degree,
                                                                               coeffs, info);
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

// A second stream per device for the weight gradients of the 32-channel layers: the one of
// layer l needs only dz[l] and act[l-1], so it runs beside the data gradient of layer l
// (which the chain below waits for), and the reduction joins the two streams.  A weight-
// gradient CTA and a data-gradient CTA fit in one SM's shared memory together.  Created
// once per device and context; the mutex is held while a call enqueues its fork and join
// (the stream and events are shared).
struct WgradSide {
  unsigned long long ctx = 0;
  cudaStream_t ss = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int kSideDevices = 64;
std::mutex g_side_mutex;
WgradSide g_side[kSideDevices];

int wgrad_side(WgradSide **out) {
  int dev = 0;
  int st = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (st != SVK_OK) return st;
  if (dev < 0 || dev >= kSideDevices) return set_error(SVK_ERR_UNSUPPORTED, "device %d out of range", dev);
  WgradSide &w = g_side[dev];
  const unsigned long long id = current_context_id();
  if (!w.ss || (id != 0 && id != w.ctx)) {  // first use, or the context was created again
    w = WgradSide{};
    st = cuda_status(cudaStreamCreateWithFlags(&w.ss, cudaStreamNonBlocking), "weight-gradient stream");
    if (st == SVK_OK) st = cuda_status(cudaEventCreateWithFlags(&w.fork, cudaEventDisableTiming), "event");
    if (st == SVK_OK) st = cuda_status(cudaEventCreateWithFlags(&w.join, cudaEventDisableTiming), "event");
    if (st != SVK_OK) {
      w = WgradSide{};
      return st;
    }
    w.ctx = id;
  }
  *out = &w;
  return SVK_OK;
}

int cnn_gradient(const float *params, const float *x, const float *target, int B, int n_out, float *grad, float *loss,
                 void *ws, size_t ws_bytes, cudaStream_t s) {
  int st = check_ws(ws, ws_bytes, B, n_out);
  if (st != SVK_OK) return st;
  const Layout L = param_layout(n_out);
  const Bufs b = bufs(ws, work_layout(B, n_out));
  const int nsm = sm_count();
  if ((st = pack(params, L, b, s, loss)) != SVK_OK) return st;
  if ((st = forward(x, L, b, B, n_out, b.out, nsm, s, target, loss)) != SVK_OK) return st;
  st = cuda_status(launch_dependent(fc_grad_kernel, n_out + (B * kCh + 255) / 256, 256, 0, s, b.dout, b.pooled,
                                    b.wq + L.fcw, b.act[kLayers - 1], grad + L.fcw, grad + L.fcb, b.dz[kLayers - 1],
                                    B, n_out),
                   "network output gradient");
  if (st != SVK_OK) return st;
  std::lock_guard<std::mutex> lock(g_side_mutex);
  WgradSide *side = nullptr;
  if ((st = wgrad_side(&side)) != SVK_OK) return st;
  bool forked = false;
  for (int li = kLayers - 1; li >= 1 && st == SVK_OK; --li) {
    // dz[li] is written (by the output gradient or the data gradient above): fork
    st = cuda_status(cudaEventRecord(side->fork, s), "fork record");
    if (st == SVK_OK) st = cuda_status(cudaStreamWaitEvent(side->ss, side->fork, 0), "fork wait");
    forked = forked || st == SVK_OK;
    if (st == SVK_OK)
      st = wgrad_tma(b.act[li - 1], 1 << kLgIn[li], b.dz[li], b.part[li], B, kLgOut[li], kStride[li], side->ss);
    if (st == SVK_OK)
      st = conv_tma<kDgrad>(b.dz[li], 1 << kLgOut[li], b.wd[li], nullptr, b.act[li - 1], b.dz[li - 1], B, kLgIn[li],
                            kStride[li], nsm, s);
  }
  if (st == SVK_OK) st = wgrad1(x, b.dz[0], b.part[0], B, s);
  if (forked) {  // joined on every path once forked (a capture must not end with the fork open)
    int js = cuda_status(cudaEventRecord(side->join, side->ss), "join record");
    if (js == SVK_OK) js = cuda_status(cudaStreamWaitEvent(s, side->join, 0), "join wait");
    if (st == SVK_OK) st = js;
  }
  if (st != SVK_OK) return st;
  WgradSet set{};
  set.row0[0] = 0;
  for (int li = 0; li < kLayers; ++li) {
    set.part[li] = b.part[li];
    set.cin[li] = kCin[li];
    set.gw[li] = grad + L.w[li];
    set.gb[li] = grad + L.b[li];
    set.nchunks[li] = wg_nchunks(B * kHout[li] * kHout[li], kCin[li]);
    set.row0[li + 1] = set.row0[li] + wg_rows(kCin[li]);
  }
  return cuda_status(launch_dependent(wgrad_reduce_kernel, set.row0[kLayers], kRedSlices * kCh, 0, s, set),
                     "network weight-gradient reduction");
}

int cnn_adam(float *params, float *m, float *v, const float *grad, int n, int step, float lr, float b1, float b2,
             float eps, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  return cuda_status(launch_dependent(adam_kernel, grid_for(n), 256, 0, s, params, m, v, grad, n, lr, b1, b2, eps, c1,
                                      c2),
                     "adam");
}

int cnn_adam_device_step(float *params, float *m, float *v, const float *grad, int n, const int *step, float lr,
                         float b1, float b2, float eps, cudaStream_t s) {
  return cuda_status(launch_dependent(adam_dstep_kernel, grid_for(n), 256, 0, s, params, m, v, grad, n, step, lr, b1,
                                      b2, eps),
                     "adam");
}

}  // namespace svk
