// svk_tc.cu -- basis form of the spatially-varying convolution on the tensor cores.
//
// By linearity of Eq. 2, (R (x) K_{x,y})(x,y) = sum_k a_k(x,y) C_k(x,y) with
// C_k = R (x) B_k.  C is a GEMM: M = pixels, N = basis stamps, K = kernel taps
// (implicit im2col).  This file computes C with tcgen05.mma (accumulators in TMEM)
// and applies a_k(x,y) (Eq. 3) and the subtraction of Eq. 1 in the epilogue.
//
// Implicit im2col without materialising it.  For a tile of 128 output pixels
// x0..x0+127 on one row and one reference row r, the A operand is
//     A(m, q) = R(r, x0 - h + m + q)      (tap u = h - q, q = 0..Lq-1)
// which depends on m + q only.  In the K-major, no-swizzle UMMA layout a core matrix
// is 8 rows (m) x 16 bytes (8 taps q), rows 16 bytes apart; core matrix (i, j) sits
// at start + i*SBO + j*LBO.  Its content R(x0 - h + 8(i+j) + rr + c) depends on i + j
// only, so with SBO = LBO = 128 bytes every core matrix is the 128-byte block
//     Hk[s] (s = i + j): row rr = R(x0 - h + 8 s + rr .. + 7)
// and the whole A tile of a reference row is the sequence of 16-byte chunks
//     chunk e (e = 8 s + rr) = R(x0 - h + e .. x0 - h + e + 7),
// one per start offset e.  Producer warps write these chunks (8x the row in bytes) from
// BF16/FP16 copies of the row; no global im2col buffer exists.
//
// Several output rows per block.  A block produces G output rows y0..y0+G-1.  The
// reference row r feeds output row y0+g through the kernel row v = y0 + g - r, so one
// A tile multiplies a B operand that stacks the basis slices of G consecutive v:
// N = G*Nb columns (Nb stamps), which keeps the MMA wide (G*49 <= 245 of 256).  The
// slices are stored in descending v, so the window for row r starts at slice
// P0 = r - y0 + h and the accumulator column of (g, k) is (G-1-g)*Nb + k.  Slices with
// |v| > h are zero rows of the table.
//
// Split precision.  R = Rh + Rl and B = Bh + Bl (BF16 or FP16 pairs); three MMAs per
// K step, Ah*Bh + Ah*Bl + Al*Bh, accumulate in the same FP32 TMEM columns.
//
// Roles (9 warps): warps 0-3 epilogue (TMEM lane quarters 0-3), warp 4 TMEM owner and
// MMA issuer (one thread), warps 5-8 producers.  All waits are bounded; a wait that
// runs out records a status word and the CTA unwinds (MMAs drained, TMEM freed).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
namespace {

constexpr int kMaxSmem = 232448;  // 227 KB opt-in shared memory per CTA on sm_100-class parts
constexpr int kEpiWarps = 4, kMmaWarp = 4, kProdWarps = 4, kFirstProdWarp = 5;
constexpr int kThreads = (kEpiWarps + 1 + kProdWarps) * 32;
constexpr int kTileM = 128;
constexpr int kMaxStages = 8;  // Hankel stages (reference rows in flight), upper bound
constexpr uint32_t kTmemCols = 512;
constexpr int kAccStride = 256;  // TMEM columns per accumulator buffer

// ----------------------------------------------------------------- plan (host+device)
struct Plan {
  int N, L, h, G, nmma;    // stamps, kernel size, half size, output rows/block, MMA N
  int nKG, nks;            // K groups of 8 taps per reference row, K steps of 16
  int S;                   // Hankel blocks per reference row (= 16 + nKG - 1)
  int seglen;              // staged row length (elements) = 8 S + 8
  int NP, nrows;           // table slices, table rows per K group
  int parts;               // 2 for split precision, 1 for plain BF16
  int NS;                  // Hankel pipeline stages
  int prec;
  size_t table_bytes;      // one table (hi or lo)
  size_t off_tab_hi, off_tab_lo, off_stage, off_stg, off_coef, off_alpha, off_bar, smem;
};

__host__ __device__ inline int rup(int v, int m) { return (v + m - 1) / m * m; }

static bool make_plan(int N, int L, int prec, int G, int NS, Plan *p) {
  Plan q{};
  q.N = N;
  q.L = L;
  q.h = (L - 1) / 2;
  q.G = G;
  q.prec = prec;
  q.NS = NS;
  q.parts = (prec == SVK_PREC_BF16) ? 1 : 2;
  q.nmma = rup(G * N, 16);
  if (q.nmma > 256 || q.nmma < 16) return false;
  const int ng = (L + 7) / 8;
  q.nks = (ng + 1) / 2;
  q.nKG = 2 * q.nks;
  q.S = kTileM / 8 + q.nKG - 1;
  q.seglen = 8 * q.S + 8;
  q.NP = L + 2 * (G - 1);
  q.nrows = rup(q.NP * N + 16, 8);
  q.table_bytes = (size_t)q.nKG * q.nrows * 16;
  size_t o = 0;
  q.off_tab_hi = o;
  o += q.table_bytes;
  q.off_tab_lo = o;
  if (q.parts == 2) o += q.table_bytes;
  o = rup((int)o, 128);
  q.off_stage = o;
  o += (size_t)NS * q.parts * q.S * 128;
  q.off_stg = o;  // per producer warp: parts x 2 copies x seglen bf16 (+16 B pad each)
  o += (size_t)kProdWarps * q.parts * 2 * rup(q.seglen * 2 + 16, 16);
  q.off_coef = o;
  o += (size_t)rup(N * 10 * 4, 16);
  q.off_alpha = o;
  o += (size_t)rup(G * N * 4 * 4, 16);
  q.off_bar = o;
  o += 8 * (2 * kMaxStages + 4 + 2) + 16;
  q.smem = o + 128;  // base alignment slack
  // more than half of an SM's shared memory: one CTA per SM, so the 512-column TMEM
  // allocation never waits for another CTA
  if (q.smem < 120 * 1024) q.smem = 120 * 1024;
  *p = q;
  return q.smem <= (size_t)kMaxSmem;
}

static bool choose_plan(int N, int L, int prec, Plan *p) {
  for (int G = 5; G >= 1; --G)
    for (int NS = kMaxStages; NS >= 4; NS -= 2)
      if (make_plan(N, L, prec, G, NS, p)) return true;
  return false;
}

// ----------------------------------------------------------------- tcgen05 wrappers
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  // K-major, no swizzle: start>>4 | LBO>>4 << 16 | SBO>>4 << 32 | version 1 << 46
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__host__ __device__ constexpr uint32_t idesc_f16(int ab_fmt, int M, int N) {
  // D = F32 (bit 4), A/B format (bits 7-9, 10-12: 0 = F16, 1 = BF16), both K-major,
  // N >> 3 at bits 17-22, M >> 4 at bits 24-28.
  return (1u << 4) | ((uint32_t)ab_fmt << 7) | ((uint32_t)ab_fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ uint32_t tmem_ld1(uint32_t taddr) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
  return r;
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void epi_bar_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Split x into hi + lo 16-bit floats; returns the two bit patterns.
template <int PREC>
__device__ __forceinline__ void split16(float x, uint16_t &hi, uint16_t &lo) {
  if (PREC == SVK_PREC_FP16X3) {
    const __half a = __float2half_rn(x);
    const __half b = __float2half_rn(x - __half2float(a));
    hi = __half_as_ushort(a);
    lo = __half_as_ushort(b);
  } else {
    const __nv_bfloat16 a = __float2bfloat16_rn(x);
    const __nv_bfloat16 b = __float2bfloat16_rn(x - __bfloat162float(a));
    hi = __bfloat16_as_ushort(a);
    lo = __bfloat16_as_ushort(b);
  }
}

// ----------------------------------------------------------------- block schedule
struct Sched {
  int nbx, nby, nblocks;
  __device__ void block(int b, int G, int &x0, int &y0) const {
    x0 = (b % nbx) * kTileM;
    y0 = (b / nbx) * G;
  }
};

// ----------------------------------------------------------------- table preparation
// Table row (K group j, row rho) holds taps q = 8j..8j+7 of stamp k = rho % N in slice
// P = rho / N (kernel row v = h + G - 1 - P); zero outside the kernel or the slices.
template <int PREC>
__global__ void tc_prep_table(const float *__restrict__ basis, Plan pl, float bscale, uint4 *th, uint4 *tl) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= pl.nKG * pl.nrows) return;
  const int j = idx / pl.nrows, rho = idx % pl.nrows;
  const int P = rho / pl.N, k = rho % pl.N, v = pl.h + pl.G - 1 - P;
  uint16_t hv[8], lv[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int q = 8 * j + c;
    float val = 0.0f;
    if (P < pl.NP && q < pl.L && v >= -pl.h && v <= pl.h)
      val = basis[(size_t)k * pl.L * pl.L + (v + pl.h) * pl.L + (pl.h - q + pl.h)] * bscale;
    split16<PREC>(val, hv[c], lv[c]);
  }
  uint4 a, b;
  a.x = hv[0] | ((uint32_t)hv[1] << 16);
  a.y = hv[2] | ((uint32_t)hv[3] << 16);
  a.z = hv[4] | ((uint32_t)hv[5] << 16);
  a.w = hv[6] | ((uint32_t)hv[7] << 16);
  b.x = lv[0] | ((uint32_t)lv[1] << 16);
  b.y = lv[2] | ((uint32_t)lv[3] << 16);
  b.z = lv[4] | ((uint32_t)lv[5] << 16);
  b.w = lv[6] | ((uint32_t)lv[7] << 16);
  th[idx] = a;
  if (tl) tl[idx] = b;
}

// ----------------------------------------------------------------- main kernel
template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
    tc_basis_kernel(const float *__restrict__ R, int pitch_R, const float *__restrict__ I, int pitch_I, int W,
                    int H, const float *__restrict__ coeffs, int degree, float *__restrict__ out, int pitch_out,
                    const uint4 *__restrict__ tab_hi, const uint4 *__restrict__ tab_lo, Plan pl, Sched sc,
                    float rscale, float out_scale, uint32_t *status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  constexpr int kParts = (PREC == SVK_PREC_BF16) ? 1 : 2;
  constexpr int kFmt = (PREC == SVK_PREC_FP16X3) ? 0 : 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = pl.N, G = pl.G, h = pl.h, T = n_terms(degree);

  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + pl.off_bar);
  const int NS = pl.NS;
  uint64_t *full = bars, *empty = bars + kMaxStages, *acc_full = bars + 2 * kMaxStages,
           *acc_empty = acc_full + 2, *tab_bar = acc_empty + 2, *drain_bar = tab_bar + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain_bar + 1);
  float *coef = reinterpret_cast<float *>(sm + pl.off_coef);
  float *alpha = reinterpret_cast<float *>(sm + pl.off_alpha);

  // ---- set-up
  if (warp == kMmaWarp) {
    tmem_alloc(tmem_slot, kTmemCols);
    if (lane == 0) {
      for (int s = 0; s < NS; ++s) {
        mbar_init(&full[s], 1);
        mbar_init(&empty[s], 1);
      }
      for (int b = 0; b < 2; ++b) {
        mbar_init(&acc_full[b], 1);
        mbar_init(&acc_empty[b], kEpiWarps * 32);
      }
      mbar_init(tab_bar, 1);
      mbar_init(drain_bar, 1);
      fence_mbar_init();
      // the basis tables, once per CTA (bulk copies of <= 32 KB)
      const uint32_t total = (uint32_t)(pl.table_bytes * kParts);
      mbar_arrive_expect_tx(tab_bar, total);
      for (int part = 0; part < kParts; ++part) {
        const unsigned char *src = reinterpret_cast<const unsigned char *>(part ? tab_lo : tab_hi);
        unsigned char *dst = sm + (part ? pl.off_tab_lo : pl.off_tab_hi);
        for (size_t o = 0; o < pl.table_bytes; o += 32768) {
          const uint32_t n = (uint32_t)((pl.table_bytes - o) < 32768 ? (pl.table_bytes - o) : 32768);
          bulk_load(dst + o, src + o, n, tab_bar);
        }
      }
    }
  }
  if (warp < kEpiWarps) {
    for (int i = threadIdx.x; i < N * 10; i += kEpiWarps * 32) {
      const int k = i / 10, t = i % 10;
      coef[i] = (t < T) ? coeffs[(size_t)k * T + t] : 0.0f;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp >= kFirstProdWarp) {
    // ================================================================ producers
    const int pw = warp - kFirstProdWarp;
    uint16_t *stg = reinterpret_cast<uint16_t *>(sm + pl.off_stg) +
                    (size_t)pw * kParts * 2 * (rup(pl.seglen * 2 + 16, 16) / 2);
    const int cstride = rup(pl.seglen * 2 + 16, 16) / 2;  // elements between staging copies
    uint32_t row_seq = 0;
    for (int b = blockIdx.x; b < sc.nblocks; b += gridDim.x) {
      int x0, y0;
      sc.block(b, G, x0, y0);
      const int r_lo = max(0, y0 - h), r_hi = min(H - 1, y0 + G - 1 + h);
      for (int r = r_lo; r <= r_hi; ++r, ++row_seq) {
        if ((int)(row_seq % kProdWarps) != pw) continue;
        const int stage = row_seq % NS;
        const uint32_t use = row_seq / NS;
        if (!mbar_wait_bounded(&empty[stage], (use & 1) ^ 1, status)) goto done;
        // stage the row segment R(r, x0 - h + e), e < seglen, as hi/lo 16-bit copies;
        // copy 1 is shifted by one element so every chunk start is 4-byte aligned
        const float *rrow = R + (size_t)r * pitch_R;
        const int xb = x0 - h;
        for (int e = lane; e < pl.seglen; e += 32) {
          const int gx = xb + e;
          const float v = (gx >= 0 && gx < W) ? rrow[gx] * rscale : 0.0f;
          uint16_t hv, lv;
          split16<PREC>(v, hv, lv);
          stg[e] = hv;
          if (e > 0) stg[cstride + e - 1] = hv;
          if (kParts == 2) {
            stg[2 * cstride + e] = lv;
            if (e > 0) stg[3 * cstride + e - 1] = lv;
          }
        }
        __syncwarp();
        unsigned char *hk = sm + pl.off_stage + (size_t)stage * kParts * pl.S * 128;
        for (int e = lane; e < 8 * pl.S; e += 32) {
#pragma unroll
          for (int part = 0; part < kParts; ++part) {
            const uint16_t *src = stg + (size_t)(2 * part + (e & 1)) * cstride + (e & ~1);
            const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
            uint4 chunk;
            chunk.x = s32[0];
            chunk.y = s32[1];
            chunk.z = s32[2];
            chunk.w = s32[3];
            *reinterpret_cast<uint4 *>(hk + (size_t)part * pl.S * 128 + (size_t)e * 16) = chunk;
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[stage]);
        __syncwarp();
      }
    }
  } else if (warp == kMmaWarp) {
    // ================================================================ MMA issuer
    if (lane == 0) {
      if (!mbar_wait_bounded(tab_bar, 0, status)) goto drain;
      {
        const uint32_t idesc = idesc_f16(kFmt, kTileM, pl.nmma);
        const uint32_t tab_h = smem_u32(sm + pl.off_tab_hi), tab_l = smem_u32(sm + pl.off_tab_lo);
        const uint32_t stage0 = smem_u32(sm + pl.off_stage);
        const uint32_t lbo_b = (uint32_t)pl.nrows * 16u;
        uint32_t row_seq = 0, blk_seq = 0;
        for (int b = blockIdx.x; b < sc.nblocks; b += gridDim.x, ++blk_seq) {
          int x0, y0;
          sc.block(b, G, x0, y0);
          const int buf = blk_seq & 1;
          if (!mbar_wait_bounded(&acc_empty[buf], ((blk_seq >> 1) & 1) ^ 1, status)) goto drain;
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(buf * kAccStride);
          uint32_t acc = 0;
          const int r_lo = max(0, y0 - h), r_hi = min(H - 1, y0 + G - 1 + h);
          for (int r = r_lo; r <= r_hi; ++r, ++row_seq) {
            const int stage = row_seq % NS;
            if (!mbar_wait_bounded(&full[stage], (row_seq / NS) & 1, status)) goto drain;
            tc_fence_after();
            const uint32_t a_h = stage0 + (uint32_t)(stage * kParts * pl.S * 128);
            const uint32_t a_l = a_h + (uint32_t)(pl.S * 128);
            const uint32_t rho0 = (uint32_t)((r - y0 + h) * N);
            for (int ks = 0; ks < pl.nks; ++ks) {
              const uint32_t boff = (uint32_t)(2 * ks) * lbo_b + rho0 * 16u;
              const uint64_t ah = sdesc(a_h + (uint32_t)ks * 256u, 128u, 128u);
              const uint64_t bh = sdesc(tab_h + boff, lbo_b, 128u);
              umma_f16(d_tmem, ah, bh, idesc, acc);
              acc = 1;
              if (kParts == 2) {
                const uint64_t al = sdesc(a_l + (uint32_t)ks * 256u, 128u, 128u);
                const uint64_t bl = sdesc(tab_l + boff, lbo_b, 128u);
                umma_f16(d_tmem, ah, bl, idesc, 1);
                umma_f16(d_tmem, al, bh, idesc, 1);
              }
            }
            umma_commit(&empty[stage]);  // stage reusable once these MMAs have read it
          }
          umma_commit(&acc_full[buf]);
        }
      }
    drain:
      // every MMA issued by this thread has completed before TMEM is released
      umma_commit(drain_bar);
      mbar_wait_bounded(drain_bar, 0, status);
    }
    __syncwarp();
  } else {
    // ================================================================ epilogue
    const int m = threadIdx.x;  // TMEM lane == pixel offset in the tile
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    uint32_t blk_seq = 0;
    for (int b = blockIdx.x; b < sc.nblocks; b += gridDim.x, ++blk_seq) {
      int x0, y0;
      sc.block(b, G, x0, y0);
      // alpha[g][k][i] = sum_j c[k][(i,j)] yt^j : a_k(x, y) = sum_i alpha[g][k][i] xt^i
      epi_bar_sync();
      for (int e = m; e < G * N; e += 128) {
        const int g = e / N, k = e % N, y = y0 + g;
        const float yt = H > 1 ? (2.0f * (float)y - (float)(H - 1)) / (float)(H - 1) : 0.0f;
        float al[4] = {0.f, 0.f, 0.f, 0.f};
        int t = 0;
        for (int i = 0; i <= degree; ++i) {
          float yj = 1.0f, s = 0.0f;
          for (int j = 0; j <= degree - i; ++j, ++t) {
            s = fmaf(coef[k * 10 + t], yj, s);
            yj *= yt;
          }
          al[i] = s;
        }
        *reinterpret_cast<float4 *>(alpha + (size_t)e * 4) = make_float4(al[0], al[1], al[2], al[3]);
      }
      epi_bar_sync();
      const int buf = blk_seq & 1;
      if (!mbar_wait_bounded(&acc_full[buf], (blk_seq >> 1) & 1, status)) break;
      tc_fence_after();
      const int x = x0 + m;
      const float xt = W > 1 ? (2.0f * (float)x - (float)(W - 1)) / (float)(W - 1) : 0.0f;
      for (int g = 0; g < G; ++g) {
        const int y = y0 + g;
        if (y >= H) break;
        const uint32_t col0 = (uint32_t)(buf * kAccStride + (G - 1 - g) * N);
        float s = 0.0f;
        // columns [col0, col0 + N): 16-column loads; the last load is moved back so it
        // never reads past column col0 + N - 1 (keeps every read inside the allocation)
        for (int kc = 0; kc < N; kc += 16) {
          const int start = (kc + 16 <= N || N < 16) ? kc : N - 16;
          uint32_t v[16];
          if (N >= 16) {
            tmem_ld16(tmem_base + lane_off + col0 + (uint32_t)start, v);
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = 0u;
            for (int e = 0; e < N; ++e) v[e] = tmem_ld1(tmem_base + lane_off + col0 + (uint32_t)e);
          }
          tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int k = start + e;
            if (k >= kc && k < N) {
              const float4 a4 = *reinterpret_cast<const float4 *>(alpha + (size_t)(g * N + k) * 4);
              const float ak = fmaf(fmaf(fmaf(a4.w, xt, a4.z), xt, a4.y), xt, a4.x);
              s = fmaf(ak, __uint_as_float(v[e]), s);
            }
          }
        }
        if (x < W) {
          float o = s * out_scale;
          if (I) o -= I[(size_t)y * pitch_I + x];
          out[(size_t)y * pitch_out + x] = o;
        }
      }
      tc_fence_before();
      mbar_arrive(&acc_empty[buf]);
    }
  }
done:
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tmem_base, kTmemCols);
}

}  // namespace

size_t tc_workspace_size(int precision, int N, int L) {
  Plan pl;
  if (!choose_plan(N, L, precision, &pl)) return 0;
  return pl.table_bytes * 2 + 256;
}

int launch_tc(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H, const float *basis, int N,
              int L, const float *coeffs, int degree, int precision, float *out, int pitch_out, void *ws,
              size_t ws_bytes, cudaStream_t s) {
  Plan pl;
  if (!choose_plan(N, L, precision, &pl))
    return set_error(SVK_ERR_UNSUPPORTED, "no tensor-core plan fits shared memory for N=%d L=%d", N, L);
  if (!ws || ws_bytes < pl.table_bytes * 2 + 256) return set_error(SVK_ERR_WORKSPACE, "tensor-core workspace too small");
  unsigned char *w = static_cast<unsigned char *>(ws);
  uint4 *th = reinterpret_cast<uint4 *>(w);
  uint4 *tl = reinterpret_cast<uint4 *>(w + pl.table_bytes);
  uint32_t *status = reinterpret_cast<uint32_t *>(w + pl.table_bytes * 2);
  cudaError_t e = cudaMemsetAsync(status, 0, 4, s);
  if (e != cudaSuccess) return cuda_status(e, "status reset");
  // FP16 operands: power-of-two scales keep R and B inside the FP16 range
  float bscale = 1.0f, rscale = 1.0f;
  if (precision == SVK_PREC_FP16X3) {
    bscale = 1024.0f;       // basis values are O(1e-3 .. 1)
    rscale = 1.0f / 16.0f;  // counts up to ~1e6 stay below 65504
  }
  const int nrow_items = pl.nKG * pl.nrows;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  Sched sc;
  sc.nbx = (W + kTileM - 1) / kTileM;
  sc.nby = (H + pl.G - 1) / pl.G;
  sc.nblocks = sc.nbx * sc.nby;
  const int grid = sc.nblocks < nsm ? sc.nblocks : nsm;
  const float out_scale = 1.0f / (bscale * rscale);
#define SVK_TC_LAUNCH(P)                                                                                       \
  do {                                                                                                         \
    tc_prep_table<P><<<(nrow_items + 255) / 256, 256, 0, s>>>(basis, pl, bscale, th, pl.parts == 2 ? tl : nullptr); \
    e = cudaFuncSetAttribute(tc_basis_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);   \
    if (e != cudaSuccess) return cuda_status(e, "tc_basis_kernel smem attribute");                             \
    tc_basis_kernel<P><<<grid, kThreads, pl.smem, s>>>(R, pitch_R, I, pitch_I, W, H, coeffs, degree, out,      \
                                                       pitch_out, th, tl, pl, sc, rscale, out_scale, status);   \
  } while (0)
  if (precision == SVK_PREC_BF16X3)
    SVK_TC_LAUNCH(SVK_PREC_BF16X3);
  else if (precision == SVK_PREC_FP16X3)
    SVK_TC_LAUNCH(SVK_PREC_FP16X3);
  else
    SVK_TC_LAUNCH(SVK_PREC_BF16);
#undef SVK_TC_LAUNCH
  return cuda_status(cudaGetLastError(), "tc_basis_kernel launch");
}

}  // namespace svk
