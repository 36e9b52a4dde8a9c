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
// K steps.  A reference row has nG = ceil(L/8) groups of 8 taps; one MMA takes two
// groups (K = 16).  Rows are consumed in pairs (r, r+1) held in consecutive pipeline
// stages.  When nG is odd the last group of r and the last group of r+1 form one MMA:
// its second core-matrix column lies one stage further in the A operand (LBO = stage
// size) and one basis slice further in the B operand (LBO = Nb * 16 bytes), so only
// ceil(L/8)*8 taps per row are multiplied instead of a multiple of 16.  A block with
// an odd row count pairs its last row with an all-zero tile that the producers write
// into the next stage (the basis table carries one slice of zero rows beyond its end for
// that pair's B window).
//
// Handshake granularity.  The tensor core queues almost nothing ahead of the issuing
// thread (measured: a delay in that thread between MMAs idles the pipe for about as
// long), and an mbarrier wait costs that thread ~300 cycles even when the phase has long
// completed, so the MMA thread waits once per `full` group of rpg = NS / 2 rows (two
// groups in flight; 8 rows = 36 MMAs per wait in the split modes where 16 stages fit).
// Its `empty` commits (cheap, no wait) come every epg = 4 rows, so a stage is handed back
// to the producers as soon as the MMAs of its 4-row group are done and no producer warp
// has to build two rows of one group back to back.  Each block's row sequence is padded
// with empty slots to a multiple of rpg.
//
// Roles (16 warps): warps 0-7 epilogue (TMEM lane quarter w % 4, output rows of parity
// w / 4), warp 8 TMEM owner and MMA issuer (one thread), warps 9-11 and 13-15 producers
// (each prefetches its next reference row into registers while it converts the current
// one), warp 12 idle (it would share the MMA warp's scheduler).  No role uses local memory:
// with ~227 KB of shared memory the L1 left for it is small.  All waits are bounded; a
// wait that runs out records a status word and the CTA unwinds (MMAs drained, TMEM
// freed).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "svk_common.cuh"
#include "svk_internal.h"
#include "svk_umma.cuh"

namespace svk {
namespace {

constexpr int kMaxSmem = 232448;  // 227 KB opt-in shared memory per CTA on sm_100-class parts
// Warp 12 shares the MMA warp's scheduler (warp % 4) and stays idle: the issuing thread
// gets that scheduler's issue slots to itself apart from two epilogue warps (measured 2 %
// faster than a seventh producer there).
constexpr int kEpiWarps = 8, kMmaWarp = 8, kProdWarps = 6, kFirstProdWarp = 9, kIdleWarp = 12;
constexpr int kSegRegs = 5;  // staged row segment: <= 160 elements = 5 per lane
constexpr int kThreads = (kEpiWarps + 1 + kProdWarps + 1) * 32;
constexpr int kTileM = 128;
constexpr int kMaxStages = 16;  // Hankel stages (reference rows in flight), upper bound
constexpr int kMaxG = 40;          // output rows per block (few stamps: the T-factored form)
constexpr uint32_t kTmemCols = 512;
constexpr int kAccStride = 256;  // TMEM columns per accumulator buffer

// ----------------------------------------------------------------- plan (host+device)
struct Plan {
  int N, L, h, G, nmma;    // stamps, kernel size, half size, output rows/block, MMA N
  int nG, nKG;             // tap groups of 8 per reference row; table groups (= nG)
  int S;                   // Hankel blocks per reference row (= 16 + nKG - 1)
  size_t stage_bytes;      // one pipeline stage (hi [+ lo] Hankel tiles)
  int seglen;              // staged row length (elements) = 8 S + 8
  int NP, nrows;           // table slices, table rows per K group (global tables)
  int parts;               // Hankel (A) parts: 2 for split precisions, 1 for plain BF16
  int tparts;              // basis-table (B) parts: 2 for the x3 splits, 1 for plain BF16
                           // and FP16x2 (whose basis is taken as FP16-exact)
  int NS;                  // Hankel pipeline stages
  int rpg, epg;            // rows per `full` group (NS / 2: two groups in flight, NS / 4 when
                           // streamed) and per `empty` group (4, or rpg when smaller)
  int stream;              // 1: basis slices streamed through a ring (below), 0: tables resident
  int xr;                  // rows a block's sequence carries beyond its reference rows (G - 1
                           // when streamed: the owners of its last window's slices)
  int M, srows;            // ring: mirror slots; shared-memory rows per K group (table or ring)
  int prec;
  size_t table_bytes;      // one global table (hi or lo)
  size_t smem_tab_bytes;   // its shared-memory copy or ring (hi or lo)
  size_t off_tab_hi, off_tab_lo, off_stage, off_stg, off_coef, off_alpha, off_alphaS, off_bar, smem;
};

__host__ __device__ inline int rup(int v, int m) { return (v + m - 1) / m * m; }

static bool make_plan(int N, int L, int prec, int G, int NS, int stream, Plan *p) {
  Plan q{};
  q.N = N;
  q.L = L;
  q.h = (L - 1) / 2;
  q.G = G;
  q.prec = prec;
  if (NS != 4 && NS != 8 && NS != 16) return false;
  q.NS = NS;
  q.stream = stream ? 1 : 0;
  q.rpg = stream ? NS / 4 : NS / 2;
  q.epg = q.rpg < 4 ? q.rpg : 4;
  q.parts = (prec == SVK_PREC_BF16) ? 1 : 2;
  q.tparts = (prec == SVK_PREC_BF16 || prec == SVK_PREC_FP16X2) ? 1 : 2;
  q.nmma = rup(G * N, 16);
  if (q.nmma > 256 || q.nmma < 16) return false;
  q.nG = (L + 7) / 8;
  q.nKG = q.nG;
  q.S = kTileM / 8 + q.nKG - 1;
  q.seglen = 8 * q.S + 8;
  if (q.seglen > 32 * kSegRegs) return false;
  q.stage_bytes = (size_t)q.parts * q.S * 128;
  q.NP = L + 2 * (G - 1);
  // slices, then zero rows: 16 for the MMA width beyond G*N and, when nG is odd, N for
  // the window one slice further that an odd last row's last tap group is paired with
  // (its A tile is zero)
  q.nrows = rup(q.NP * N + 16 + ((q.nG & 1) ? N : 0), 8);
  q.table_bytes = (size_t)q.nKG * q.nrows * 16;
  if (stream) {
    // the MMA of a group of rpg rows reads the slices of the next group's first
    // G - 1 + (nG & 1) rows and no further, so it waits for one group ahead of it; the
    // producers fill that group while the tensor core runs the one before (NS / rpg = 4)
    if (NS < 8 || G - 1 + (q.nG & 1) > q.rpg) return false;
    q.xr = G - 1;
    // slot k holds the slice of the row in stage k; a window (and the paired window one
    // slot further) covers ceil(nmma / N) slots from its row's slot on, so the first M
    // slots are mirrored after the last and every window is contiguous
    q.M = (q.nmma + N - 1) / N - 1;
    q.srows = rup((NS + q.M) * N, 8);
  } else {
    q.xr = 0;
    q.M = 0;
    q.srows = q.nrows;
  }
  q.smem_tab_bytes = (size_t)q.nKG * q.srows * 16;

  size_t o = 0;
  q.off_tab_hi = o;
  o += q.smem_tab_bytes;
  q.off_tab_lo = o;
  if (q.tparts == 2) o += q.smem_tab_bytes;
  o = rup((int)o, 128);
  q.off_stage = o;
  o += (size_t)NS * q.stage_bytes;
  q.off_stg = o;  // per producer warp: parts x 2 copies x seglen bf16 (+16 B pad each)
  o += (size_t)kProdWarps * q.parts * 2 * rup(q.seglen * 2 + 16, 16);
  q.off_coef = o;
  o += (size_t)rup(N * 10 * 4, 16);
  q.off_alpha = o;
  o += (size_t)rup(G * N * 4 * 4, 16);
  q.off_alphaS = o;  // G x 4 powers of xt x 64 load slots (only the 16..64-stamp epilogue)
  if (N >= 16 && N <= 64) o += (size_t)G * 64 * 16;
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
  // the widest MMA (most output rows per block) that fits, with resident tables and the
  // most stages when they fit, else with the slices streamed (large L, whose tables
  // leave no room for wide blocks); the autotuner replaces this default by measurement
  for (int G = kMaxG; G >= 1; --G) {
    for (int NS = kMaxStages; NS >= 4; NS /= 2)
      if (make_plan(N, L, prec, G, NS, 0, p)) return true;
    for (int NS = kMaxStages; NS >= 8; NS /= 2)
      if (make_plan(N, L, prec, G, NS, 1, p)) return true;
  }
  return false;
}

__device__ __forceinline__ void epi_bar_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Named barrier 1 over the 256 epilogue threads that also ORs a predicate: every epilogue
// thread gets the same answer, so a decision to give up (a bounded wait that ran out in
// any of them) is taken by all of them together and none is left at a barrier the others
// have abandoned.
__device__ __forceinline__ bool epi_bar_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, 256, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

// Split x into hi + lo 16-bit floats; returns the two bit patterns.
template <int PREC>
__device__ __forceinline__ void split16(float x, uint16_t &hi, uint16_t &lo) {
  if (PREC == SVK_PREC_FP16X3 || PREC == SVK_PREC_FP16X2) {
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

// ----------------------------------------------------------------- frames and blocks
// A launch processes a set of frames that share one plan (same N, L, precision): every
// frame's blocks are numbered consecutively from its block0, and each persistent CTA
// takes a contiguous range of that block space.  The set travels as a __grid_constant__
// kernel parameter, so a launch (or a CUDA graph of launches) needs no descriptor copy.
constexpr int kMaxFrames = 64;

struct FrameDesc {
  const float *R, *I;
  float *out;
  const float *coeffs;
  const uint4 *tab_hi, *tab_lo;  // this frame's basis tables (shared by frames with one basis)
  int W, H, pitch_R, pitch_I, pitch_out, degree;
  int y_begin, y_end;  // output rows of this launch (a band of the frame, or all of it)
  int r_begin, r_end;  // frame rows R holds (row r at R + (r - r_begin) * pitch_R); others read as 0
  int nbx, block0;  // blocks per band of G rows; first block of the frame in the set
  float rscale, out_scale;
};

struct FrameSet {
  int n, nblocks;
  FrameDesc fr[kMaxFrames];
};

__device__ __forceinline__ int advance_frame(const FrameSet &fs, int f, int b) {
  while (f + 1 < fs.n && b >= fs.fr[f + 1].block0) ++f;
  return f;
}

__device__ __forceinline__ void block_origin(const FrameDesc &fd, int b, int G, int &x0, int &y0) {
  const int lb = b - fd.block0;
  x0 = (lb % fd.nbx) * kTileM;
  y0 = fd.y_begin + (lb / fd.nbx) * G;
}

__device__ __forceinline__ void cta_block_range(const FrameSet &fs, int &b0, int &b1) {
  b0 = (int)((long long)blockIdx.x * fs.nblocks / gridDim.x);
  b1 = (int)((long long)(blockIdx.x + 1) * fs.nblocks / gridDim.x);
}

// The CTA's sequence of reference rows: for each of its blocks the rows
// max(0, y0-h) .. min(H-1, y0+G-1+h), then xr slots that only carry basis slices (streamed
// plans), padded with empty slots to a multiple of the rows per handshake group.
struct RowIt {
  int b, b_end, f, i, n, nseq, r_lo, x0, y0, rpg, xr;
  __device__ void set_block(const FrameSet &fs, int bb, int G, int h) {
    b = bb;
    i = 0;
    if (b < b_end) {
      f = advance_frame(fs, f, b);
      block_origin(fs.fr[f], b, G, x0, y0);
      r_lo = max(0, y0 - h);
      n = min(fs.fr[f].H - 1, y0 + G - 1 + h) - r_lo + 1;
      nseq = (n + xr + rpg - 1) & ~(rpg - 1);  // rpg is a power of two
    }
  }
  __device__ void next(const FrameSet &fs, int G, int h) {
    if (++i >= nseq) set_block(fs, b + 1, G, h);
  }
  __device__ bool valid() const { return b < b_end; }
  __device__ bool real() const { return i < n; }
  __device__ int row() const { return r_lo + i; }
};

// ----------------------------------------------------------------- table preparation
// Table row (K group j, row rho) holds taps q = 8j..8j+7 of stamp k = rho % N in slice
// P = rho / N (kernel row v = h + G - 1 - P); zero outside the kernel or the slices.
template <int PREC>
__global__ void tc_prep_table(const float *__restrict__ basis, Plan pl, float bscale, uint4 *th, uint4 *tl) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
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

// The epilogue's dot products for one pixel and output row: s[p] = sum over the slots of
// alpha[p][slot] * C[slot] for the powers p < NPOW of xt (the others are zero), the slots
// taken four at a time (q < NQ) as packed f32x2 pairs: P[p] accumulates slots 4q, 4q+2 in
// its low half and 4q+1, 4q+3 in its high half.  The coefficients are broadcast
// shared-memory loads (four wavefronts per 16 bytes), so slots and powers that carry
// nothing are not read.
template <int NPOW, int NQ>
__device__ __forceinline__ void slot_dots(const uint32_t (&v)[64], const float *ag, float (&s)[4]) {
  uint64_t P[4] = {0, 0, 0, 0};
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const uint64_t c01 = f2_pack(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]));
    const uint64_t c23 = f2_pack(__uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
#pragma unroll
    for (int p = 0; p < NPOW; ++p) {
      const ulonglong2 A = *reinterpret_cast<const ulonglong2 *>(ag + 64 * p + 4 * q);
      P[p] = f2_fma(A.x, c01, P[p]);
      P[p] = f2_fma(A.y, c23, P[p]);
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    float l = 0.0f, u = 0.0f;
    if (p < NPOW) f2_unpack(P[p], l, u);
    s[p] = l + u;
  }
}

// The same dot products with one output row's columns spread over four lanes.  The
// 16x256b TMEM loads start on a multiple of 8 columns, so the row's columns c0 .. c0+N-1
// are read from ca = c0 rounded down, in NREP = ceil((c0 - ca + N) / 8) repetitions of 8
// (slot s = column ca + s; the coefficients of stamp k sit at slot k + c0 - ca, zeros
// elsewhere).  Lane t gets slots 8r + 2(t%4), 8r + 2(t%4) + 1 (r < NREP) of the four
// pixels t/4 + 8j (j < 4) of its warp's lane quarter, so it reads 2 NREP coefficients per
// power instead of all 52 (8-byte loads, the warp's four distinct pairs in one wavefront),
// and the four lanes of a pixel group add their partial sums in two shuffle steps, after
// which lane t holds the sums of pixel t/4 + 8(t%4).  The pixels come in two halves (TMEM
// lanes 0..15 and 16..31 of the quarter, pixels j = 2hh, 2hh + 1), one load and wait
// each, so only one half's columns are live at a time.
template <int NPOW, int NREP>
__device__ __forceinline__ void quad_dots(uint32_t ca, bool in_range, const float *ag, int q, float (&s)[4]) {
  float K[2][NPOW];
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    uint32_t v[4 * NREP];
    if (in_range) {
      const uint32_t ta = ca + ((uint32_t)(16 * hh) << 16);
      tmem_ld256x4(ta, &v[0]);
      if (NREP == 8) {
        tmem_ld256x4(ta + 32u, &v[16]);
      } else {
        tmem_ld256x2(ta + 32u, &v[16]);
        tmem_ld256x1(ta + 48u, &v[24]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4 * NREP; ++i) v[i] = 0u;
    }
    tmem_ld_wait();
    uint64_t P[2][NPOW];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int p = 0; p < NPOW; ++p) P[j][p] = 0;
#pragma unroll
    for (int r = 0; r < NREP; ++r) {
      uint64_t A[NPOW];
#pragma unroll
      for (int p = 0; p < NPOW; ++p) A[p] = *reinterpret_cast<const uint64_t *>(ag + 64 * p + 8 * r + 2 * q);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const uint64_t c = f2_pack(__uint_as_float(v[4 * r + 2 * j]), __uint_as_float(v[4 * r + 2 * j + 1]));
#pragma unroll
        for (int p = 0; p < NPOW; ++p) P[j][p] = f2_fma(A[p], c, P[j][p]);
      }
    }
    // lanes q and q^1 swap the pixel of this half they do not keep (pixel parity q & 1)
#pragma unroll
    for (int p = 0; p < NPOW; ++p) {
      float l0, u0, l1, u1;
      f2_unpack(P[0][p], l0, u0);
      f2_unpack(P[1][p], l1, u1);
      const float s0 = l0 + u0, s1 = l1 + u1;
      const float mine = (q & 1) ? s1 : s0, other = (q & 1) ? s0 : s1;
      K[hh][p] = mine + __shfl_xor_sync(0xffffffffu, other, 1);
    }
  }
  // then lanes q and q^2 (half q >> 1): lane q ends with pixel j = q summed over its lanes
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    s[p] = 0.0f;
    if (p < NPOW) {
      const float mine = (q >> 1) ? K[1][p] : K[0][p];
      const float other = (q >> 1) ? K[0][p] : K[1][p];
      s[p] = mine + __shfl_xor_sync(0xffffffffu, other, 2);
    }
  }
}

// First column of output row g's accumulators, its offset from the 8-column boundary
// below, and the 8-column repetitions that cover its N columns from that boundary.
__host__ __device__ inline int quad_col(int G, int N, int g) { return (G - 1 - g) * N; }
__host__ __device__ inline int quad_off(int G, int N, int g) { return quad_col(G, N, g) & 7; }
__host__ __device__ inline int quad_reps(int G, int N, int g) { return (quad_off(G, N, g) + N + 7) >> 3; }

// ----------------------------------------------------------------- main kernel
// STREAM: the plan streams its basis slices (pl.stream); a template parameter, so the
// resident-table kernel carries none of the streamed bookkeeping in its issuing loop
template <int PREC, bool STREAM>
__global__ void __launch_bounds__(kThreads, 1)
    tc_basis_kernel(const __grid_constant__ FrameSet fs, const Plan pl, uint32_t *status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  // Hankel (A) parts and basis-table (B) parts: the x3 splits multiply Ah Bh + Ah Bl + Al Bh,
  // FP16x2 (an FP16-exact basis) Ah B + Al B, plain BF16 A B
  constexpr int kParts = (PREC == SVK_PREC_BF16) ? 1 : 2;
  constexpr int kPartsB = (PREC == SVK_PREC_BF16 || PREC == SVK_PREC_FP16X2) ? 1 : 2;
  constexpr int kFmt = (PREC == SVK_PREC_FP16X3 || PREC == SVK_PREC_FP16X2) ? 0 : 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = pl.N, G = pl.G, h = pl.h, NS = pl.NS;

  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + pl.off_bar);
  uint64_t *full = bars, *empty = bars + kMaxStages, *acc_full = bars + 2 * kMaxStages,
           *acc_empty = acc_full + 2, *tab_bar = acc_empty + 2, *drain_bar = tab_bar + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain_bar + 1);
  float *coef = reinterpret_cast<float *>(sm + pl.off_coef);
  float *alpha = reinterpret_cast<float *>(sm + pl.off_alpha);
  float *alphaS = reinterpret_cast<float *>(sm + pl.off_alphaS);
  dep_trigger();  // launched by launch_dependent: the next kernel may start launching
  const bool fast = (N >= 16 && N <= 64);
  // 49..52 stamps (the 49 of three Gaussians of degrees 6, 4, 2 among them): slot k carries
  // column k, loaded as three 16-column loads and one 4-column load (slots N..51 read
  // columns of the next group or the MMA padding, with zero coefficients), when those
  // columns lie inside the accumulator buffer; other stamp counts use four 16-column loads
  const bool exact = N >= 49 && N <= 52 && (G - 1) * N + 52 <= kAccStride;
  // Streamed plans (whose slice copies add to the shared-memory traffic) with 49..56
  // stamps whose output rows' column windows (from the 8-column boundary at or below the
  // row's first column, 7 or 8 repetitions of 8) lie inside the MMA's columns (those past
  // G*N hold exact zeros, products of the table's zero rows): the four-lane form of the dot
  // products (quad_dots), a quarter of the coefficient reads for about 45 % more epilogue
  // instructions.  Measured per 2048^2 frame: 2-4 % faster at L = 25 and 31 (streamed),
  // 3 % slower at L = 19 with resident tables, where the epilogue warps that share the
  // MMA-issuing thread's scheduler delay it.
  bool quad = STREAM && N >= 49 && N <= 56;
  for (int g = 0; g < G && quad; ++g)
    quad = (quad_col(G, N, g) & ~7) + 8 * quad_reps(G, N, g) <= pl.nmma;
  int b_begin, b_end;
  cta_block_range(fs, b_begin, b_end);

  // ---- set-up
  if (warp == kMmaWarp) {
    tmem_alloc(tmem_slot, kTmemCols);
    if (lane == 0) {
      for (int q = 0; q < NS / pl.rpg; ++q) mbar_init(&full[q], pl.rpg);  // one arrival per row of the group
      for (int q = 0; q < NS / pl.epg; ++q) mbar_init(&empty[q], 1);       // one commit per group
      for (int b = 0; b < 2; ++b) {
        mbar_init(&acc_full[b], 1);
        mbar_init(&acc_empty[b], kEpiWarps * 32);
      }
      mbar_init(tab_bar, 1);
      mbar_init(drain_bar, 1);
      fence_mbar_init();
    }
  }
  if (STREAM) {
    // the ring starts as zeros: slots a window reads beyond its slices (the MMA columns
    // past G*N, the partner window of an odd last row, whose A tile is zero) always hold
    // finite values
    for (size_t o = (size_t)threadIdx.x * 16; o < pl.smem_tab_bytes * kPartsB; o += (size_t)kThreads * 16)
      *reinterpret_cast<uint4 *>(sm + pl.off_tab_hi + o) = make_uint4(0u, 0u, 0u, 0u);
    fence_proxy_async_smem();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // set-up done (shared memory and TMEM only); global memory from here on, once the
  // kernel before this one in the stream has completed
  dep_wait();

  if (warp == kIdleWarp) {
    goto done;
  } else if (warp >= kFirstProdWarp) {
    // ================================================================ producers
    // P = min(kProdWarps, NS) warps take the rows in turn.  A warp about to fill group q
    // waits for the `empty` group that used its stages NS slots earlier to drain; that group
    // cannot be consumed again before this warp refills it, so its barrier is never more
    // than one phase ahead of the parity this warp waits for, and the parity wait cannot
    // alias a phase two uses ahead.
    const int pw = warp - kFirstProdWarp - (warp > kIdleWarp ? 1 : 0), nprod = kProdWarps < NS ? kProdWarps : NS;
    if (pw >= nprod) goto done;
    const int cstride = rup(pl.seglen * 2 + 16, 16) / 2;  // elements between staging copies
    uint16_t *stg = reinterpret_cast<uint16_t *>(sm + pl.off_stg) + (size_t)pw * kParts * 2 * cstride;
    // stage slot and its phase parity, stepped without divisions (NS, rpg and epg are
    // powers of two; nprod <= NS, so a step wraps at most once)
    const int rshift = __ffs(pl.rpg) - 1, eshift = __ffs(pl.epg) - 1;
    uint32_t stage = (uint32_t)pw, sph = 0;
    RowIt it;
    it.rpg = pl.rpg;
    it.xr = STREAM ? pl.xr : 0;
    it.b_end = b_end;
    it.f = 0;
    it.set_block(fs, b_begin, G, h);
    for (int k = 0; k < pw && it.valid(); ++k) it.next(fs, G, h);
    float cur[kSegRegs], nxt[kSegRegs];
    auto load_row = [&](const RowIt &ri, float (&v)[kSegRegs]) {
      const FrameDesc &fd = fs.fr[ri.f];
      const int r = ri.row();
      const bool held = r >= fd.r_begin && r < fd.r_end;
      const float *rrow = fd.R + (size_t)(held ? r - fd.r_begin : 0) * fd.pitch_R;
      const int xb = ri.x0 - h;
#pragma unroll
      for (int j = 0; j < kSegRegs; ++j) {
        const int e = lane + 32 * j, gx = xb + e;
        v[j] = (held && e < pl.seglen && gx >= 0 && gx < fd.W) ? __ldg(rrow + gx) * fd.rscale : 0.0f;
      }
    };
    if (it.valid() && it.real()) load_row(it, cur);
    while (it.valid()) {
      RowIt nx = it;
      for (int k = 0; k < nprod && nx.valid(); ++k) nx.next(fs, G, h);
      if (nx.valid() && nx.real()) load_row(nx, nxt);  // in flight while this row is built
      const int grp = (int)stage >> rshift;
      // every lane waits; the warp leaves together if any lane's wait ran out (the
      // warp-synchronous code below must not run with part of the warp gone)
      const bool ok = mbar_wait_bounded(&empty[stage >> eshift], sph ^ 1, status);
      if (__any_sync(0xffffffffu, !ok)) goto done;
      if (it.real()) {
        // hi/lo 16-bit copies of the segment; copy 1 is shifted by one element so every
        // 8-element chunk starts on a 4-byte boundary in one of the two copies
#pragma unroll
        for (int j = 0; j < kSegRegs; ++j) {
          const int e = lane + 32 * j;
          if (e < pl.seglen && SVK_CHECK(3 * cstride + e < kParts * 2 * cstride + (kParts == 1 ? 2 * cstride : 0), status, 1)) {
            uint16_t hv, lv;
            split16<PREC>(cur[j], hv, lv);
            stg[e] = hv;
            if (e > 0) stg[cstride + e - 1] = hv;
            if (kParts == 2) {
              stg[2 * cstride + e] = lv;
              if (e > 0) stg[3 * cstride + e - 1] = lv;
            }
          }
        }
        __syncwarp();
        unsigned char *hk = sm + pl.off_stage + (size_t)stage * pl.stage_bytes;
        // chunk e (e < 8 S <= 152): elements e .. e + 7; all loads issued before the stores
        uint4 chunk[kSegRegs][kParts];
#pragma unroll
        for (int j = 0; j < kSegRegs; ++j) {
          const int e = lane + 32 * j;
#pragma unroll
          for (int part = 0; part < kParts; ++part) {
            if (e < 8 * pl.S) {
              const uint32_t *s32 =
                  reinterpret_cast<const uint32_t *>(stg + (size_t)(2 * part + (e & 1)) * cstride + (e & ~1));
              chunk[j][part] = make_uint4(s32[0], s32[1], s32[2], s32[3]);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < kSegRegs; ++j) {
          const int e = lane + 32 * j;
#pragma unroll
          for (int part = 0; part < kParts; ++part)
            if (e < 8 * pl.S &&
                SVK_CHECK((size_t)part * pl.S * 128 + (size_t)e * 16 + 16 <= pl.stage_bytes && stage < (uint32_t)NS, status, 2))
              *reinterpret_cast<uint4 *>(hk + (size_t)part * pl.S * 128 + (size_t)e * 16) = chunk[j][part];
        }
        fence_proxy_async_smem();
      } else if (it.i == it.n && (it.n & 1) && (pl.nG & 1)) {
        // the slot after an odd last row: an all-zero tile, the partner of that row's
        // last tap group in the paired K step
        unsigned char *hk = sm + pl.off_stage + (size_t)stage * pl.stage_bytes;
        for (int o = lane * 16; o < (int)pl.stage_bytes; o += 32 * 16)
          if (SVK_CHECK(stage < (uint32_t)NS, status, 3)) *reinterpret_cast<uint4 *>(hk + o) = make_uint4(0u, 0u, 0u, 0u);
        fence_proxy_async_smem();
      }
      __syncwarp();
      if (!STREAM) {
        if (lane == 0) mbar_arrive(&full[grp]);
      } else {
        // the slice this row's slot holds (slice P0 + i of the block's table, the last of
        // the window of row i - G + 1) copied by the bulk-copy engine, in every K group and
        // part, and again into the mirror slot; the row's arrival then also waits for those
        // bytes
        const int t = it.r_lo - it.y0 + h + it.i;
        const int ncopy = t < pl.NP ? kPartsB * pl.nKG * ((int)stage < pl.M ? 2 : 1) : 0;
        if (lane == 0) {
          if (ncopy) mbar_arrive_expect_tx(&full[grp], (uint32_t)(ncopy * N * 16));
          else mbar_arrive(&full[grp]);
        }
        __syncwarp();
        if (lane < ncopy) {
          const int c = lane % (kPartsB * pl.nKG), part = c / pl.nKG, kg = c % pl.nKG;
          const uint4 *src = (part ? fs.fr[it.f].tab_lo : fs.fr[it.f].tab_hi) + (size_t)kg * pl.nrows + (size_t)t * N;
          const size_t slot = lane < kPartsB * pl.nKG ? stage : stage + NS;  // copy 2: the mirror
          const size_t dst = (part ? pl.off_tab_lo : pl.off_tab_hi) + ((size_t)kg * pl.srows + slot * N) * 16;
          if (SVK_CHECK(dst + (size_t)N * 16 <= (part ? pl.off_tab_lo : pl.off_tab_hi) + pl.smem_tab_bytes &&
                            (slot + 1) * N <= (size_t)pl.srows && ((size_t)t + 1) * N <= (size_t)pl.nrows,
                        status, 8))
            bulk_load(sm + dst, src, (uint32_t)(N * 16), &full[grp]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < kSegRegs; ++j) cur[j] = nxt[j];
      it = nx;
      stage += (uint32_t)nprod;
      if (stage >= (uint32_t)NS) {
        stage -= (uint32_t)NS;
        sph ^= 1;
      }
    }
  } else if (warp == kMmaWarp) {
    // ================================================================ MMA issuer
    // Descriptors are built once; the start-address field is linear (units of 16 bytes),
    // so every MMA's descriptors are a base descriptor plus an offset: the issuing
    // thread spends a few integer instructions per MMA instead of rebuilding them.
    uint32_t drain_phase = 0;
    if (lane == 0) {
      {
        const uint32_t idesc = idesc_f16(kFmt, kTileM, pl.nmma);
        const uint32_t lbo_b = (uint32_t)pl.srows * 16u, sbytes = (uint32_t)pl.stage_bytes;
        const uint64_t dA = sdesc(smem_u32(sm + pl.off_stage), 128u, 128u);
        const uint64_t dB = sdesc(smem_u32(sm + pl.off_tab_hi), lbo_b, 128u);
        const uint64_t dAx = sdesc(smem_u32(sm + pl.off_stage) + (uint32_t)(pl.nG - 1) * 128u, sbytes, 128u);
        const uint64_t dBx = sdesc(smem_u32(sm + pl.off_tab_hi) + (uint32_t)(pl.nG - 1) * lbo_b, (uint32_t)N * 16u, 128u);
        const uint64_t oBl = (uint64_t)((pl.off_tab_lo - pl.off_tab_hi) >> 4);  // hi -> lo table
        const uint64_t oAl = (uint64_t)((pl.S * 128) >> 4);                     // hi -> lo Hankel
        const uint64_t oKs_a = 256u >> 4, oKs_b = (uint64_t)(2u * lbo_b) >> 4;  // one K step
        const uint64_t oStage = sbytes >> 4, oSlice = (uint64_t)N;              // N rows x 16 B
        const int inrow = (pl.nG - (pl.nG & 1)) / 2;  // K steps a paired row takes on its own
        // The thread issues the MMAs back to back and the tensor core queues almost nothing
        // ahead of it, so its bookkeeping between MMAs stays free of divisions: the stage
        // of the next row pair and its phase parity, and the block origin, are stepped.
        uint32_t sa = 0, sph = 0, blk_seq = 0, acc = 0, d_tmem = 0, tab_phase = 0;
        const uint32_t rmask = (uint32_t)pl.rpg - 1u, emask = (uint32_t)pl.epg - 1u;
        const int rshift = __ffs(pl.rpg) - 1, eshift = __ffs(pl.epg) - 1;
        const uint4 *loaded = nullptr;
        // the frame's basis tables into shared memory, once every MMA that reads the
        // tables now there has completed (frames with one basis share their tables)
        auto load_tables = [&](const FrameDesc &fd) -> bool {
          if (fd.tab_hi == loaded) return true;
          if (loaded) {
            umma_commit(drain_bar);
            if (!mbar_wait_bounded(drain_bar, drain_phase, status)) return false;
            drain_phase ^= 1;
          }
          mbar_arrive_expect_tx(tab_bar, (uint32_t)(pl.table_bytes * kPartsB));
          for (int part = 0; part < kPartsB; ++part) {
            const unsigned char *src = reinterpret_cast<const unsigned char *>(part ? fd.tab_lo : fd.tab_hi);
            unsigned char *dst = sm + (part ? pl.off_tab_lo : pl.off_tab_hi);
            for (size_t o = 0; o < pl.table_bytes; o += 32768) {
              const uint32_t n = (uint32_t)((pl.table_bytes - o) < 32768 ? (pl.table_bytes - o) : 32768);
              bulk_load(dst + o, src + o, n, tab_bar);
            }
          }
          if (!mbar_wait_bounded(tab_bar, tab_phase, status)) return false;
          tab_phase ^= 1;
          loaded = fd.tab_hi;
          return true;
        };
        // K steps [0, nsteps) of the row whose Hankel tile is at descriptor a and whose
        // basis window starts at descriptor b
        auto row_mmas = [&](uint64_t a, uint64_t b, int nsteps) {
          for (int ks = 0; ks < nsteps; ++ks, a += oKs_a, b += oKs_b) {
            if (kParts == 2 && kPartsB == 2) {  // A hi read once for its two products
              umma_f16_fill(d_tmem, a, b, idesc, acc);
              umma_f16_lastuse(d_tmem, a, b + oBl, idesc, 1);
              umma_f16(d_tmem, a + oAl, b, idesc, 1);
            } else if (kParts == 2) {  // FP16x2: A hi and lo against the one B
              umma_f16(d_tmem, a, b, idesc, acc);
              umma_f16(d_tmem, a + oAl, b, idesc, 1);
            } else {
              umma_f16(d_tmem, a, b, idesc, acc);
            }
            acc = 1;
          }
        };
        int f = 0, x0 = 0, y0 = 0;
        // streamed plans wait one group ahead (its first rows hold the slices this group's
        // windows end with): the CTA's first group before its first block
        if (STREAM && b_begin < b_end)
          if (!mbar_wait_bounded(&full[0], 0, status)) goto drain;
        for (int b = b_begin; b < b_end; ++b, ++blk_seq) {
          if (b == b_begin || (f + 1 < fs.n && b >= fs.fr[f + 1].block0)) {
            f = advance_frame(fs, f, b);
            block_origin(fs.fr[f], b, G, x0, y0);
          } else {  // the next block of the same frame: one tile to the right, or the next band
            x0 += kTileM;
            if (x0 >= fs.fr[f].nbx * kTileM) {
              x0 = 0;
              y0 += G;
            }
          }
          const FrameDesc &fd = fs.fr[f];
          if (!STREAM && !load_tables(fd)) goto drain;
          const int buf = blk_seq & 1;
          if (!mbar_wait_bounded(&acc_empty[buf], ((blk_seq >> 1) & 1) ^ 1, status)) goto drain;
          tc_fence_after();
          d_tmem = tmem_base + (uint32_t)(buf * kAccStride);
          acc = 0;
          const int r_lo = max(0, y0 - h), n = min(fd.H - 1, y0 + G - 1 + h) - r_lo + 1;
          const int nseq = (n + (STREAM ? pl.xr : 0) + pl.rpg - 1) & ~(pl.rpg - 1);
          // resident tables: the window of row r_lo + i starts at slice r_lo + i - y0 + h of
          // the table; streamed: at the slot of the row's own stage
          const uint64_t bw0 = STREAM ? dB : dB + (uint64_t)(r_lo - y0 + h) * oSlice;
          const uint64_t bx0 = STREAM ? dBx : dBx + (uint64_t)(r_lo - y0 + h) * oSlice;
          for (int i = 0; i < nseq; i += 2) {  // stages sa, sa + 1
            if ((sa & rmask) == 0) {
              if (!STREAM) {
                if (!mbar_wait_bounded(&full[sa >> rshift], sph, status)) goto drain;
              } else if (b + 1 < b_end || i + pl.rpg < nseq) {  // the next group, if any
                uint32_t na = sa + (uint32_t)pl.rpg, nph = sph;
                if (na >= (uint32_t)NS) {
                  na -= (uint32_t)NS;
                  nph ^= 1;
                }
                if (!mbar_wait_bounded(&full[na >> rshift], nph, status)) goto drain;
              }
            }
            // shared-memory operands: ordered by the producers' proxy fence + mbarrier
            // the pair's two stages inside the ring; the B window of the pair's first row (and
            // the slice after it, read by the paired last tap groups) inside the table or ring
            const uint32_t wrow = STREAM ? sa : (uint32_t)(r_lo + i - y0 + h);
            if (!SVK_CHECK(sa + 1 < (uint32_t)NS && (i >= n || (r_lo + i - y0 + h >= 0 &&
                               (wrow + ((i + 1 < n || (pl.nG & 1)) ? 1 : 0)) * N + pl.nmma <= (uint32_t)pl.srows)),
                           status, 5))
              goto drain;
            const uint64_t a = dA + (uint64_t)sa * oStage;
            const uint64_t bw = bw0 + (uint64_t)(STREAM ? sa : (uint32_t)i) * oSlice;  // window of row r_lo + i
            if (i < n) {
              // rows r_lo + i and r_lo + i + 1 (for an odd last row the second is the
              // producers' all-zero tile): each row's full K steps, then their last tap
              // groups together in one K step when nG is odd
              row_mmas(a, bw, inrow);
              if (i + 1 < n) row_mmas(a + oStage, bw + oSlice, inrow);
              if (pl.nG & 1) {
                const uint64_t ax = dAx + (uint64_t)sa * oStage;
                const uint64_t bx = bx0 + (uint64_t)(STREAM ? sa : (uint32_t)i) * oSlice;
                if (kParts == 2 && kPartsB == 2) {
                  umma_f16_fill(d_tmem, ax, bx, idesc, acc);
                  umma_f16_lastuse(d_tmem, ax, bx + oBl, idesc, 1);
                  umma_f16(d_tmem, ax + oAl, bx, idesc, 1);
                } else if (kParts == 2) {
                  umma_f16(d_tmem, ax, bx, idesc, acc);
                  umma_f16(d_tmem, ax + oAl, bx, idesc, 1);
                } else {
                  umma_f16(d_tmem, ax, bx, idesc, acc);
                }
                acc = 1;
              }
            }
            if (((sa + 2u) & emask) == 0) umma_commit(&empty[sa >> eshift]);
            sa += 2;
            if (sa == (uint32_t)NS) {
              sa = 0;
              sph ^= 1;
            }
          }
          umma_commit(&acc_full[buf]);
        }
      }
    drain:
      // every MMA issued by this thread has completed before TMEM is released
      umma_commit(drain_bar);
      mbar_wait_bounded(drain_bar, drain_phase, status);
    }
    __syncwarp();
  } else {
    // ================================================================ epilogue
    // Eight warps: warp w reads TMEM lane quarter w % 4 (pixels 32 (w % 4) ..) and the
    // output rows g of parity w / 4, so two warps share each scheduler and one's TMEM
    // wait overlaps the other's arithmetic.
    const int et = threadIdx.x;  // 0 .. 255
    // m: the pixel (TMEM lane) whose output this thread writes; in the four-lane form the
    // lane that ends with pixel t/4 + 8(t%4) of the quarter
    const int m = (warp & 3) * 32 + (quad ? (lane >> 2) + 8 * (lane & 3) : lane), par = warp >> 2;
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    uint32_t blk_seq = 0;
    int f = 0, coef_frame = -1;
    float inext[3];
    auto load_I = [&](int b, int fi, float (&v)[3]) {
      int xq = 0, yq = 0;
      const bool ok = b < b_end;
      const FrameDesc &fq = fs.fr[fi];
      if (ok) block_origin(fq, b, G, xq, yq);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int g = par + 2 * j;
        v[j] = (ok && fq.I && g < G && yq + g < fq.y_end && xq + m < fq.W)
                   ? __ldg(fq.I + (size_t)(yq + g) * fq.pitch_I + xq + m) : 0.0f;
      }
    };
    if (b_begin < b_end) load_I(b_begin, advance_frame(fs, 0, b_begin), inext);
    for (int b = b_begin; b < b_end; ++b, ++blk_seq) {
      f = advance_frame(fs, f, b);
      const FrameDesc &fd = fs.fr[f];
      int x0, y0;
      block_origin(fd, b, G, x0, y0);
      const int degree = fd.degree;
      epi_bar_sync();
      if (f != coef_frame) {  // this frame's coefficients c[k][t], packed per stamp
        const int T = n_terms(degree);
        for (int i = et; i < N * 10; i += kEpiWarps * 32) {
          const int k = i / 10, t = i % 10;
          coef[i] = (t < T) ? fd.coeffs[(size_t)k * T + t] : 0.0f;
        }
        coef_frame = f;
      }
      if (fast)
        for (int e = et; e < G * 64; e += kEpiWarps * 32)
          *reinterpret_cast<float4 *>(alphaS + (size_t)e * 4) = make_float4(0.f, 0.f, 0.f, 0.f);
      epi_bar_sync();
      // alpha[g][k][i] = sum_j c[k][(i,j)] yt^j, so a_k(x, y0+g) = sum_i alpha[g][k][i] xt^i
      for (int e = et; e < G * N; e += kEpiWarps * 32) {
        const int g = e / N, k = e % N, y = y0 + g;
        const float yt = fd.H > 1 ? (2.0f * (float)y - (float)(fd.H - 1)) / (float)(fd.H - 1) : 0.0f;
        const float *ck = coef + k * 10;  // packed (i outer, j inner) for i + j <= degree
        const float y2 = yt * yt, y3 = y2 * yt;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (degree == 0) {
          a0 = ck[0];
        } else if (degree == 1) {
          a0 = ck[0] + ck[1] * yt;
          a1 = ck[2];
        } else if (degree == 2) {
          a0 = ck[0] + ck[1] * yt + ck[2] * y2;
          a1 = ck[3] + ck[4] * yt;
          a2 = ck[5];
        } else {
          a0 = ck[0] + ck[1] * yt + ck[2] * y2 + ck[3] * y3;
          a1 = ck[4] + ck[5] * yt + ck[6] * y2;
          a2 = ck[7] + ck[8] * yt;
          a3 = ck[9];
        }
        *reinterpret_cast<float4 *>(alpha + (size_t)e * 4) = make_float4(a0, a1, a2, a3);
        if (exact || quad) {  // the same coefficients at slot k (four-lane form: k + row offset)
          float *as = alphaS + (size_t)g * 256 + k + (quad ? quad_off(G, N, g) : 0);  // [g][power of xt][slot]
          as[0] = a0;
          as[64] = a1;
          as[128] = a2;
          as[192] = a3;
        } else if (fast) {
          // the same coefficients at the TMEM-load slot that carries column k
          // (load i covers columns min(16 i, N - 16) .. + 15; each column used once)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int st = min(16 * i, N - 16), slot = k - st;
            if (16 * i < N && slot >= 0 && slot < 16 && k >= 16 * i) {
              float *as = alphaS + (size_t)g * 256 + 16 * i + slot;  // [g][power of xt][slot]
              as[0] = a0;
              as[64] = a1;
              as[128] = a2;
              as[192] = a3;
            }
          }
        }
      }
      epi_bar_sync();
      const int buf = blk_seq & 1;
      const int x = x0 + m;
      const float xt = fd.W > 1 ? (2.0f * (float)x - (float)(fd.W - 1)) / (float)(fd.W - 1) : 0.0f;
      // I of this block was loaded during the previous block; start the next block's loads
      float ival[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) ival[j] = inext[j];
      if (b + 1 < b_end) load_I(b + 1, advance_frame(fs, f, b + 1), inext);
      // each thread times its own wait; the epilogue gives up only as a whole (the TMEM
      // loads are warp-aligned and the named barriers count all 256 threads)
      const bool ok = mbar_wait_bounded(&acc_full[buf], (blk_seq >> 1) & 1, status);
      if (epi_bar_any(!ok)) break;
      tc_fence_after();
      const uint32_t tbase = tmem_base + lane_off + (uint32_t)(buf * kAccStride);
#pragma unroll 1
      for (int j = 0;; ++j) {
        const int g = par + 2 * j;
        if (g >= G || y0 + g >= fd.y_end) break;
        // rows beyond the first three per warp (plans with G > 6) read I here
        const float iv = j == 0 ? ival[0] : j == 1 ? ival[1] : j == 2 ? ival[2]
                       : (fd.I && x < fd.W ? __ldg(fd.I + (size_t)(y0 + g) * fd.pitch_I + x) : 0.0f);
        const uint32_t c0 = tbase + (uint32_t)((G - 1 - g) * N);
        // sum_k a_k C_k = sum_i xt^i (sum_k alpha[g][k][i] C_k): four independent dot
        // products over the accumulator columns, then Horner in xt
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        if (quad) {
          // the row's columns from the 8-column boundary below c0, TMEM lanes 0..15 and
          // 16..31 of the quarter
          const float *ag = alphaS + (size_t)g * 256;
          const int off = quad_off(G, N, g), nrep = quad_reps(G, N, g);
          const uint32_t ca = c0 - (uint32_t)off;
          const bool in_range = SVK_CHECK((quad_col(G, N, g) - off) % 8 == 0 && quad_col(G, N, g) - off + 8 * nrep <= pl.nmma &&
                                              off + N <= 8 * nrep && nrep <= 8,
                                          status, 4);
          float sv[4];
          if (nrep == 8) {
            if (degree >= 3) quad_dots<4, 8>(ca, in_range, ag, lane & 3, sv);
            else quad_dots<3, 8>(ca, in_range, ag, lane & 3, sv);  // degree <= 2: no xt^3 term
          } else {
            if (degree >= 3) quad_dots<4, 7>(ca, in_range, ag, lane & 3, sv);
            else quad_dots<3, 7>(ca, in_range, ag, lane & 3, sv);
          }
          s0 = sv[0];
          s1 = sv[1];
          s2 = sv[2];
          s3 = sv[3];
        } else if (fast) {
          // 16 <= N <= 64, one wait for all loads.  Exact slots: columns 0..51.  Otherwise
          // four 16-column loads, the last one moved back to end at column N - 1, zeros at
          // its repeated slots.
          uint32_t v[64];
          if (exact) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
              if (SVK_CHECK((G - 1 - g) * N + 16 * i + 16 <= kAccStride, status, 4))
                tmem_ld16p(c0 + (uint32_t)(16 * i), &v[16 * i]);
            if (SVK_CHECK((G - 1 - g) * N + 52 <= kAccStride, status, 4)) tmem_ld4p(c0 + 48u, &v[48]);
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int st = 16 * i < N ? min(16 * i, N - 16) : 0;  // unused slots re-read chunk 0
              if (SVK_CHECK((G - 1 - g) * N + st + 16 <= kAccStride, status, 4)) tmem_ld16p(c0 + (uint32_t)st, &v[16 * i]);
            }
          }
          tmem_ld_wait();
          const float *ag = alphaS + (size_t)g * 256;
          float sv[4];
          if (exact) {
            if (degree >= 3) slot_dots<4, 13>(v, ag, sv);
            else slot_dots<3, 13>(v, ag, sv);  // degree <= 2: no xt^3 term
          } else {
            if (degree >= 3) slot_dots<4, 16>(v, ag, sv);
            else slot_dots<3, 16>(v, ag, sv);
          }
          s0 = sv[0];
          s1 = sv[1];
          s2 = sv[2];
          s3 = sv[3];
        } else {
          const float4 *a4 = reinterpret_cast<const float4 *>(alpha) + (size_t)g * N;
          const int nfull = N >> 4, tail = N & 15;
          for (int cc = 0; cc < nfull; ++cc) {
            uint32_t v[16];
            tmem_ld16(c0 + (uint32_t)(cc * 16), v);
            tmem_ld_wait();
            const float4 *ap = a4 + cc * 16;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float4 a = ap[e];
              const float cv = __uint_as_float(v[e]);
              s0 = fmaf(a.x, cv, s0);
              s1 = fmaf(a.y, cv, s1);
              s2 = fmaf(a.z, cv, s2);
              s3 = fmaf(a.w, cv, s3);
            }
          }
          for (int e = 0; e < tail; ++e) {  // the last N mod 16 columns, one per load
            const uint32_t u = tmem_ld1(c0 + (uint32_t)(nfull * 16 + e));
            const float4 a = a4[nfull * 16 + e];
            tmem_ld_wait();  // the loaded value is used only after the wait
            const float cv = __uint_as_float(u);
            s0 = fmaf(a.x, cv, s0);
            s1 = fmaf(a.y, cv, s1);
            s2 = fmaf(a.z, cv, s2);
            s3 = fmaf(a.w, cv, s3);
          }
        }
        const float sres = fmaf(fmaf(fmaf(s3, xt, s2), xt, s1), xt, s0);
        if (x < fd.W) fd.out[(size_t)(y0 + g) * fd.pitch_out + x] = sres * fd.out_scale - iv;
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

// ================================================================== host side
namespace {

std::mutex g_tune_mutex;
// (N, L, prec) -> (G, stages, streamed): plans set by the autotuner or svk_set_plan
std::map<std::tuple<int, int, int>, std::tuple<int, int, int>> g_tuned;

bool plan_for(int N, int L, int prec, Plan *pl) {
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(std::make_tuple(N, L, prec));
    if (it != g_tuned.end() &&
        make_plan(N, L, prec, std::get<0>(it->second), std::get<1>(it->second), std::get<2>(it->second), pl))
      return true;
  }
  return choose_plan(N, L, prec, pl);
}

void prec_scales(int prec, float &bscale, float &rscale) {
  bscale = 1.0f;
  rscale = 1.0f;
  if (prec == SVK_PREC_FP16X3 || prec == SVK_PREC_FP16X2) {
    bscale = 1024.0f;       // basis values are O(1e-3 .. 1)
    rscale = 1.0f / 16.0f;  // counts up to ~1e6 stay below 65504
  }
}

// Workspace of one launch over `n` frames that share a plan: one table pair per distinct
// basis pointer, then a status word.
size_t set_workspace(const svk_frame *fr, int n, const Plan &pl) {
  int distinct = 0;
  for (int i = 0; i < n; ++i) {
    bool seen = false;
    for (int j = 0; j < i; ++j) seen |= fr[j].basis == fr[i].basis;
    distinct += seen ? 0 : 1;
  }
  return (size_t)distinct * pl.table_bytes * 2 + 256;
}

template <int P>
int launch_set_prec(const svk_frame *fr, int n, const Plan &pl, unsigned char *ws, const int *rows, const int *held,
                    bool prep, cudaStream_t s) {
  static FrameSet fs;  // built on the host, passed by value as the kernel parameter
  static std::mutex fs_mutex;
  std::lock_guard<std::mutex> lock(fs_mutex);
  float bscale, rscale;
  prec_scales(P, bscale, rscale);
  fs.n = n;
  int blocks = 0, ntab = 0;
  const int nrow_items = pl.nKG * pl.nrows;
  for (int i = 0; i < n; ++i) {
    FrameDesc &d = fs.fr[i];
    d.R = fr[i].R;
    d.I = fr[i].I;
    d.out = fr[i].D;
    d.coeffs = fr[i].coeffs;
    d.W = fr[i].W;
    d.H = fr[i].H;
    d.pitch_R = fr[i].pitch_R;
    d.pitch_I = fr[i].pitch_I;
    d.pitch_out = fr[i].pitch_D;
    d.degree = fr[i].degree;
    d.y_begin = rows ? rows[2 * i] : 0;
    d.y_end = rows ? rows[2 * i + 1] : fr[i].H;
    d.r_begin = held ? held[2 * i] : 0;
    d.r_end = held ? held[2 * i + 1] : fr[i].H;
    d.nbx = (fr[i].W + kTileM - 1) / kTileM;
    d.block0 = blocks;
    blocks += d.nbx * ((d.y_end - d.y_begin + pl.G - 1) / pl.G);
    d.rscale = rscale;
    d.out_scale = 1.0f / (bscale * rscale);
    int same = -1;
    for (int j = 0; j < i; ++j)
      if (fr[j].basis == fr[i].basis) same = j;
    if (same >= 0) {
      d.tab_hi = fs.fr[same].tab_hi;
      d.tab_lo = fs.fr[same].tab_lo;
    } else {
      uint4 *th = reinterpret_cast<uint4 *>(ws + (size_t)ntab * pl.table_bytes * 2);
      uint4 *tl = reinterpret_cast<uint4 *>(ws + (size_t)ntab * pl.table_bytes * 2 + pl.table_bytes);
      if (prep) {
        const cudaError_t pe = launch_dependent(tc_prep_table<P>, (nrow_items + 255) / 256, 256, 0, s, fr[i].basis, pl,
                                                bscale, th, pl.tparts == 2 ? tl : nullptr);
        if (pe != cudaSuccess) return cuda_status(pe, "tc_prep_table launch");
      }
      d.tab_hi = th;
      d.tab_lo = tl;
      ++ntab;
    }
  }
  fs.nblocks = blocks;
  // the library's sticky status word (svk_device_status); the workspace word if it
  // cannot be resolved
  uint32_t *status = device_status_word();
  if (!status) status = reinterpret_cast<uint32_t *>(ws + (size_t)ntab * pl.table_bytes * 2);
  auto kern = pl.stream ? tc_basis_kernel<P, true> : tc_basis_kernel<P, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return cuda_status(e, "tc_basis_kernel smem attribute");
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = blocks < nsm ? blocks : nsm;
  if (grid > 0) return cuda_status(launch_dependent(kern, grid, kThreads, pl.smem, s, fs, pl, status), "tc_basis_kernel launch");
  return SVK_OK;
}

// rows: per frame the output rows [rows[2i], rows[2i+1]) (multiples of G apart from the
// frame's last row), or NULL for whole frames; held: per frame the rows of the frame its R
// buffer holds (R points at row held[2i]), or NULL for whole frames; prep = false reuses
// the basis tables an earlier launch with the same plan, basis and workspace prepared.
int launch_set(const svk_frame *fr, int n, int prec, const Plan &pl, void *ws, size_t ws_bytes, cudaStream_t s,
               const int *rows = nullptr, bool prep = true, const int *held = nullptr) {
  if (n < 1 || n > kMaxFrames) return set_error(SVK_ERR_ARG, "frame set of %d (1..%d)", n, kMaxFrames);
  if (!ws || ws_bytes < set_workspace(fr, n, pl)) return set_error(SVK_ERR_WORKSPACE, "tensor-core workspace too small");
  unsigned char *w = static_cast<unsigned char *>(ws);
  if (prec == SVK_PREC_BF16X3) return launch_set_prec<SVK_PREC_BF16X3>(fr, n, pl, w, rows, held, prep, s);
  if (prec == SVK_PREC_FP16X3) return launch_set_prec<SVK_PREC_FP16X3>(fr, n, pl, w, rows, held, prep, s);
  if (prec == SVK_PREC_FP16X2) return launch_set_prec<SVK_PREC_FP16X2>(fr, n, pl, w, rows, held, prep, s);
  return launch_set_prec<SVK_PREC_BF16>(fr, n, pl, w, rows, held, prep, s);
}

// Frames of a batch grouped by (N, L): launches of up to kMaxFrames frames each.
struct BatchPlan {
  std::vector<std::vector<int>> sets;
  std::vector<Plan> plans;
  size_t ws = 0;
};

int plan_batch(const svk_frame *fr, int n, int prec, BatchPlan *bp) {
  std::map<std::pair<int, int>, std::vector<int>> groups;
  std::vector<std::pair<int, int>> order;
  for (int i = 0; i < n; ++i) {
    const auto key = std::make_pair(fr[i].N, fr[i].L);
    if (!groups.count(key)) order.push_back(key);
    groups[key].push_back(i);
  }
  for (const auto &key : order) {
    Plan pl;
    if (!plan_for(key.first, key.second, prec, &pl))
      return set_error(SVK_ERR_UNSUPPORTED, "no tensor-core plan for N=%d L=%d", key.first, key.second);
    const auto &idx = groups[key];
    for (size_t o = 0; o < idx.size(); o += kMaxFrames) {
      std::vector<int> set(idx.begin() + o, idx.begin() + std::min(idx.size(), o + kMaxFrames));
      std::vector<svk_frame> tmp;
      for (int i : set) tmp.push_back(fr[i]);
      bp->ws += (set_workspace(tmp.data(), (int)tmp.size(), pl) + 255) & ~size_t(255);
      bp->sets.push_back(set);
      bp->plans.push_back(pl);
    }
  }
  return SVK_OK;
}

__global__ void tune_fill_kernel(float *p, size_t n, float base, float amp, uint32_t seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t x = (uint32_t)i * 2654435761u + seed;
    x ^= x >> 13;
    x *= 0x5bd1e995u;
    x ^= x >> 15;
    p[i] = base + amp * ((float)(x & 0xFFFFFF) / 16777216.0f - 0.5f);
  }
}

}  // namespace

size_t tc_workspace_size(int precision, int N, int L) {
  Plan pl;
  if (!plan_for(N, L, precision, &pl)) return 0;
  return pl.table_bytes * 2 + 256;
}

int launch_tc(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H, const float *basis, int N,
              int L, const float *coeffs, int degree, int precision, float *out, int pitch_out, void *ws,
              size_t ws_bytes, cudaStream_t s, int y_begin, int y_end, bool prep, int r_begin, int r_end) {
  Plan pl;
  if (!plan_for(N, L, precision, &pl))
    return set_error(SVK_ERR_UNSUPPORTED, "no tensor-core plan fits shared memory for N=%d L=%d", N, L);
  svk_frame f{};
  f.R = R;
  f.pitch_R = pitch_R;
  f.I = I;
  f.pitch_I = pitch_I;
  f.D = out;
  f.pitch_D = pitch_out;
  f.W = W;
  f.H = H;
  f.basis = basis;
  f.N = N;
  f.L = L;
  f.coeffs = coeffs;
  f.degree = degree;
  const int rows[2] = {y_begin, y_end < 0 ? H : y_end};
  const int held[2] = {r_begin, r_end < 0 ? H : r_end};
  return launch_set(&f, 1, precision, pl, ws, ws_bytes, s, rows, prep, held);
}

int tc_rows_per_block(int N, int L, int precision) {
  Plan pl;
  return plan_for(N, L, precision, &pl) ? pl.G : 0;
}

namespace {
// K_t = sum_k c[k][t] B_k (FP64 sums, stored FP32) and the T x T identity coefficients
// that make the epilogue's polynomial sum_t m_t C_t.  Blocks of 64 threads: each thread's
// sum is a chain of N dependent FP64 multiply-adds, so the outputs are spread over many
// SMs rather than sharing a few SMs' FP64 pipes.
__global__ void tform_combine_kernel(const float *__restrict__ basis, const float *__restrict__ coeffs, int N, int T,
                                     int LL, float *__restrict__ Kt, float *__restrict__ ident) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < T * LL) {
    const int t = idx / LL, i = idx % LL;
    double acc = 0.0;
    // eight stamps' loads in flight at a time (a plain loop waits for each load in turn);
    // the sum is taken in the same order
    for (int k0 = 0; k0 < N; k0 += 8) {
      float cv[8], bv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = k0 + j;
        cv[j] = k < N ? coeffs[(size_t)k * T + t] : 0.0f;
        bv[j] = k < N ? basis[(size_t)k * LL + i] : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (k0 + j < N) acc += (double)cv[j] * (double)bv[j];
    }
    Kt[idx] = (float)acc;
  }
  if (idx < T * T) ident[idx] = (idx / T == idx % T) ? 1.0f : 0.0f;
}

size_t tform_head_bytes(int T, int L) { return ((size_t)T * L * L * 4 + (size_t)T * T * 4 + 255) & ~size_t(255); }
}  // namespace

size_t tform_workspace_size(int precision, int L, int degree) {
  const int T = n_terms(degree);
  if (precision == SVK_PREC_FP32) return tform_head_bytes(T, L);  // K_t and identity; FFMA path
  Plan pl;
  if (!plan_for(T, L, precision, &pl)) return 0;
  return tform_head_bytes(T, L) + pl.table_bytes * 2 + 256;
}

int launch_tform(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H, const float *basis, int N,
                 int L, const float *coeffs, int degree, int precision, float *out, int pitch_out, void *ws,
                 size_t ws_bytes, cudaStream_t s, int y_begin, int y_end, bool prep, int r_begin, int r_end) {
  const int T = n_terms(degree);
  if (precision == SVK_PREC_FP32) {
    // FFMA pipe: the T convolutions R (x) K_t accumulated per pixel, combined with the
    // pixel's monomials in the epilogue
    const size_t head = tform_head_bytes(T, L);
    if (!ws || ws_bytes < head) return set_error(SVK_ERR_WORKSPACE, "T-form workspace too small");
    float *Kt = static_cast<float *>(ws);
    float *ident = Kt + (size_t)T * L * L;
    const int n = T * L * L > T * T ? T * L * L : T * T;
    if (prep) tform_combine_kernel<<<(n + 63) / 64, 64, 0, s>>>(basis, coeffs, N, T, L * L, Kt, ident);
    return launch_tform_fp32(R, pitch_R, I, pitch_I, W, H, Kt, T, L, out, pitch_out, s, y_begin,
                             y_end < 0 ? H : y_end, r_begin, r_end);
  }
  Plan pl;
  if (!plan_for(T, L, precision, &pl))
    return set_error(SVK_ERR_UNSUPPORTED, "no tensor-core plan for T=%d L=%d", T, L);
  const size_t head = tform_head_bytes(T, L);
  if (!ws || ws_bytes < head + pl.table_bytes * 2 + 256) return set_error(SVK_ERR_WORKSPACE, "T-form workspace too small");
  unsigned char *w = static_cast<unsigned char *>(ws);
  float *Kt = reinterpret_cast<float *>(w);
  float *ident = Kt + (size_t)T * L * L;
  const int n = T * L * L > T * T ? T * L * L : T * T;
  if (prep) tform_combine_kernel<<<(n + 63) / 64, 64, 0, s>>>(basis, coeffs, N, T, L * L, Kt, ident);
  svk_frame f{};
  f.R = R;
  f.pitch_R = pitch_R;
  f.I = I;
  f.pitch_I = pitch_I;
  f.D = out;
  f.pitch_D = pitch_out;
  f.W = W;
  f.H = H;
  f.basis = Kt;
  f.N = T;
  f.L = L;
  f.coeffs = ident;
  f.degree = degree;
  const int rows[2] = {y_begin, y_end < 0 ? H : y_end};
  const int held[2] = {r_begin, r_end < 0 ? H : r_end};
  return launch_set(&f, 1, precision, pl, w + head, ws_bytes - head, s, rows, prep, held);
}

size_t batch_workspace_size(const svk_frame *frames, int n, int precision) {
  BatchPlan bp;
  if (plan_batch(frames, n, precision, &bp) != SVK_OK) return 0;
  return bp.ws;
}

int launch_batch(const svk_frame *frames, int n, int precision, void *ws, size_t ws_bytes, cudaStream_t s) {
  BatchPlan bp;
  int st = plan_batch(frames, n, precision, &bp);
  if (st != SVK_OK) return st;
  if (!ws || ws_bytes < bp.ws) return set_error(SVK_ERR_WORKSPACE, "batch workspace of %zu bytes needed", bp.ws);
  unsigned char *w = static_cast<unsigned char *>(ws);
  size_t off = 0;
  for (size_t k = 0; k < bp.sets.size(); ++k) {
    std::vector<svk_frame> tmp;
    for (int i : bp.sets[k]) tmp.push_back(frames[i]);
    const size_t need = set_workspace(tmp.data(), (int)tmp.size(), bp.plans[k]);
    st = launch_set(tmp.data(), (int)tmp.size(), precision, bp.plans[k], w + off, need, s);
    if (st != SVK_OK) return st;
    off += (need + 255) & ~size_t(255);
  }
  return SVK_OK;
}

int autotune_tc(int N, int L, int degree, int precision, int W, int H, int *G_out, int *stages_out, cudaStream_t s) {
  const int T = n_terms(degree);
  const size_t px = (size_t)W * H;
  float *R = nullptr, *I = nullptr, *D = nullptr, *B = nullptr, *C = nullptr;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  for (int G = 1; G <= kMaxG; ++G)
    for (int NS = 4; NS <= kMaxStages; NS *= 2)
      for (int sm = 0; sm < 2; ++sm) {
        Plan pl;
        if (make_plan(N, L, precision, G, NS, sm, &pl) && pl.table_bytes * 2 + 256 > ws_bytes)
          ws_bytes = pl.table_bytes * 2 + 256;
      }
  if (ws_bytes == 0) return set_error(SVK_ERR_UNSUPPORTED, "no tensor-core plan for N=%d L=%d", N, L);
  cudaError_t e = cudaMallocAsync(&R, px * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&I, px * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&D, px * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&B, (size_t)N * L * L * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&C, (size_t)N * T * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&ws, ws_bytes, s);
  int st = cuda_status(e, "autotune buffers");
  float best = 1e30f;
  int bestG = 0, bestNS = 0, bestSM = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == SVK_OK) {
    tune_fill_kernel<<<256, 256, 0, s>>>(R, px, 1500.0f, 1000.0f, 1u);
    tune_fill_kernel<<<256, 256, 0, s>>>(I, px, 1500.0f, 1000.0f, 2u);
    tune_fill_kernel<<<64, 256, 0, s>>>(B, (size_t)N * L * L, 0.0f, 0.1f, 3u);
    tune_fill_kernel<<<8, 256, 0, s>>>(C, (size_t)N * T, 0.0f, 0.2f, 4u);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    svk_frame f{};
    f.R = R;
    f.pitch_R = W;
    f.I = I;
    f.pitch_I = W;
    f.D = D;
    f.pitch_D = W;
    f.W = W;
    f.H = H;
    f.basis = B;
    f.N = N;
    f.L = L;
    f.coeffs = C;
    f.degree = degree;
    for (int G = kMaxG; G >= 1 && st == SVK_OK; --G)
      for (int v = 0; v < 6 && st == SVK_OK; ++v) {  // resident 16, 8, 4 stages; streamed 16, 8
        const int sm = v >= 3, NS = sm ? kMaxStages >> (v - 3) : kMaxStages >> v;
        Plan pl;
        if (!make_plan(N, L, precision, G, NS, sm, &pl)) continue;
        st = launch_set(&f, 1, precision, pl, ws, ws_bytes, s);  // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && st == SVK_OK; ++r) st = launch_set(&f, 1, precision, pl, ws, ws_bytes, s);
        cudaEventRecord(e1, s);
        if (st == SVK_OK) st = cuda_status(cudaEventSynchronize(e1), "autotune timing");
        float ms = 0.0f;
        if (st == SVK_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (st == SVK_OK && ms < best) {
          best = ms;
          bestG = G;
          bestNS = NS;
          bestSM = sm;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  cudaFreeAsync(R, s);
  cudaFreeAsync(I, s);
  cudaFreeAsync(D, s);
  cudaFreeAsync(B, s);
  cudaFreeAsync(C, s);
  cudaFreeAsync(ws, s);
  if (st != SVK_OK) return st;
  if (bestG == 0) return set_error(SVK_ERR_UNSUPPORTED, "autotune found no plan");
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[std::make_tuple(N, L, precision)] = std::make_tuple(bestG, bestNS, bestSM);
  }
  if (G_out) *G_out = bestG;
  if (stages_out) *stages_out = bestNS;
  return SVK_OK;
}

int set_tc_plan(int N, int L, int precision, int G, int stages, int streamed) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  const auto key = std::make_tuple(N, L, precision);
  if (G == 0) {  // back to the default plan
    g_tuned.erase(key);
    return SVK_OK;
  }
  Plan pl;
  if (!make_plan(N, L, precision, G, stages, streamed, &pl))
    return set_error(SVK_ERR_UNSUPPORTED, "no tensor-core plan G=%d stages=%d streamed=%d for N=%d L=%d", G, stages,
                     streamed, N, L);
  g_tuned[key] = std::make_tuple(G, stages, streamed ? 1 : 0);
  return SVK_OK;
}

int get_tc_plan(int N, int L, int precision, int *G, int *stages, int *streamed) {
  Plan pl;
  if (!plan_for(N, L, precision, &pl)) return set_error(SVK_ERR_UNSUPPORTED, "no tensor-core plan for N=%d L=%d", N, L);
  if (G) *G = pl.G;
  if (stages) *stages = pl.NS;
  if (streamed) *streamed = pl.stream;
  return SVK_OK;
}

}  // namespace svk
