// svk_stamps.cu -- choice of the star stamps the least-squares fit runs over.
//
// Sec. 2 fits the coefficients over stamps around isolated stars and leaves the rule
// open.  The rule implemented here:
//   peak        R(p) - sky >= threshold and R(p) > R(q) for every in-frame 8-neighbour q
//   selectable  margin <= x <= W-1-margin (likewise y), R(p) < saturation, and no other
//               peak q with max(|dx|,|dy|) <= iso_radius has
//               R(q) - sky >= iso_frac * (R(p) - sky)
//   order       R(p) descending, then the row-major index y*W + x ascending.
// Differences and products are rounded to float32 one operation at a time (no
// contraction), so each decision is reproducible.
//
// Four steps on the stream, none of which needs the host to know a count:
//   1. peak_kernel     one thread per pixel: peak map (1 byte/pixel), selectable-position
//                      candidates appended to a list (order of arrival is irrelevant);
//   2. isolate_kernel  one warp per candidate: its lanes scan the window of the peak map
//                      and it appends a 64-bit sort key (inverted order-preserving bits of
//                      R(p), then the index) for each isolated one;
//   3. the keys, padded to the next power of two of their count read on the device, in
//      order: when at most kLocalSort stamps are wanted, a bitonic top-k -- chunks of
//      kLocalSort keys sorted in shared memory, then rounds that merge pairs of chunks
//      keeping the smaller half (one launch per round, log2 of the chunk capacity rounds);
//      otherwise a full bitonic sort.  The host launches the passes or rounds for the
//      largest possible count, and those beyond the actual count return at once;
//   4. output_kernel   the first max_stamps keys -> (x, y), and the counts.
// Capacity: two peaks are never 8-neighbours, so a frame holds at most
// ceil(W/2) * ceil(H/2) peaks; every buffer is sized for that.  The kernels are launched as
// programmatic dependents, so the sort's passes beyond the actual count, which return at
// once, cost little more than their launch.
#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
namespace {

constexpr int kLocalSort = 2048;  // keys sorted in shared memory by one block
constexpr int kGridStride = 152 * 8;

enum Counter { kSel = 0, kCand = 1, kPeaks = 2 };

struct SelectLayout {
  size_t off_pk, off_cnt, off_cand, off_keys, total;
  long long cap, cap_p2;
};

long long next_pow2(long long v) {
  long long p = 1;
  while (p < v) p <<= 1;
  return p;
}

SelectLayout select_layout(int W, int H) {
  SelectLayout l{};
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  l.cap = (long long)((W + 1) / 2) * ((H + 1) / 2);
  l.cap_p2 = next_pow2(l.cap < 2 ? 2 : l.cap);
  if (l.cap_p2 < kLocalSort) l.cap_p2 = kLocalSort;
  size_t o = 0;
  l.off_pk = o;
  o += up((size_t)W * H);
  l.off_cnt = o;
  o += 256;
  l.off_cand = o;
  o += up((size_t)l.cap * 4);
  l.off_keys = o;
  o += (size_t)l.cap_p2 * 8;
  l.total = o;
  return l;
}

__device__ __forceinline__ uint32_t dev_next_pow2(uint32_t v) {
  uint32_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

__global__ void peak_kernel(const float *__restrict__ R, int W, int H, int pitch, float sky, float thr, float sat,
                            int margin, unsigned char *__restrict__ pk, int *__restrict__ cand, int *cnt) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W) return;
  const float v = R[(size_t)y * pitch + x];
  bool peak = __fsub_rn(v, sky) >= thr;
  for (int dy = -1; dy <= 1 && peak; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      const int yy = y + dy, xx = x + dx;
      if ((dy || dx) && yy >= 0 && yy < H && xx >= 0 && xx < W && !(v > R[(size_t)yy * pitch + xx])) peak = false;
    }
  pk[(size_t)y * W + x] = peak ? 1 : 0;
  if (!peak) return;
  atomicAdd(&cnt[kPeaks], 1);
  if (x >= margin && x <= W - 1 - margin && y >= margin && y <= H - 1 - margin && v < sat)
    cand[atomicAdd(&cnt[kCand], 1)] = y * W + x;
}

__device__ __forceinline__ unsigned long long sort_key(float v, uint32_t idx) {
  uint32_t u = __float_as_uint(v);
  if (u == 0x80000000u) u = 0;                      // -0 ranks with +0
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // ascending in v
  return ((unsigned long long)(~u) << 32) | idx;    // descending v, then ascending index
}

__global__ void isolate_kernel(const float *__restrict__ R, int W, int H, int pitch, float sky, float frac, int rad,
                               const unsigned char *__restrict__ pk, const int *__restrict__ cand, int *cnt,
                               unsigned long long *__restrict__ keys) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  const int n = cnt[kCand];
  const int lane = threadIdx.x & 31;
  // one warp per candidate: the lanes take the window's pixels in row-major order (runs of
  // a row are consecutive bytes of the peak map), the warp stops at the first hit
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
    const int idx = cand[i], y = idx / W, x = idx % W;
    const float v = R[(size_t)y * pitch + x];
    const float bar = __fmul_rn(frac, __fsub_rn(v, sky));
    const int y0 = max(0, y - rad), y1 = min(H - 1, y + rad), x0 = max(0, x - rad), x1 = min(W - 1, x + rad);
    const int wx = x1 - x0 + 1, total = (y1 - y0 + 1) * wx;
    bool hit = false;
    for (int e0 = 0; e0 < total; e0 += 32) {
      const int e = e0 + lane;
      if (e < total) {
        const int yy = y0 + e / wx, xx = x0 + e % wx;
        hit = pk[(size_t)yy * W + xx] && (yy != y || xx != x) && __fsub_rn(R[(size_t)yy * pitch + xx], sky) >= bar;
      }
      if (__any_sync(0xffffffffu, hit)) break;
    }
    const bool any_hit = __any_sync(0xffffffffu, hit);  // every lane votes
    if (lane == 0 && !any_hit) keys[atomicAdd(&cnt[kSel], 1)] = sort_key(v, (uint32_t)idx);
    __syncwarp();
  }
}

__global__ void pad_kernel(unsigned long long *keys, const int *cnt) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  const uint32_t n = (uint32_t)cnt[kSel], np2 = dev_next_pow2(n);
  for (uint32_t i = n + blockIdx.x * blockDim.x + threadIdx.x; i < np2; i += gridDim.x * blockDim.x) keys[i] = ~0ull;
}

// One compare-exchange stage (k, j) of the bitonic network over the padded keys.
__global__ void bitonic_global(unsigned long long *keys, const int *cnt, uint32_t k, uint32_t j) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  const uint32_t np2 = dev_next_pow2((uint32_t)cnt[kSel]);
  if (k > np2) return;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np2; i += gridDim.x * blockDim.x) {
    const uint32_t l = i ^ j;
    if (l <= i) continue;
    const unsigned long long a = keys[i], b = keys[l];
    const bool up = (i & k) == 0;
    if ((a > b) == up) {
      keys[i] = b;
      keys[l] = a;
    }
  }
}

// Stages k = k_lo .. k_hi (doubling) with j < kLocalSort, in shared memory: each block
// holds one kLocalSort-key segment (pairs (i, i ^ j) never leave it for j < kLocalSort).
// chunk_dir: every segment ascending (directions from the index within the segment; the
// top-k path), else the directions of the whole-array network.
__global__ void __launch_bounds__(kLocalSort / 2) bitonic_local(unsigned long long *keys, const int *cnt,
                                                                uint32_t k_lo, uint32_t k_hi, int chunk_dir) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  __shared__ unsigned long long s[kLocalSort];
  const uint32_t np2 = dev_next_pow2((uint32_t)cnt[kSel]);
  const uint32_t base = blockIdx.x * kLocalSort;
  if (k_lo > np2 || base >= np2) return;
  const uint32_t len = np2 - base < (uint32_t)kLocalSort ? np2 - base : (uint32_t)kLocalSort;
  for (uint32_t t = threadIdx.x; t < len; t += blockDim.x) s[t] = keys[base + t];
  __syncthreads();
  for (uint32_t k = k_lo; k <= k_hi && k <= np2; k <<= 1)
    for (uint32_t j = (k >> 1) < (uint32_t)(kLocalSort / 2) ? (k >> 1) : (uint32_t)(kLocalSort / 2); j > 0; j >>= 1) {
      for (uint32_t t = threadIdx.x; t < len; t += blockDim.x) {
        const uint32_t l = t ^ j;
        if (l > t && l < len) {
          const unsigned long long a = s[t], b = s[l];
          const bool up = ((chunk_dir ? t : base + t) & k) == 0;
          if ((a > b) == up) {
            s[t] = b;
            s[l] = a;
          }
        }
      }
      __syncthreads();
    }
  for (uint32_t t = threadIdx.x; t < len; t += blockDim.x) keys[base + t] = s[t];
}

// Round r of the top-k: block b merges the ascending chunks c = b 2^r and c + 2^(r-1) (in
// chunks of kLocalSort keys).  C_i = min(A_i, B_{m-1-i}) are the m smallest keys of the two
// and form a bitonic sequence (the first stage of Batcher's bitonic merge of A with B
// reversed); the rest of that merge sorts them ascending into chunk c.  A chunk without a
// partner (or beyond the padded count) stays as it is.
__global__ void __launch_bounds__(kLocalSort / 2) topk_merge(unsigned long long *keys, const int *cnt, uint32_t r) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  __shared__ unsigned long long s[kLocalSort];
  const uint32_t np2 = dev_next_pow2((uint32_t)cnt[kSel]);
  const uint32_t nch = np2 <= (uint32_t)kLocalSort ? 1u : np2 / kLocalSort;
  const uint32_t c = blockIdx.x << r, pc = c + (1u << (r - 1));
  if (pc >= nch) return;
  unsigned long long *A = keys + (size_t)c * kLocalSort;
  const unsigned long long *Bc = keys + (size_t)pc * kLocalSort;
  for (uint32_t t = threadIdx.x; t < (uint32_t)kLocalSort; t += blockDim.x) {
    const unsigned long long a = A[t], b = Bc[kLocalSort - 1 - t];
    s[t] = a < b ? a : b;
  }
  __syncthreads();
  for (uint32_t j = kLocalSort / 2; j > 0; j >>= 1) {
    for (uint32_t t = threadIdx.x; t < (uint32_t)kLocalSort; t += blockDim.x) {
      const uint32_t l = t ^ j;
      if (l > t) {
        const unsigned long long a = s[t], b = s[l];
        if (a > b) {
          s[t] = b;
          s[l] = a;
        }
      }
    }
    __syncthreads();
  }
  for (uint32_t t = threadIdx.x; t < (uint32_t)kLocalSort; t += blockDim.x) A[t] = s[t];
}

__global__ void output_kernel(const unsigned long long *keys, const int *cnt, int W, int max_stamps, int *xy,
                              int *counts) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  const int n = min(cnt[kSel], max_stamps);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t idx = (uint32_t)(keys[i] & 0xFFFFFFFFull);
    xy[2 * i] = (int)(idx % (uint32_t)W);
    xy[2 * i + 1] = (int)(idx / (uint32_t)W);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    counts[0] = n;
    counts[1] = cnt[kPeaks];
  }
}

}  // namespace

size_t select_workspace_size(int W, int H) { return select_layout(W, H).total; }

int launch_select(const float *R, int W, int H, int pitch, float sky, float threshold, float saturation, int margin,
                  int iso_radius, float iso_frac, int max_stamps, int *xy, int *counts, void *ws, size_t ws_bytes,
                  cudaStream_t s) {
  const SelectLayout l = select_layout(W, H);
  if (ws_bytes < l.total) return set_error(SVK_ERR_WORKSPACE, "stamp-selection workspace too small");
  unsigned char *w = static_cast<unsigned char *>(ws);
  unsigned char *pk = w + l.off_pk;
  int *cnt = reinterpret_cast<int *>(w + l.off_cnt);
  int *cand = reinterpret_cast<int *>(w + l.off_cand);
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(w + l.off_keys);
  int st = cuda_status(cudaMemsetAsync(cnt, 0, 16, s), "clear counters");
  if (st != SVK_OK) return st;
  cudaError_t e = launch_dependent(peak_kernel, dim3((W + 255) / 256, H), 256, 0, s, R, W, H, pitch, sky, threshold,
                                   saturation, margin, pk, cand, cnt);
  if (e == cudaSuccess)
    e = launch_dependent(isolate_kernel, kGridStride, 256, 0, s, R, W, H, pitch, sky, iso_frac, iso_radius, pk, cand,
                         cnt, keys);
  if (e == cudaSuccess) e = launch_dependent(pad_kernel, kGridStride, 256, 0, s, keys, cnt);
  const uint32_t P = (uint32_t)l.cap_p2, nloc = P / kLocalSort;
  if (max_stamps <= kLocalSort) {  // top-k: log2(nloc) merge rounds instead of the full network
    if (e == cudaSuccess)
      e = launch_dependent(bitonic_local, nloc, kLocalSort / 2, 0, s, keys, cnt, 2u, (uint32_t)kLocalSort, 1);
    for (uint32_t r = 1; (nloc >> r) >= 1 && e == cudaSuccess; ++r)
      e = launch_dependent(topk_merge, nloc >> r, kLocalSort / 2, 0, s, keys, (const int *)cnt, r);
  } else {
    if (e == cudaSuccess)
      e = launch_dependent(bitonic_local, nloc, kLocalSort / 2, 0, s, keys, cnt, 2u, (uint32_t)kLocalSort, 0);
    for (uint32_t k = 2 * kLocalSort; k <= P && e == cudaSuccess; k <<= 1) {
      for (uint32_t j = k >> 1; j >= (uint32_t)kLocalSort && e == cudaSuccess; j >>= 1)
        e = launch_dependent(bitonic_global, kGridStride, 256, 0, s, keys, cnt, k, j);
      if (e == cudaSuccess) e = launch_dependent(bitonic_local, nloc, kLocalSort / 2, 0, s, keys, cnt, k, k, 0);
    }
  }
  if (e == cudaSuccess)
    e = launch_dependent(output_kernel, kGridStride / 8, 256, 0, s, keys, (const int *)cnt, W, max_stamps, xy, counts);
  return cuda_status(e, "stamp selection launch");
}

}  // namespace svk
