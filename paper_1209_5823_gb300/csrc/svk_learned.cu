// svk_learned.cu -- the data side of the coefficient network (row A9): stamps cut from
// images and normalised for its input, standardisation of its targets and outputs, the
// residual check that decides whether its coefficients are kept or handed to the FP64 fit,
// and the pieces of a training step that run on the device (batch draw, row gather, step
// bookkeeping), so a captured training step is library kernels only.  The training-step
// kernels are launched as programmatic dependents (launch_dependent), like the network's.
#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
namespace {

// out[s * stride + v * size + u] = (img(cx - size/2 + u, cy - size/2 + v) - offset) / divisor,
// img read as 0 outside the frame.  One thread per output value.
__global__ void cut_stamps_kernel(const float *__restrict__ img, int W, int H, int pitch, const int *__restrict__ xy,
                                  int n, int size, float offset, float divisor, float *__restrict__ out,
                                  long long stride) {
  const long long per = (long long)size * size;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= per * n) return;
  const int s = (int)(idx / per), p = (int)(idx % per);
  const int half = size / 2;
  const int x = xy[2 * s] - half + p % size, y = xy[2 * s + 1] - half + p / size;
  const float v = (x >= 0 && x < W && y >= 0 && y < H) ? __ldg(img + (size_t)y * pitch + x) : 0.0f;
  out[(size_t)s * stride + p] = __fdiv_rn(v - offset, divisor);
}

// Per stamp: sum over its pixels of (D - mean)^2 in FP64, the mean taken over the stamp
// (D read as 0 outside the frame).  One block per stamp; two passes over the stamp.
__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

__global__ void __launch_bounds__(256) stamp_residual_kernel(const float *__restrict__ D, int W, int H, int pitch,
                                                             const int *__restrict__ xy, int size,
                                                             double *__restrict__ part) {
  __shared__ double red[32];
  const int s = blockIdx.x, half = size / 2, per = size * size;
  const int x0 = xy[2 * s] - half, y0 = xy[2 * s + 1] - half;
  auto val = [&](int p) -> double {
    const int x = x0 + p % size, y = y0 + p / size;
    return (x >= 0 && x < W && y >= 0 && y < H) ? (double)D[(size_t)y * pitch + x] : 0.0;
  };
  double sum = 0.0;
  for (int p = threadIdx.x; p < per; p += blockDim.x) sum += val(p);
  const double mean = block_sum(sum, red) / (double)per;
  double sq = 0.0;
  for (int p = threadIdx.x; p < per; p += blockDim.x) {
    const double d = val(p) - mean;
    sq = fma(d, d, sq);
  }
  const double t = block_sum(sq, red);
  if (threadIdx.x == 0) part[s] = t;
}

// The stamps' sums in order, the noise floor and the decision (one block).
__global__ void __launch_bounds__(256) stamp_residual_final(const double *__restrict__ part, int n, int size,
                                                            const float *__restrict__ k0, int LL, double noise,
                                                            double ref_noise, double ratio, const int *field_info,
                                                            double *out, int *fallback) {
  __shared__ double red[32];
  // the stamps' sums in a fixed order: thread t adds stamps t, t + 256, ... then the block
  // reduction combines the threads in a fixed tree
  double a = 0.0;
  for (int s = threadIdx.x; s < n; s += blockDim.x) a += part[s];
  const double tot = block_sum(a, red);
  double k2 = 0.0;
  for (int i = threadIdx.x; i < LL; i += blockDim.x) k2 = fma((double)k0[i], (double)k0[i], k2);
  const double ksum = block_sum(k2, red);
  if (threadIdx.x == 0) {
    const double chi2 = tot / ((double)n * size * size);
    const double floor = noise * noise + ref_noise * ref_noise * ksum;
    out[0] = chi2;
    out[1] = floor;
    const bool failed = field_info && *field_info >= 0;
    *fallback = (failed || !(chi2 <= ratio * floor)) ? 1 : 0;
  }
}

// out[r][c] = (in[r][c] - mean[c]) / std[c], or mean[c] + std[c] * in[r][c] (inverse).
__global__ void standardise_kernel(const float *__restrict__ in, long long rows, int cols,
                                   const float *__restrict__ mean, const float *__restrict__ sd, int inverse,
                                   float *__restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int c = (int)(idx % cols);
  out[idx] = inverse ? fmaf(sd[c], in[idx], mean[c]) : __fdiv_rn(in[idx] - mean[c], sd[c]);
}

// SplitMix64 finaliser (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): a bijective mix of a 64-bit counter.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// idx[i] in [0, n) for draw (step, i): counter = seed + step * batch + i through
// SplitMix64, reduced to the range by a 32 x 32 -> 64-bit multiply of its high word.
__global__ void draw_batch_kernel(uint64_t seed, const int *__restrict__ step, int n, int batch,
                                  long long *__restrict__ idx) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  const uint64_t ctr = seed + (uint64_t)(uint32_t)(*step) * (uint64_t)batch + (uint64_t)i;
  const uint64_t r = splitmix64(ctr);
  idx[i] = (long long)(((r >> 32) * (uint64_t)(uint32_t)n) >> 32);
}

// dst row i = src row idx[i] (rows of `words` 32-bit words).
__global__ void gather_rows_kernel(const uint32_t *__restrict__ src, long long words, const long long *__restrict__ idx,
                                   int n, uint32_t *__restrict__ dst) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  const int r = blockIdx.y;
  if (r >= n) return;
  const uint32_t *s = src + (size_t)idx[r] * words;
  uint32_t *d = dst + (size_t)r * words;
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (long long)gridDim.x * blockDim.x)
    d[w] = s[w];
}

__global__ void step_end_kernel(const float *__restrict__ loss, int *__restrict__ step, float *__restrict__ hist,
                                int len) {
  dep_trigger();  // launched by launch_dependent: wait for the previous kernel first
  dep_wait();
  const int s = *step;
  hist[(unsigned)s % (unsigned)len] = *loss;
  *step = s + 1;
}

}  // namespace

int launch_cut_stamps(const float *img, int W, int H, int pitch, const int *xy, int n, int size, float offset,
                      float divisor, float *out, long long stride, cudaStream_t s) {
  const long long total = (long long)size * size * n;
  if (total == 0) return SVK_OK;
  cut_stamps_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(img, W, H, pitch, xy, n, size, offset, divisor,
                                                                     out, stride);
  return cuda_status(cudaGetLastError(), "cut_stamps_kernel launch");
}

size_t stamp_residual_workspace_size(int n) { return ((size_t)(n > 0 ? n : 1) * sizeof(double) + 255) & ~size_t(255); }

int launch_stamp_residual(const float *D, int W, int H, int pitch, const int *xy, int n, int size, const float *basis0,
                          int L, double noise, double ref_noise, double ratio, const int *field_info, double *out,
                          int *fallback, void *ws, size_t ws_bytes, cudaStream_t s) {
  if (!ws || ws_bytes < stamp_residual_workspace_size(n))
    return set_error(SVK_ERR_WORKSPACE, "stamp residual workspace too small");
  double *part = static_cast<double *>(ws);
  stamp_residual_kernel<<<n, 256, 0, s>>>(D, W, H, pitch, xy, size, part);
  stamp_residual_final<<<1, 256, 0, s>>>(part, n, size, basis0, L * L, noise, ref_noise, ratio, field_info, out,
                                         fallback);
  return cuda_status(cudaGetLastError(), "stamp residual launch");
}

int launch_standardise(const float *in, long long rows, int cols, const float *mean, const float *sd, int inverse,
                       float *out, cudaStream_t s) {
  const long long total = rows * cols;
  if (total == 0) return SVK_OK;
  standardise_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(in, rows, cols, mean, sd, inverse, out);
  return cuda_status(cudaGetLastError(), "standardise_kernel launch");
}

int launch_draw_batch(unsigned long long seed, const int *step, int n, int batch, long long *idx, cudaStream_t s) {
  return cuda_status(launch_dependent(draw_batch_kernel, (batch + 255) / 256, 256, 0, s, (uint64_t)seed, step, n, batch,
                                      idx),
                     "draw_batch_kernel launch");
}

int launch_gather_rows(const void *src, long long row_bytes, const long long *idx, int n, void *dst, cudaStream_t s) {
  const long long words = row_bytes / 4;
  const int bx = (int)((words + 255) / 256 < 64 ? (words + 255) / 256 : 64);
  return cuda_status(launch_dependent(gather_rows_kernel, dim3(bx, n), 256, 0, s, static_cast<const uint32_t *>(src),
                                      words, idx, n, static_cast<uint32_t *>(dst)),
                     "gather_rows_kernel launch");
}

int launch_step_end(const float *loss, int *step, float *hist, int len, cudaStream_t s) {
  return cuda_status(launch_dependent(step_end_kernel, 1, 1, 0, s, loss, step, hist, len), "step_end_kernel launch");
}

}  // namespace svk
