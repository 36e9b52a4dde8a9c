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
// Weights are used rounded to BF16 (the FP32 master copy is what Adam updates);
// activations and all accumulations are FP32.  Convolution is cross-correlation.
// Parameter order (flat FP32): per conv layer w[Cout][Cin][3][3], b[Cout]; then the
// linear layer w[n_out][32], b[n_out].
#include <cuda_bf16.h>

#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
namespace {

constexpr int kIn = 64, kCh = 32, kLayers = 4;
constexpr int kCin[kLayers] = {2, kCh, kCh, kCh};
constexpr int kStride[kLayers] = {2, 2, 2, 1};
constexpr int kHin[kLayers] = {kIn, kIn / 2, kIn / 4, kIn / 8};
constexpr int kHout[kLayers] = {32, 16, 8, 8};

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

struct Work {
  size_t wq, act[kLayers], da0, da1, pooled, dpooled, out, dout, total;  // float offsets
};

Work work_layout(int B, int n_out) {
  Work w;
  size_t o = 0;
  auto take = [&](size_t n) {
    const size_t at = o;
    o += (n + 63) & ~size_t(63);
    return at;
  };
  w.wq = take(param_layout(n_out).total);
  size_t maxact = 0;
  for (int i = 0; i < kLayers; ++i) {
    const size_t n = (size_t)B * kCh * kHout[i] * kHout[i];
    w.act[i] = take(n);
    maxact = n > maxact ? n : maxact;
  }
  w.da0 = take(maxact);
  w.da1 = take(maxact);
  w.pooled = take((size_t)B * kCh);
  w.dpooled = take((size_t)B * kCh);
  w.out = take((size_t)B * n_out);
  w.dout = take((size_t)B * n_out);
  w.total = o;
  return w;
}

__global__ void quantize_kernel(const float *__restrict__ p, float *__restrict__ q, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    q[i] = __bfloat162float(__float2bfloat16_rn(p[i]));
}

// out[b][o][y][x] = relu(bias[o] + sum_{c,dy,dx} w[o][c][dy][dx] in[b][c][s y+dy-1][s x+dx-1])
template <int CIN>
__global__ void conv_fwd_kernel(const float *__restrict__ in, const float *__restrict__ w, const float *__restrict__ bias,
                                float *__restrict__ out, int B, int Hin, int Hout, int stride) {
  __shared__ float ws[kCh * CIN * 9];
  for (int i = threadIdx.x; i < kCh * CIN * 9; i += blockDim.x) ws[i] = w[i];
  __syncthreads();
  const int n = B * kCh * Hout * Hout;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const int x = idx % Hout, y = (idx / Hout) % Hout, o = (idx / (Hout * Hout)) % kCh, b = idx / (kCh * Hout * Hout);
    float acc = bias[o];
    const float *ib = in + (size_t)b * CIN * Hin * Hin;
    for (int c = 0; c < CIN; ++c) {
      const float *ic = ib + (size_t)c * Hin * Hin;
      const float *wc = ws + (o * CIN + c) * 9;
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        const int yy = stride * y + dy - 1;
        if (yy < 0 || yy >= Hin) continue;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const int xx = stride * x + dx - 1;
          if (xx >= 0 && xx < Hin) acc = fmaf(wc[dy * 3 + dx], ic[yy * Hin + xx], acc);
        }
      }
    }
    out[idx] = fmaxf(acc, 0.0f);
  }
}

// dL/din (through this layer) given dL/dout and the layer's post-ReLU output:
// dz = dout * (out > 0); din[b][c][y][x] = sum_{o,dy,dx} w[o][c][dy][dx] dz[b][o][yo][xo]
// with s yo + dy - 1 = y, s xo + dx - 1 = x.
template <int CIN>
__global__ void conv_bwd_data_kernel(const float *__restrict__ dout, const float *__restrict__ act_out,
                                     const float *__restrict__ w, float *__restrict__ din, int B, int Hin, int Hout,
                                     int stride) {
  __shared__ float ws[kCh * CIN * 9];
  for (int i = threadIdx.x; i < kCh * CIN * 9; i += blockDim.x) ws[i] = w[i];
  __syncthreads();
  const int n = B * CIN * Hin * Hin;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const int x = idx % Hin, y = (idx / Hin) % Hin, c = (idx / (Hin * Hin)) % CIN, b = idx / (CIN * Hin * Hin);
    float acc = 0.0f;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
      const int ty = y + 1 - dy;
      if (ty < 0 || ty % stride) continue;
      const int yo = ty / stride;
      if (yo >= Hout) continue;
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int tx = x + 1 - dx;
        if (tx < 0 || tx % stride) continue;
        const int xo = tx / stride;
        if (xo >= Hout) continue;
        for (int o = 0; o < kCh; ++o) {
          const size_t oi = (((size_t)b * kCh + o) * Hout + yo) * Hout + xo;
          const float dz = act_out[oi] > 0.0f ? dout[oi] : 0.0f;
          acc = fmaf(ws[(o * CIN + c) * 9 + dy * 3 + dx], dz, acc);
        }
      }
    }
    din[idx] = acc;
  }
}

// dw[o][c][dy][dx] = sum_{b,y,x} dz[b][o][y][x] in[b][c][s y+dy-1][s x+dx-1]; one CTA per
// (o, c), and the c == 0 CTA also forms db[o] = sum dz.
__global__ void conv_bwd_weight_kernel(const float *__restrict__ dout, const float *__restrict__ act_out,
                                       const float *__restrict__ in, float *__restrict__ dw, float *__restrict__ db,
                                       int B, int Cin, int Hin, int Hout, int stride) {
  const int o = blockIdx.x / Cin, c = blockIdx.x % Cin;
  float acc[10];
#pragma unroll
  for (int t = 0; t < 10; ++t) acc[t] = 0.0f;
  const int npos = B * Hout * Hout;
  for (int p = threadIdx.x; p < npos; p += blockDim.x) {
    const int x = p % Hout, y = (p / Hout) % Hout, b = p / (Hout * Hout);
    const size_t oi = (((size_t)b * kCh + o) * Hout + y) * Hout + x;
    const float dz = act_out[oi] > 0.0f ? dout[oi] : 0.0f;
    if (dz == 0.0f) continue;
    const float *ic = in + ((size_t)b * Cin + c) * Hin * Hin;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
      const int yy = stride * y + dy - 1;
      if (yy < 0 || yy >= Hin) continue;
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int xx = stride * x + dx - 1;
        if (xx >= 0 && xx < Hin) acc[dy * 3 + dx] = fmaf(dz, ic[yy * Hin + xx], acc[dy * 3 + dx]);
      }
    }
    acc[9] += dz;
  }
  __shared__ float red[32][10];
#pragma unroll
  for (int t = 0; t < 10; ++t)
    for (int s = 16; s > 0; s >>= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], s);
  const int wi = threadIdx.x >> 5, li = threadIdx.x & 31;
  if (li == 0)
#pragma unroll
    for (int t = 0; t < 10; ++t) red[wi][t] = acc[t];
  __syncthreads();
  if (threadIdx.x < 10) {
    float s = 0.0f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i][threadIdx.x];
    if (threadIdx.x < 9) dw[((size_t)o * Cin + c) * 9 + threadIdx.x] = s;
    else if (c == 0) db[o] = s;
  }
}

// pooled[b][c] = mean over the 8x8 positions; out[b][j] = fcb[j] + sum_c fcw[j][c] pooled[b][c]
__global__ void pool_fc_kernel(const float *__restrict__ act, const float *__restrict__ fcw,
                               const float *__restrict__ fcb, float *__restrict__ pooled, float *__restrict__ out,
                               int n_out) {
  __shared__ float pl[kCh];
  const int b = blockIdx.x;
  if (threadIdx.x < kCh) {
    const float *a = act + ((size_t)b * kCh + threadIdx.x) * 64;
    float s = 0.0f;
    for (int i = 0; i < 64; ++i) s += a[i];
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

// linear layer gradients and dL/dpooled; then dL/dact4 = dpooled / 64 at every position
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

__global__ void unpool_kernel(const float *__restrict__ dpooled, float *__restrict__ da, int B) {
  const int n = B * kCh * 64;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    da[i] = dpooled[i / 64] * (1.0f / 64.0f);
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

template <int CIN>
void conv_fwd(const float *in, const float *w, const float *b, float *out, int B, int li, cudaStream_t s) {
  const size_t n = (size_t)B * kCh * kHout[li] * kHout[li];
  conv_fwd_kernel<CIN><<<grid_for(n), 256, 0, s>>>(in, w, b, out, B, kHin[li], kHout[li], kStride[li]);
}

// forward: x -> act[0..3] -> pooled -> out (weights already quantised into wq)
void forward(const float *x, const float *wq, const Layout &L, const Work &Wk, float *ws, int B, int n_out,
             cudaStream_t s) {
  const float *in = x;
  for (int li = 0; li < kLayers; ++li) {
    float *out = ws + Wk.act[li];
    if (li == 0) conv_fwd<2>(in, wq + L.w[li], wq + L.b[li], out, B, li, s);
    else conv_fwd<kCh>(in, wq + L.w[li], wq + L.b[li], out, B, li, s);
    in = out;
  }
  pool_fc_kernel<<<B, 64, 0, s>>>(ws + Wk.act[kLayers - 1], wq + L.fcw, wq + L.fcb, ws + Wk.pooled, ws + Wk.out, n_out);
}

int check_ws(void *ws, size_t ws_bytes, int B, int n_out) {
  if (!ws || ws_bytes < work_layout(B, n_out).total * sizeof(float))
    return set_error(SVK_ERR_WORKSPACE, "network workspace too small");
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
size_t cnn_workspace_size(int B, int n_out) { return work_layout(B, n_out).total * sizeof(float); }

int cnn_forward(const float *params, const float *x, int B, int n_out, float *out, void *ws_v, size_t ws_bytes,
                cudaStream_t s) {
  int st = check_ws(ws_v, ws_bytes, B, n_out);
  if (st != SVK_OK) return st;
  const Layout L = param_layout(n_out);
  const Work Wk = work_layout(B, n_out);
  float *ws = static_cast<float *>(ws_v);
  quantize_kernel<<<grid_for(L.total), 256, 0, s>>>(params, ws + Wk.wq, (int)L.total);
  forward(x, ws + Wk.wq, L, Wk, ws, B, n_out, s);
  cudaError_t e = cudaMemcpyAsync(out, ws + Wk.out, sizeof(float) * B * n_out, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_status(e, "network output copy");
  return cuda_status(cudaGetLastError(), "network forward");
}

int cnn_gradient(const float *params, const float *x, const float *target, int B, int n_out, float *grad, float *loss,
                 void *ws_v, size_t ws_bytes, cudaStream_t s) {
  int st = check_ws(ws_v, ws_bytes, B, n_out);
  if (st != SVK_OK) return st;
  const Layout L = param_layout(n_out);
  const Work Wk = work_layout(B, n_out);
  float *ws = static_cast<float *>(ws_v);
  const float *wq = ws + Wk.wq;
  quantize_kernel<<<grid_for(L.total), 256, 0, s>>>(params, ws + Wk.wq, (int)L.total);
  forward(x, wq, L, Wk, ws, B, n_out, s);
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), s);
  if (e != cudaSuccess) return cuda_status(e, "loss reset");
  const int n = B * n_out;
  mse_kernel<<<grid_for(n), 256, 0, s>>>(ws + Wk.out, target, ws + Wk.dout, loss, n);
  fc_bwd_kernel<<<grid_for((size_t)(n_out * kCh > B * kCh ? n_out * kCh : B * kCh)), 256, 0, s>>>(
      ws + Wk.dout, ws + Wk.pooled, wq + L.fcw, grad + L.fcw, grad + L.fcb, ws + Wk.dpooled, B, n_out);
  float *da = ws + Wk.da0, *dnext = ws + Wk.da1;
  unpool_kernel<<<grid_for((size_t)B * kCh * 64), 256, 0, s>>>(ws + Wk.dpooled, da, B);
  for (int li = kLayers - 1; li >= 0; --li) {
    const float *in = li == 0 ? x : ws + Wk.act[li - 1];
    const float *aout = ws + Wk.act[li];
    conv_bwd_weight_kernel<<<kCh * kCin[li], 256, 0, s>>>(da, aout, in, grad + L.w[li], grad + L.b[li], B, kCin[li],
                                                         kHin[li], kHout[li], kStride[li]);
    if (li > 0) {
      const size_t nin = (size_t)B * kCin[li] * kHin[li] * kHin[li];
      conv_bwd_data_kernel<kCh><<<grid_for(nin), 256, 0, s>>>(da, aout, wq + L.w[li], dnext, B, kHin[li], kHout[li],
                                                             kStride[li]);
      float *t = da;
      da = dnext;
      dnext = t;
    }
  }
  return cuda_status(cudaGetLastError(), "network gradient");
}

int cnn_adam(float *params, float *m, float *v, const float *grad, int n, int step, float lr, float b1, float b2,
             float eps, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  adam_kernel<<<grid_for(n), 256, 0, s>>>(params, m, v, grad, n, lr, b1, b2, eps, c1, c2);
  return cuda_status(cudaGetLastError(), "adam");
}

}  // namespace svk
