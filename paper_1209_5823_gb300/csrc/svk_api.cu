// svk_api.cu -- the C ABI entry points declared in include/svk.h: argument checks on the
// host, workspace handling and dispatch to the kernels of the other translation units.
#include <cudaTypedefs.h>
#include <cmath>
#include <mutex>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {

static thread_local char g_err[512] = "";

int set_error(int status, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return status;
}

int cuda_status(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return SVK_OK;
  return set_error(SVK_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

const char *last_error() { return g_err; }

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool encode_tmap_2d_f32(CUtensorMap *map, const float *base, int W, int H, int pitch, int box_w,
                        int box_h) {
  auto fn = encode_fn();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0 || ((size_t)pitch * 4) % 16 != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
  cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool encode_tmap_nhwc32_bf16(CUtensorMap *map, const void *base, int S, int B, int box_x, int box_y, int box_b,
                             int estride) {
  auto fn = encode_fn();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
  cuuint64_t dims[4] = {32, (cuuint64_t)S, (cuuint64_t)S, (cuuint64_t)B};
  cuuint64_t strides[3] = {64, (cuuint64_t)S * 64, (cuuint64_t)S * S * 64};
  cuuint32_t box[4] = {32, (cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)box_b};
  cuuint32_t estr[4] = {1, (cuuint32_t)estride, (cuuint32_t)estride, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool encode_tmap_stamps_f32(CUtensorMap *map, const float *base, int S, int C, int B, int box_y) {
  auto fn = encode_fn();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0 || (S * 4) % 16 != 0) return false;
  cuuint64_t dims[4] = {(cuuint64_t)S, (cuuint64_t)S, (cuuint64_t)C, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)S * 4, (cuuint64_t)S * S * 4, (cuuint64_t)C * S * S * 4};
  cuuint32_t box[4] = {(cuuint32_t)S, (cuuint32_t)box_y, (cuuint32_t)C, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int ScopedWorkspace::acquire(size_t bytes, void *user_ws, size_t user_bytes, cudaStream_t s) {
  if (bytes == 0) return SVK_OK;
  if (user_ws) {
    if (user_bytes < bytes)
      return set_error(SVK_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", user_bytes, bytes);
    ptr = user_ws;
    return SVK_OK;
  }
  if (user_bytes != 0) return set_error(SVK_ERR_ARG, "ws_bytes > 0 with a NULL workspace");
  stream = s;
  cudaError_t e = cudaMallocAsync(&ptr, bytes, s);
  if (e != cudaSuccess) {
    ptr = nullptr;
    return cuda_status(e, "cudaMallocAsync(workspace)");
  }
  owned = true;
  return SVK_OK;
}

ScopedWorkspace::~ScopedWorkspace() {
  if (owned && ptr) cudaFreeAsync(ptr, stream);
}

// The driver's id of the calling thread's current context, or 0 when there is none or it
// cannot be read.  Ids are unique for the life of the process: a context destroyed (by
// cudaDeviceReset, for instance) and created again gets a new id even where the driver
// hands out the same handle.
unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int symbol_address(SymbolAddressCache &cache, const void *symbol, const char *what, void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= SymbolAddressCache::kMaxDevices)
    return set_error(SVK_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, SymbolAddressCache::kMaxDevices);
  std::lock_guard<std::mutex> lock(cache.mu);
  const unsigned long long id = current_context_id();
  if (!cache.addr[dev] || id == 0 || id != cache.ctx[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, symbol);  // creates the device's context if there is none yet
    if (e != cudaSuccess) return cuda_status(e, what);
    cache.addr[dev] = p;
    cache.ctx[dev] = current_context_id();
  }
  *out = cache.addr[dev];
  return SVK_OK;
}

// Sticky device status word: the library's bounded device waits record a timeout here
// (kernels get its address as their status pointer); svk_device_status reads and clears it.
__device__ uint32_t g_device_status;

uint32_t *device_status_word() {
  static SymbolAddressCache cache;
  void *p = nullptr;
  if (symbol_address(cache, reinterpret_cast<const void *>(&g_device_status), "cudaGetSymbolAddress(status word)",
                     &p) != SVK_OK)
    return nullptr;
  return static_cast<uint32_t *>(p);
}

}  // namespace svk

using namespace svk;

// An NVTX range named after the entry point around each call that queues GPU work, so a
// timeline tool shows the library's calls (the calls cost nothing without a tool).
namespace {
struct CallRange {
  explicit CallRange(const char *name) { nvtxRangePushA(name); }
  ~CallRange() { nvtxRangePop(); }
};
}  // namespace

static int check_conv_args(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H,
                           const float *basis, int N, int L, const float *coeffs, int degree,
                           int method, int precision, int edge, const float *out, int pitch_out,
                           bool need_I) {
  if (!R || !basis || !coeffs || !out || (need_I && !I))
    return set_error(SVK_ERR_ARG, "NULL image, basis, coefficient or output pointer");
  if (W < 1 || H < 1 || W > 65535 || H > 65535) return set_error(SVK_ERR_ARG, "bad frame size %dx%d", W, H);
  if (pitch_R < W || pitch_out < W || (need_I && pitch_I < W))
    return set_error(SVK_ERR_ARG, "pitch smaller than W");
  if (L < 1 || L > 31 || (L % 2) == 0) return set_error(SVK_ERR_ARG, "kernel size L=%d must be odd in [1,31]", L);
  if (N < 1 || N > 4096) return set_error(SVK_ERR_ARG, "N=%d out of range", N);
  if (degree < 0 || degree > 3) return set_error(SVK_ERR_ARG, "degree=%d out of range [0,3]", degree);
  if (edge != SVK_EDGE_ZERO) return set_error(SVK_ERR_ARG, "unknown edge mode %d", edge);
  if (method == SVK_METHOD_DIRECT) {
    if (precision != SVK_PREC_FP32)
      return set_error(SVK_ERR_UNSUPPORTED, "the direct method computes in FP32 only");
  } else if (method == SVK_METHOD_BASIS || method == SVK_METHOD_TFORM) {
    const bool tc = precision == SVK_PREC_BF16X3 || precision == SVK_PREC_FP16X3 || precision == SVK_PREC_BF16 ||
                    (precision == SVK_PREC_FP16X2 && method == SVK_METHOD_BASIS);
    if (!tc && !(method == SVK_METHOD_TFORM && precision == SVK_PREC_FP32))
      return set_error(SVK_ERR_UNSUPPORTED, "precision %d not built for method %d", precision, method);
    if (method == SVK_METHOD_BASIS && N > 256)
      return set_error(SVK_ERR_UNSUPPORTED, "basis method supports N <= 256 (got %d)", N);
  } else {
    return set_error(SVK_ERR_ARG, "unknown method %d", method);
  }
  return SVK_OK;
}

static int run_conv(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H,
                    const float *basis, int N, int L, const float *coeffs, int degree, int method,
                    int precision, int edge, float *out, int pitch_out, void *ws, size_t ws_bytes,
                    void *stream, bool need_I) {
  int st = check_conv_args(R, pitch_R, I, pitch_I, W, H, basis, N, L, coeffs, degree, method, precision,
                           edge, out, pitch_out, need_I);
  if (st != SVK_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (method == SVK_METHOD_DIRECT)
    return launch_direct(R, pitch_R, need_I ? I : nullptr, pitch_I, W, H, basis, N, L, coeffs, degree, out,
                         pitch_out, s);
  ScopedWorkspace w;
  if (method == SVK_METHOD_TFORM) {
    const size_t need = tform_workspace_size(precision, L, degree);
    st = w.acquire(need, ws, ws_bytes, s);
    if (st != SVK_OK) return st;
    return launch_tform(R, pitch_R, need_I ? I : nullptr, pitch_I, W, H, basis, N, L, coeffs, degree, precision, out,
                        pitch_out, w.ptr, need, s);
  }
  st = w.acquire(tc_workspace_size(precision, N, L), ws, ws_bytes, s);
  if (st != SVK_OK) return st;
  return launch_tc(R, pitch_R, need_I ? I : nullptr, pitch_I, W, H, basis, N, L, coeffs, degree, precision,
                   out, pitch_out, w.ptr, tc_workspace_size(precision, N, L), s);
}

extern "C" {

const char *svk_last_error(void) { return svk::last_error(); }

int svk_version(void) { return SVK_VERSION; }

int svk_gauss_basis_count(int n_gauss, const int *deg) {
  if (n_gauss < 1 || !deg) return -1;
  int n = 0;
  for (int g = 0; g < n_gauss; ++g) {
    if (deg[g] < 0 || deg[g] > 10) return -1;
    n += (deg[g] + 1) * (deg[g] + 2) / 2;
  }
  return n;
}

int svk_round_basis_fp16(float *basis, long long n, void *stream) {
  CallRange range("svk_round_basis_fp16");
  if (n < 0 || (n > 0 && !basis)) return set_error(SVK_ERR_ARG, "bad basis rounding arguments");
  return launch_round_basis_fp16(basis, n, static_cast<cudaStream_t>(stream));
}

int svk_build_basis(int kind, int L, int n_gauss, const double *sigma, const int *deg, int normalize,
                    float *basis_out, int *n_basis_out, void *stream) {
  CallRange range("svk_build_basis");
  if (!basis_out) return set_error(SVK_ERR_ARG, "NULL basis_out");
  if (L < 1 || L > 63 || (L % 2) == 0) return set_error(SVK_ERR_ARG, "L=%d must be odd in [1,63]", L);
  if (normalize != SVK_NORM_NONE && normalize != SVK_NORM_ALARD)
    return set_error(SVK_ERR_ARG, "unknown normalisation %d", normalize);
  int N;
  if (kind == SVK_BASIS_GAUSS) {
    if (n_gauss < 1 || n_gauss > 16 || !sigma || !deg) return set_error(SVK_ERR_ARG, "bad Gaussian list");
    for (int g = 0; g < n_gauss; ++g)
      if (!(sigma[g] > 0.0) || deg[g] < 0 || deg[g] > 10) return set_error(SVK_ERR_ARG, "bad sigma/deg[%d]", g);
    N = svk_gauss_basis_count(n_gauss, deg);
  } else if (kind == SVK_BASIS_DELTA) {
    N = L * L;
  } else {
    return set_error(SVK_ERR_ARG, "unknown basis kind %d", kind);
  }
  if (n_basis_out) *n_basis_out = N;
  return launch_build_basis(kind, L, n_gauss, sigma, deg, normalize, basis_out, N,
                            static_cast<cudaStream_t>(stream));
}

size_t svk_workspace_size(int method, int precision, int W, int H, int N, int L, int degree) {
  (void)W;
  (void)H;
  (void)degree;
  if (method == SVK_METHOD_BASIS) return tc_workspace_size(precision, N, L);
  if (method == SVK_METHOD_TFORM) return tform_workspace_size(precision, L, degree);
  return 0;
}

int svk_convolve(const float *R, int W, int H, int pitch_R, const float *basis, int N, int L,
                 const float *coeffs, int degree, int method, int precision, int edge, float *out,
                 int pitch_out, void *workspace, size_t ws_bytes, void *stream) {
  CallRange range("svk_convolve");
  return run_conv(R, pitch_R, nullptr, 0, W, H, basis, N, L, coeffs, degree, method, precision, edge, out,
                  pitch_out, workspace, ws_bytes, stream, false);
}

int svk_difference(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H,
                   const float *basis, int N, int L, const float *coeffs, int degree, int method,
                   int precision, int edge, float *D, int pitch_D, void *workspace, size_t ws_bytes,
                   void *stream) {
  CallRange range("svk_difference");
  return run_conv(R, pitch_R, I, pitch_I, W, H, basis, N, L, coeffs, degree, method, precision, edge, D,
                  pitch_D, workspace, ws_bytes, stream, true);
}

static int check_batch(const svk_frame *frames, int n_frames, int precision) {
  if (!frames || n_frames < 1) return set_error(SVK_ERR_ARG, "empty frame list");
  for (int i = 0; i < n_frames; ++i) {
    const svk_frame &f = frames[i];
    const int st = check_conv_args(f.R, f.pitch_R, f.I, f.I ? f.pitch_I : f.W, f.W, f.H, f.basis, f.N, f.L, f.coeffs,
                                   f.degree, SVK_METHOD_BASIS, precision, SVK_EDGE_ZERO, f.D, f.pitch_D, false);
    if (st != SVK_OK) {
      char msg[512];
      snprintf(msg, sizeof(msg), "%s", svk::last_error());
      return set_error(st, "frame %d: %s", i, msg);
    }
  }
  return SVK_OK;
}

size_t svk_batch_workspace_size(const svk_frame *frames, int n_frames, int precision) {
  if (check_batch(frames, n_frames, precision) != SVK_OK) return 0;
  return batch_workspace_size(frames, n_frames, precision);
}

int svk_difference_batch(const svk_frame *frames, int n_frames, int precision, void *workspace, size_t ws_bytes,
                         void *stream) {
  CallRange range("svk_difference_batch");
  int st = check_batch(frames, n_frames, precision);
  if (st != SVK_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScopedWorkspace w;
  const size_t need = batch_workspace_size(frames, n_frames, precision);
  st = w.acquire(need, workspace, ws_bytes, s);
  if (st != SVK_OK) return st;
  return launch_batch(frames, n_frames, precision, w.ptr, need, s);
}

int svk_autotune(int N, int L, int degree, int precision, int W, int H, int *G_out, int *stages_out, void *stream) {
  CallRange range("svk_autotune");
  if (precision != SVK_PREC_BF16X3 && precision != SVK_PREC_FP16X3 && precision != SVK_PREC_BF16 &&
      precision != SVK_PREC_FP16X2)
    return set_error(SVK_ERR_UNSUPPORTED, "autotune covers the tensor-core precisions only");
  if (N < 1 || N > 256 || L < 1 || L > 31 || (L % 2) == 0 || degree < 0 || degree > 3 || W < 1 || H < 1 ||
      W > 65535 || H > 65535)
    return set_error(SVK_ERR_ARG, "bad autotune problem");
  return autotune_tc(N, L, degree, precision, W, H, G_out, stages_out, static_cast<cudaStream_t>(stream));
}

static bool tc_plan_args(int N, int L, int precision) {
  return (precision == SVK_PREC_BF16X3 || precision == SVK_PREC_FP16X3 || precision == SVK_PREC_BF16 ||
          precision == SVK_PREC_FP16X2) && N >= 1 &&
         N <= 256 && L >= 1 && L <= 31 && (L % 2) == 1;
}

int svk_tc_plan(int N, int L, int precision, int *G, int *stages, int *streamed) {
  if (!tc_plan_args(N, L, precision)) return set_error(SVK_ERR_ARG, "bad tensor-core plan query");
  return get_tc_plan(N, L, precision, G, stages, streamed);
}

int svk_set_plan(int N, int L, int precision, int G, int stages, int streamed) {
  if (!tc_plan_args(N, L, precision) || G < 0) return set_error(SVK_ERR_ARG, "bad tensor-core plan");
  return set_tc_plan(N, L, precision, G, stages, streamed);
}

int svk_cnn_param_count(int n_out) { return (n_out < 1 || n_out > 256) ? -1 : cnn_param_count(n_out); }

size_t svk_cnn_workspace_size(int batch, int n_out) {
  if (batch < 1 || batch > 4096 || n_out < 1 || n_out > 256) return 0;
  return cnn_workspace_size(batch, n_out);
}

static int check_cnn(const void *params, const void *x, int batch, int n_out) {
  if (!params || !x) return set_error(SVK_ERR_ARG, "NULL network parameter or input pointer");
  if (batch < 1 || batch > 4096 || n_out < 1 || n_out > 256)
    return set_error(SVK_ERR_ARG, "batch %d / n_out %d out of range", batch, n_out);
  return SVK_OK;
}

int svk_cnn_forward(const float *params, const float *x, int batch, int n_out, float *out, void *workspace,
                    size_t ws_bytes, void *stream) {
  CallRange range("svk_cnn_forward");
  int st = check_cnn(params, x, batch, n_out);
  if (st != SVK_OK) return st;
  if (!out) return set_error(SVK_ERR_ARG, "NULL output");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScopedWorkspace w;
  const size_t need = cnn_workspace_size(batch, n_out);
  st = w.acquire(need, workspace, ws_bytes, s);
  if (st != SVK_OK) return st;
  return cnn_forward(params, x, batch, n_out, out, w.ptr, need, s);
}

int svk_cnn_gradient(const float *params, const float *x, const float *target, int batch, int n_out, float *grad,
                     float *loss, void *workspace, size_t ws_bytes, void *stream) {
  CallRange range("svk_cnn_gradient");
  int st = check_cnn(params, x, batch, n_out);
  if (st != SVK_OK) return st;
  if (!target || !grad || !loss) return set_error(SVK_ERR_ARG, "NULL target, gradient or loss pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScopedWorkspace w;
  const size_t need = cnn_workspace_size(batch, n_out);
  st = w.acquire(need, workspace, ws_bytes, s);
  if (st != SVK_OK) return st;
  return cnn_gradient(params, x, target, batch, n_out, grad, loss, w.ptr, need, s);
}

int svk_cnn_adam(float *params, float *m, float *v, const float *grad, int n_params, int step, float lr, float beta1,
                 float beta2, float eps, void *stream) {
  CallRange range("svk_cnn_adam");
  if (!params || !m || !v || !grad || n_params < 1 || step < 1)
    return set_error(SVK_ERR_ARG, "bad optimiser arguments");
  return cnn_adam(params, m, v, grad, n_params, step, lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream));
}

int svk_cnn_adam_device_step(float *params, float *m, float *v, const float *grad, int n_params, const int *step,
                             float lr, float beta1, float beta2, float eps, void *stream) {
  CallRange range("svk_cnn_adam_device_step");
  if (!params || !m || !v || !grad || !step || n_params < 1) return set_error(SVK_ERR_ARG, "bad optimiser arguments");
  return cnn_adam_device_step(params, m, v, grad, n_params, step, lr, beta1, beta2, eps,
                              static_cast<cudaStream_t>(stream));
}

int svk_cnn_field_fit(const float *local, const int *xy, const float *weights, int S, int N, int W, int H, int degree,
                      double *coeffs, int *info, void *stream) {
  CallRange range("svk_cnn_field_fit");
  if (!local || !xy || !coeffs || !info || S < 1 || N < 1 || W < 1 || H < 1 || degree < 0 || degree > 3)
    return set_error(SVK_ERR_ARG, "bad field-fit arguments");
  return cnn_field_fit(local, xy, weights, S, N, W, H, degree, coeffs, info, static_cast<cudaStream_t>(stream));
}

size_t svk_fit_workspace_size(int n_stamps, int stamp_size, int N, int L, int degree, int bg_degree) {
  return fit_workspace_size(n_stamps, stamp_size, N, L, degree, bg_degree);
}

int svk_fit_coeffs(const float *R, const float *I, int W, int H, int pitch, const int *stamp_xy,
                   int n_stamps, int stamp_size, const float *basis, int N, int L, int degree,
                   int bg_degree, const float *weight, double *coeffs_out, double *chi2_out,
                   int *info_out, void *workspace, size_t ws_bytes, int sync, void *stream) {
  CallRange range("svk_fit_coeffs");
  if (!R || !I || !stamp_xy || !basis || !coeffs_out || !info_out)
    return set_error(SVK_ERR_ARG, "NULL pointer argument");
  if (W < 1 || H < 1 || W > 65535 || H > 65535 || pitch < W) return set_error(SVK_ERR_ARG, "bad frame size/pitch");
  if (n_stamps < 1 || stamp_size < 1 || stamp_size > 127 || (stamp_size % 2) == 0)
    return set_error(SVK_ERR_ARG, "bad stamp list (n=%d, size=%d)", n_stamps, stamp_size);
  if (L < 1 || L > 31 || (L % 2) == 0) return set_error(SVK_ERR_ARG, "L=%d must be odd in [1,31]", L);
  if (degree < 0 || degree > 3 || bg_degree < -1 || bg_degree > 3)
    return set_error(SVK_ERR_ARG, "degree %d / bg_degree %d out of range", degree, bg_degree);
  const int M = N * n_terms(degree) + n_terms(bg_degree);
  if (N < 1 || M > 1024) return set_error(SVK_ERR_ARG, "M=%d unknowns out of range [1,1024]", M);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScopedWorkspace w;
  const size_t need = fit_workspace_size(n_stamps, stamp_size, N, L, degree, bg_degree);
  int st = w.acquire(need, workspace, ws_bytes, s);
  if (st != SVK_OK) return st;
  st = launch_fit(R, I, W, H, pitch, stamp_xy, n_stamps, stamp_size, basis, N, L, degree, bg_degree, weight,
                  coeffs_out, chi2_out, info_out, w.ptr, need, s);
  if (st != SVK_OK || !sync) return st;
  st = cuda_status(cudaStreamSynchronize(s), "svk_fit_coeffs sync");
  if (st != SVK_OK) return st;
  int info = -1;
  st = cuda_status(cudaMemcpy(&info, info_out, sizeof(int), cudaMemcpyDeviceToHost), "read info");
  if (st != SVK_OK) return st;
  if (info >= 0) return set_error(SVK_ERR_NOT_SPD, "normal matrix not positive definite at pivot %d", info);
  return SVK_OK;
}

size_t svk_fit_moments_count(int N, int degree, int bg_degree) {
  if (N < 1 || N > 64 || degree < 0 || degree > 3 || bg_degree < -1 || bg_degree > 3) return 0;
  return fit_moments_count(N, degree, bg_degree);
}

size_t svk_fit_moments_workspace_size(int n_stamps, int stamp_size, int N) {
  if (n_stamps < 0 || stamp_size < 1 || N < 1) return 0;
  return fit_moments_workspace_size(n_stamps, stamp_size, N);
}

int svk_fit_moments(const float *R, const float *I, const float *weight, int W, int H, int pitch, int row_begin,
                    int row_end, const int *stamp_xy, int n_stamps, int stamp_size, const float *basis, int N, int L,
                    int degree, int bg_degree, double *moments, int accumulate, void *workspace, size_t ws_bytes,
                    void *stream) {
  CallRange range("svk_fit_moments");
  if (!R || !I || !basis || !moments || (n_stamps > 0 && !stamp_xy))
    return set_error(SVK_ERR_ARG, "NULL pointer argument");
  if (W < 1 || H < 1 || W > 65535 || H > 65535 || pitch < W) return set_error(SVK_ERR_ARG, "bad frame size/pitch");
  if (row_begin < 0 || row_end > H || row_begin >= row_end)
    return set_error(SVK_ERR_ARG, "held rows [%d, %d) not inside the frame's %d rows", row_begin, row_end, H);
  if (n_stamps < 0 || stamp_size < 1 || stamp_size > 127 || (stamp_size % 2) == 0)
    return set_error(SVK_ERR_ARG, "bad stamp list (n=%d, size=%d)", n_stamps, stamp_size);
  if (L < 1 || L > 31 || (L % 2) == 0) return set_error(SVK_ERR_ARG, "L=%d must be odd in [1,31]", L);
  if (N < 1 || N > 64) return set_error(SVK_ERR_UNSUPPORTED, "the fit supports 1 <= N <= 64 basis stamps (got %d)", N);
  if (degree < 0 || degree > 3 || bg_degree < -1 || bg_degree > 3)
    return set_error(SVK_ERR_ARG, "degree %d / bg_degree %d out of range", degree, bg_degree);
  if (N * n_terms(degree) + n_terms(bg_degree) > 1024) return set_error(SVK_ERR_ARG, "more than 1024 unknowns");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_stamps == 0) {  // no pixels: the moments are zero (or unchanged)
    if (accumulate) return SVK_OK;
    return cuda_status(cudaMemsetAsync(moments, 0, fit_moments_count(N, degree, bg_degree) * sizeof(double), s),
                       "moments reset");
  }
  ScopedWorkspace w;
  const size_t need = fit_moments_workspace_size(n_stamps, stamp_size, N);
  int st = w.acquire(need, workspace, ws_bytes, s);
  if (st != SVK_OK) return st;
  return launch_fit_moments(R, I, weight, W, H, pitch, row_begin, row_end, stamp_xy, n_stamps, stamp_size, basis, N,
                            L, degree, bg_degree, moments, accumulate != 0, w.ptr, need, s);
}

size_t svk_fit_solve_workspace_size(int N, int degree, int bg_degree) {
  if (N < 1 || N > 64 || degree < 0 || degree > 3 || bg_degree < -1 || bg_degree > 3) return 0;
  return fit_solve_workspace_size(N, degree, bg_degree);
}

int svk_fit_solve(const double *moments, int N, int degree, int bg_degree, double *coeffs_out, double *chi2_out,
                  int *info_out, void *workspace, size_t ws_bytes, int sync, void *stream) {
  CallRange range("svk_fit_solve");
  if (!moments || !coeffs_out || !info_out) return set_error(SVK_ERR_ARG, "NULL pointer argument");
  if (N < 1 || N > 64) return set_error(SVK_ERR_UNSUPPORTED, "the fit supports 1 <= N <= 64 basis stamps (got %d)", N);
  if (degree < 0 || degree > 3 || bg_degree < -1 || bg_degree > 3)
    return set_error(SVK_ERR_ARG, "degree %d / bg_degree %d out of range", degree, bg_degree);
  if (N * n_terms(degree) + n_terms(bg_degree) > 1024) return set_error(SVK_ERR_ARG, "more than 1024 unknowns");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScopedWorkspace w;
  const size_t need = fit_solve_workspace_size(N, degree, bg_degree);
  int st = w.acquire(need, workspace, ws_bytes, s);
  if (st != SVK_OK) return st;
  st = launch_fit_solve(moments, N, degree, bg_degree, coeffs_out, chi2_out, info_out, w.ptr, need, s);
  if (st != SVK_OK || !sync) return st;
  st = cuda_status(cudaStreamSynchronize(s), "svk_fit_solve sync");
  if (st != SVK_OK) return st;
  int info = -1;
  st = cuda_status(cudaMemcpy(&info, info_out, sizeof(int), cudaMemcpyDeviceToHost), "read info");
  if (st != SVK_OK) return st;
  if (info >= 0) return set_error(SVK_ERR_NOT_SPD, "normal matrix not positive definite at pivot %d", info);
  return SVK_OK;
}

int svk_band_rows(int method, int precision, int N, int L, int degree) {
  if (L < 1 || L > 31 || (L % 2) == 0 || N < 1 || N > 4096 || degree < 0 || degree > 3) return 0;
  if (method == SVK_METHOD_DIRECT && precision != SVK_PREC_FP32) return 0;
  if (method != SVK_METHOD_DIRECT && method != SVK_METHOD_BASIS && method != SVK_METHOD_TFORM) return 0;
  return band_granule(method, precision, N, L, degree);
}

int svk_difference_rows(const float *R, int pitch_R, int r_begin, int r_end, const float *I, int pitch_I, float *D,
                        int pitch_D, int W, int H, int y_begin, int y_end, const float *basis, int N, int L,
                        const float *coeffs, int degree, int method, int precision, int edge, void *workspace,
                        size_t ws_bytes, void *stream) {
  CallRange range("svk_difference_rows");
  const bool need_I = I != nullptr;
  int st = check_conv_args(R, pitch_R, I, pitch_I, W, H, basis, N, L, coeffs, degree, method, precision, edge, D,
                           pitch_D, need_I);
  if (st != SVK_OK) return st;
  if (y_begin < 0 || y_end > H || y_begin >= y_end)
    return set_error(SVK_ERR_ARG, "output rows [%d, %d) not inside the frame's %d rows", y_begin, y_end, H);
  const int gran = band_granule(method, precision, N, L, degree);
  if (gran < 1) return set_error(SVK_ERR_UNSUPPORTED, "no plan for this method, N=%d, L=%d", N, L);
  if (y_begin % gran != 0 || (y_end % gran != 0 && y_end != H))
    return set_error(SVK_ERR_ARG, "band [%d, %d) not aligned to %d rows (svk_band_rows)", y_begin, y_end, gran);
  const int h = (L - 1) / 2;
  const int need_lo = y_begin - h > 0 ? y_begin - h : 0, need_hi = y_end + h < H ? y_end + h : H;
  if (r_begin < 0 || r_end > H || r_begin > need_lo || r_end < need_hi)
    return set_error(SVK_ERR_ARG, "R holds rows [%d, %d); the band needs [%d, %d)", r_begin, r_end, need_lo, need_hi);
  // the kernels index I and D by frame row and touch only rows [y_begin, y_end)
  const float *If = need_I ? reinterpret_cast<const float *>(reinterpret_cast<uintptr_t>(I) -
                                                            (uintptr_t)y_begin * (uintptr_t)pitch_I * sizeof(float))
                           : nullptr;
  float *Df = reinterpret_cast<float *>(reinterpret_cast<uintptr_t>(D) -
                                        (uintptr_t)y_begin * (uintptr_t)pitch_D * sizeof(float));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (method == SVK_METHOD_DIRECT)
    return launch_direct(R, pitch_R, If, pitch_I, W, H, basis, N, L, coeffs, degree, Df, pitch_D, s, y_begin, y_end,
                         r_begin, r_end);
  ScopedWorkspace w;
  if (method == SVK_METHOD_TFORM) {
    const size_t need = tform_workspace_size(precision, L, degree);
    if ((st = w.acquire(need, workspace, ws_bytes, s)) != SVK_OK) return st;
    return launch_tform(R, pitch_R, If, pitch_I, W, H, basis, N, L, coeffs, degree, precision, Df, pitch_D, w.ptr,
                        need, s, y_begin, y_end, true, r_begin, r_end);
  }
  const size_t need = tc_workspace_size(precision, N, L);
  if ((st = w.acquire(need, workspace, ws_bytes, s)) != SVK_OK) return st;
  return launch_tc(R, pitch_R, If, pitch_I, W, H, basis, N, L, coeffs, degree, precision, Df, pitch_D, w.ptr, need,
                   s, y_begin, y_end, true, r_begin, r_end);
}

int svk_cut_stamps(const float *img, int W, int H, int pitch, const int *xy, int n, int size, float offset,
                   float divisor, float *out, long long stamp_stride, void *stream) {
  CallRange range("svk_cut_stamps");
  if (!img || !out || (n > 0 && !xy)) return set_error(SVK_ERR_ARG, "NULL pointer argument");
  if (W < 1 || H < 1 || pitch < W) return set_error(SVK_ERR_ARG, "bad image size/pitch");
  if (n < 0 || size < 1 || size > 1024) return set_error(SVK_ERR_ARG, "bad stamp count %d / size %d", n, size);
  if (stamp_stride < (long long)size * size) return set_error(SVK_ERR_ARG, "stamp stride below size * size");
  if (!(divisor != 0.0f) || !std::isfinite(divisor) || !std::isfinite(offset))
    return set_error(SVK_ERR_ARG, "offset/divisor must be finite and divisor non-zero");
  return launch_cut_stamps(img, W, H, pitch, xy, n, size, offset, divisor, out, stamp_stride,
                           static_cast<cudaStream_t>(stream));
}

size_t svk_stamp_residual_workspace_size(int n) { return n < 1 ? 0 : stamp_residual_workspace_size(n); }

int svk_stamp_residual(const float *D, int W, int H, int pitch, const int *xy, int n, int size, const float *basis0,
                       int L, double noise_sigma, double ref_noise_sigma, double ratio, const int *field_info,
                       double *out, int *fallback_out, void *workspace, size_t ws_bytes, void *stream) {
  CallRange range("svk_stamp_residual");
  if (!D || !xy || !basis0 || !out || !fallback_out) return set_error(SVK_ERR_ARG, "NULL pointer argument");
  if (W < 1 || H < 1 || pitch < W) return set_error(SVK_ERR_ARG, "bad image size/pitch");
  if (n < 1 || size < 1 || size > 1024) return set_error(SVK_ERR_ARG, "bad stamp count %d / size %d", n, size);
  if (L < 1 || L > 63 || (L % 2) == 0) return set_error(SVK_ERR_ARG, "L=%d must be odd in [1,63]", L);
  if (!(noise_sigma >= 0.0) || !(ref_noise_sigma >= 0.0) || !(ratio > 0.0))
    return set_error(SVK_ERR_ARG, "noise levels must be >= 0 and the ratio > 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScopedWorkspace w;
  const size_t need = stamp_residual_workspace_size(n);
  int st = w.acquire(need, workspace, ws_bytes, s);
  if (st != SVK_OK) return st;
  return launch_stamp_residual(D, W, H, pitch, xy, n, size, basis0, L, noise_sigma, ref_noise_sigma, ratio, field_info,
                               out, fallback_out, w.ptr, need, s);
}

int svk_cnn_standardise(const float *in, long long rows, int cols, const float *mean, const float *sd, int inverse,
                        float *out, void *stream) {
  if (!in || !mean || !sd || !out) return set_error(SVK_ERR_ARG, "NULL pointer argument");
  if (rows < 0 || cols < 1) return set_error(SVK_ERR_ARG, "bad shape %lld x %d", rows, cols);
  return launch_standardise(in, rows, cols, mean, sd, inverse != 0, out, static_cast<cudaStream_t>(stream));
}

int svk_cnn_draw_batch(unsigned long long seed, const int *step, int n, int batch, long long *idx_out, void *stream) {
  if (!step || !idx_out) return set_error(SVK_ERR_ARG, "NULL pointer argument");
  if (n < 1 || batch < 1) return set_error(SVK_ERR_ARG, "n=%d and batch=%d must be positive", n, batch);
  return launch_draw_batch(seed, step, n, batch, idx_out, static_cast<cudaStream_t>(stream));
}

int svk_gather_rows(const void *src, long long row_bytes, const long long *idx, int n, void *dst, void *stream) {
  if (!src || !idx || !dst) return set_error(SVK_ERR_ARG, "NULL pointer argument");
  if (row_bytes < 4 || row_bytes % 4 != 0) return set_error(SVK_ERR_ARG, "row_bytes must be a positive multiple of 4");
  if (n < 0 || n > 65535) return set_error(SVK_ERR_ARG, "n=%d rows out of range [0, 65535]", n);
  if (n == 0) return SVK_OK;
  return launch_gather_rows(src, row_bytes, idx, n, dst, static_cast<cudaStream_t>(stream));
}

int svk_cnn_step_end(const float *loss, int *step, float *history, int history_len, void *stream) {
  if (!loss || !step || !history) return set_error(SVK_ERR_ARG, "NULL pointer argument");
  if (history_len < 1) return set_error(SVK_ERR_ARG, "history_len must be >= 1");
  return launch_step_end(loss, step, history, history_len, static_cast<cudaStream_t>(stream));
}

size_t svk_host_workspace_size(int method, int precision, int W, int H, int N, int L, int degree) {
  if (W < 1 || H < 1 || W > 65535 || H > 65535) return 0;
  return host_workspace_size(method, precision, W, H, N, L, degree);
}

int svk_difference_host(const float *R, const float *I, float *D, int W, int H, int pitch, const float *basis, int N,
                        int L, const float *coeffs, int degree, int method, int precision, int n_bands,
                        void *workspace, size_t ws_bytes, void *stream) {
  CallRange range("svk_difference_host");
  int st = check_conv_args(R, pitch, I, pitch, W, H, basis, N, L, coeffs, degree, method, precision, SVK_EDGE_ZERO,
                           D, pitch, true);
  if (st != SVK_OK) return st;
  if (n_bands < 1) return set_error(SVK_ERR_ARG, "n_bands=%d must be >= 1", n_bands);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScopedWorkspace w;
  const size_t need = host_workspace_size(method, precision, W, H, N, L, degree);
  st = w.acquire(need, workspace, ws_bytes, s);
  if (st != SVK_OK) return st;
  return launch_host(R, I, D, W, H, pitch, basis, N, L, coeffs, degree, method, precision, n_bands, w.ptr, need, s);
}

static int check_host_frames(const svk_frame *frames, int n, int method, int precision) {
  if (!frames || n < 1) return set_error(SVK_ERR_ARG, "no frames");
  for (int f = 0; f < n; ++f) {
    const svk_frame &F = frames[f];
    int st = check_conv_args(F.R, F.pitch_R, F.I, F.pitch_I, F.W, F.H, F.basis, F.N, F.L, F.coeffs, F.degree, method,
                             precision, SVK_EDGE_ZERO, F.D, F.pitch_D, true);
    if (st != SVK_OK) {
      char msg[sizeof(g_err)];  // the message is rewritten into g_err below
      snprintf(msg, sizeof(msg), "%s", last_error());
      return set_error(st, "frame %d: %s", f, msg);
    }
  }
  return SVK_OK;
}

size_t svk_host_batch_workspace_size(const svk_frame *frames, int n_frames, int method, int precision) {
  if (check_host_frames(frames, n_frames, method, precision) != SVK_OK) return 0;
  return host_batch_workspace_size(frames, n_frames, method, precision);
}

int svk_difference_host_batch(const svk_frame *frames, int n_frames, int method, int precision, int n_bands,
                              void *workspace, size_t ws_bytes, void *stream) {
  CallRange range("svk_difference_host_batch");
  int st = check_host_frames(frames, n_frames, method, precision);
  if (st != SVK_OK) return st;
  if (n_bands < 1) return set_error(SVK_ERR_ARG, "n_bands=%d must be >= 1", n_bands);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScopedWorkspace w;
  const size_t need = host_batch_workspace_size(frames, n_frames, method, precision);
  st = w.acquire(need, workspace, ws_bytes, s);
  if (st != SVK_OK) return st;
  return launch_host_batch(frames, n_frames, method, precision, n_bands, w.ptr, need, s);
}

int svk_device_status(int reset, void *stream) {
  uint32_t *w = device_status_word();
  if (!w) return set_error(SVK_ERR_CUDA, "device status word not available");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  int st = cuda_status(cudaMemcpyAsync(&v, w, 4, cudaMemcpyDeviceToHost, s), "read device status");
  if (st == SVK_OK) st = cuda_status(cudaStreamSynchronize(s), "device status sync");
  if (st != SVK_OK) return st;
  if (reset && v != 0) {
    if ((st = cuda_status(cudaMemsetAsync(w, 0, 4, s), "clear device status")) != SVK_OK) return st;
    if ((st = cuda_status(cudaStreamSynchronize(s), "device status sync")) != SVK_OK) return st;
  }
  if (v & kDevIndex)
    return set_error(SVK_ERR_INDEX,
                     "a device index check failed (debug build; check sites 0x%x; the access was skipped, results invalid)",
                     v >> 8);
  if (v & kDevTimeout)
    return set_error(SVK_ERR_TIMEOUT, "a bounded device wait gave up (results since the last check are invalid)");
  return v == 0 ? SVK_OK : set_error(SVK_ERR_CUDA, "device status 0x%x", v);
}

int svk_selftest_bounded_wait(unsigned long long limit_ns, unsigned long long *waited_ns, void *stream) {
  if (limit_ns < 1000ull || limit_ns > 10000000000ull)
    return set_error(SVK_ERR_ARG, "limit %llu ns out of range [1 us, 10 s]", limit_ns);
  return selftest_bounded_wait(limit_ns, waited_ns, static_cast<cudaStream_t>(stream));
}

int svk_measure_fma_peak(int kind, double *flops_per_s, void *stream) {
  if (!flops_per_s) return set_error(SVK_ERR_ARG, "NULL pointer argument");
  if (kind < SVK_FMA_FP32 || kind > SVK_FMA_FP32X2) return set_error(SVK_ERR_ARG, "unknown FMA kind");
  return measure_fma_peak(kind, flops_per_s, static_cast<cudaStream_t>(stream));
}

size_t svk_select_workspace_size(int W, int H) {
  if (W < 1 || H < 1 || W > 65535 || H > 65535 || (long long)W * H >= (1ll << 31)) return 0;
  return select_workspace_size(W, H);
}

int svk_select_stamps(const float *R, int W, int H, int pitch, float sky, float threshold, float saturation,
                      int margin, int iso_radius, float iso_frac, int max_stamps, int *stamp_xy_out, int *counts_out,
                      void *workspace, size_t ws_bytes, void *stream) {
  CallRange range("svk_select_stamps");
  if (!R || !counts_out || (max_stamps > 0 && !stamp_xy_out)) return set_error(SVK_ERR_ARG, "NULL pointer argument");
  if (W < 1 || H < 1 || W > 65535 || H > 65535 || (long long)W * H >= (1ll << 31) || pitch < W)
    return set_error(SVK_ERR_ARG, "bad frame size/pitch");
  if (margin < 0 || iso_radius < 0 || iso_radius > 1024 || max_stamps < 0)
    return set_error(SVK_ERR_ARG, "margin %d / iso_radius %d / max_stamps %d out of range", margin, iso_radius,
                     max_stamps);
  if (!(iso_frac >= 0.0f) || !std::isfinite(iso_frac) || !std::isfinite(sky) || std::isnan(threshold) ||
      std::isnan(saturation))
    return set_error(SVK_ERR_ARG, "sky, threshold, saturation and iso_frac must be numbers (iso_frac >= 0)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScopedWorkspace w;
  const size_t need = select_workspace_size(W, H);
  int st = w.acquire(need, workspace, ws_bytes, s);
  if (st != SVK_OK) return st;
  return launch_select(R, W, H, pitch, sky, threshold, saturation, margin, iso_radius, iso_frac, max_stamps,
                       stamp_xy_out, counts_out, w.ptr, need, s);
}

}  // extern "C"
