/*
 * svk.h -- C ABI of the spatially-varying kernel (SVK) image-subtraction library.
 *
 * The library computes the difference image of Optimal Image Subtraction,
 *     D = (R (x) K_{x,y}) - I                                   (Eq. 1)
 *     K_{x,y} = sum_k a_k(x,y) B_k                               (Eq. 2)
 *     a_k(x,y) = sum_t c[k][t] m_t(xt, yt)                       (Eq. 3, order d)
 * on one GB300 GPU (sm_103a), with hand-written CUDA kernels, and fits the
 * coefficients c by least squares over star stamps (Sec. 2).
 *
 * Conventions shared by every entry point:
 *   - Images are row-major float32, x = column (contiguous), y = row; pitches are in
 *     ELEMENTS and must be >= W.
 *   - Kernel size L is odd, h = (L - 1) / 2; basis stamps are stored
 *     basis[k][v + h][u + h] (row = y offset v, column = x offset u), float32.
 *   - (x) is a true convolution: (R (x) K)(x,y) = sum_{u,v} K(u,v) R(x - u, y - v),
 *     R is zero outside the frame, and the kernel is formed at the OUTPUT pixel.
 *   - Polynomial coordinates are normalised over the frame:
 *     xt = (2x - (W - 1)) / (W - 1) (0 when W == 1), likewise yt with H.
 *   - Monomials m_t = xt^i yt^j with i + j <= d, i outer, j inner; T = (d+1)(d+2)/2.
 *     For d = 2 this is 1, yt, yt^2, xt, xt yt, xt^2 (the terms of Eq. 3).
 *   - Coefficients are float32 c[N][T] (row-major) on the device.
 *   - Every pointer named "device" must be device memory of the current CUDA device;
 *     the caller owns all buffers; the library never frees them.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is
 *     asynchronous on that stream unless its comment says otherwise.
 *   - Return value: SVK_OK or an error code; svk_last_error() gives a message
 *     (thread-local).  Argument errors are detected on the host before any launch
 *     and leave outputs untouched.
 */
#ifndef SVK_H
#define SVK_H

#include <stddef.h>

#if defined(__GNUC__)
#define SVK_API __attribute__((visibility("default")))
#else
#define SVK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define SVK_VERSION 1

/* status codes */
#define SVK_OK 0
#define SVK_ERR_ARG 1         /* invalid argument (host-side check)                      */
#define SVK_ERR_CUDA 2        /* a CUDA runtime/driver call failed                        */
#define SVK_ERR_NOT_SPD 3     /* normal matrix not positive definite (info = pivot)       */
#define SVK_ERR_TIMEOUT 4     /* a bounded device-side wait ran out                       */
#define SVK_ERR_UNSUPPORTED 5 /* valid request the library does not implement              */
#define SVK_ERR_WORKSPACE 6   /* caller workspace too small                               */
#define SVK_ERR_INDEX 7       /* a device index check failed (debug builds, SVK_DEBUG)     */

/* basis kinds (Sec. 2: Gaussian function basis and Dirac delta function basis) */
#define SVK_BASIS_GAUSS 0
#define SVK_BASIS_DELTA 1

/* basis normalisation */
#define SVK_NORM_NONE 0  /* raw stamps                                                    */
#define SVK_NORM_ALARD 1 /* GAUSS: B_0 unit sum; even-even stamps made zero-sum by        */
                         /* subtracting (sum) B_0; stamps k >= 1 scaled to unit L2 norm.  */
                         /* DELTA: stamps other than the centre tap become                */
                         /* delta_k - delta_centre.                                       */

/* convolution methods */
#define SVK_METHOD_DIRECT 0 /* kernel formed per pixel on the CUDA cores (FP32 FFMA)      */
#define SVK_METHOD_BASIS 1  /* R (x) B_k for all k as an implicit-im2col GEMM on the       */
                            /* tensor cores (tcgen05, TMEM accumulators), then a fused     */
                            /* polynomial epilogue sum_k a_k(x,y) C_k(x,y) (- I)           */
#define SVK_METHOD_TFORM 2  /* the same result by linearity of Eq. 2 and 3 as              */
                            /* sum_t m_t(xt,yt) (R (x) K_t)(x,y) (- I), K_t = sum_k c[k][t] */
                            /* B_k: T = (d+1)(d+2)/2 convolutions instead of N; any N       */
                            /* (delta bases included); on the tensor cores with the         */
                            /* precisions of SVK_METHOD_BASIS, or on the CUDA cores with    */
                            /* SVK_PREC_FP32 (the T convolutions accumulated per pixel)     */

/* arithmetic of the contraction */
#define SVK_PREC_FP32 0   /* DIRECT, TFORM: FP32 FFMA on the CUDA cores                   */
#define SVK_PREC_BF16X3 1 /* BASIS, TFORM: R and B split hi + lo in BF16, hi*hi + hi*lo + lo*hi, */
                          /* FP32 accumulation                                            */
#define SVK_PREC_FP16X3 2 /* BASIS, TFORM: the same split in FP16 (power-of-two prescaled) */
#define SVK_PREC_BF16 3   /* BASIS, TFORM: plain BF16 operands, FP32 accumulation (one MMA) */
#define SVK_PREC_FP16X2 4 /* BASIS: R split hi + lo in FP16 (power-of-two prescaled), the     */
                          /* basis taken as FP16-exact (its values x 1024 rounded to FP16),  */
                          /* hi*B + lo*B: two MMAs; FP32-level accuracy for a basis that      */
                          /* svk_round_basis_fp16 made exact (otherwise the convolution is    */
                          /* with that rounding of the basis)                                  */

#define SVK_EDGE_ZERO 0 /* R is zero outside the frame (the only mode)                    */

/* Message of the last error on this host thread ("" if none). */
SVK_API const char *svk_last_error(void);

/* SVK_VERSION of the loaded library. */
SVK_API int svk_version(void);

/* Number of Gaussian-basis stamps for n_gauss Gaussians of polynomial degrees deg[]
 * (sum of (d+1)(d+2)/2), or -1 on bad arguments.  Host only, no CUDA call. */
SVK_API int svk_gauss_basis_count(int n_gauss, const int *deg);

/*
 * Tabulate basis stamps B_k on the L x L grid (Sec. 2, Eq. 2; the Gaussian basis of
 * Alard & Lupton and the delta basis of Miller et al.), in FP64 on the device,
 * stored as float32.
 *   kind        SVK_BASIS_GAUSS: for Gaussian g (sigma[g] px) and (p, q) with
 *               p + q <= deg[g] (p outer, q inner),
 *               B(u,v) = exp(-(u^2 + v^2) / (2 sigma_g^2)) u^p v^q;
 *               N = svk_gauss_basis_count(n_gauss, deg), Gaussian-major.
 *               SVK_BASIS_DELTA: N = L*L, B_k = delta at tap k = (v+h) L + (u+h);
 *               sigma / deg / n_gauss ignored.
 *   L           odd kernel size, 1 <= L <= 63.
 *   sigma, deg  HOST arrays of n_gauss entries (sigma > 0, 0 <= deg <= 10).
 *   normalize   SVK_NORM_NONE or SVK_NORM_ALARD.
 *   basis_out   device float32 [N][L][L]; must hold N*L*L floats.
 *   n_basis_out HOST int receiving N (may be NULL).
 */
SVK_API int svk_build_basis(int kind, int L, int n_gauss, const double *sigma, const int *deg,
                    int normalize, float *basis_out, int *n_basis_out, void *stream);

/*
 * Round n basis values in place so that 1024 b is exactly an FP16 value:
 * b <- fp16_rn(1024 b) / 1024.  A basis so rounded is a basis like any other (any B_k
 * defines Eq. 2's kernel family); SVK_PREC_FP16X2 then multiplies it without a low part
 * (two MMAs per K step instead of three) at the accuracy of the x3 splits.  Values beyond
 * +-64 saturate to FP16's range.  basis: device float32, n >= 0.  Asynchronous on
 * `stream`; SVK_ERR_ARG on a NULL pointer with n > 0.
 */
SVK_API int svk_round_basis_fp16(float *basis, long long n, void *stream);

/*
 * Bytes of device workspace that svk_convolve / svk_difference need for this request.
 * A call may pass workspace == NULL with ws_bytes == 0, in which case the library makes
 * a stream-ordered allocation of this size for the duration of the call.
 */
SVK_API size_t svk_workspace_size(int method, int precision, int W, int H, int N, int L, int degree);

/*
 * out = R (x) K_{x,y}  (Eq. 1 without the subtraction; Eq. 2 and 3 for K).
 *   R        device float32 [H][pitch_R]
 *   W, H     frame size (>= 1 each; W, H <= 65535)
 *   basis    device float32 [N][L][L] (1 <= N <= 4096, odd 1 <= L <= 31)
 *   coeffs   device float32 [N][T], T = (degree+1)(degree+2)/2, 0 <= degree <= 3
 *   method   SVK_METHOD_DIRECT (precision SVK_PREC_FP32), SVK_METHOD_BASIS (precision
 *            SVK_PREC_BF16X3 / FP16X3 / BF16; N <= 256) or SVK_METHOD_TFORM (the same
 *            precisions or SVK_PREC_FP32; any N)
 *   edge     SVK_EDGE_ZERO
 *   out      device float32 [H][pitch_out]; must not overlap R
 *   workspace, ws_bytes   device scratch of at least svk_workspace_size() bytes, or
 *            NULL / 0 (library allocates on `stream`).
 * Errors: SVK_ERR_ARG (bad sizes, even L, NULL pointers, pitch < W),
 * SVK_ERR_UNSUPPORTED (method/precision pair not built), SVK_ERR_WORKSPACE,
 * SVK_ERR_CUDA.
 */
SVK_API int svk_convolve(const float *R, int W, int H, int pitch_R, const float *basis, int N, int L,
                 const float *coeffs, int degree, int method, int precision, int edge,
                 float *out, int pitch_out, void *workspace, size_t ws_bytes, void *stream);

/*
 * D = (R (x) K_{x,y}) - I  (Eq. 1), the subtraction fused into the convolution.
 * Arguments as svk_convolve, plus I (device float32 [H][pitch_I]) and D (device
 * float32 [H][pitch_D]; must not overlap R or I).
 */
SVK_API int svk_difference(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H,
                   const float *basis, int N, int L, const float *coeffs, int degree, int method,
                   int precision, int edge, float *D, int pitch_D, void *workspace,
                   size_t ws_bytes, void *stream);

/*
 * D = (R (x) K_{x,y}) - I by the tensor-core basis form, allocating no device memory.
 * The paper has no counterpart: this is an interface for callers that cannot allocate --
 * a host application that owns the whole device heap, a pipeline that must not
 * allocate (or risk a failed allocation) once it is running, or a caller with no way
 * to pass a workspace.  Arguments as svk_difference with method SVK_METHOD_BASIS
 * (precision SVK_PREC_BF16X3 / FP16X3 / BF16) and no workspace.
 * Scratch: one 512 KiB __device__ array inside this library, held on every device that
 * loads it until the process exits; requests needing more return SVK_ERR_WORKSPACE.
 * The first call on a device looks up the array's device address (again after that
 * device's context was replaced, e.g. by cudaDeviceReset); make that first call before
 * any stream capture.  All calls share the array and it
 * keeps the last call's contents, so calls that overlap on the GPU race: serialise them.
 */
SVK_API int svk_difference_noalloc(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H,
                                   const float *basis, int N, int L, const float *coeffs, int degree,
                                   int precision, int edge, float *D, int pitch_D, void *stream);

/*
 * One frame of a batch: D = (R (x) K_{x,y}) - I (I may be NULL: D = R (x) K_{x,y}).
 * Pointers are device memory; field meanings as in svk_difference.
 */
typedef struct svk_frame {
  const float *R;
  int pitch_R;
  const float *I;
  int pitch_I;
  float *D;
  int pitch_D;
  int W, H;
  const float *basis;
  int N, L;
  const float *coeffs;
  int degree;
} svk_frame;

/* Bytes of device workspace svk_difference_batch needs for these frames (0 on error). */
SVK_API size_t svk_batch_workspace_size(const svk_frame *frames, int n_frames, int precision);

/*
 * A night's batch of uneven frames (Sec. 3: a wide-field camera delivers many tiles per
 * exposure) by the tensor-core basis form.  Frames are grouped by (N, L); each group
 * runs as persistent launches over up to 64 frames whose blocks are split into
 * contiguous ranges per CTA, every frame with its own size, degree, coefficients and
 * basis (frames sharing one basis pointer share its tables).  `frames` is a HOST array
 * of n_frames >= 1 descriptors, read during the call.  With a workspace the call issues
 * only kernel launches and memsets on `stream`, so it can be captured in a CUDA graph
 * and replayed.  Errors as svk_difference, checked for every frame before any launch.
 */
SVK_API int svk_difference_batch(const svk_frame *frames, int n_frames, int precision, void *workspace,
                                 size_t ws_bytes, void *stream);

/*
 * Time every tensor-core plan that fits shared memory -- output rows per block G (up to
 * 256 MMA columns, G * N <= 256), pipeline stages 4, 8 or 16, basis tables resident in
 * shared memory or their slices streamed through a ring beside the stages -- on a
 * synthetic W x H frame for (N, L, degree, precision), keep the fastest for later calls
 * with that (N, L, precision) in this process, and report it through G_out / stages_out
 * (nullable; svk_tc_plan also reports whether the tables are streamed).  Allocates its
 * test buffers on `stream` and synchronises it.
 */
SVK_API int svk_autotune(int N, int L, int degree, int precision, int W, int H, int *G_out, int *stages_out,
                         void *stream);

/*
 * The tensor-core plan later calls with (N, L, precision) use: output rows per block G,
 * pipeline stages, and streamed = 1 when the basis slices stream through a shared-memory
 * ring (each reference row's slot carries the slice its window ends with) instead of
 * resident tables.  Without svk_autotune or svk_set_plan: the most output rows per block
 * that fit, resident tables preferred.  Outputs nullable.  SVK_ERR_UNSUPPORTED when no plan
 * fits (N, L).  Host-only: no device work.
 */
SVK_API int svk_tc_plan(int N, int L, int precision, int *G, int *stages, int *streamed);

/*
 * Set the plan for later calls with (N, L, precision) in this process, as svk_autotune
 * would (e.g. a plan an earlier process tuned); G = 0 restores the default.
 * SVK_ERR_UNSUPPORTED when the plan does not fit shared memory or breaks the streamed
 * ring's rules (stages 8 or 16, G - 1 + (ceil(L/8) odd) <= stages / 4).  Workspace sizes
 * follow the plan: query them after setting it.  Host-only: no device work.
 */
SVK_API int svk_set_plan(int N, int L, int precision, int G, int stages, int streamed);

/*
 * Coefficient network.  A small CNN predicts, from a (R, I) star-stamp pair, the local
 * kernel coefficients a_k (Eq. 3 evaluated at the stamp; Eq. 2 combines them with the
 * basis), as a fast stand-in for the least-squares fit of Sec. 2, whose result is the
 * reference for the network's error and its fallback.  Input x: device float32
 * [batch][2][64][64] (channel 0 R, channel 1 I, both already normalised by the caller);
 * output float32 [batch][n_out].
 * Architecture: four 3x3 convolutions (2->32 stride 2, 32->32 stride 2, 32->32 stride 2,
 * 32->32 stride 1, zero padding 1, ReLU), global average pooling, linear 32 -> n_out.
 * Parameters: one float32 vector of svk_cnn_param_count(n_out) values (FP32 master
 * copy).  Precision: weights are used rounded to BF16; the input, every post-ReLU
 * activation and every pre-activation gradient are stored in BF16; all sums accumulate
 * in FP32 (the convolutions on the tensor cores, BF16 x BF16 -> FP32).  The gradient is
 * deterministic (fixed-order reductions, no atomics); the loss is summed with atomics.
 * 1 <= n_out <= 256, 1 <= batch <= 4096.  workspace: device memory of
 * svk_cnn_workspace_size(batch, n_out) bytes, 256-byte aligned, owned by the caller
 * (SVK_ERR_WORKSPACE when smaller, SVK_ERR_ARG when misaligned; NULL: the library
 * allocates one on the stream).
 */
SVK_API int svk_cnn_param_count(int n_out);
SVK_API size_t svk_cnn_workspace_size(int batch, int n_out);
SVK_API int svk_cnn_forward(const float *params, const float *x, int batch, int n_out, float *out, void *workspace,
                            size_t ws_bytes, void *stream);
/* Mean squared error against target [batch][n_out] into *loss (device float) and its
 * gradient with respect to every parameter into grad (device float [param_count]).  The
 * weight gradients of the 32-channel layers run on a library stream forked from and joined
 * back into `stream` within the call (events; capturable in a CUDA graph once a first call
 * has run outside the capture), so all of the call's work is ordered on `stream`. */
SVK_API int svk_cnn_gradient(const float *params, const float *x, const float *target, int batch, int n_out,
                             float *grad, float *loss, void *workspace, size_t ws_bytes, void *stream);
/* One Adam step (bias-corrected, step >= 1) on the FP32 parameters with moments m, v. */
SVK_API int svk_cnn_adam(float *params, float *m, float *v, const float *grad, int n_params, int step, float lr,
                         float beta1, float beta2, float eps, void *stream);
/* The same step with the step count read from device memory (*step: device int32, >= 1
 * when the kernel runs; the bias corrections 1 - beta^step are formed on the device), so
 * that a training step can be captured once as a CUDA graph and replayed while the count
 * advances.  Errors: SVK_ERR_ARG for NULL pointers or n_params < 1. */
SVK_API int svk_cnn_adam_device_step(float *params, float *m, float *v, const float *grad, int n_params,
                                     const int *step, float lr, float beta1, float beta2, float eps, void *stream);
/*
 * Coefficient field from local predictions: for stamps s at (x_s, y_s) of a W x H frame
 * with local coefficients local[s][k] (device float32 [S][N]) and optional weights
 * (device float32 [S] or NULL), the FP64 least-squares c[k][t] of
 * a_k(x, y) = sum_t c[k][t] m_t(xt, yt) (Eq. 3 with the coordinate reading of svk_convolve)
 * into coeffs (device double [N][T]); *info = -1, or the failing pivot (coeffs zero).
 */
SVK_API int svk_cnn_field_fit(const float *local, const int *xy, const float *weights, int S, int N, int W, int H,
                              int degree, double *coeffs, int *info, void *stream);

/*
 * Square stamps of an image (row A9: the network's input and the residual check both look
 * at stamps around stars, the stamps over which Sec. 2 fits the kernel):
 *   out[s * stamp_stride + v * size + u] = (img(cx_s - size/2 + u, cy_s - size/2 + v) - offset) / divisor
 * with img read as 0 outside the W x H frame, u, v = 0 .. size - 1.
 *   img    device float32 [H][pitch];  xy: device int32 [n][2] = (cx, cy)
 *   out    device float32, stamp s at out + s * stamp_stride (stamp_stride >= size^2; pass
 *          2 size^2 and out + c size^2 to fill channel c of an [n][2][size][size] input)
 *   offset, divisor: the affine normalisation (0 and 1 for raw counts; divisor != 0)
 * Errors: SVK_ERR_ARG (host checks).  Asynchronous on `stream`.
 */
SVK_API int svk_cut_stamps(const float *img, int W, int H, int pitch, const int *xy, int n, int size, float offset,
                           float divisor, float *out, long long stamp_stride, void *stream);

/* Bytes of device workspace svk_stamp_residual needs (0 when n < 1). */
SVK_API size_t svk_stamp_residual_workspace_size(int n);

/*
 * The check that keeps or rejects the network's coefficients for a frame (row A9, the FP64
 * fit as fallback): with D = (R (x) K) - I made from them,
 *   chi2_per_px = mean over the n stamps and their size^2 pixels of (D - mean_stamp(D))^2
 *                 (D read as 0 outside the frame; each stamp's mean removed, the background
 *                 not being part of the prediction)
 *   floor       = noise_sigma^2 + ref_noise_sigma^2 * sum(K0^2)   (basis0: K0 [L][L], the
 *                 unit-sum first stamp standing in for the kernel)
 *   fallback    = 1 when chi2_per_px > ratio * floor or *field_info >= 0 (the field fit
 *                 failed; field_info nullable), else 0
 * out: device double [2] = {chi2_per_px, floor}; fallback_out: device int [1].  FP64 sums
 * in a fixed order (deterministic).  Asynchronous on `stream`.
 */
SVK_API int svk_stamp_residual(const float *D, int W, int H, int pitch, const int *xy, int n, int size,
                               const float *basis0, int L, double noise_sigma, double ref_noise_sigma, double ratio,
                               const int *field_info, double *out, int *fallback_out, void *workspace,
                               size_t ws_bytes, void *stream);

/*
 * Standardisation of the network's targets and outputs: out[r][c] = (in[r][c] - mean[c]) /
 * sd[c], or with `inverse` non-zero out[r][c] = mean[c] + sd[c] * in[r][c].  Device float32
 * [rows][cols] (in may equal out); mean, sd: device float32 [cols].
 */
SVK_API int svk_cnn_standardise(const float *in, long long rows, int cols, const float *mean, const float *sd,
                                int inverse, float *out, void *stream);

/*
 * Training batch drawn on the device: idx_out[i] (device int64 [batch]) uniform in [0, n)
 * for i < batch, from the counter seed + step * batch + i (step read from device memory
 * when the kernel runs) mixed by SplitMix64 and reduced by a multiply-shift.  A captured
 * training step that advances *step draws a new batch at every replay, and the draws of a
 * run are fixed by (seed, step): resuming from a saved step reproduces them.
 */
SVK_API int svk_cnn_draw_batch(unsigned long long seed, const int *step, int n, int batch, long long *idx_out,
                               void *stream);

/*
 * Row gather: row i of dst = row idx[i] of src, for i < n (rows of row_bytes bytes, a
 * multiple of 4; n <= 65535).  Device pointers; the caller keeps idx in range.
 */
SVK_API int svk_gather_rows(const void *src, long long row_bytes, const long long *idx, int n, void *dst,
                            void *stream);

/*
 * End of a training step on the device: history[*step % history_len] = *loss, then
 * *step += 1 (device pointers; for a captured step that keeps its losses on the device).
 */
SVK_API int svk_cnn_step_end(const float *loss, int *step, float *history, int history_len, void *stream);

/*
 * Bytes of device workspace svk_fit_coeffs needs.
 */
SVK_API size_t svk_fit_workspace_size(int n_stamps, int stamp_size, int N, int L, int degree,
                              int bg_degree);

/*
 * Optimal Image Subtraction least-squares fit of the coefficients (Sec. 2: least squares
 * on Eq. 1 over isolated-star stamps, K decomposed on the basis).  Model at a stamp
 * pixel:  sum_k sum_t c[k][t] m_t(xt,yt) C_k(x,y) + sum_j g_j m_j(xt,yt),  with
 * C_k = R (x) B_k (computed in FP32 on the device); minimise
 * sum w (model - I)^2 through the normal equations A c = b, and solve them by an FP64
 * Cholesky factorisation on the device.  A and b are FP64; their sums over the stamp
 * pixels are taken in double-float arithmetic (pairs of float32, about 48 significant
 * bits, error-free two-sums) within each run of pixels a CTA handles and in FP64 across
 * them (the order of the FP64 additions across CTAs is not fixed, so repeated calls may
 * differ in the last bits).
 *   R, I       device float32 [H][pitch] (same pitch)
 *   stamp_xy   device int32 [n_stamps][2] = (x, y) centres; stamps are
 *              stamp_size x stamp_size (odd); pixels outside the frame are skipped
 *   basis      device float32 [N][L][L]; degree 0..3; bg_degree -1 (none) .. 3
 *   weight     device float32 [H][pitch] per-pixel weight, or NULL (unit weight)
 *   coeffs_out device double [M], M = N*T + Tbg: c[k][t] at k*T + t, then g_j
 *   chi2_out   device double [1] (nullable): sum w (model - I)^2 at the solution
 *   info_out   device int [1]: -1 on success, else the first non-positive pivot
 *   workspace  device scratch of svk_fit_workspace_size() bytes, or NULL / 0.
 * Limits: 1 <= M <= 1024, n_stamps >= 1, stamp_size <= 127.
 * The factorisation outcome is only known on the device: this call returns SVK_OK
 * once the work is queued; *info_out >= 0 after the stream completes means the normal
 * matrix was not positive definite (coeffs_out is then left at zero).  When `sync` is
 * non-zero the call synchronises the stream and returns SVK_ERR_NOT_SPD in that case.
 */
SVK_API int svk_fit_coeffs(const float *R, const float *I, int W, int H, int pitch, const int *stamp_xy,
                   int n_stamps, int stamp_size, const float *basis, int N, int L, int degree,
                   int bg_degree, const float *weight, double *coeffs_out, double *chi2_out,
                   int *info_out, void *workspace, size_t ws_bytes, int sync, void *stream);

/*
 * The fit in two parts, so that the stamps can be split over several GPUs (one process
 * each): every GPU accumulates the moments of its own stamps, the moment arrays are summed
 * over the GPUs (an all-reduce of FP64 sums), and every GPU solves the same normal
 * equations.  The paper fits on one machine (Sec. 2); its two-GPU split of the image
 * (Sec. 4) and the multi-GPU outlook (Sec. 6) motivate this split of the fit's one
 * exchange step.
 *
 * Moments: with the extended columns E = [C_0 .. C_{N-1}, I, 1] of a stamp pixel p,
 *   S[(e1 * (N+2) + e2) * n_mu + mu] = sum_p w(p) E_e1(p) E_e2(p) mu(xt_p, yt_p)   (e1 <= e2)
 * for the n_mu monomials mu of degree <= 2 max(degree, bg_degree) (x exponent outer, y
 * inner); entries with e1 > e2 stay zero.  Every entry of A and b (svk_fit_coeffs) is one
 * of them, so summing S over disjoint stamp sets sums the normal equations.
 * svk_fit_moments_count() doubles (0 on bad arguments).
 */
SVK_API size_t svk_fit_moments_count(int N, int degree, int bg_degree);

/* Bytes of device workspace svk_fit_moments needs (C_k at the stamp pixels). */
SVK_API size_t svk_fit_moments_workspace_size(int n_stamps, int stamp_size, int N);

/*
 * Moments S (above) of the stamps' pixels, written to `moments` (device double
 * [svk_fit_moments_count]) or, when `accumulate` is non-zero, added to it.
 *   R, I, weight  device float32 buffers holding the frame rows [row_begin, row_end) of the
 *                 W x H frame (each pointer at row row_begin, one pitch); weight nullable.
 *                 Pass 0, H for whole frames.  Pixels outside the frame or outside the held
 *                 rows add nothing, so a GPU holding a band of the frame passes the stamps
 *                 whose pixels and kernel halo (stamp_size/2 + L/2 rows each side) it holds.
 *   stamp_xy      device int32 [n_stamps][2], frame coordinates; n_stamps may be 0.
 * Other arguments as svk_fit_coeffs (1 <= N <= 64).  Asynchronous on `stream`.
 */
SVK_API int svk_fit_moments(const float *R, const float *I, const float *weight, int W, int H, int pitch,
                            int row_begin, int row_end, const int *stamp_xy, int n_stamps, int stamp_size,
                            const float *basis, int N, int L, int degree, int bg_degree, double *moments,
                            int accumulate, void *workspace, size_t ws_bytes, void *stream);

/* Bytes of device workspace svk_fit_solve needs (A and b). */
SVK_API size_t svk_fit_solve_workspace_size(int N, int degree, int bg_degree);

/*
 * The normal equations assembled from the moments S, solved by the FP64 Cholesky of
 * svk_fit_coeffs.  coeffs_out, info_out and `sync` as svk_fit_coeffs; chi2_out (nullable)
 * receives sum w (model - I)^2 computed from the moments, S_II - b.c (A c = b at the
 * solution), rather than by a second pass over the pixels.  Asynchronous on `stream`.
 */
SVK_API int svk_fit_solve(const double *moments, int N, int degree, int bg_degree, double *coeffs_out,
                          double *chi2_out, int *info_out, void *workspace, size_t ws_bytes, int sync,
                          void *stream);

/*
 * Row alignment of svk_difference_rows bands for a method: the output-row block of its
 * kernel (12 direct, 16 T-form FP32, the plan's G rows on the tensor cores); 0 when the
 * arguments have no plan.  svk_autotune may change the tensor-core value.
 */
SVK_API int svk_band_rows(int method, int precision, int N, int L, int degree);

/*
 * Output rows [y_begin, y_end) of D = (R (x) K_{x,y}) - I for the W x H frame, from buffers
 * that hold only part of it: the unit of work of a row-band split of one frame over
 * several GPUs (Sec. 4 splits an image between two GPUs; here by row bands).  Coordinates
 * are normalised over the whole frame, so the rows equal those of svk_difference on the
 * whole frame bit for bit.
 *   R        device float32, frame rows [r_begin, r_end) (R points at row r_begin), with
 *            r_begin <= max(0, y_begin - h) and r_end >= min(H, y_end + h), h = (L-1)/2
 *   I, D     device float32, frame rows [y_begin, y_end) (pointers at row y_begin); I may
 *            be NULL (D = R (x) K)
 *   y_begin  a multiple of svk_band_rows(); y_end a multiple of it or H
 * Other arguments, workspace and errors as svk_difference (SVK_ERR_ARG for a band or held
 * range that breaks the rules above).
 */
SVK_API int svk_difference_rows(const float *R, int pitch_R, int r_begin, int r_end, const float *I, int pitch_I,
                                float *D, int pitch_D, int W, int H, int y_begin, int y_end, const float *basis,
                                int N, int L, const float *coeffs, int degree, int method, int precision, int edge,
                                void *workspace, size_t ws_bytes, void *stream);

/*
 * Bytes of device workspace svk_difference_host needs: device copies of R, I and D
 * (W * H * 4 bytes each, rounded up to 256) plus svk_workspace_size() of the method.
 */
SVK_API size_t svk_host_workspace_size(int method, int precision, int W, int H, int N, int L, int degree);

/*
 * D = (R (x) K_{x,y}) - I (Eq. 1) for images in HOST memory: the end-to-end call of a
 * pipeline whose frames live on the host.  The frame is cut into n_bands row bands
 * (at most 16; boundaries are rounded to the method's block of output rows); band b's
 * rows of I and the rows of R it reads are copied in on an internal stream, the band is
 * computed on `stream` by `method` / `precision` (as svk_difference), and its rows of D
 * are copied out on a second internal stream, so copies overlap computation.
 *   R, I       HOST float32 [H][pitch] (page-locked memory lets the copies overlap the
 *              computation; pageable memory works but serialises them)
 *   D          HOST float32 [H][pitch] (output; written when the stream reaches the end
 *              of this call)
 *   basis, coeffs   DEVICE, as for svk_difference
 *   workspace  device scratch of svk_host_workspace_size() bytes, or NULL / 0 (then
 *              allocated on the stream and released after the call).
 * Asynchronous on `stream`: the call returns once the work is queued; `stream` waits for
 * the last copy, so synchronising it (or an event recorded on it after the call) makes D
 * valid.  Calls from several host threads are serialised while they queue work (the two
 * internal copy streams of a device are shared).
 */
SVK_API int svk_difference_host(const float *R, const float *I, float *D, int W, int H, int pitch,
                                const float *basis, int N, int L, const float *coeffs, int degree, int method,
                                int precision, int n_bands, void *workspace, size_t ws_bytes, void *stream);

/* Bytes of device workspace svk_difference_host_batch needs for these frames: two
 * staging sets, each holding R, I and D of the largest frame and the method's tables
 * (0 on error). */
SVK_API size_t svk_host_batch_workspace_size(const svk_frame *frames, int n_frames, int method, int precision);

/*
 * A sequence of frames whose images live in HOST memory (a night streamed from the
 * host): D_f = (R_f (x) K_f) - I_f (Eq. 1) for every frame, as svk_difference_host does
 * for one, with the frames pipelined: frames alternate between two device staging sets,
 * so frame f+1's copies in and frame f-1's copies out overlap frame f's computation, and
 * within a frame the n_bands row bands are pipelined as in svk_difference_host.
 *   frames     HOST array of n_frames >= 1 descriptors (read during the call): R, I and D
 *              are HOST float32 [H][pitch_*] (page-locked for overlap), basis and coeffs
 *              DEVICE, each frame with its own size, N, L and degree.
 *   workspace  device scratch of svk_host_batch_workspace_size() bytes, or NULL / 0
 *              (then allocated on the stream and released after the call).
 * Asynchronous on `stream` like svk_difference_host: every D is written when the stream
 * reaches the end of the call.  Errors as svk_difference_host, checked for every frame
 * before any work is queued.
 */
SVK_API int svk_difference_host_batch(const svk_frame *frames, int n_frames, int method, int precision, int n_bands,
                                      void *workspace, size_t ws_bytes, void *stream);

/*
 * The library's sticky device status: every bounded device wait that gives up (after
 * ~2 s, e.g. a copy that never lands) records SVK_ERR_TIMEOUT there and its kernel
 * unwinds, so results computed since the last check are invalid.  A library built with
 * SVK_DEBUG also checks shared-memory, tensor-memory and descriptor indices in its
 * kernels and records SVK_ERR_INDEX (the access skipped) instead of trapping.
 * Synchronises `stream`, returns SVK_OK, SVK_ERR_INDEX or SVK_ERR_TIMEOUT, and clears the
 * word when `reset` is non-zero.
 */
SVK_API int svk_device_status(int reset, void *stream);

/*
 * Self-test of the bounded waits of the library's pipelined kernels (failure detection
 * without a fault): one device thread waits on an mbarrier that nothing ever arrives at,
 * with the same bounded wait the kernels use (sleep-hinted try_wait, limit `limit_ns`,
 * 1 us .. 10 s).  The wait gives up, records the timeout in a status word and returns;
 * the call synchronises `stream`, stores the measured wait in *waited_ns (nullable) and
 * returns SVK_ERR_TIMEOUT -- the expected result.  Any other status means the mechanism
 * is broken.  The context stays usable.  Tooling with no counterpart in the paper.
 */
SVK_API int svk_selftest_bounded_wait(unsigned long long limit_ns, unsigned long long *waited_ns, void *stream);

/*
 * Measured multiply-add throughput of the current device, in FLOP/s (2 per FMA), for
 * kind SVK_FMA_FP32 (scalar FP32 FFMA), SVK_FMA_FP64 (FP64 DFMA) or SVK_FMA_FP32X2
 * (packed fma.rn.f32x2, two FP32 multiply-adds per instruction).  These are the
 * denominators of the direct form's roofline (FP32 ALU bound: the larger of the two FP32
 * kinds) and of the fit's normal-equation accumulation (FP64).  Tooling with no
 * counterpart in the paper.  Synchronous: launches one warm-up and one timed kernel
 * (~30 ms) on `stream` and waits for them; allocates a small scratch buffer.  Any other
 * kind: SVK_ERR_ARG.
 *   flops_per_s  host double [1] (output).
 */
#define SVK_FMA_FP32 0
#define SVK_FMA_FP64 1
#define SVK_FMA_FP32X2 2
SVK_API int svk_measure_fma_peak(int kind, double *flops_per_s, void *stream);

/*
 * Bytes of device workspace svk_select_stamps needs for a W x H frame (about 4 bytes
 * per pixel: a peak map and buffers for the largest possible number of peaks).
 */
SVK_API size_t svk_select_workspace_size(int W, int H);

/*
 * Stamp centres for svk_fit_coeffs (Sec. 2: the fit runs over isolated stars; the
 * paper leaves the selection rule open, this is the library's rule):
 *   peak        R(p) - sky >= threshold and R(p) > R(q) for every in-frame 8-neighbour q
 *               (a flat top has no peak);
 *   selectable  margin <= x <= W-1-margin and margin <= y <= H-1-margin, R(p) <
 *               saturation, and no other peak q with max(|dx|, |dy|) <= iso_radius has
 *               R(q) - sky >= iso_frac * (R(p) - sky);
 *   order       R(p) descending, equal values by y*W + x ascending.
 * Differences and products are rounded to float32 one at a time.
 *   R             device float32 [H][pitch]; W * H < 2^31, W, H <= 65535
 *   sky, threshold, saturation   counts (threshold above sky; saturation is a level of R)
 *   margin >= 0, 0 <= iso_radius <= 1024, iso_frac >= 0 (finite)
 *   stamp_xy_out  device int32 [max_stamps][2]: (x, y) of the first selectable peaks in
 *                 the order above (may be NULL when max_stamps == 0); entries past the
 *                 selected count are left untouched
 *   counts_out    device int32 [2]: {number written = min(selectable, max_stamps),
 *                 number of peaks}
 *   workspace     device scratch of svk_select_workspace_size(W, H) bytes, or NULL / 0
 *                 (then allocated on the stream and released after the call).
 * Asynchronous: the counts are known on the device only; the stamp list can be passed to
 * svk_fit_coeffs once the caller has read counts_out[0].
 */
SVK_API int svk_select_stamps(const float *R, int W, int H, int pitch, float sky, float threshold, float saturation,
                              int margin, int iso_radius, float iso_frac, int max_stamps, int *stamp_xy_out,
                              int *counts_out, void *workspace, size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SVK_H */
