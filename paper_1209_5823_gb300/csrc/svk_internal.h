// svk_internal.h -- launchers behind the C ABI (one translation unit each).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "svk.h"

namespace svk {

// Direct form (svk_direct.cu): kernel of Eq. 2 formed at every output pixel, FP32 FFMA.
// I may be NULL (plain convolution).  Arguments already validated.
// y_begin / y_end: the output rows to compute (-1 = to the last row); band starts must
// be multiples of direct_rows(L), the kernel's block height (12 rows).
// r_begin / r_end: the frame rows R holds (R points at row r_begin; -1 = to the last row);
// rows outside them read as zero (a band of output rows needs rows y_begin - h .. y_end + h - 1).
// I and out are indexed by frame row.
int direct_rows(int L);
int launch_direct(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H,
                  const float *basis, int N, int L, const float *coeffs, int degree, float *out,
                  int pitch_out, cudaStream_t s, int y_begin = 0, int y_end = -1, int r_begin = 0,
                  int r_end = -1);

// T-factored form on the CUDA cores (svk_direct.cu): D = sum_t m_t (R (x) K_t) - I for
// the T in {1, 3, 6, 10} stamps Kt [T][L][L]; bands as for launch_direct, block height
// tform_fp32_rows(L) (16 rows).
int tform_fp32_rows(int L);
int launch_tform_fp32(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H, const float *Kt, int T,
                      int L, float *out, int pitch_out, cudaStream_t s, int y_begin = 0, int y_end = -1,
                      int r_begin = 0, int r_end = -1);

// Basis tabulation (svk_basis.cu).
int launch_round_basis_fp16(float *basis, long long n, cudaStream_t s);
int launch_build_basis(int kind, int L, int n_gauss, const double *sigma, const int *deg,
                       int normalize, float *basis_out, int N, cudaStream_t s);

// Tensor-core basis form (svk_tc.cu).
size_t tc_workspace_size(int precision, int N, int L);
// y_begin / y_end: the output rows to compute (a band of the frame; -1 = to the last
// row); prep = false reuses the tables an earlier call with the same arguments and
// workspace prepared.  Band starts other than 0 must be multiples of
// tc_rows_per_block(N or T, L, precision).
int launch_tc(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H,
              const float *basis, int N, int L, const float *coeffs, int degree, int precision,
              float *out, int pitch_out, void *ws, size_t ws_bytes, cudaStream_t s,
              int y_begin = 0, int y_end = -1, bool prep = true, int r_begin = 0, int r_end = -1);
int tc_rows_per_block(int N, int L, int precision);  // 0 when no plan fits

size_t tform_workspace_size(int precision, int L, int degree);
int launch_tform(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H, const float *basis, int N,
                 int L, const float *coeffs, int degree, int precision, float *out, int pitch_out, void *ws,
                 size_t ws_bytes, cudaStream_t s, int y_begin = 0, int y_end = -1, bool prep = true,
                 int r_begin = 0, int r_end = -1);
int launch_batch(const svk_frame *frames, int n, int precision, void *ws, size_t ws_bytes, cudaStream_t s);
size_t batch_workspace_size(const svk_frame *frames, int n, int precision);
int autotune_tc(int N, int L, int degree, int precision, int W, int H, int *G_out, int *stages_out, cudaStream_t s);
int set_tc_plan(int N, int L, int precision, int G, int stages, int streamed);
int get_tc_plan(int N, int L, int precision, int *G, int *stages, int *streamed);

// Least-squares fit (svk_fit.cu).
size_t fit_workspace_size(int n_stamps, int stamp_size, int N, int L, int degree, int bg_degree);
int launch_fit(const float *R, const float *I, int W, int H, int pitch, const int *stamp_xy,
               int n_stamps, int stamp_size, const float *basis, int N, int L, int degree,
               int bg_degree, const float *weight, double *coeffs_out, double *chi2_out,
               int *info_out, void *ws, size_t ws_bytes, cudaStream_t s);
// The fit in two parts (the moments can be summed over stamp subsets, e.g. over GPUs):
// the FP64 moments S of the stamps' pixels, R / I / weight holding frame rows
// [row_begin, row_end) (pointers at row row_begin; pixels outside them add nothing) ...
size_t fit_moments_count(int N, int degree, int bg_degree);
size_t fit_moments_workspace_size(int n_stamps, int stamp_size, int N);
int launch_fit_moments(const float *R, const float *I, const float *weight, int W, int H, int pitch, int row_begin,
                       int row_end, const int *stamp_xy, int n_stamps, int stamp_size, const float *basis, int N, int L,
                       int degree, int bg_degree, double *moments, bool accumulate, void *ws, size_t ws_bytes,
                       cudaStream_t s);
// ... and the normal equations assembled from S, Cholesky, substitution, chi^2 from S.
size_t fit_solve_workspace_size(int N, int degree, int bg_degree);
int launch_fit_solve(const double *moments, int N, int degree, int bg_degree, double *coeffs_out, double *chi2_out,
                     int *info_out, void *ws, size_t ws_bytes, cudaStream_t s);

// Output-row block of a method (svk_host.cu): band starts are multiples of it (0: no plan).
int band_granule(int method, int precision, int N, int L, int degree);

// The difference image from host buffers, pipelined over row bands (svk_host.cu).
size_t host_workspace_size(int method, int precision, int W, int H, int N, int L, int degree);
int launch_host(const float *R, const float *I, float *D, int W, int H, int pitch, const float *basis, int N, int L,
                const float *coeffs, int degree, int method, int precision, int n_bands, void *ws, size_t ws_bytes,
                cudaStream_t s);
size_t host_batch_workspace_size(const svk_frame *frames, int n, int method, int precision);
int launch_host_batch(const svk_frame *frames, int n, int method, int precision, int n_bands, void *ws,
                      size_t ws_bytes, cudaStream_t s);

// Stamp selection (svk_stamps.cu).
size_t select_workspace_size(int W, int H);
int launch_select(const float *R, int W, int H, int pitch, float sky, float threshold, float saturation, int margin,
                  int iso_radius, float iso_frac, int max_stamps, int *xy, int *counts, void *ws, size_t ws_bytes,
                  cudaStream_t s);

// Self-test of the bounded device waits (svk_selftest.cu); returns SVK_ERR_TIMEOUT when
// the wait gave up as designed.
int selftest_bounded_wait(unsigned long long limit_ns, unsigned long long *waited_ns, cudaStream_t s);

// Measured FMA throughput (svk_peaks.cu).
int measure_fma_peak(int kind, double *flops_per_s, cudaStream_t s);  // SVK_FMA_*

// Coefficient network (svk_cnn.cu).
int cnn_param_count(int n_out);
size_t cnn_workspace_size(int B, int n_out);
int cnn_forward(const float *params, const float *x, int B, int n_out, float *out, void *ws, size_t ws_bytes,
                cudaStream_t s);
int cnn_gradient(const float *params, const float *x, const float *target, int B, int n_out, float *grad, float *loss,
                 void *ws, size_t ws_bytes, cudaStream_t s);
int cnn_adam(float *params, float *m, float *v, const float *grad, int n, int step, float lr, float b1, float b2,
             float eps, cudaStream_t s);
int cnn_adam_device_step(float *params, float *m, float *v, const float *grad, int n, const int *step, float lr,
                         float b1, float b2, float eps, cudaStream_t s);
int cnn_field_fit(const float *local, const int *xy, const float *wts, int S, int N, int W, int H, int degree,
                  double *coeffs, int *info, cudaStream_t s);

// The data side of the coefficient network (svk_learned.cu).
int launch_cut_stamps(const float *img, int W, int H, int pitch, const int *xy, int n, int size, float offset,
                      float divisor, float *out, long long stride, cudaStream_t s);
size_t stamp_residual_workspace_size(int n);
int launch_stamp_residual(const float *D, int W, int H, int pitch, const int *xy, int n, int size, const float *basis0,
                          int L, double noise, double ref_noise, double ratio, const int *field_info, double *out,
                          int *fallback, void *ws, size_t ws_bytes, cudaStream_t s);
int launch_standardise(const float *in, long long rows, int cols, const float *mean, const float *sd, int inverse,
                       float *out, cudaStream_t s);
int launch_draw_batch(unsigned long long seed, const int *step, int n, int batch, long long *idx, cudaStream_t s);
int launch_gather_rows(const void *src, long long row_bytes, const long long *idx, int n, void *dst, cudaStream_t s);
int launch_step_end(const float *loss, int *step, float *hist, int len, cudaStream_t s);

}  // namespace svk
