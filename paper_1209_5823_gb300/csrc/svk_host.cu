// svk_host.cu -- the difference image of Eq. 1 from host buffers.
//
// The frame is cut into row bands.  Band b's rows of I and the rows of R it reads (its
// rows plus h halo rows below; the rows above arrived with the earlier bands) are copied
// in on one stream, the band is computed, and its rows of D are copied out on another
// stream, so the copies of one band overlap the computation of its neighbours.  Bands are
// computed alternately on the caller's stream and on a second compute stream, so one
// band's last blocks overlap the next band's first ones instead of idling SMs.  The
// basis tables are prepared once, before the bands.  Events order the streams; the
// caller's stream waits for the last copy, so the whole call is one asynchronous
// operation on it.  Band boundaries are multiples of the kernel's output-row block, so a
// band's blocks never straddle two bands.
#include <mutex>

#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
namespace {

constexpr int kMaxBands = 16;
constexpr int kMaxDevices = 64;

struct HostStreams {
  bool ready = false;
  cudaStream_t h2d = nullptr, d2h = nullptr, comp = nullptr, comp0 = nullptr;
  cudaEvent_t start = nullptr, end = nullptr, in[kMaxBands] = {}, out[kMaxBands] = {};
  // frame pipeline of the batch call: tables ready, compute-stream join, per staging set
  // "computation done" and "copies out done", and the final joins
  cudaEvent_t prep = nullptr, jc = nullptr, comp_done[2] = {}, d2h_done[2] = {}, join[3] = {};
};

std::mutex g_host_mutex;  // held while a call enqueues its work (streams and events are shared)
HostStreams g_host[kMaxDevices];

int host_streams(int dev, HostStreams **hs) {
  if (dev < 0 || dev >= kMaxDevices) return set_error(SVK_ERR_UNSUPPORTED, "device %d out of range", dev);
  HostStreams &h = g_host[dev];
  if (!h.ready) {
    int st = cuda_status(cudaStreamCreateWithFlags(&h.h2d, cudaStreamNonBlocking), "copy-in stream");
    if (st == SVK_OK) st = cuda_status(cudaStreamCreateWithFlags(&h.d2h, cudaStreamNonBlocking), "copy-out stream");
    if (st == SVK_OK) st = cuda_status(cudaStreamCreateWithFlags(&h.comp, cudaStreamNonBlocking), "compute stream");
    if (st == SVK_OK) st = cuda_status(cudaStreamCreateWithFlags(&h.comp0, cudaStreamNonBlocking), "compute stream");
    cudaEvent_t *evs[] = {&h.start, &h.end, &h.prep, &h.jc, &h.comp_done[0], &h.comp_done[1], &h.d2h_done[0],
                          &h.d2h_done[1], &h.join[0], &h.join[1], &h.join[2]};
    for (cudaEvent_t *e : evs)
      if (st == SVK_OK) st = cuda_status(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "event");
    for (int b = 0; b < kMaxBands && st == SVK_OK; ++b) {
      st = cuda_status(cudaEventCreateWithFlags(&h.in[b], cudaEventDisableTiming), "event");
      if (st == SVK_OK) st = cuda_status(cudaEventCreateWithFlags(&h.out[b], cudaEventDisableTiming), "event");
    }
    if (st != SVK_OK) return st;
    h.ready = true;
  }
  *hs = &h;
  return SVK_OK;
}

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

size_t method_ws(int method, int precision, int N, int L, int degree) {
  if (method == SVK_METHOD_BASIS) return tc_workspace_size(precision, N, L);
  if (method == SVK_METHOD_TFORM) return tform_workspace_size(precision, L, degree);
  return 0;
}

// Band boundaries yb[0..nb]: multiples of gran, at most kMaxBands bands, none empty.
int band_bounds(int H, int gran, int n_bands, int *yb) {
  int nb = 0;
  const int want = n_bands < 1 ? 1 : (n_bands > kMaxBands ? kMaxBands : n_bands);
  yb[0] = 0;
  for (int b = 1; b < want; ++b) {
    const int y = (int)((long long)b * H / want) / gran * gran;
    if (y > yb[nb] && y < H) yb[++nb] = y;
  }
  yb[++nb] = H;
  return nb;
}

// One staging set of the batch call: planes R, I, D at fixed offsets, each the size of the
// largest frame (so a frame's R and I never overlap the D plane whose copies out may
// still be running for the set's previous frame), then the method's tables.
void stage_sizes(const svk_frame *fr, int n, int method, int precision, size_t *plane_bytes, size_t *tables_bytes) {
  size_t a = 0, t = 0;
  for (int f = 0; f < n; ++f) {
    const size_t v = up256((size_t)fr[f].W * fr[f].H * sizeof(float));
    const size_t m = up256(method_ws(method, precision, fr[f].N, fr[f].L, fr[f].degree));
    a = v > a ? v : a;
    t = m > t ? m : t;
  }
  *plane_bytes = a;
  *tables_bytes = t;
}

}  // namespace

// Output-row block of the method: band boundaries are multiples of it (0: no plan).
int band_granule(int method, int precision, int N, int L, int degree) {
  if (method == SVK_METHOD_DIRECT) return direct_rows(L);
  if (method == SVK_METHOD_TFORM && precision == SVK_PREC_FP32) return tform_fp32_rows(L);
  return tc_rows_per_block(method == SVK_METHOD_TFORM ? n_terms(degree) : N, L, precision);
}

size_t host_workspace_size(int method, int precision, int W, int H, int N, int L, int degree) {
  return 3 * up256((size_t)W * H * sizeof(float)) + method_ws(method, precision, N, L, degree);
}

size_t host_batch_workspace_size(const svk_frame *fr, int n, int method, int precision) {
  size_t a = 0, t = 0;
  stage_sizes(fr, n, method, precision, &a, &t);
  return 2 * (3 * a + t);
}

// Frames pipelined through two staging sets: frame f uses set f & 1.  Its copies in wait
// only for the computation that last read that set (frame f - 2), its computation for the
// copies out that last read that set's D; so frame f + 1's copies in and frame f - 1's
// copies out run while frame f computes.  Within a frame the bands are pipelined as in
// launch_host, on the two internal compute streams.
int launch_host_batch(const svk_frame *fr, int n, int method, int precision, int n_bands, void *ws, size_t ws_bytes,
                      cudaStream_t s) {
  size_t plane = 0, tb = 0;
  stage_sizes(fr, n, method, precision, &plane, &tb);
  const size_t set_bytes = 3 * plane + tb;
  if (ws_bytes < 2 * set_bytes) return set_error(SVK_ERR_WORKSPACE, "host batch workspace too small");
  int dev = 0;
  int st = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (st != SVK_OK) return st;
  std::lock_guard<std::mutex> lock(g_host_mutex);
  HostStreams *hs = nullptr;
  if ((st = host_streams(dev, &hs)) != SVK_OK) return st;
  if ((st = cuda_status(cudaEventRecord(hs->start, s), "event record")) != SVK_OK) return st;
  auto frames = [&]() -> int {
    int e;
    cudaStream_t all[4] = {hs->h2d, hs->d2h, hs->comp0, hs->comp};
    for (cudaStream_t x : all)
      if ((e = cuda_status(cudaStreamWaitEvent(x, hs->start, 0), "stream wait")) != SVK_OK) return e;
    for (int f = 0; f < n; ++f) {
      const svk_frame &F = fr[f];
      const int k = f & 1, W = F.W, H = F.H, h = (F.L - 1) / 2;
      unsigned char *base = static_cast<unsigned char *>(ws) + (size_t)k * set_bytes;
      float *Rd = reinterpret_cast<float *>(base), *Id = reinterpret_cast<float *>(base + plane);
      float *Dd = reinterpret_cast<float *>(base + 2 * plane);
      void *mws = base + 3 * plane;
      const size_t row = (size_t)W * sizeof(float);
      const int gran = band_granule(method, precision, F.N, F.L, F.degree);
      if (gran < 1) return set_error(SVK_ERR_UNSUPPORTED, "no tensor-core plan for frame %d", f);
      int yb[kMaxBands + 1];
      const int nb = band_bounds(H, gran, n_bands, yb);
      if (f >= 2) {  // staging set k was last used by frame f - 2
        if ((e = cuda_status(cudaStreamWaitEvent(hs->h2d, hs->comp_done[k], 0), "stream wait")) != SVK_OK) return e;
        if ((e = cuda_status(cudaStreamWaitEvent(hs->comp0, hs->d2h_done[k], 0), "stream wait")) != SVK_OK) return e;
      }
      e = SVK_OK;
      if (method == SVK_METHOD_TFORM)  // this frame's tables (a launch over no rows)
        e = launch_tform(Rd, W, Id, W, W, H, F.basis, F.N, F.L, F.coeffs, F.degree, precision, Dd, W, mws, tb,
                         hs->comp0, 0, 0, true);
      else if (method == SVK_METHOD_BASIS)
        e = launch_tc(Rd, W, Id, W, W, H, F.basis, F.N, F.L, F.coeffs, F.degree, precision, Dd, W, mws, tb, hs->comp0,
                      0, 0, true);
      if (e != SVK_OK) return e;
      if ((e = cuda_status(cudaEventRecord(hs->prep, hs->comp0), "event record")) != SVK_OK) return e;
      if ((e = cuda_status(cudaStreamWaitEvent(hs->comp, hs->prep, 0), "stream wait")) != SVK_OK) return e;
      int r_done = 0;
      for (int b = 0; b < nb; ++b) {
        const int y0 = yb[b], y1 = yb[b + 1];
        const int r_need = y1 + h < H ? y1 + h : H;
        if (r_need > r_done) {
          e = cuda_status(cudaMemcpy2DAsync(Rd + (size_t)r_done * W, row, F.R + (size_t)r_done * F.pitch_R,
                                            (size_t)F.pitch_R * sizeof(float), row, (size_t)(r_need - r_done),
                                            cudaMemcpyHostToDevice, hs->h2d),
                          "copy R in");
          if (e != SVK_OK) return e;
          r_done = r_need;
        }
        e = cuda_status(cudaMemcpy2DAsync(Id + (size_t)y0 * W, row, F.I + (size_t)y0 * F.pitch_I,
                                          (size_t)F.pitch_I * sizeof(float), row, (size_t)(y1 - y0),
                                          cudaMemcpyHostToDevice, hs->h2d),
                        "copy I in");
        if (e != SVK_OK) return e;
        if ((e = cuda_status(cudaEventRecord(hs->in[b], hs->h2d), "event record")) != SVK_OK) return e;
        cudaStream_t cs = (b & 1) ? hs->comp : hs->comp0;
        if ((e = cuda_status(cudaStreamWaitEvent(cs, hs->in[b], 0), "stream wait")) != SVK_OK) return e;
        if (method == SVK_METHOD_DIRECT)
          e = launch_direct(Rd, W, Id, W, W, H, F.basis, F.N, F.L, F.coeffs, F.degree, Dd, W, cs, y0, y1);
        else if (method == SVK_METHOD_TFORM)
          e = launch_tform(Rd, W, Id, W, W, H, F.basis, F.N, F.L, F.coeffs, F.degree, precision, Dd, W, mws, tb, cs,
                           y0, y1, false);
        else
          e = launch_tc(Rd, W, Id, W, W, H, F.basis, F.N, F.L, F.coeffs, F.degree, precision, Dd, W, mws, tb, cs, y0,
                        y1, false);
        if (e != SVK_OK) return e;
        if ((e = cuda_status(cudaEventRecord(hs->out[b], cs), "event record")) != SVK_OK) return e;
        if ((e = cuda_status(cudaStreamWaitEvent(hs->d2h, hs->out[b], 0), "stream wait")) != SVK_OK) return e;
        e = cuda_status(cudaMemcpy2DAsync(F.D + (size_t)y0 * F.pitch_D, (size_t)F.pitch_D * sizeof(float),
                                          Dd + (size_t)y0 * W, row, row, (size_t)(y1 - y0), cudaMemcpyDeviceToHost,
                                          hs->d2h),
                        "copy D out");
        if (e != SVK_OK) return e;
      }
      // frame end: both compute streams done -> comp_done[k]; its copies out -> d2h_done[k]
      if ((e = cuda_status(cudaEventRecord(hs->jc, hs->comp), "event record")) != SVK_OK) return e;
      if ((e = cuda_status(cudaStreamWaitEvent(hs->comp0, hs->jc, 0), "stream wait")) != SVK_OK) return e;
      if ((e = cuda_status(cudaEventRecord(hs->comp_done[k], hs->comp0), "event record")) != SVK_OK) return e;
      if ((e = cuda_status(cudaEventRecord(hs->d2h_done[k], hs->d2h), "event record")) != SVK_OK) return e;
    }
    return SVK_OK;
  };
  st = frames();
  // join every internal stream into the caller's stream, whatever happened above
  cudaEventRecord(hs->join[0], hs->h2d);
  cudaEventRecord(hs->join[1], hs->comp);
  cudaEventRecord(hs->join[2], hs->comp0);
  cudaEventRecord(hs->end, hs->d2h);
  cudaStreamWaitEvent(s, hs->join[0], 0);
  cudaStreamWaitEvent(s, hs->join[1], 0);
  cudaStreamWaitEvent(s, hs->join[2], 0);
  const int jst = cuda_status(cudaStreamWaitEvent(s, hs->end, 0), "stream join");
  return st != SVK_OK ? st : jst;
}


int launch_host(const float *R, const float *I, float *D, int W, int H, int pitch, const float *basis, int N, int L,
                const float *coeffs, int degree, int method, int precision, int n_bands, void *ws, size_t ws_bytes,
                cudaStream_t s) {
  const int h = (L - 1) / 2;
  const int gran = band_granule(method, precision, N, L, degree);
  if (gran < 1) return set_error(SVK_ERR_UNSUPPORTED, "no tensor-core plan for N=%d L=%d", N, L);
  int yb[kMaxBands + 1];
  const int nb = band_bounds(H, gran, n_bands, yb);

  const size_t frame = up256((size_t)W * H * sizeof(float));
  unsigned char *w = static_cast<unsigned char *>(ws);
  float *Rd = reinterpret_cast<float *>(w), *Id = reinterpret_cast<float *>(w + frame);
  float *Dd = reinterpret_cast<float *>(w + 2 * frame);
  void *mws = w + 3 * frame;
  const size_t mws_bytes = ws_bytes - 3 * frame;
  const size_t row = (size_t)W * sizeof(float), hrow = (size_t)pitch * sizeof(float);

  int dev = 0;
  int st = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (st != SVK_OK) return st;
  std::lock_guard<std::mutex> lock(g_host_mutex);
  HostStreams *hs = nullptr;
  if ((st = host_streams(dev, &hs)) != SVK_OK) return st;
  // the copies start after the caller's earlier work on its stream (the workspace may be
  // in use there); the tables are prepared there first (a launch over no rows)
  if (method == SVK_METHOD_TFORM)
    st = launch_tform(Rd, W, Id, W, W, H, basis, N, L, coeffs, degree, precision, Dd, W, mws, mws_bytes, s, 0, 0, true);
  else if (method == SVK_METHOD_BASIS)
    st = launch_tc(Rd, W, Id, W, W, H, basis, N, L, coeffs, degree, precision, Dd, W, mws, mws_bytes, s, 0, 0, true);
  if (st != SVK_OK) return st;
  if ((st = cuda_status(cudaEventRecord(hs->start, s), "event record")) != SVK_OK) return st;
  // Queue the bands; whatever happens, the caller's stream then waits for all three
  // internal streams, so nothing queued on them outlives the call's stream order (the
  // workspace may be released on `s` right after it).
  auto bands = [&]() -> int {
    int e;
    if ((e = cuda_status(cudaStreamWaitEvent(hs->h2d, hs->start, 0), "stream wait")) != SVK_OK) return e;
    if ((e = cuda_status(cudaStreamWaitEvent(hs->d2h, hs->start, 0), "stream wait")) != SVK_OK) return e;
    if ((e = cuda_status(cudaStreamWaitEvent(hs->comp, hs->start, 0), "stream wait")) != SVK_OK) return e;
    int r_done = 0;  // rows of R already on their way
    for (int b = 0; b < nb; ++b) {
      const int y0 = yb[b], y1 = yb[b + 1];
      const int r_need = y1 + h < H ? y1 + h : H;
      if (r_need > r_done) {
        e = cuda_status(cudaMemcpy2DAsync(Rd + (size_t)r_done * W, row, R + (size_t)r_done * pitch, hrow, row,
                                          (size_t)(r_need - r_done), cudaMemcpyHostToDevice, hs->h2d),
                        "copy R in");
        if (e != SVK_OK) return e;
        r_done = r_need;
      }
      e = cuda_status(cudaMemcpy2DAsync(Id + (size_t)y0 * W, row, I + (size_t)y0 * pitch, hrow, row,
                                        (size_t)(y1 - y0), cudaMemcpyHostToDevice, hs->h2d),
                      "copy I in");
      if (e != SVK_OK) return e;
      if ((e = cuda_status(cudaEventRecord(hs->in[b], hs->h2d), "event record")) != SVK_OK) return e;
      cudaStream_t cs = (b & 1) ? hs->comp : s;
      if ((e = cuda_status(cudaStreamWaitEvent(cs, hs->in[b], 0), "stream wait")) != SVK_OK) return e;
      if (method == SVK_METHOD_DIRECT)
        e = launch_direct(Rd, W, Id, W, W, H, basis, N, L, coeffs, degree, Dd, W, cs, y0, y1);
      else if (method == SVK_METHOD_TFORM)
        e = launch_tform(Rd, W, Id, W, W, H, basis, N, L, coeffs, degree, precision, Dd, W, mws, mws_bytes, cs, y0,
                         y1, false);
      else
        e = launch_tc(Rd, W, Id, W, W, H, basis, N, L, coeffs, degree, precision, Dd, W, mws, mws_bytes, cs, y0, y1,
                      false);
      if (e != SVK_OK) return e;
      if ((e = cuda_status(cudaEventRecord(hs->out[b], cs), "event record")) != SVK_OK) return e;
      if ((e = cuda_status(cudaStreamWaitEvent(hs->d2h, hs->out[b], 0), "stream wait")) != SVK_OK) return e;
      e = cuda_status(cudaMemcpy2DAsync(D + (size_t)y0 * pitch, hrow, Dd + (size_t)y0 * W, row, row,
                                        (size_t)(y1 - y0), cudaMemcpyDeviceToHost, hs->d2h),
                      "copy D out");
      if (e != SVK_OK) return e;
    }
    return SVK_OK;
  };
  st = bands();
  // join (the events' earlier waits were captured when they were queued, so re-recording
  // them here is safe)
  cudaEventRecord(hs->in[0], hs->h2d);
  cudaEventRecord(hs->out[0], hs->comp);
  cudaEventRecord(hs->end, hs->d2h);
  cudaStreamWaitEvent(s, hs->in[0], 0);
  cudaStreamWaitEvent(s, hs->out[0], 0);
  const int jst = cuda_status(cudaStreamWaitEvent(s, hs->end, 0), "stream join");
  return st != SVK_OK ? st : jst;
}

}  // namespace svk
