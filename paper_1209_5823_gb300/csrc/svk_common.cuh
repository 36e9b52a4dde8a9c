// svk_common.cuh -- helpers shared by the SVK CUDA translation units: host-side error
// reporting, tensor-map encoding through the driver entry point, and thin inline-PTX
// wrappers for mbarriers, TMA (cp.async.bulk) and bounded waits.  Written for sm_103a.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "svk.h"

namespace svk {

// ------------------------------------------------------------------ host side
int set_error(int status, const char *fmt, ...);  // records the message, returns status
int cuda_status(cudaError_t e, const char *what); // SVK_OK or SVK_ERR_CUDA with message
const char *last_error();

// 2-D float32 tensor map over an image [H][pitch] with a (box_w x box_h) box, zero fill
// out of bounds.  Returns false when the driver refuses (alignment, sizes).
bool encode_tmap_2d_f32(CUtensorMap *map, const float *base, int W, int H, int pitch,
                        int box_w, int box_h);

// 4-D BF16 tensor map over NHWC activations [B][S][S][32] (64-byte pixels), 64-byte
// swizzle, zero fill out of bounds; the box is 32 channels x box_x x box_y x box_b with
// traversal stride `estride` along x and y.  False when the driver refuses.
bool encode_tmap_nhwc32_bf16(CUtensorMap *map, const void *base, int S, int B, int box_x, int box_y, int box_b,
                             int estride);

// 4-D float32 tensor map over the network's input stamps [B][C][S][S] (rows of S floats),
// no swizzle, zero fill out of bounds; box: S columns x box_y rows x C channels x 1 stamp.
bool encode_tmap_stamps_f32(CUtensorMap *map, const float *base, int S, int C, int B, int box_y);

// Device-memory allocation on a stream for calls that received no workspace.
struct ScopedWorkspace {
  void *ptr = nullptr;
  cudaStream_t stream = nullptr;
  bool owned = false;
  int acquire(size_t bytes, void *user_ws, size_t user_bytes, cudaStream_t s);
  ~ScopedWorkspace();
};

__host__ __device__ inline int n_terms(int d) { return d < 0 ? 0 : (d + 1) * (d + 2) / 2; }

// Device status word written by kernels (0 = fine; bits OR-ed in): a bounded wait that
// gave up, or (debug builds only, SVK_DEBUG) an index check that failed.
enum DeviceStatus : uint32_t { kDevOk = 0, kDevTimeout = 1, kDevIndex = 2 };

// Address of the library's sticky device status word on the current device (the
// kernels' status pointer), or NULL if it cannot be resolved.
uint32_t *device_status_word();

// The driver's id of the calling thread's current context (unique for the life of the
// process), or 0 when there is none or it cannot be read.
unsigned long long current_context_id();

// Device addresses of a file-scope __device__ variable, one per device ordinal, each
// remembered with the context it was looked up in.  In host code such a variable's name
// is only a host-side stand-in, so its device address comes from cudaGetSymbolAddress
// with the device current; it is looked up again whenever the device's current context
// differs from the remembered one (after a cudaDeviceReset, for instance).
struct SymbolAddressCache {
  static constexpr int kMaxDevices = 64;
  std::mutex mu;
  void *addr[kMaxDevices] = {};
  unsigned long long ctx[kMaxDevices] = {};
};
int symbol_address(SymbolAddressCache &cache, const void *symbol, const char *what, void **out);

// ------------------------------------------------------------------ device side
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait with a suspend-time hint: a waiting thread sleeps until the phase completes
// (or the hint expires) instead of spinning, so it leaves issue slots to the warps that
// share its scheduler.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar` for at most `limit_ns` nanoseconds.  On expiry the
// wait records kDevTimeout in *status (if given) and returns false; the caller then
// unwinds without touching the data the barrier guards.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t *status,
                                                  uint64_t limit_ns = 2000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait_sleep(bar, parity, 100000u)) return true;
    if (globaltimer_ns() - t0 > limit_ns) {
      if (status) atomicOr(status, (uint32_t)kDevTimeout);
      return false;
    }
  }
}

// Index checks of the debug build (compiled with -DSVK_DEBUG, see build.py): SVK_CHECK(c, st, id)
// is `c`, and when `c` is false it also records kDevIndex in *st, so the caller skips the
// access it guards and the host learns of it through svk_device_status; a release build
// compiles it to `true` (no check, no cost).  No check traps.
// Each check site has a number (1..23) whose bit 8 + id is OR-ed in beside kDevIndex, so
// the status word names the sites that fired.
#ifdef SVK_DEBUG
__device__ __forceinline__ bool svk_check(bool c, uint32_t *status, int id) {
  if (!c && status) atomicOr(status, (uint32_t)kDevIndex | (1u << (8 + id)));
  return c;
}
#define SVK_CHECK(c, st, id) (::svk::svk_check((c), (st), (id)))
#else
// release builds: always true, the condition never evaluated (it is only named, so the
// values it checks do not read as unused)
#define SVK_CHECK(c, st, id) (true || (c))
#endif

// 2-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// 4-D tiled TMA load of one box into shared memory, completing on `bar` (coordinates
// innermost first; the innermost one must be a multiple of 16 bytes).
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size multiple of 16).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Packed FP32 pairs (low, high) in one 64-bit register: one fma.rn.f32x2 performs two
// independent round-to-nearest FP32 multiply-adds, one per half.
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Programmatic dependent launch.  A kernel launched by launch_dependent() may start while
// the kernel before it in the stream is still running; dep_wait() blocks until that kernel
// has completed and its writes are visible, so a kernel calls it before its first access
// to global memory.  dep_trigger() lets the next such kernel start launching (it still
// waits in its own dep_wait()).  In a kernel launched the ordinary way both are no-ops in
// effect: there is nothing to wait for.
__device__ __forceinline__ void dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch `kernel` on `s` with programmatic stream serialization (see dep_wait); also
// captured into CUDA graphs as a programmatic dependency.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args &&...args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace svk
