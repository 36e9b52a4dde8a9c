// svk_noalloc.cu -- svk_difference_noalloc: the tensor-core difference image for callers
// that cannot allocate device memory.
//
// Who needs it: programs whose device memory is owned by someone else -- a host
// application or framework that reserves the whole GPU heap at start-up and forbids
// cudaMalloc afterwards, a real-time survey pipeline that must not allocate (and so
// cannot fail an allocation) once observing has started, or a caller whose own API has
// no place to pass a workspace.  svk_difference either takes a caller workspace or
// allocates one on the stream; this entry point does neither.
//
// Its scratch is one file-scope __device__ array of kNoAllocScratchBytes (512 KiB).
// Every GPU that loads this library holds that array until the process exits.  The
// tensor-core path keeps its basis tables in shared memory, so no plan's workspace can
// exceed it; a request that would is rejected with SVK_ERR_WORKSPACE.  All calls share
// the array and it keeps the last call's contents: calls that overlap on the GPU (two
// streams, or two host threads) race on it and must be serialised by the caller.
#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
namespace {

constexpr size_t kNoAllocScratchBytes = 512 * 1024;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

SymbolAddressCache g_scratch_addr;

// Device address of the scratch array on the current device.  In host code the array's
// name is only a host-side stand-in, so its address is looked up with the device current
// (the first call on a device, and again after that device's context was replaced) and
// cached per device.
int scratch_address(void **out) {
  return symbol_address(g_scratch_addr, reinterpret_cast<const void *>(g_noalloc_scratch),
                        "cudaGetSymbolAddress(no-allocation scratch)", out);
}

}  // namespace
}  // namespace svk

extern "C" int svk_difference_noalloc(const float *R, int pitch_R, const float *I, int pitch_I, int W, int H,
                                      const float *basis, int N, int L, const float *coeffs, int degree,
                                      int precision, int edge, float *D, int pitch_D, void *stream) {
  using namespace svk;
  if (precision != SVK_PREC_BF16X3 && precision != SVK_PREC_FP16X3 && precision != SVK_PREC_BF16 &&
      precision != SVK_PREC_FP16X2)
    return set_error(SVK_ERR_UNSUPPORTED, "svk_difference_noalloc runs the tensor-core basis form only (precision %d)",
                     precision);
  const size_t need = svk_workspace_size(SVK_METHOD_BASIS, precision, W, H, N, L, degree);
  if (need > kNoAllocScratchBytes)
    return set_error(SVK_ERR_WORKSPACE, "request needs %zu bytes of scratch; the no-allocation scratch holds %zu",
                     need, kNoAllocScratchBytes);
  void *scratch = nullptr;
  int st = scratch_address(&scratch);
  if (st != SVK_OK) return st;
  // the caller-workspace path of svk_difference: the status word it clears and the
  // basis tables it rewrites on every call are all this entry point's state
  return svk_difference(R, pitch_R, I, pitch_I, W, H, basis, N, L, coeffs, degree, SVK_METHOD_BASIS, precision, edge,
                        D, pitch_D, scratch, kNoAllocScratchBytes, stream);
}
