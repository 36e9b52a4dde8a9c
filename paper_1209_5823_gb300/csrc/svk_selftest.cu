// svk_selftest.cu -- self-test of the bounded device waits that every pipelined kernel of
// the library uses (mbar_wait_bounded): one thread waits on an mbarrier that nothing ever
// arrives at.  The wait must give up after its limit, record the timeout in the status
// word and return, leaving the context usable.  No fault, trap or endless loop is involved.
#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
namespace {

__global__ void wait_for_nothing_kernel(unsigned long long limit_ns, uint32_t *status, unsigned long long *waited) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);  // expects one arrival; none comes
  fence_mbar_init();
  const uint64_t t0 = globaltimer_ns();
  const bool done = mbar_wait_bounded(&bar, 0, status, limit_ns);
  *waited = globaltimer_ns() - t0;
  if (done) *status = 0xFFFFFFFFu;  // the phase completed: impossible without an arrival
}

}  // namespace

int selftest_bounded_wait(unsigned long long limit_ns, unsigned long long *waited_ns, cudaStream_t s) {
  ScopedWorkspace w;
  int st = w.acquire(16, nullptr, 0, s);
  if (st != SVK_OK) return st;
  uint32_t *status = static_cast<uint32_t *>(w.ptr);
  unsigned long long *waited = reinterpret_cast<unsigned long long *>(static_cast<unsigned char *>(w.ptr) + 8);
  if ((st = cuda_status(cudaMemsetAsync(w.ptr, 0, 16, s), "status reset")) != SVK_OK) return st;
  wait_for_nothing_kernel<<<1, 32, 0, s>>>(limit_ns, status, waited);
  if ((st = cuda_status(cudaGetLastError(), "self-test launch")) != SVK_OK) return st;
  uint32_t hs = 0;
  unsigned long long hw = 0;
  if ((st = cuda_status(cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, s), "read status")) != SVK_OK) return st;
  if ((st = cuda_status(cudaMemcpyAsync(&hw, waited, 8, cudaMemcpyDeviceToHost, s), "read time")) != SVK_OK) return st;
  if ((st = cuda_status(cudaStreamSynchronize(s), "self-test sync")) != SVK_OK) return st;
  if (waited_ns) *waited_ns = hw;
  if (hs == kDevTimeout)
    return set_error(SVK_ERR_TIMEOUT, "bounded wait gave up after %llu ns (limit %llu ns)", hw, limit_ns);
  return set_error(SVK_ERR_CUDA, "bounded-wait self-test: unexpected status 0x%x", hs);
}

}  // namespace svk
