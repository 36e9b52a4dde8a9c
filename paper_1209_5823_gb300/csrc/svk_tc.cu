// svk_tc.cu -- tensor-core basis form (placeholder until the tcgen05 path lands).
#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
size_t tc_workspace_size(int, int, int) { return 0; }
int launch_tc(const float *, int, const float *, int, int, int, const float *, int, int, const float *, int, int,
              float *, int, void *, size_t, cudaStream_t) {
  return set_error(SVK_ERR_UNSUPPORTED, "basis method not built yet");
}
}  // namespace svk
