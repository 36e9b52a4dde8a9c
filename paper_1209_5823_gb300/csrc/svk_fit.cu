// svk_fit.cu -- least-squares fit (placeholder).
#include "svk_common.cuh"
#include "svk_internal.h"

namespace svk {
size_t fit_workspace_size(int, int, int, int, int, int) { return 0; }
int launch_fit(const float *, const float *, int, int, int, const int *, int, int, const float *, int, int, int,
               int, const float *, double *, double *, int *, void *, size_t, cudaStream_t) {
  return set_error(SVK_ERR_UNSUPPORTED, "fit not built yet");
}
}  // namespace svk
