// Float-float regular-pair assembly (placeholder until the FP32-pipe kernel lands).
#include "fosb_internal.h"

namespace fosb {
cudaError_t launch_efie_regular_ff(const DevMesh&, double, double*, int64_t, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace fosb
