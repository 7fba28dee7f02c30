// Persistent FT-GCR kernel instances for at most 8 Krylov directions.
#include "ftgcr_instances.h"
#include "ftgcr_phases.cuh"

namespace ftgcr {
const void* persistent_kernel_k8(bool fp64) {
  return fp64 ? (const void*)k_ftgcr_persistent<double, 8, false> : (const void*)k_ftgcr_persistent<float, 8, false>;
}
}  // namespace ftgcr
