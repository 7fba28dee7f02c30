// Persistent FT-GCR kernel instance with split rounds (mixed path) for at
// most 8 Krylov directions.
#include "ftgcr_instances.h"
#include "ftgcr_phases.cuh"

namespace ftgcr {
const void* persistent_kernel_k8_split() { return (const void*)k_ftgcr_persistent<float, 8, true>; }
}  // namespace ftgcr
