// Persistent FT-GCR kernel instance for wide-row FP64 solves, whose line
// solve reads its factors from global memory, for at most 8 Krylov
// directions.
#include "ftgcr_instances.h"
#include "ftgcr_phases.cuh"

namespace ftgcr {
const void* persistent_kernel_k8_wide64() { return (const void*)k_ftgcr_persistent<double, 8, true>; }
}  // namespace ftgcr
