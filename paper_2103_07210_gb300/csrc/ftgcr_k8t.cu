// Persistent FT-GCR kernel instance with streamed step rounds (mixed path,
// HBM-resident solves) beside the split rounds, for at most 8 Krylov
// directions.
#include "ftgcr_instances.h"
#include "ftgcr_phases.cuh"

namespace ftgcr {
const void* persistent_kernel_k8_stream() { return (const void*)k_ftgcr_persistent<float, 8, 2>; }
}  // namespace ftgcr
