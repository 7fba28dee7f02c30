// Entry points of the persistent-kernel instances compiled in separate
// translation units (one per compile-time direction bound).
#pragma once

namespace ftgcr {
const void* persistent_kernel_k4(bool fp64);
const void* persistent_kernel_k8(bool fp64);
const void* persistent_kernel_k16(bool fp64);
inline const void* persistent_kernel_ptr(int kb, bool fp64) {
  if (kb == 4) return persistent_kernel_k4(fp64);
  if (kb == 8) return persistent_kernel_k8(fp64);
  return persistent_kernel_k16(fp64);
}
}  // namespace ftgcr
