// Entry points of the persistent-kernel instances compiled in separate
// translation units (one per compile-time direction bound and round layout).
#pragma once

namespace ftgcr {
const void* persistent_kernel_k4(bool fp64);
const void* persistent_kernel_k8(bool fp64);
const void* persistent_kernel_k16(bool fp64);
const void* persistent_kernel_k4_split();
const void* persistent_kernel_k8_split();
const void* persistent_kernel_k16_split();
const void* persistent_kernel_k4_wide64();
const void* persistent_kernel_k8_wide64();
const void* persistent_kernel_k16_wide64();
const void* persistent_kernel_k4_stream();
const void* persistent_kernel_k8_stream();
const void* persistent_kernel_k16_stream();
// wide 1: the instance for wide-row solves (mixed path: split rounds; FP64
// path: line-solve factors read from global memory); wide 2 (mixed path): the
// split-round instance with the streamed step rounds
inline const void* persistent_kernel_ptr(int kb, bool fp64, int wide) {
  if (wide == 2 && !fp64) {
    if (kb == 4) return persistent_kernel_k4_stream();
    if (kb == 8) return persistent_kernel_k8_stream();
    return persistent_kernel_k16_stream();
  }
  if (wide && !fp64) {
    if (kb == 4) return persistent_kernel_k4_split();
    if (kb == 8) return persistent_kernel_k8_split();
    return persistent_kernel_k16_split();
  }
  if (wide) {
    if (kb == 4) return persistent_kernel_k4_wide64();
    if (kb == 8) return persistent_kernel_k8_wide64();
    return persistent_kernel_k16_wide64();
  }
  if (kb == 4) return persistent_kernel_k4(fp64);
  if (kb == 8) return persistent_kernel_k8(fp64);
  return persistent_kernel_k16(fp64);
}
}  // namespace ftgcr
