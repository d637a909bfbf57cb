// Device-side bounds checks of the checked build (compiled with
// -DVECKM_CHECKED; build.build(checked=True) writes libveckm_checked.so).
//
// VK_CHECK(cond) guards an access whose index the kernel computed from data
// (a pixel from the sorted records, a slot from an atomic counter, a bucket
// from an event): in the checked build a false condition is counted in a
// device word of the translation unit, the line of the first one is kept,
// and the caller skips the access; in the normal build VK_CHECK is `true`
// and compiles away.  veckm_debug_checks() reads and clears the words of
// every translation unit.  This stands in for a memory checker: it reports
// an index that would have left its buffer instead of letting the access
// happen.
#pragma once
#include <cuda_runtime.h>

#ifdef VECKM_CHECKED
namespace veckm {
namespace {
// [0]: violations, [1]: source line of the first
__device__ int g_check[2];

__device__ __noinline__ bool check_fail(int line) {
  if (atomicAdd(&g_check[0], 1) == 0) g_check[1] = line;
  return false;
}
}  // namespace
}  // namespace veckm
#define VK_CHECK(cond) ((cond) ? true : ::veckm::check_fail(__LINE__))
// Host reader of this translation unit's words: the violation count (and the
// first line in *line), then both are cleared; -1 if reading failed.
#define VK_CHECK_READER(name)                                                        \
  int name(int *line) {                                                              \
    int h[2] = {0, 0};                                                               \
    if (cudaMemcpyFromSymbol(h, ::veckm::g_check, sizeof(h)) != cudaSuccess) return -1; \
    const int z[2] = {0, 0};                                                         \
    if (cudaMemcpyToSymbol(::veckm::g_check, z, sizeof(z)) != cudaSuccess) return -1;   \
    if (line) *line = h[1];                                                          \
    return h[0];                                                                     \
  }
#else
#define VK_CHECK(cond) true
#define VK_CHECK_READER(name) \
  int name(int *line) {       \
    if (line) *line = 0;      \
    return 0;                 \
  }
#endif
