// The combine step of the partitioned sweep (Sec. 3, Eq. 1 with its
// constraints split over ranks): every rank's one-sweep partial next domain
// is D^(k-1) AND the supports on its share of C_x, so D^(k) is the AND of the
// partials, and the loop's two decisions (a domain changed, a domain is
// empty: Algorithm 1's #Vals comparison and wipe-out test) are read off the
// combined words.
#include <string>

#include "rac_internal.h"

namespace rac {
namespace {

__global__ void __launch_bounds__(256) rac_combine_kernel(const uint32_t *__restrict__ parts,
                                                          int32_t n_parts, int64_t n,
                                                          const uint32_t *prev, uint32_t *next,
                                                          int32_t *flags) {
  bool changed = false, empty = false;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < n; x += stride) {
    const uint32_t p = prev[x];
    uint32_t w = p;
    for (int32_t g = 0; g < n_parts; ++g) w &= __ldg(parts + g * n + x);
    next[x] = w;
    changed |= w != p;
    empty |= w == 0u;
  }
  const bool c = __any_sync(0xffffffffu, changed);
  const bool e = __any_sync(0xffffffffu, empty);
  if ((threadIdx.x & 31) == 0) {
    if (c) atomicOr(flags, 1);
    if (e) atomicOr(flags + 1, 1);
  }
}

}  // namespace
}  // namespace rac

using namespace rac;

extern "C" rac_status rac_combine_partials(int32_t n_parts, int32_t n_vars,
                                           const uint32_t *partials, const uint32_t *dom_prev,
                                           uint32_t *dom_next, int32_t *flags,
                                           rac_stream_t stream) try {
  set_error("");
  if (n_parts < 1 || n_vars < 0) {
    set_error("rac_combine_partials: need n_parts >= 1 and n_vars >= 0");
    return RAC_EINVAL;
  }
  if (!flags || (n_vars > 0 && (!partials || !dom_prev || !dom_next))) {
    set_error("rac_combine_partials: NULL argument");
    return RAC_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(flags, 0, 2 * sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "rac_combine_partials: clearing the flags");
  if (n_vars == 0) return RAC_OK;
  // n_vars words per part: a few thousand CTAs of 256 threads at most
  const int64_t blocks = (int64_t(n_vars) + 255) / 256;
  const unsigned grid = unsigned(blocks < 4096 ? blocks : 4096);
  rac_combine_kernel<<<grid, 256, 0, s>>>(partials, n_parts, int64_t(n_vars), dom_prev, dom_next,
                                          flags);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rac_combine_partials: launch");
  return RAC_OK;
} RAC_CATCH_STATUS
