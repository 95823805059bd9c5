// rac_enforce_noalloc: rac_enforce for callers that cannot allocate device
// memory at call time.
//
// Some callers of this library cannot call cudaMalloc when they enforce:
// processes whose device memory is entirely reserved by another allocator
// (a framework's caching pool that holds the whole card, so a direct
// cudaMalloc fails or fragments it), and latency-bound loops that cannot
// absorb the device-wide synchronisation cudaMalloc and cudaFree may imply.
// This entry point takes its scratch from one fixed array compiled into the
// library instead of from a per-stream workspace, so it allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kScratchWords words = 311,808 bytes, about 305 KiB) until
// the process exits.  All calls share it and it keeps the previous call's
// contents, so each call first resets, on its stream, what the kernel
// expects: the sync words (including the sticky error word) and flag slots
// to zero and the scratch domain buffer to all ones (cudaMemsetAsync, which
// allocates nothing).  Because the error word is cleared too, a call whose
// bounded wait ran out does not poison the next one, unlike the per-stream
// workspace of rac_enforce.  Two calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on the array and give
// undefined results.
//
// Host code must not use the array's name as a device address: in host code
// it is a stand-in.  The first call on each device, with that device current,
// looks the real address up with cudaGetSymbolAddress and keeps it; that
// first call should come before any stream capture.  Only the bit-packed
// kernel runs here (RAC_KERNEL_TENSOR is refused with RAC_ENOTSUP).
#include <mutex>
#include <string>

#include "rac_internal.h"

namespace rac {
namespace {

constexpr int kNoallocMaxVars = RAC_NOALLOC_MAX_VARS;
constexpr int kNoallocMaxBlocks = (kNoallocMaxVars + 31) / 32;
// word layout: [0, 64) sync words | any[3] wipe[3] | chg[3][nb] | chgU[3][nb] | pad | bufB[n]
constexpr int kSyncWords = 64;
constexpr int kFlagWords = 6 + 6 * kNoallocMaxBlocks;
constexpr int kBufOffset = ((kSyncWords + kFlagWords + 63) / 64) * 64;
constexpr int kScratchWords = kBufOffset + kNoallocMaxVars;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];
static_assert(sizeof(g_noalloc_scratch) == 311808, "the documented size of the scratch array");
static_assert(sizeof(Sync) <= kSyncWords * sizeof(uint32_t), "the sync words fit their slot");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
uint32_t *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device).
rac_status scratch_on_current_device(uint32_t **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "rac_enforce_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("rac_enforce_noalloc: device ordinal out of range");
    return RAC_ENOTSUP;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return cuda_fail(e, "rac_enforce_noalloc: cudaGetSymbolAddress of the scratch array");
    g_scratch_ptr[dev] = static_cast<uint32_t *>(p);
  }
  *out = g_scratch_ptr[dev];
  return RAC_OK;
}

}  // namespace
}  // namespace rac

using namespace rac;

extern "C" rac_status rac_enforce_noalloc(const rac_network *net, const uint32_t *dom_in,
                                          uint32_t *dom_out, int32_t *iterations,
                                          int32_t *status, int32_t max_sweeps, uint32_t flags,
                                          rac_stream_t stream) try {
  set_error("");
  if (!net || !dom_in || !dom_out || !iterations || !status) {
    set_error("rac_enforce_noalloc: NULL argument");
    return RAC_EINVAL;
  }
  if (flags & RAC_KERNEL_TENSOR) {
    set_error("rac_enforce_noalloc: only the bit-packed kernel runs without allocation "
              "(RAC_KERNEL_TENSOR needs rac_enforce)");
    return RAC_ENOTSUP;
  }
  if (flags & ~uint32_t(RAC_STOP_ON_WIPEOUT | RAC_INCREMENTAL | RAC_TEST_WITHHOLD_ARRIVAL)) {
    set_error("rac_enforce_noalloc: unknown flag");
    return RAC_EINVAL;
  }
  if (net->n > kNoallocMaxVars) {
    set_error("rac_enforce_noalloc: the network has " + std::to_string(net->n) +
              " variables; the static scratch array holds at most " +
              std::to_string(kNoallocMaxVars) + " (use rac_enforce)");
    return RAC_EINVAL;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "rac_enforce_noalloc: cudaGetDevice");
  if (dev != net->device) {
    set_error("rac_enforce_noalloc: the current CUDA device is not the network's device");
    return RAC_EINVAL;
  }
  uint32_t *scratch = nullptr;
  rac_status rc = scratch_on_current_device(&scratch);
  if (rc != RAC_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  LaunchParams P = {};
  P.net = net_dev(net);
  P.n_states = 1;
  P.contiguous = 1;
  P.dom_in = dom_in;
  P.dom_out = dom_out;
  P.iterations = iterations;
  P.status = status;
  P.sync = reinterpret_cast<Sync *>(scratch);
  P.any = scratch + kSyncWords;
  P.wipe = P.any + 3;
  P.chg = P.wipe + 3;
  P.chgU = P.chg + 3 * size_t(net->nb);
  P.bufB = scratch + kBufOffset;
  P.flag_stride = 1;
  P.max_sweeps = max_sweeps;
  const int64_t bound = int64_t(net->n) * net->d + 2;
  P.sweep_bound = int32_t(bound < 0xFFFFF0 ? bound : 0xFFFFF0);
  P.flags = flags;
  P.wait_limit_ns = wait_limit_for(flags);
  P.seed_var = -1;
  P.seed_keep = 0xFFFFFFFFu;
  P.n_first = int32_t(net->first.size() < size_t(kMaxFirst) ? net->first.size() : kMaxFirst);
  for (int32_t i = 0; i < P.n_first; ++i) P.first[i] = net->first[size_t(i)];
  // what the kernel expects to find: sync words and flags zero, the scratch
  // domain buffer all ones (a previous call may have left anything there)
  e = cudaMemsetAsync(scratch, 0, size_t(kBufOffset) * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.bufB, 0xFF, size_t(net->n) * sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "rac_enforce_noalloc: resetting the scratch array");
  return launch_bits(P, s);
} RAC_CATCH_STATUS
