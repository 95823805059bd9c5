// rac_search: the backtrack search of Algorithm 2 driven by a host loop
// inside the library.  Every assignment is one launch of the bit-packed
// kernel seeded with the assigned variable (Proposition 2, as
// rac_assign_enforce); the kernel writes the child state, its sweep count
// and status straight into pinned host memory and then a completion number
// (the instance the host entry point uses), so the loop waits on that word
// and never synchronises the stream.  The levels' states stay on the device;
// the host keeps a copy of each for the variable choice.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <string>
#include <vector>

#include "rac_internal.h"

namespace rac {
namespace {

// Smallest domain of size > 1, lowest index; -1 when all are singletons.
int choose_variable(const uint32_t *dom, int n) {
  int best = -1, best_size = 33;
  for (int x = 0; x < n; ++x) {
    const int size = __builtin_popcount(dom[x]);
    if (size > 1 && size < best_size) {
      best = x;
      best_size = size;
    }
  }
  return best;
}

struct SearchBuffers {
  // device, n words per level (level k: the state after k assignments), in
  // blocks of levels allocated as the search deepens
  std::vector<uint32_t *> blocks;
  std::vector<uint32_t *> levels;
  int32_t *res = nullptr;   // device: iterations, status
  uint32_t *pin = nullptr;  // pinned host: n words, iterations, status, completion
  uint32_t *pin_dev = nullptr;
  ~SearchBuffers() {
    for (uint32_t *p : blocks) cudaFree(p);
    cudaFree(res);
    cudaFreeHost(pin);
  }
};

}  // namespace
}  // namespace rac

using namespace rac;

extern "C" rac_status rac_search(const rac_network *net, const uint32_t *dom0, int64_t max_nodes,
                                 uint32_t flags, rac_stream_t stream, uint32_t *solution,
                                 int32_t *found, int32_t *exhausted, int64_t *nodes,
                                 int32_t *root, int32_t *steps, int64_t step_cap) try {
  set_error("");
  if (!net || !dom0 || !solution || !found || !exhausted || !nodes || !root ||
      max_nodes < 0 || step_cap < 0 || (step_cap > 0 && !steps)) {
    set_error("rac_search: NULL argument or negative count");
    return RAC_EINVAL;
  }
  if (flags & ~uint32_t(RAC_STOP_ON_WIPEOUT | RAC_INCREMENTAL)) {
    set_error("rac_search: unknown flag (it takes RAC_STOP_ON_WIPEOUT, RAC_INCREMENTAL)");
    return RAC_EINVAL;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "rac_search: cudaGetDevice");
  if (dev != net->device) {
    set_error("rac_search: the current CUDA device is not the network's device");
    return RAC_EINVAL;
  }
  *found = 0;
  *exhausted = 0;
  *nodes = 0;
  const int n = net->n;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  rac_status rc = RAC_OK;
  Workspace *w = get_workspace(net, s, 1, 0, &rc);
  if (!w) return rc;

  SearchBuffers buf;
  const size_t words = size_t(n);
  // levels come in blocks (the first of up to 64 MiB, then doubling), so the
  // loop seldom allocates (an allocation waits for the device)
  auto level_buffer = [&](size_t k) -> uint32_t * {
    while (buf.levels.size() <= k) {
      const size_t have = buf.levels.size();
      size_t count = have ? have : std::max<size_t>(1, (size_t(64) << 20) / (words * 4 + 1));
      count = std::min(count, size_t(n) + 1 - std::min(have, size_t(n)));
      count = std::max<size_t>(count, 1);
      uint32_t *p = nullptr;
      if (cudaMalloc(&p, count * words * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      buf.blocks.push_back(p);
      for (size_t i = 0; i < count; ++i) buf.levels.push_back(p + i * words);
    }
    return buf.levels[k];
  };
  void *pd = nullptr;
  if (!level_buffer(0) || cudaMalloc(&buf.res, 2 * sizeof(int32_t)) != cudaSuccess ||
      cudaMallocHost(&buf.pin, (words + 3) * sizeof(uint32_t)) != cudaSuccess ||
      cudaHostGetDevicePointer(&pd, buf.pin, 0) != cudaSuccess) {
    cudaGetLastError();
    set_error("rac_search: out of memory for the search buffers");
    return RAC_ENOMEM;
  }
  buf.pin_dev = static_cast<uint32_t *>(pd);
  volatile uint32_t *done = buf.pin + words + 2;
  *done = w->host_seq;  // the number of launches with host results this workspace completed

  // One launch (the root's full enforcement, or an assignment's seeded one)
  // with its results in the pinned buffer; waits for its completion word.
  auto run = [&](const uint32_t *in, uint32_t *out, int var, int value) -> rac_status {
    LaunchParams P = base_params(net, w, 1, 0, flags);
    P.contiguous = 1;
    P.dom_in = in;
    P.dom_out = out;
    P.iterations = buf.res;
    P.status = buf.res + 1;
    P.host_out = buf.pin_dev;
    P.host_done = buf.pin_dev + words + 2;
    if (var >= 0) {
      P.seed_var = var;
      P.seed_keep = 1u << value;
    }
    rac_status r = launch_bits(P, s);
    if (r != RAC_OK) return r;
    const uint32_t want = w->host_seq + 1u;
    const auto t0 = std::chrono::steady_clock::now();
    const auto limit = std::chrono::nanoseconds(2 * wait_limit_for(flags) + 1000000000ull);
    bool seen = false;
    for (uint32_t i = 0;; ++i) {
      if (*done == want) {
        seen = true;
        break;
      }
      if ((i & 255u) == 0u && std::chrono::steady_clock::now() - t0 > limit) break;
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    if (!seen) {
      const cudaError_t er = cudaStreamSynchronize(s);
      if (er != cudaSuccess) return cuda_fail(er, "rac_search: cudaStreamSynchronize");
    }
    w->host_seq = *done;
    return RAC_OK;
  };
  const int32_t *pin_res = reinterpret_cast<const int32_t *>(buf.pin + words);

  // the root: tensorAC(Vars, all)
  e = cudaMemcpyAsync(buf.levels[0], dom0, words * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "rac_search: copy of the initial domains");
  if ((rc = run(buf.levels[0], buf.levels[0], -1, 0)) != RAC_OK) return rc;
  root[0] = pin_res[0];
  root[1] = pin_res[1];
  if (root[1] != RAC_OK) return RAC_OK;

  // depth-first: per level its state (host copy), its variable and the next
  // value to try
  std::vector<std::vector<uint32_t>> host(1, std::vector<uint32_t>(buf.pin, buf.pin + words));
  std::vector<int> var_at(1, choose_variable(host[0].data(), n));
  std::vector<int> next_val(1, 0);
  if (var_at[0] < 0) {
    std::copy(host[0].begin(), host[0].end(), solution);
    *found = 1;
    return RAC_OK;
  }
  size_t level = 0;
  for (;;) {
    const int var = var_at[level];
    const uint32_t dv = host[level][size_t(var)];
    int value = next_val[level];
    while (value < net->d && !((dv >> value) & 1u)) ++value;
    if (value >= net->d) {  // every value of var tried: back to the parent
      if (level == 0) return RAC_OK;
      --level;
      continue;
    }
    next_val[level] = value + 1;
    if (*nodes >= max_nodes) {
      *exhausted = 1;
      return RAC_OK;
    }
    uint32_t *child = level_buffer(level + 1);
    if (!child) {
      set_error("rac_search: out of device memory for a search level");
      return RAC_ENOMEM;
    }
    if ((rc = run(buf.levels[level], child, var, value)) != RAC_OK) return rc;
    const int32_t its = pin_res[0], st = pin_res[1];
    if (*nodes < step_cap) {
      int32_t *rec = steps + 5 * *nodes;
      rec[0] = int32_t(level);
      rec[1] = var;
      rec[2] = value;
      rec[3] = its;
      rec[4] = st;
    }
    ++*nodes;
    if (st != RAC_OK) continue;  // wipe-out (or a failed wait): the next value
    if (host.size() <= level + 1) {
      host.emplace_back(words);
      var_at.push_back(-1);
      next_val.push_back(0);
    }
    std::copy(buf.pin, buf.pin + words, host[level + 1].begin());
    const int nv = choose_variable(host[level + 1].data(), n);
    if (nv < 0) {  // every domain a singleton: a solution
      std::copy(host[level + 1].begin(), host[level + 1].end(), solution);
      *found = 1;
      return RAC_OK;
    }
    ++level;
    var_at[level] = nv;
    next_val[level] = 0;
  }
} RAC_CATCH_STATUS
