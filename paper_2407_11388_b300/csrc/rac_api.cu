// Host side of librac: argument checking, the bit-packed relation layout,
// per-stream workspaces and the extern "C" entry points declared in rac.h.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include <atomic>
#include <chrono>

#include "rac_internal.h"

namespace rac {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string &msg) { g_last_error = msg; }
void set_error_nothrow(const char *msg) noexcept {
  try {
    g_last_error = msg;
  } catch (...) {
  }
}

rac_status cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return RAC_ECUDA;
}

rac_status persistent_shape(LaunchCache &cache, const void *func, int threads, size_t smem,
                            const char *what, int *per_sm, int *sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device index beyond the supported range");
    return RAC_ENOTSUP;
  }
  std::lock_guard<std::mutex> lock(cache.mu);
  if (cache.per_sm[dev] == 0) {
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return cuda_fail(e, what);
    int p = 0, n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, func, threads, smem);
    if (e != cudaSuccess) return cuda_fail(e, what);
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (p < 1) {
      set_error(std::string(what) + ": the kernel does not fit on an SM");
      return RAC_ECUDA;
    }
    cache.sms[dev] = n;
    cache.per_sm[dev] = p;
  }
  *per_sm = cache.per_sm[dev];
  *sms = cache.sms[dev];
  return RAC_OK;
}

NetDev net_dev(const rac_network *net) {
  NetDev N;
  N.n = net->n;
  N.d = net->d;
  N.dp = net->dp;
  N.q = net->q;
  N.packed = net->packed;
  N.rw = net->rw;
  N.nb = net->nb;
  N.rows_per_slab = net->rows_per_slab;
  N.n_slabs = int32_t(net->n_slabs);
  N.max_ctas = net->max_ctas;
  const size_t tiles = size_t(net->tc_tiles);
  N.tc_ops = net->d_tc;
  N.tc_pm = net->d_tc ? net->d_tc + tiles * kTcStoreWordsPerTile : nullptr;
  N.tc_ij = net->d_tc ? N.tc_pm + tiles * 32 : nullptr;
  N.tc_tiles = net->tc_tiles;
  N.rel = static_cast<const uint4 *>(net->d_rel);
  N.slabs = net->d_slabs;
  N.slab_feat = net->d_slab_feat;
  return N;
}

void free_workspace(Workspace *w) {
  if (!w) return;
  cudaFree(w->bufB);
  cudaFree(w->flags);
  cudaFree(w->sync);
  cudaFree(w->state_off);
  cudaFree(w->res_idx);
  cudaFree(w->host_dom);
  cudaFreeHost(w->host_pin);
  if (w->host_graph) cudaGraphExecDestroy(w->host_graph);
  if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
  cudaFree(w->pend);
  cudaFree(w->pend_slab);
  cudaFree(w->pcount);
  delete w;
}

namespace {
size_t flag_words(int states, int nb) {
  return size_t(6) * states + size_t(3) * states * nb + size_t(3) * nb;
}
}  // namespace

Workspace *get_workspace(const rac_network *cnet, cudaStream_t stream, int n_states, int n_items,
                         rac_status *rc) {
  rac_network *net = const_cast<rac_network *>(cnet);
  std::lock_guard<std::mutex> lock(net->mu);
  Workspace *&w = net->ws[stream];
  if (w && w->cap_states >= n_states && w->cap_items >= n_items) return w;
  // grow: the old workspace may still be in use by work queued on `stream`
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    *rc = cuda_fail(e, "cudaStreamSynchronize before workspace growth");
    return nullptr;
  }
  const int states = std::max(n_states, w ? w->cap_states : 0);
  const int items = std::max(n_items, w ? w->cap_items : 0);
  free_workspace(w);
  w = new (std::nothrow) Workspace();
  if (!w) {
    set_error("out of host memory");
    *rc = RAC_ENOMEM;
    return nullptr;
  }
  w->cap_states = states;
  w->cap_items = items;
  w->nb = net->nb;
  w->n = net->n;
  const size_t nwords = size_t(states) * size_t(net->n);
  bool ok = cudaMalloc(&w->bufB, std::max<size_t>(nwords, 1) * 4) == cudaSuccess &&
            cudaMalloc(&w->flags, flag_words(states, net->nb) * 4) == cudaSuccess &&
            cudaMalloc(&w->sync, sizeof(Sync)) == cudaSuccess &&
            cudaMalloc(&w->state_off, std::max(items, 1) * sizeof(int64_t)) == cudaSuccess &&
            cudaMalloc(&w->res_idx, std::max(items, 1) * sizeof(int32_t)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_workspace(w);
    w = nullptr;
    set_error("device allocation of the enforcement workspace failed");
    *rc = RAC_ENOMEM;
    return nullptr;
  }
  // the state every launch expects: scratch domains all ones, flags and
  // sync words zero
  e = cudaMemset(w->sync, 0, sizeof(Sync));
  if (e == cudaSuccess) e = cudaMemset(w->flags, 0, flag_words(states, net->nb) * 4);
  if (e == cudaSuccess) e = cudaMemset(w->bufB, 0xFF, std::max<size_t>(nwords, 1) * 4);
  if (e != cudaSuccess) {
    free_workspace(w);
    w = nullptr;
    *rc = cuda_fail(e, "cudaMemset of the workspace");
    return nullptr;
  }
  return w;
}

namespace {

bool check_device(const rac_network *net) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != net->device) {
    set_error("the current CUDA device is not the network's device");
    return false;
  }
  return true;
}

}  // namespace

LaunchParams base_params(const rac_network *net, Workspace *w, int n_states, int32_t max_sweeps,
                         uint32_t flags) {
  LaunchParams P = {};
  P.net = net_dev(net);
  P.n_states = n_states;
  P.bufB = w->bufB;
  // flag slots are strided by the workspace's capacity, not by this launch's
  // state count, so launches of different sizes agree on where they are
  const size_t cap = size_t(w->cap_states);
  P.any = w->flags;
  P.wipe = P.any + 3 * cap;
  P.chg = P.wipe + 3 * cap;
  P.chgU = P.chg + 3 * cap * net->nb;
  P.sync = w->sync;
  P.flag_stride = w->cap_states;
  P.max_sweeps = max_sweeps;
  const int64_t bound = int64_t(net->n) * net->d + 2;
  P.sweep_bound = int32_t(std::min<int64_t>(bound, 0xFFFFF0));
  P.flags = flags;
  P.wait_limit_ns = wait_limit_for(flags);
  P.seed_var = -1;
  P.seed_keep = 0xFFFFFFFFu;
  P.n_first = int32_t(std::min<size_t>(net->first.size(), kMaxFirst));
  for (int32_t i = 0; i < P.n_first; ++i) P.first[i] = net->first[size_t(i)];
  return P;
}

namespace {

constexpr uint32_t kKnownFlags =
    RAC_STOP_ON_WIPEOUT | RAC_INCREMENTAL | RAC_KERNEL_TENSOR | RAC_TEST_WITHHOLD_ARRIVAL;

rac_status launch_for(const LaunchParams &P, uint32_t flags, cudaStream_t s) {
  return (flags & RAC_KERNEL_TENSOR) ? launch_tc(P, s) : launch_bits(P, s);
}

// The tensor-core kernel reads the network's operand store: build it (once)
// before the launch parameters are taken from the network.
rac_status prepare_for(const rac_network *net, uint32_t flags, cudaStream_t s) {
  return (flags & RAC_KERNEL_TENSOR) ? ensure_tc_store(net, s) : RAC_OK;
}

// Largest power of two rows (<= 32) whose slab fits one ring stage, for rw
// words per stored relation.
int rows_per_slab_for(int rw) {
  int rows = 32;
  while (rows > 1 && size_t(rows) * 32 * rw * 4 > size_t(kSlabRelBytes)) rows >>= 1;
  return rows;
}

}  // namespace
}  // namespace rac

using namespace rac;

extern "C" {

const char *rac_last_error(void) { return rac::g_last_error.c_str(); }

rac_status rac_create_network(int32_t n_vars, int32_t d, int64_t n_cons, const int32_t *scope,
                              const uint32_t *rel_bits, uint32_t layout_flags,
                              rac_network **out) try {
  set_error("");
  if (!out) {
    set_error("out is NULL");
    return RAC_EINVAL;
  }
  *out = nullptr;
  if (n_vars < 1 || n_vars > 2000000) {
    set_error("n_vars must be in [1, 2000000]");
    return RAC_EINVAL;
  }
  if (d < 1 || d > 32) {
    set_error("d must be in [1, 32]");
    return RAC_EINVAL;
  }
  if (n_cons < 0 || (n_cons > 0 && (!scope || !rel_bits))) {
    set_error("n_cons < 0 or NULL scope / rel_bits");
    return RAC_EINVAL;
  }
  if (n_cons > int64_t(n_vars) * (n_vars - 1) / 2) {
    set_error("more constraints than pairs of variables (each pair takes at most one)");
    return RAC_EINVAL;
  }
  if (layout_flags & ~(RAC_LAYOUT_BITS | RAC_LAYOUT_FP8 | RAC_LAYOUT_PACKED |
                       RAC_LAYOUT_ROWS_MASK | RAC_LAYOUT_MAX_CTAS_MASK)) {
    set_error("unknown layout flag");
    return RAC_EINVAL;
  }
  const uint32_t full = d == 32 ? 0xFFFFFFFFu : ((1u << d) - 1u);
  const int nb = (n_vars + 31) / 32;
  const int dp = (d + 3) & ~3;
  const int q = dp / 4;
  // packed rows for d <= 28 (at d > 28 a row of 4q = 32 bits is a whole word)
  const bool packed = (layout_flags & RAC_LAYOUT_PACKED) && q < 8;
  const int rw = packed ? packed_words(q) : dp;  // words per stored relation
  int rows = rows_per_slab_for(rw);
  if (const uint32_t code = (layout_flags & RAC_LAYOUT_ROWS_MASK) >> 8) {
    if (code < 2 || code > 6) {
      // l = 0 would give a 2-word tile header: relations and tile sizes that
      // are not multiples of the 16 bytes a bulk copy moves
      set_error("RAC_LAYOUT_ROWS(l) takes 1 <= l <= 5");
      return RAC_EINVAL;
    }
    rows = 1 << (code - 1);
    if (size_t(rows) * 32 * rw * 4 > size_t(kSlabRelBytes)) {
      set_error("a tile of " + std::to_string(rows) + " rows of width " + std::to_string(d) +
                " does not fit the 32 KiB staging buffer");
      return RAC_EINVAL;
    }
  }

  // orient every constraint as (lo, hi) and sort by (I, J, i, j)
  std::vector<std::pair<uint64_t, int64_t>> order;
  try {
    order.resize(size_t(n_cons));
  } catch (const std::bad_alloc &) {
    set_error("out of host memory");
    return RAC_ENOMEM;
  }
  for (int64_t c = 0; c < n_cons; ++c) {
    const int32_t x = scope[2 * c], y = scope[2 * c + 1];
    if (x < 0 || x >= n_vars || y < 0 || y >= n_vars || x == y) {
      set_error("constraint " + std::to_string(c) + " has a bad scope");
      return RAC_EINVAL;
    }
    for (int a = 0; a < d; ++a)
      if (rel_bits[c * d + a] & ~full) {
        set_error("constraint " + std::to_string(c) + " sets a relation bit >= d");
        return RAC_EINVAL;
      }
    const uint32_t lo = uint32_t(std::min(x, y)), hi = uint32_t(std::max(x, y));
    const uint64_t key = ((uint64_t(lo >> 5) * uint64_t(nb) + (hi >> 5)) << 10) |
                         (uint64_t(lo & 31u) << 5) | (hi & 31u);
    order[size_t(c)] = {key, c};
  }
  std::sort(order.begin(), order.end());
  for (size_t i = 1; i < order.size(); ++i)
    if (order[i].first == order[i - 1].first) {
      set_error("two constraints on the same pair of variables (constraints " +
                std::to_string(order[i - 1].second) + " and " + std::to_string(order[i].second) +
                ")");
      return RAC_EINVAL;
    }

  // slabs: (I, J, i / rows), each a header followed by its relations
  std::vector<SlabDesc> slabs;
  std::vector<float2> slab_feat;  // tightness, density
  std::vector<uint32_t> relw;
  const size_t hdr = size_t(2) * rows;  // pm[rows] + roff[rows], a multiple of 4 words (rows >= 2)
  try {
    size_t i = 0;
    while (i < order.size()) {
      const uint64_t key = order[i].first;
      const uint64_t tile = key >> 10;
      const uint32_t row_group = uint32_t((key >> 5) & 31u) / uint32_t(rows);
      const uint32_t I = uint32_t(tile / uint64_t(nb)), J = uint32_t(tile % uint64_t(nb));
      const uint32_t row0 = row_group * uint32_t(rows);
      size_t j = i;
      while (j < order.size() && (order[j].first >> 10) == tile &&
             uint32_t((order[j].first >> 5) & 31u) / uint32_t(rows) == row_group)
        ++j;
      const size_t count = j - i;
      const size_t base = relw.size();
      // the record padded to whole 16-byte units (packed rows only)
      const size_t rec_words = (hdr + count * size_t(rw) + 3) & ~size_t(3);
      relw.resize(base + rec_words, 0u);
      uint32_t *pm = relw.data() + base;
      uint32_t *roff = pm + rows;
      uint32_t *rel = pm + hdr;
      for (size_t t = i; t < j; ++t) {
        const uint32_t ri = uint32_t((order[t].first >> 5) & 31u) - row0;
        pm[ri] |= 1u << uint32_t(order[t].first & 31u);
      }
      uint32_t acc = 0;
      for (int r = 0; r < rows; ++r) {
        roff[r] = acc;
        acc += uint32_t(__builtin_popcount(pm[r]));
      }
      // Inside a slab row the relations are stored chunk-major (whole-word
      // rows: 16-byte chunk c, rows 4c..4c+3, of the row's t-th relation sits
      // at chunk c * cnt + t of the row) or word-major (packed rows: word w
      // of the t-th relation at word w * cnt + t), so the lanes of a warp,
      // one relation each, read consecutive chunks or words (no shared-memory
      // bank conflict).
      uint32_t pk[32];
      for (size_t t = i; t < j; ++t) {
        const uint32_t ri = uint32_t((order[t].first >> 5) & 31u) - row0;
        const uint32_t cnt = uint32_t(__builtin_popcount(pm[ri]));
        const uint32_t rank = uint32_t(t - i) - roff[ri];
        uint32_t *row_base = rel + size_t(roff[ri]) * rw;
        // relation rows in the (lo, hi) orientation
        const int64_t c = order[t].second;
        const bool swap = scope[2 * c] > scope[2 * c + 1];
        if (packed) std::fill(pk, pk + rw, 0u);
        for (int a = 0; a < dp; ++a) {
          uint32_t w = 0;
          if (a < d && !swap) {
            w = rel_bits[c * d + a];
          } else if (a < d) {
            for (int b = 0; b < d; ++b) w |= ((rel_bits[c * d + b] >> a) & 1u) << b;
          }
          if (!packed) {
            row_base[(size_t(a / 4) * cnt + rank) * 4 + (a % 4)] = w;
          } else if (w != 0u) {  // row a at bits [dp a, dp a + dp) of the stream
            const int off = a * dp, wd = off >> 5, sh = off & 31;
            pk[wd] |= w << sh;
            if (sh + dp > 32) pk[wd + 1] |= w >> (32 - sh);
          }
        }
        if (packed)
          for (int wd = 0; wd < rw; ++wd) row_base[size_t(wd) * cnt + rank] = pk[wd];
      }
      // the slab's tightness (disallowed fraction of its d x d relation bits)
      // and density (constraints / (rows x 32))
      uint64_t allowed = 0;
      for (size_t t = i; t < j; ++t) {
        const int64_t c = order[t].second;
        for (int a = 0; a < d; ++a) allowed += uint64_t(__builtin_popcount(rel_bits[c * d + a]));
      }
      slab_feat.push_back(make_float2(
          float(1.0 - double(allowed) / (double(count) * double(d) * double(d))),
          float(double(count) / (double(rows) * 32.0))));
      SlabDesc sd;
      sd.rel_off16 = uint32_t(base / 4);
      sd.nbytes = uint32_t(rec_words * 4);
      sd.ij = I | (J << 16);
      sd.rows = row0 | (uint32_t(rows) << 8);
      slabs.push_back(sd);
      i = j;
    }
  } catch (const std::bad_alloc &) {
    set_error("out of host memory");
    return RAC_ENOMEM;
  }
  if (relw.size() / 4 > 0xFFFFFFFFull) {
    set_error("relation store too large");
    return RAC_ENOTSUP;
  }

  rac_network *net = new (std::nothrow) rac_network();
  if (!net) {
    set_error("out of host memory");
    return RAC_ENOMEM;
  }
  net->n = n_vars;
  net->d = d;
  net->dp = dp;
  net->q = q;
  net->packed = packed ? 1 : 0;
  net->rw = rw;
  net->nb = nb;
  net->rows_per_slab = rows;
  net->max_ctas = int32_t(layout_flags >> 16);
  net->m = n_cons;
  net->n_slabs = int64_t(slabs.size());
  net->first.assign(slabs.begin(), slabs.begin() + std::min<size_t>(slabs.size(), kMaxFirst));
  net->rel_bytes = relw.size() * 4;
  cudaError_t e = cudaGetDevice(&net->device);
  auto fail = [&](cudaError_t err, const char *what) {
    rac_status rc = err == cudaErrorMemoryAllocation ? RAC_ENOMEM : cuda_fail(err, what);
    if (rc == RAC_ENOMEM) set_error(std::string(what) + ": out of device memory");
    rac_destroy(net);
    return rc;
  };
  if (e != cudaSuccess) return fail(e, "cudaGetDevice");
  auto upload = [&](void **dst, const void *src, size_t bytes) -> cudaError_t {
    cudaError_t er = cudaMalloc(dst, std::max<size_t>(bytes, 16));
    if (er != cudaSuccess) return er;
    if (bytes) er = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    return er;
  };
  if ((e = upload(&net->d_rel, relw.data(), relw.size() * 4)) != cudaSuccess)
    return fail(e, "upload of the relation slabs");
  if ((e = upload(reinterpret_cast<void **>(&net->d_slabs), slabs.data(),
                  slabs.size() * sizeof(SlabDesc))) != cudaSuccess)
    return fail(e, "upload of the slab table");
  if ((e = upload(reinterpret_cast<void **>(&net->d_slab_feat), slab_feat.data(),
                  slab_feat.size() * sizeof(float2))) != cudaSuccess)
    return fail(e, "upload of the slab features");
  if (layout_flags & RAC_LAYOUT_FP8) {
    const rac_status rc = ensure_tc_store(net, nullptr);
    if (rc != RAC_OK) {
      const std::string msg = rac_last_error();
      rac_destroy(net);
      set_error(msg);
      return rc;
    }
  }
  *out = net;
  return RAC_OK;
} RAC_CATCH_STATUS

rac_status rac_create_network_u8(int32_t n_vars, int32_t d, int64_t n_cons, const int32_t *scope,
                                 const uint8_t *rel, uint32_t layout_flags, rac_network **out) try {
  set_error("");
  if (!out) {
    set_error("out is NULL");
    return RAC_EINVAL;
  }
  *out = nullptr;
  if (d < 1 || d > 32) {
    set_error("d must be in [1, 32]");
    return RAC_EINVAL;
  }
  if (n_cons < 0 || (n_cons > 0 && (!scope || !rel))) {
    set_error("n_cons < 0 or NULL scope / rel");
    return RAC_EINVAL;
  }
  if (n_vars < 1 || n_vars > 2000000 || n_cons > int64_t(n_vars) * (n_vars - 1) / 2) {
    set_error("n_vars outside [1, 2000000] or more constraints than pairs of variables");
    return RAC_EINVAL;
  }
  // row a of constraint c becomes one word: bit b = R_xy[a][b]
  std::vector<uint32_t> words;
  try {
    words.resize(size_t(n_cons) * size_t(d));
  } catch (const std::bad_alloc &) {
    set_error("out of host memory");
    return RAC_ENOMEM;
  }
  const size_t dd = size_t(d);
  for (size_t r = 0; r < words.size(); ++r) {
    const uint8_t *row = rel + r * dd;
    uint32_t w = 0u, bad = 0u;
    for (size_t b = 0; b < dd; ++b) {
      w |= uint32_t(row[b] & 1u) << b;
      bad |= row[b] & ~1u;
    }
    if (bad) {
      set_error("constraint " + std::to_string(r / dd) + " has a relation entry other than 0 or 1");
      return RAC_EINVAL;
    }
    words[r] = w;
  }
  return rac_create_network(n_vars, d, n_cons, scope, n_cons > 0 ? words.data() : nullptr,
                            layout_flags, out);
} RAC_CATCH_STATUS

void rac_destroy(rac_network *net) try {
  if (!net) return;
  for (auto &kv : net->ws) free_workspace(kv.second);
  net->ws.clear();
  cudaFree(net->d_tc);
  cudaFree(net->d_rel);
  cudaFree(net->d_slabs);
  cudaFree(net->d_slab_feat);
  delete net;
} RAC_CATCH_VOID

int32_t rac_network_info(const rac_network *net, int64_t *info, int32_t n_info) try {
  if (!net || !info || n_info <= 0) return 0;
  const int64_t v[7] = {net->n, net->d, net->m, int64_t(net->rel_bytes), net->n_slabs,
                        net->rows_per_slab, net->rw};
  const int32_t k = std::min<int32_t>(n_info, 7);
  for (int32_t i = 0; i < k; ++i) info[i] = v[i];
  return k;
} RAC_CATCH_ZERO

rac_status rac_enforce(const rac_network *net, const uint32_t *dom_in, uint32_t *dom_out,
                       int32_t *iterations, int32_t *status, int32_t max_sweeps, uint32_t flags,
                       rac_stream_t stream) try {
  set_error("");
  if (!net || !dom_in || !dom_out || !iterations || !status) {
    set_error("NULL argument");
    return RAC_EINVAL;
  }
  if (flags & ~kKnownFlags) {
    set_error("unknown flag");
    return RAC_EINVAL;
  }
  if (!check_device(net)) return RAC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  rac_status rc = prepare_for(net, flags, s);
  if (rc != RAC_OK) return rc;
  Workspace *w = get_workspace(net, s, 1, 0, &rc);
  if (!w) return rc;
  LaunchParams P = base_params(net, w, 1, max_sweeps, flags);
  P.contiguous = 1;
  P.dom_in = dom_in;
  P.dom_out = dom_out;
  P.iterations = iterations;
  P.status = status;
  return launch_for(P, flags, s);
} RAC_CATCH_STATUS

rac_status rac_assign_enforce(const rac_network *net, const uint32_t *dom_in, uint32_t *dom_out,
                              int32_t var, int32_t value, int32_t *iterations, int32_t *status,
                              int32_t max_sweeps, uint32_t flags, rac_stream_t stream) try {
  set_error("");
  if (!net || !dom_in || !dom_out || !iterations || !status) {
    set_error("NULL argument");
    return RAC_EINVAL;
  }
  if (var < 0 || var >= net->n || value < 0 || value >= net->d) {
    set_error("assignment out of range");
    return RAC_EINVAL;
  }
  if (flags & ~kKnownFlags) {
    set_error("unknown flag");
    return RAC_EINVAL;
  }
  if (flags & RAC_KERNEL_TENSOR) {
    set_error("the seeded first sweep of an assignment runs on the bit-packed kernel only");
    return RAC_ENOTSUP;
  }
  if (!check_device(net)) return RAC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  rac_status rc = RAC_OK;
  Workspace *w = get_workspace(net, s, 1, 0, &rc);
  if (!w) return rc;
  LaunchParams P = base_params(net, w, 1, max_sweeps, flags);
  P.contiguous = 1;
  P.dom_in = dom_in;
  P.dom_out = dom_out;
  P.iterations = iterations;
  P.status = status;
  P.seed_var = var;
  P.seed_keep = 1u << value;
  return launch_bits(P, s);
} RAC_CATCH_STATUS

rac_status rac_enforce_batch(const rac_network *const *nets, int32_t n_nets, int32_t n_items,
                             const int32_t *item_net, const int64_t *item_dom_off,
                             const uint32_t *dom_in, uint32_t *dom_out, int32_t *iterations,
                             int32_t *status, int32_t max_sweeps, uint32_t flags,
                             rac_stream_t stream) try {
  set_error("");
  if (n_items < 0 || n_nets < 0) {
    set_error("negative count");
    return RAC_EINVAL;
  }
  if (n_items == 0) return RAC_OK;
  if (!nets || !item_net || !item_dom_off || !dom_in || !dom_out || !iterations || !status) {
    set_error("NULL argument");
    return RAC_EINVAL;
  }
  if (flags & ~kKnownFlags) {
    set_error("unknown flag");
    return RAC_EINVAL;
  }
  std::vector<std::vector<int32_t>> groups(size_t(std::max(n_nets, 1)));
  for (int32_t i = 0; i < n_items; ++i) {
    const int32_t k = item_net[i];
    if (k < 0 || k >= n_nets || !nets[k]) {
      set_error("item " + std::to_string(i) + " names a bad network");
      return RAC_EINVAL;
    }
    if (item_dom_off[i] < 0) {
      set_error("item " + std::to_string(i) + " has a negative offset");
      return RAC_EINVAL;
    }
    groups[size_t(k)].push_back(i);
  }
  for (int32_t k = 0; k < n_nets; ++k)
    if (!groups[size_t(k)].empty() && !check_device(nets[k])) return RAC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int32_t used_nets = 0;
  for (int32_t k = 0; k < n_nets; ++k) used_nets += groups[size_t(k)].empty() ? 0 : 1;
  if (used_nets > 1 && (flags & RAC_KERNEL_TENSOR)) {
    set_error("the tensor-core kernel takes the states of one network per call");
    return RAC_ENOTSUP;
  }
  const size_t chunk = (flags & RAC_KERNEL_TENSOR) ? size_t(kTensorMaxStates)
                                                   : size_t(kMaxStatesPerLaunch);
  if (used_nets > 1)  // one persistent launch over all networks
    return enforce_batch_multi(nets, n_nets, n_items, item_net, item_dom_off, dom_in, dom_out,
                               iterations, status, max_sweeps, flags, s);
  std::vector<int64_t> off;
  std::vector<int32_t> idx;
  for (int32_t k = 0; k < n_nets; ++k) {
    const std::vector<int32_t> &g = groups[size_t(k)];
    if (!g.empty()) {
      const rac_status rc = prepare_for(nets[k], flags, s);
      if (rc != RAC_OK) return rc;
    }
    for (size_t base = 0; base < g.size(); base += chunk) {
      const int cnt = int(std::min<size_t>(chunk, g.size() - base));
      rac_status rc = RAC_OK;
      Workspace *w = get_workspace(nets[k], s, cnt, cnt, &rc);
      if (!w) return rc;
      off.assign(size_t(cnt), 0);
      idx.assign(size_t(cnt), 0);
      for (int j = 0; j < cnt; ++j) {
        off[size_t(j)] = item_dom_off[g[base + j]];
        idx[size_t(j)] = g[base + j];
      }
      cudaError_t e = cudaMemcpyAsync(w->state_off, off.data(), cnt * sizeof(int64_t),
                                      cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(w->res_idx, idx.data(), cnt * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail(e, "upload of the item table");
      // pageable sources: the copies above are staged before they return
      LaunchParams P = base_params(nets[k], w, cnt, max_sweeps, flags);
      P.contiguous = 0;
      P.state_off = w->state_off;
      P.res_idx = w->res_idx;
      P.dom_in = dom_in;
      P.dom_out = dom_out;
      P.iterations = iterations;
      P.status = status;
      // a later chunk on this workspace is stream-ordered after this launch
      rc = launch_for(P, flags, s);
      if (rc != RAC_OK) return rc;
    }
  }
  return RAC_OK;
} RAC_CATCH_STATUS

rac_status rac_enforce_host(const rac_network *net, int32_t n_states, const uint32_t *dom_in,
                            uint32_t *dom_out, int32_t *iterations, int32_t *status,
                            int32_t max_sweeps, uint32_t flags, rac_stream_t stream) try {
  set_error("");
  if (!net || !dom_in || !dom_out || !iterations || !status || n_states < 0) {
    set_error("NULL argument or negative state count");
    return RAC_EINVAL;
  }
  if (flags & ~kKnownFlags) {
    set_error("unknown flag");
    return RAC_EINVAL;
  }
  if (n_states == 0) return RAC_OK;
  if (!check_device(net)) return RAC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t words = size_t(n_states) * net->n;
  // One launch of the bit-packed kernel writes its results straight into the
  // pinned staging buffer at its end (posted writes, no separate copy out);
  // the tensor-core kernel and calls of several launches copy them out.
  const bool direct = !(flags & RAC_KERNEL_TENSOR) && n_states <= kMaxStatesPerLaunch;
  // pinned staging: [input words][result words][iterations][status][completion word]
  const size_t total = 2 * words + 2 * size_t(n_states) + 1;
  rac_status rc = prepare_for(net, flags, s);
  if (rc != RAC_OK) return rc;
  Workspace *w0 = get_workspace(net, s, std::min<int32_t>(n_states, kMaxStatesPerLaunch), 0, &rc);
  if (!w0) return rc;
  if (w0->host_cap < total) {
    cudaError_t er = cudaStreamSynchronize(s);
    if (er != cudaSuccess) return cuda_fail(er, "cudaStreamSynchronize");
    if (w0->host_graph) cudaGraphExecDestroy(w0->host_graph);
    w0->host_graph = nullptr;
    w0->graph_states = -1;
    cudaFree(w0->host_dom);
    cudaFreeHost(w0->host_pin);
    w0->host_dom = nullptr;
    w0->host_pin = nullptr;
    w0->host_pin_dev = nullptr;
    w0->host_cap = 0;
    void *dp = nullptr;
    if (cudaMalloc(&w0->host_dom, total * 4) != cudaSuccess ||
        cudaMallocHost(&w0->host_pin, total * 4) != cudaSuccess ||
        cudaHostGetDevicePointer(&dp, w0->host_pin, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(w0->host_dom);
      cudaFreeHost(w0->host_pin);
      w0->host_dom = nullptr;
      w0->host_pin = nullptr;
      set_error("out of memory for the host-path staging buffers");
      return RAC_ENOMEM;
    }
    w0->host_pin_dev = static_cast<uint32_t *>(dp);
    w0->host_cap = total;
  }
  uint32_t *d_dom = w0->host_dom;
  int32_t *d_res = reinterpret_cast<int32_t *>(d_dom + words);
  uint32_t *pin = w0->host_pin;
  uint32_t *pin_res = pin + words;  // results: domains, then iterations and status
  // the work of one call on `q`
  auto enqueue = [&](cudaStream_t q) -> rac_status {
    cudaError_t e = cudaMemcpyAsync(d_dom, pin, words * 4, cudaMemcpyHostToDevice, q);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    if (direct) {
      LaunchParams P = base_params(net, w0, n_states, max_sweeps, flags);
      P.contiguous = 1;
      P.dom_in = d_dom;
      P.dom_out = d_dom;
      P.iterations = d_res;
      P.status = d_res + n_states;
      P.host_out = w0->host_pin_dev + words;
      if (n_states < 4) P.host_done = w0->host_pin_dev + (total - 1);
      return launch_for(P, flags, q);
    }
    // the launches (state chunks), one copy out
    const int32_t chunk = (flags & RAC_KERNEL_TENSOR) ? kTensorMaxStates : kMaxStatesPerLaunch;
    for (int32_t base = 0; base < n_states; base += chunk) {
      const int cnt = std::min<int32_t>(chunk, n_states - base);
      LaunchParams P = base_params(net, w0, cnt, max_sweeps, flags);
      P.contiguous = 1;
      P.dom_in = d_dom + size_t(base) * net->n;
      P.dom_out = d_dom + size_t(base) * net->n;
      P.iterations = d_res + base;
      P.status = d_res + n_states + base;
      const rac_status r = launch_for(P, flags, q);
      if (r != RAC_OK) return r;
    }
    e = cudaMemcpyAsync(pin_res, d_dom, (words + 2 * size_t(n_states)) * 4,
                        cudaMemcpyDeviceToHost, q);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    return RAC_OK;
  };
  // the caller's buffers meet only host copies
  std::memcpy(pin, dom_in, words * 4);
  // this call's completion word (its place depends on n_states) starts at
  // the number of launches with host results the workspace has completed
  // (Sync::done_seq on the device), whatever an earlier call left there
  reinterpret_cast<volatile uint32_t *>(w0->host_pin)[total - 1] = w0->host_seq;
  const bool same = w0->graph_states == n_states && w0->graph_max_sweeps == max_sweeps &&
                    w0->graph_flags == flags;
  if (same && w0->host_graph) {
    const cudaError_t e = cudaGraphLaunch(w0->host_graph, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphLaunch of the host path");
  } else {
    // the first call of this shape runs eagerly (it also sets up the kernel
    // attributes), then records the same work as a graph for the next calls;
    // a shape whose capture failed keeps running eagerly
    rc = enqueue(s);
    if (rc == RAC_OK && !same) {
      if (w0->host_graph) cudaGraphExecDestroy(w0->host_graph);
      w0->host_graph = nullptr;
      w0->graph_states = -1;
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      bool ok = w0->cap_stream ||
                cudaStreamCreateWithFlags(&w0->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
      ok = ok && cudaStreamBeginCapture(w0->cap_stream, cudaStreamCaptureModeThreadLocal) ==
                     cudaSuccess;
      if (ok) {
        const rac_status r = enqueue(w0->cap_stream);
        ok = cudaStreamEndCapture(w0->cap_stream, &g) == cudaSuccess && r == RAC_OK;
        ok = ok && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
      }
      if (g) cudaGraphDestroy(g);
      if (!ok) {
        cudaGetLastError();
        if (ge) cudaGraphExecDestroy(ge);
        ge = nullptr;
      }
      w0->host_graph = ge;
      w0->graph_states = n_states;
      w0->graph_max_sweeps = max_sweeps;
      w0->graph_flags = flags;
      set_error("");
    }
  }
  // One direct launch: wait for its completion word in pinned memory (the
  // last CTA writes it after every result is in host memory) instead of
  // synchronising the stream; the kernel's exit may still be in flight, and
  // later work on `stream` is ordered after it.  A word that does not come
  // within the time limit (the launch failed) falls back to synchronising.
  bool seen = false;
  const bool done_word = direct && n_states < 4;  // the launches that publish one
  if (done_word && rc == RAC_OK) {
    const volatile uint32_t *done = w0->host_pin + (total - 1);
    const uint32_t want = w0->host_seq + 1u;
    const auto t0 = std::chrono::steady_clock::now();
    const auto limit = std::chrono::nanoseconds(2 * wait_limit_for(flags) + 1000000000ull);
    for (uint32_t i = 0;; ++i) {
      if (*done == want) {
        seen = true;
        break;
      }
      if ((i & 255u) == 0u && std::chrono::steady_clock::now() - t0 > limit) break;
    }
    std::atomic_thread_fence(std::memory_order_acquire);
  }
  if (!seen) {
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && rc == RAC_OK) rc = cuda_fail(e, "cudaStreamSynchronize");
  }
  if (done_word)
    w0->host_seq = *reinterpret_cast<volatile uint32_t *>(w0->host_pin + (total - 1));
  if (rc == RAC_OK) {
    std::memcpy(dom_out, pin_res, words * 4);
    std::memcpy(iterations, pin_res + words, size_t(n_states) * 4);
    std::memcpy(status, pin_res + words + n_states, size_t(n_states) * 4);
  }
  return rc;
} RAC_CATCH_STATUS

rac_status rac_enforce_learned(const rac_network *net, int32_t n_states, const uint32_t *dom_in,
                               uint32_t *dom_out, int32_t *sweeps, int32_t *status,
                               int32_t max_sweeps, uint32_t flags, const rac_predictor *pred,
                               float threshold, int32_t min_scored, const rac_trace *trace,
                               rac_stream_t stream) try {
  set_error("");
  if (!net || n_states < 0) {
    set_error("NULL network or negative state count");
    return RAC_EINVAL;
  }
  if (n_states > 0 && (!dom_in || !dom_out || !sweeps || !status)) {
    set_error("NULL argument");
    return RAC_EINVAL;
  }
  if (flags & ~(RAC_STOP_ON_WIPEOUT | RAC_INCREMENTAL | RAC_VERIFY_FULL |
                RAC_TEST_WITHHOLD_ARRIVAL)) {
    set_error("unknown flag (rac_enforce_learned takes RAC_STOP_ON_WIPEOUT, RAC_VERIFY_FULL)");
    return RAC_EINVAL;
  }
  if (trace && (trace->capacity < 0 ||
                (trace->capacity > 0 && (!trace->features || !trace->label || !trace->where ||
                                         !trace->count)))) {
    set_error("trace: negative capacity, or records without features / label / where / count");
    return RAC_EINVAL;
  }
  if (!check_device(net)) return RAC_EINVAL;
  if (pred && predictor_device(pred) != net->device) {
    set_error("the predictor lives on another device than the network");
    return RAC_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (trace) {
    cudaError_t e = cudaSuccess;
    if (trace->count) e = cudaMemsetAsync(trace->count, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess && trace->evaluated)
      e = cudaMemsetAsync(trace->evaluated, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the trace counters");
  }
  for (int32_t base = 0; base < n_states; base += kMaxStatesPerLaunch) {
    const int cnt = std::min<int32_t>(kMaxStatesPerLaunch, n_states - base);
    rac_status rc = RAC_OK;
    Workspace *w = get_workspace(net, s, cnt, 0, &rc);
    if (!w) return rc;
    if (pred && !(flags & RAC_VERIFY_FULL) && !w->pend) {
      // the launch clears them in its first sweep: no initialisation needed
      const size_t slabs = size_t(std::max<int64_t>(net->n_slabs, 1));
      if (cudaMalloc(&w->pend, slabs * size_t(w->cap_states)) != cudaSuccess ||
          cudaMalloc(&w->pend_slab, slabs * sizeof(int32_t)) != cudaSuccess ||
          cudaMalloc(&w->pcount, size_t(w->cap_states) * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of the pending-pair arrays failed");
        return RAC_ENOMEM;
      }
    }
    // Proposition-2 bookkeeping (changed-variable union) is what both the
    // gated sweeps and the trace mode start from
    LaunchParams P = base_params(net, w, cnt, max_sweeps, flags | RAC_INCREMENTAL);
    // a gated sweep that removes nothing is followed by a full sweep, so at
    // most twice the |D| + 1 sweeps of Proposition 1 (plus one)
    const int64_t bound = 2 * (int64_t(net->n) * net->d + 2);
    P.sweep_bound = int32_t(std::min<int64_t>(bound, 0xFFFFF0));
    P.contiguous = 1;
    P.dom_in = dom_in + size_t(base) * net->n;
    P.dom_out = dom_out + size_t(base) * net->n;
    P.iterations = sweeps + base;
    P.status = status + base;
    P.mlp = pred ? predictor_pack(pred) : nullptr;
    P.mlp_thr = threshold;
    P.mlp_min_scored = min_scored;
    if (pred && !(flags & RAC_VERIFY_FULL)) {
      P.pend = w->pend;
      P.pend_slab = w->pend_slab;
      P.pcount = w->pcount;
      cudaError_t e = cudaMemsetAsync(w->pcount, 0, size_t(cnt) * sizeof(int32_t), s);
      if (e != cudaSuccess) return cuda_fail(e, "clearing the pending counts");
    }
    if (trace) {
      P.tr_x = trace->features;
      P.tr_y = trace->label;
      P.tr_z = trace->logit;
      P.tr_w = trace->where;
      P.tr_cap = trace->capacity;
      P.tr_count = trace->count;
      P.tr_evals = trace->evaluated;
      P.tr_state_base = base;
    }
    rc = launch_bits(P, s);
    if (rc != RAC_OK) return rc;
  }
  return RAC_OK;
} RAC_CATCH_STATUS

}  // extern "C"
