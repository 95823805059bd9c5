// Internal types shared by the host side of librac and its kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "rac.h"

namespace rac {

// ---------------------------------------------------------------------------
// Bit-packed relation layout ("slabs").
//
// Variables are grouped in blocks of 32.  Each constraint is stored once, as
// R_lo,hi with lo < hi (rows = values of lo, bit b of a row = value b of hi),
// in tile (I, J) = (lo / 32, hi / 32), I <= J.  A tile is cut into slabs of
// `rows_per_slab` consecutive rows (values of i = lo % 32); inside a slab the
// relations are stored row by row, and inside a row by increasing column
// j = hi % 32, present pairs only.  A relation occupies dp = round_up(d, 4)
// words (row a in word a, rows >= d zero), so every relation and every slab
// starts on a 16-byte boundary and a slab is one contiguous bulk copy.
// ---------------------------------------------------------------------------
struct SlabDesc {
  uint32_t rel_off16;  // offset of the slab's first relation, 16-byte units
  uint32_t nbytes;     // bytes of relations in the slab (multiple of 16)
  uint32_t I, J;       // row block (x = 32 I + i) and column block (y = 32 J + j)
  uint32_t row0;       // first row i of the slab inside block I
  uint32_t nrows;      // rows of the slab
  uint32_t meta_off;   // index of the slab's first row in pmask / roff
  uint32_t pad;
};
static_assert(sizeof(SlabDesc) == 32, "SlabDesc is 32 bytes");

constexpr int kConsumerWarps = 8;
constexpr int kThreads = (kConsumerWarps + 1) * 32;  // 8 consumer warps + 1 producer warp
constexpr int kStageBytes = 32768;                   // largest slab
constexpr int kStages = 5;                           // bulk-copy ring depth
constexpr int kMaxStatesPerLaunch = 1024;

struct NetDev {
  int32_t n, d, dp, q, nb, rows_per_slab, n_slabs;
  const uint4 *rel;
  const SlabDesc *slabs;
  const uint32_t *pmask;  // per slab row: columns j present in the row
  const uint32_t *roff;   // per slab row: index of the row's first relation in the slab
};

struct Sync {
  uint32_t bar0;        // phase-0 arrivals (split barrier before the first removals)
  uint32_t bar_main;    // one arrival per CTA per sweep, monotone within a launch
  uint32_t exit_count;  // the last CTA out resets all four words
  uint32_t err;         // kErr* bits
};

constexpr uint32_t kErrGridWait = 1u;
constexpr uint32_t kErrCopyWait = 2u;
constexpr uint32_t kErrSweepBound = 4u;

struct LaunchParams {
  NetDev net;
  int32_t n_states;
  int32_t contiguous;        // state s at word s*n of dom_in/dom_out, results at index s
  const uint32_t *dom_in;
  uint32_t *dom_out;
  const int64_t *state_off;  // (contiguous == 0) word offset of state s
  const int32_t *res_idx;    // (contiguous == 0) result slot of state s
  uint32_t *bufB;            // n_states x n scratch words
  int32_t *iterations;
  int32_t *status;
  uint32_t *any;             // [3][n_states] some value removed in the sweep
  uint32_t *wipe;            // [3][n_states] some domain emptied in the sweep
  uint32_t *chg;             // [3][n_states][nb] variables that lost a value
  uint32_t *chgU;            // [3][nb] union of chg over the states
  Sync *sync;
  int32_t max_sweeps;        // <= 0: none
  int32_t sweep_bound;       // hard bound (|D| + 2), a safety net only
  uint32_t flags;
};

// Per-(network, stream) scratch.
struct Workspace {
  int cap_states = 0;
  int nb = 0;
  int n = 0;
  uint32_t *bufB = nullptr;
  uint32_t *flags = nullptr;  // any | wipe | chg | chgU
  Sync *sync = nullptr;
  int64_t *state_off = nullptr;
  int32_t *res_idx = nullptr;
  int cap_items = 0;
  uint32_t *host_dom = nullptr;  // staging for rac_enforce_host
  int32_t *host_res = nullptr;
  size_t host_cap = 0;
  size_t host_res_cap = 0;
};

}  // namespace rac

struct rac_network {
  int32_t n = 0, d = 0, dp = 0, q = 0, nb = 0, rows_per_slab = 0;
  int64_t m = 0;
  int64_t n_slabs = 0;
  size_t rel_bytes = 0;
  int device = 0;
  void *d_rel = nullptr;
  rac::SlabDesc *d_slabs = nullptr;
  uint32_t *d_pmask = nullptr;
  uint32_t *d_roff = nullptr;
  std::mutex mu;
  std::unordered_map<cudaStream_t, rac::Workspace *> ws;
};

namespace rac {
void set_error(const std::string &msg);
rac_status cuda_fail(cudaError_t e, const char *what);
NetDev net_dev(const rac_network *net);
// Launch the bit-packed kernel for P (grid sized by the callee).
rac_status launch_bits(const LaunchParams &P, cudaStream_t stream);
Workspace *get_workspace(const rac_network *net, cudaStream_t stream, int n_states, int n_items,
                         rac_status *rc);
void free_workspace(Workspace *w);
}  // namespace rac
