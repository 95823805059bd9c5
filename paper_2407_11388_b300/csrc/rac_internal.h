// Internal types shared by the host side of librac and its kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <new>
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
// `rows_per_slab` consecutive rows (values of i = lo % 32).  A slab is one
// contiguous, 16-byte aligned record of the relation store:
//   header:    pm[rows]   bit j set iff the pair (32 I + row0 + r, 32 J + j)
//                         is constrained,
//              roff[rows] index of row r's first relation in the slab,
//   relations: row by row; a row's cnt relations (present pairs only, by
//              increasing column j) take cnt * rw words each.  Whole-word
//              rows (the default): rw = dp = round_up(d, 4), relation row a
//              in word a, stored chunk-major: 16-byte chunk c (relation
//              rows 4c..4c+3, rows >= d zero) of the row's t-th relation is
//              chunk c*cnt + t.  Packed rows (RAC_LAYOUT_PACKED, d <= 28):
//              relation row a in bits [dp a, dp a + dp) of the relation's
//              rw = packed_words(q) words (bit i of the stream = bit i % 32
//              of word i / 32), stored word-major: word w of the row's t-th
//              relation is word w*cnt + t.  The record is padded to 16 bytes.
// so one bulk copy brings everything a slab's evaluation needs.
// ---------------------------------------------------------------------------
struct SlabDesc {
  uint32_t rel_off16;  // offset of the slab record, 16-byte units
  uint32_t nbytes;     // bytes of the record (header + relations), multiple of 16
  uint32_t ij;         // I | J << 16: row block (x = 32 I + i), column block (y = 32 J + j)
  uint32_t rows;       // row0 | nrows << 8
};
static_assert(sizeof(SlabDesc) == 16, "SlabDesc is 16 bytes");

constexpr int kGroupWarps = 4;                        // warps that evaluate one slab together
constexpr int kGroups = 3;                            // slabs evaluated at the same time
// 13 warps: at most 4 per SM sub-partition, so 128 registers per thread fit
constexpr int kConsumerWarps = kGroupWarps * kGroups;
constexpr int kThreads = (kConsumerWarps + 1) * 32;  // + 1 producer warp

constexpr int kSlabRelBytes = 32768;                 // relation bytes of the largest slab
constexpr int kStageBytes = kSlabRelBytes + 256;     // + header (at most 32 rows x 2 words)
// Bulk-copy ring depth: a multiple of kGroups, so that every stage is always
// consumed by the same group (position p goes to stage p % kStages and group
// p % kGroups).  A stage shared by two groups could let one group test the
// next round's phase parity while the current round is still filling, and a
// parity test cannot tell those two phases apart.
constexpr int kStages = 6;
// A plain sweep streams each CTA's first kStaticSlabs slabs (cta, cta + G,
// ...) from its own descriptor list, then claims the rest from a grid-wide
// counter in batches of kClaimBatch, so that CTAs whose slabs are quicker
// take more and the sweep's last CTA ends about one batch after the others.
constexpr int kStaticSlabs = kStages;
constexpr int kClaimBatch = 2;
constexpr int kMaxStatesPerLaunch = 1024;
constexpr int kDescCache = 200;   // slab descriptors a CTA keeps in shared memory
constexpr int kDomWords = 5040;   // domain words a CTA keeps in shared memory per sweep

// Words of one relation with packed rows: 4q rows of 4q bits (rows >= d and
// bits >= d zero), rounded up to whole words.
__host__ __device__ constexpr int packed_words(int q) { return (16 * q * q + 31) / 32; }

struct NetDev {
  int32_t n, d, dp, q, nb, rows_per_slab, n_slabs;
  int32_t packed;  // 1: packed relation rows (RAC_LAYOUT_PACKED), 0: whole-word rows
  int32_t rw;      // words per stored relation: packed_words(q) or dp
  int32_t max_ctas;  // > 0: grid cap of the network's launches (RAC_LAYOUT_MAX_CTAS)
  // operand store of the tensor-core kernel (RAC_LAYOUT_FP8; null until
  // built): per tile holding a constraint, kTcStoreWordsPerTile relation
  // words (both orientations, in the kernel's unit order), 32 presence rows
  // and the tile's I | J << 16
  const uint32_t *tc_ops;
  const uint32_t *tc_pm;
  const uint32_t *tc_ij;
  int32_t tc_tiles;
  const uint4 *rel;
  const SlabDesc *slabs;
  const float2 *slab_feat;  // per slab: (tightness, density), the predictor's f3 and f4
};

// Launch-to-launch state of a workspace.  Between launches the scratch
// domain buffer is all ones and every flag slot the next launch writes
// before clearing it is zero.  Barrier k of a launch uses slot (base + k) % 3
// of the barrier words and of the per-sweep flag arrays; during sweep k the
// slot of sweep k+1 is cleared, and after its last sweep K a launch sets
// base += K, so the next launch starts on the slot its predecessor cleared
// last -- no CTA has to reset anything on its way out.
struct Sync {
  unsigned long long bar[3];  // sweep barrier words, four 16-bit counts: arrivals |
                              // CTAs that removed values << 16 | CTAs that emptied
                              // a domain << 32 | CTAs that failed a wait << 48
  uint32_t base;
  uint32_t err;  // kErr* bits; sticky: a failed launch poisons the workspace
  // host entry point: CTAs done writing their results into host memory in
  // this launch (the last one resets it), and the number of such launches
  // completed on the workspace (the last CTA publishes it to the host)
  uint32_t done_cta;
  uint32_t done_seq;
  // dynamic slab claims of a plain sweep (slot as bar): slabs beyond the
  // first kStaticSlabs per CTA go to whichever producer asks first
  uint32_t claim[3];
};
constexpr int kBarCountBits = 16;  // grids of at most 65535 CTAs

constexpr uint32_t kErrGridWait = 1u;
constexpr uint32_t kErrCopyWait = 2u;

constexpr int kMaxFirst = 160;  // per-CTA first slab descriptors passed with the launch
constexpr uint64_t kWaitLimitNs = 2000000000ull;      // 2 s
constexpr uint64_t kTestWaitLimitNs = 50000000ull;    // 50 ms under RAC_TEST_WITHHOLD_ARRIVAL
inline uint64_t wait_limit_for(uint32_t flags) {
  return (flags & RAC_TEST_WITHHOLD_ARRIVAL) ? kTestWaitLimitNs : kWaitLimitNs;
}

struct LaunchParams {
  NetDev net;
  int32_t n_states;
  int32_t contiguous;        // state s at word s*n of dom_in/dom_out, results at index s
  const uint32_t *dom_in;
  uint32_t *dom_out;
  const int64_t *state_off;  // (contiguous == 0) word offset of state s
  const int32_t *res_idx;    // (contiguous == 0) result slot of state s
  uint32_t *bufB;            // n_states x n scratch words (all ones between launches)
  int32_t *iterations;
  int32_t *status;
  // optional (contiguous launches): the results also written to host memory
  // at the end -- n_states x n domain words, then iterations, then status
  uint32_t *host_out;
  // optional, with host_out: host word that receives Sync::done_seq once
  // every CTA's results are in host memory (the caller waits on it instead
  // of synchronising the stream)
  uint32_t *host_done;
  uint32_t *any;             // [3][flag_stride] some value removed in the sweep
  uint32_t *wipe;            // [3][flag_stride] some domain emptied in the sweep
  uint32_t *chg;             // [3][flag_stride][nb] variables that lost a value
  uint32_t *chgU;            // [3][nb] union of chg over the states
  Sync *sync;
  int32_t flag_stride;       // state capacity of the workspace (>= n_states)
  int32_t max_sweeps;        // <= 0: none
  int32_t sweep_bound;       // hard bound (|D| + 2), a safety net only
  uint32_t flags;
  uint64_t wait_limit_ns;    // every device-side wait gives up after this long
  int32_t seed_var;          // >= 0: the search's assignment (one state only): the
  uint32_t seed_keep;        //   input domain of seed_var is ANDed with seed_keep, and
                             //   sweep 1 examines only the constraints on seed_var
  // learned gating (rac_enforce_learned): with mlp set, sweep k >= 2 of a
  // state in the gated phase evaluates a Proposition-2 candidate slab only if
  // the predictor's logit exceeds mlp_thr; a gated sweep that removes nothing
  // is followed by a full sweep, and only a full sweep that removes nothing
  // ends the state
  const uint4 *mlp;          // the predictor's fragment-packed weights
  float mlp_thr;
  int32_t mlp_min_scored;    // a 32-state chunk is scored only with this many gated candidates
  // pending (slab, state) pairs: candidates a gated sweep skipped and no
  // sweep has evaluated since (RAC_VERIFY_FULL off).  pend[sl * flag_stride
  // + s] is owned by the CTA that owns slab sl; pend_slab[sl] counts the
  // slab's pending states, pcount[s] the state's pending slabs.
  uint8_t *pend;
  int32_t *pend_slab;
  int32_t *pcount;
  // trace records (tr_count set): one per Proposition-2 candidate of sweep
  // k >= 2 -- features [8], label (1 removed / 0 not / -1 skipped), logit,
  // where [4] = k (| 1 << 30 in the gated phase), state, tile I | J << 16,
  // rows row0 | nrows << 8
  float *tr_x, *tr_y, *tr_z;
  int32_t *tr_w;
  int64_t tr_cap;
  unsigned long long *tr_count;  // records offered (may exceed tr_cap)
  unsigned long long *tr_evals;  // (slab, state) evaluations executed
  int32_t tr_state_base;         // added to the state index of a record
  int32_t n_first;           // CTAs whose first slab descriptor is in `first`
  SlabDesc first[kMaxFirst];
};

// ---------------------------------------------------------------------------
// Batched launch: many networks, each with its own states, in one persistent
// launch.  Global slab g belongs to job j iff slab_base[j] <= g <
// slab_base[j+1]; states are numbered job by job.
// ---------------------------------------------------------------------------
struct BatchJob {
  const uint4 *rel;
  const SlabDesc *slabs;
  int32_t n, d, q, nb;
  int32_t n_slabs, slab_base;    // first global slab index of the job
  int32_t n_states, state_base;  // first state of the job
  int64_t u_off;                 // offset of the job's words in a chgU slot
  int32_t lcode;                 // relation layout: q (whole-word rows), 16 + q (packed rows)
  int32_t pad;
};
static_assert(sizeof(BatchJob) == 64, "BatchJob is 64 bytes");

struct BatchSync {
  unsigned long long bar[3];   // end-of-sweep barrier words (as Sync::bar)
  unsigned long long bar2[3];  // decision barrier words: arrivals | running states << 32
  uint32_t base;
  uint32_t err;
};


struct BatchParams {
  const BatchJob *jobs;
  int32_t n_jobs, total_slabs, total_states;
  const int64_t *state_off;    // word offset of state t in dom_in / dom_out
  const int64_t *scratch_off;  // word offset of state t in bufB
  const int64_t *chg_off;      // word offset of state t inside a chg slot
  const int32_t *res_idx;      // result index of state t
  const uint32_t *dom_in;
  uint32_t *dom_out;
  uint32_t *bufB;              // all ones between launches
  int32_t *iterations;
  int32_t *status;
  uint32_t *any, *wipe;        // [3][total_states]
  uint32_t *chg;               // [3][chg_slot_words]
  uint32_t *chgU;              // [3][u_slot_words]
  uint32_t *st_info;           // [total_states], zero between launches
  uint32_t *job_alive;         // [3][n_jobs] some state of the job still runs
  const int32_t *state_job;    // job of state t
  const int32_t *chg_state;    // state whose words hold word i of a chg slot
  int64_t chg_slot_words, u_slot_words;
  BatchSync *sync;
  int32_t max_sweeps;
  uint32_t flags;
  uint64_t wait_limit_ns;
  uint32_t rel_evict_first;    // the relation stores exceed L2: stream them evict-first
  uint32_t any_packed;         // some job's relation rows are packed (RAC_LAYOUT_PACKED)
};
constexpr size_t kEvictFirstBytes = size_t(96) << 20;  // relation bytes above which streams go evict-first

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
  // rac_enforce_host: device staging (domains, then iterations and status,
  // host_cap words in all), a pinned host copy of it, and the CUDA graph of
  // the copy in, the launches and the copy out for one (state count, sweep
  // cap, flags), captured on cap_stream and replayed on the caller's stream
  uint32_t *host_dom = nullptr;
  uint32_t *host_pin = nullptr;
  uint32_t *host_pin_dev = nullptr;  // the device's address of host_pin
  size_t host_cap = 0;
  uint32_t host_seq = 0;             // the last completion number seen in host_pin
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t host_graph = nullptr;
  int32_t graph_states = -1, graph_max_sweeps = 0;
  uint32_t graph_flags = 0;
  // learned gating: pending pairs (allocated on the first learned call)
  uint8_t *pend = nullptr;       // [n_slabs][cap_states]
  int32_t *pend_slab = nullptr;  // [n_slabs]
  int32_t *pcount = nullptr;     // [cap_states]
};

}  // namespace rac

struct rac_network {
  int32_t n = 0, d = 0, dp = 0, q = 0, nb = 0, rows_per_slab = 0;
  int32_t packed = 0, rw = 0;  // packed relation rows; words per stored relation
  int32_t max_ctas = 0;  // RAC_LAYOUT_MAX_CTAS, 0: none
  // the tensor-core kernel's operand store (RAC_LAYOUT_FP8, or built by the
  // first RAC_KERNEL_TENSOR call under mu): relation words, then presence
  // rows, then tile coordinates, in one allocation
  mutable uint32_t *d_tc = nullptr;
  mutable size_t tc_bytes = 0;
  mutable int32_t tc_tiles = 0;
  int64_t m = 0;
  int64_t n_slabs = 0;
  size_t rel_bytes = 0;
  int device = 0;
  void *d_rel = nullptr;
  rac::SlabDesc *d_slabs = nullptr;
  float2 *d_slab_feat = nullptr;      // per slab: tightness, density
  std::vector<rac::SlabDesc> first;  // host copy of the first kMaxFirst descriptors
  mutable std::mutex mu;
  std::unordered_map<cudaStream_t, rac::Workspace *> ws;
};

namespace rac {
// One-time, per-device launch set-up of a persistent kernel: raises its
// dynamic shared-memory limit to `smem` and measures how many CTAs of
// `threads` threads fit on an SM.  Safe for concurrent callers on any device.
constexpr int kMaxDevices = 64;
struct LaunchCache {
  std::mutex mu;
  int per_sm[kMaxDevices] = {};
  int sms[kMaxDevices] = {};
};
rac_status persistent_shape(LaunchCache &cache, const void *func, int threads, size_t smem,
                            const char *what, int *per_sm, int *sms);
void set_error(const std::string &msg);
void set_error_nothrow(const char *msg) noexcept;
rac_status cuda_fail(cudaError_t e, const char *what);
NetDev net_dev(const rac_network *net);
// Launch parameters of n_states states of net on workspace w: the flag
// slots, sync words and first slab descriptors; the caller sets the domain,
// result and seed fields.
LaunchParams base_params(const rac_network *net, Workspace *w, int n_states, int32_t max_sweeps,
                         uint32_t flags);
// Launch the bit-packed kernel for P (grid sized by the callee).
rac_status launch_bits(const LaunchParams &P, cudaStream_t stream);
// Launch the tensor-core kernel for P (at most 128 states; P.net.tc_ops set).
rac_status launch_tc(const LaunchParams &P, cudaStream_t stream);
constexpr int kTensorMaxStates = 128;
// The tensor-core kernel's relation words of one 32 x 32-variable tile: two
// directions x 8 units x 32 groups x 4 relations x 32 rows.
constexpr int kTcStoreWordsPerTile = 2 * 8 * 32 * 128;
// Builds net's tensor-core operand store if it has none yet (thread-safe;
// the first call allocates and fills it on `stream` and waits).
rac_status ensure_tc_store(const rac_network *net, cudaStream_t stream);
const uint4 *predictor_pack(const rac_predictor *p);  // fragment-packed weights
int predictor_device(const rac_predictor *p);
Workspace *get_workspace(const rac_network *net, cudaStream_t stream, int n_states, int n_items,
                         rac_status *rc);
void free_workspace(Workspace *w);
rac_status enforce_batch_multi(const rac_network *const *nets, int32_t n_nets, int32_t n_items,
                               const int32_t *item_net, const int64_t *item_dom_off,
                               const uint32_t *dom_in, uint32_t *dom_out, int32_t *iterations,
                               int32_t *status, int32_t max_sweeps, uint32_t flags,
                               cudaStream_t s);
}  // namespace rac

// The extern "C" entry points are function-try-blocks that end in one of
// these, so that no C++ exception (a failed host allocation inside a
// std::vector or std::string, a length error on an absurd size) crosses the
// C ABI: a status-returning call reports it as an error code.
#define RAC_CATCH_STATUS                                        \
  catch (const std::bad_alloc &) {                              \
    rac::set_error_nothrow("out of host memory");               \
    return RAC_ENOMEM;                                          \
  }                                                             \
  catch (...) {                                                 \
    rac::set_error_nothrow("unexpected host-side exception");   \
    return RAC_EINVAL;                                          \
  }
#define RAC_CATCH_ZERO \
  catch (...) {        \
    return 0;          \
  }
#define RAC_CATCH_VOID \
  catch (...) {        \
  }
