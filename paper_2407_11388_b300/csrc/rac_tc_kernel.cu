// Kernel (b): the support counts of Eq. 1 on the 5th-generation tensor cores
// (tcgen05.mma kind::f8f6f4, E5M2 0/1 operands, FP32 accumulation in tensor
// memory), for up to 128 domain states of one network, swept to the fixpoint
// in one persistent cooperative launch.
//
// For a relation R_xy and a state s the counts of Fig. 1 are
//   forward  Sup_xy[a](s) = sum_b R[a][b] D_s[y][b]
//   reverse  Sup_yx[b](s) = sum_a R[a][b] D_s[x][a]
// and only whether a count is positive matters (the clamp of the paper's
// listing).  The relation rows are the MMA's M axis and the states its N
// axis, so every tensor-memory lane quarter (and every SM sub-partition)
// works whatever the number of states:
//   M = 128 rows: four relations x 32 rows (rows >= d are zero), their FP8
//       entries written straight into tensor memory by the A-operand warps
//       (tcgen05.st) from the relation's bit words -- no shared-memory copy;
//   K = 32 values of the other variable;
//   N = the running states, rounded up to 16 (at most 128): one MMA per
//       group, because an MMA of this shape costs the same whatever N up to
//       128 (about 100 SM cycles).
// Entries are 2.0 or 0 on both sides, so a count is 4 x the number of
// supports, an exact small integer in FP32, and its bits are non-zero iff it
// is.  The epilogue folds a constraint into the running AND over C_x with
// one unsigned minimum per (row, state): the minimum over the row's
// constraints is non-zero iff every count is.  After a unit's 32 constraints
// a warp ballot per state gathers the rows' kept bits, and removals follow
// kernel (a) (atomicAnd into the next domain buffer, change marks; an
// emptied domain is found by the next sweep's owner step).
//
// Work: the network's variables form blocks of 32; a constraint lies in tile
// (I, J) = (min/32, max/32).  An item is one direction of one tile: forward
// (rows x of block I against the 32 variables y of block J) or reverse (rows
// y of block J against the x of block I).  Its 8 units take four variables
// each (one MMA row group of 128), and a unit's 32 groups are the 32
// variables of the other block, one MMA each, whose B operands (the other
// variable's domain words of every running state, expanded to E5M2) are
// built once per item in shared memory.  Items are claimed from a grid-wide
// counter.
//
// Roles (one CTA per SM, 704 threads):
//   warps 0-3   A operands: lane quarter q = warp; lane a writes row a of
//               the group's relation q into a 16-slot ring of tensor-memory
//               A tiles (8 columns each), four groups per store wait;
//   warps 4-19  epilogue: lane quarter warp % 4 and 32 state columns each
//               (part (warp - 4) / 4), every group (parts beyond the running
//               states idle);
//   warp 20     lane 0 issues the MMAs (three accumulators of 128 columns)
//               and commits their completion to the A slots and accumulators;
//   warp 21     claims items, publishes them through a two-deep queue and
//               streams each unit's 16 KiB of relation words into a
//               three-stage ring (cp.async.bulk).
// Every role waits on mbarriers only; the consumer warps meet on a named
// barrier four times per item (the B operands are rebuilt per item).  Every
// wait is bounded, and one that runs out aborts the launch (RAC_EBARRIER).
#include <algorithm>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {
namespace {

using namespace dev;

// warp roles (see the file comment)
constexpr int kTcAWarps = 4;                             // warps 0-3
constexpr int kTcEpiParts = 4;                           // epilogue warps per lane quarter
constexpr int kTcEpiWarp0 = kTcAWarps;                   // warps 4-19
constexpr int kTcEpiWarps = 4 * kTcEpiParts;
constexpr int kTcMmaWarp = kTcEpiWarp0 + kTcEpiWarps;    // warp 20
constexpr int kTcConsumerWarps = kTcMmaWarp + 1;         // warps 0-20
constexpr int kTcThreads = (kTcConsumerWarps + 1) * 32;  // + warp 21, the producer
constexpr int kTcCT = kTcConsumerWarps * 32;             // consumer threads

constexpr int kTcMaxStates = kTensorMaxStates;  // 128
constexpr int kNMax = 128;                      // N: one column per state
static_assert(kNMax >= kTcMaxStates && kNMax == 32 * kTcEpiParts, "a part per 32 columns");
constexpr int kAccSlots = 3, kAccCols = 128;  // accumulators: 3 x 128 columns
constexpr int kASlots = 16, kACols = 8;       // A tiles: 128 lanes x 32 bytes
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kACol0 = kAccSlots * kAccCols;
static_assert(kACol0 + kASlots * kACols <= kTmemCols, "tensor memory of one CTA");
constexpr int kGroups = 32;                 // groups (constraint columns) per unit
// groups per batch: the A warps store a batch's tiles before one wait
constexpr int kBatch = 4;
static_assert(kGroups % kBatch == 0 && kASlots % kBatch == 0, "batches");
constexpr int kUnitWords = kGroups * 128;   // a unit's relation words
constexpr uint32_t kUnitBytes = kUnitWords * 4;
constexpr int kRing = 3;
constexpr int kBTileBytes = (kNMax / 8) * 256;  // one variable's B tile
constexpr int kBSetBytes = 32 * kBTileBytes;    // the item's 32 variables
constexpr int kDStride = 33;                    // staged domain words, padded
static_assert(kTcStoreWordsPerTile == 2 * 8 * kUnitWords, "store layout");

// E5M2 entries 2.0 (0x40, bit 6) on both sides: a count is 4 x the supports
constexpr int kOneBit = 6;
// instruction descriptor: FP32 accumulator, E5M2 A and B, K-major, M = 128
__device__ __forceinline__ uint32_t idesc_for(int ncols) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(ncols >> 3) << 17) |
         (uint32_t(128 >> 4) << 24);
}

// Four bits (bit i of nib) -> four bytes, each 1 << t or 0.  The four
// shifted copies of nib land at distinct bit positions (7 i + t for bit i),
// so the product has no carries.
__device__ __forceinline__ uint32_t spread4(uint32_t nib, int t) {
  return (nib * (0x00204081u << t)) & (0x01010101u << t);
}

struct TcSmem {
  uint8_t bset[kBSetBytes];          // B tiles of the item's 32 variables
  uint32_t ring[kRing][kUnitWords];  // relation words of a unit
  uint32_t dstage[kNMax][kDStride];  // domain words of the item's 32 variables
  uint64_t ring_full[kRing], ring_empty[kRing];
  uint64_t a_full[kASlots], a_empty[kASlots];
  uint64_t acc_full[kAccSlots], acc_empty[kAccSlots];
  uint64_t item_full[2], item_empty[2];
  int32_t item_q[2];
  int32_t cur_item;
  uint32_t active;  // units of the current item with a constraint
  uint32_t pm[32];  // presence rows of the current item's tile
  uint32_t tmem_base;
  uint32_t mma_issued, ring_issued;
  uint32_t base, poisoned, abort, failed, all_done;
  uint32_t any_total, wipe_total, cta_any, cta_wipe;
  int32_t n_slots, ncols;
  uint8_t slot_state[kNMax];
  uint32_t st_info[kTcMaxStates];
  uint8_t any_loc[kTcMaxStates], wipe_loc[kTcMaxStates];
};
static_assert(sizeof(TcSmem) + 1024 <= 232448, "shared memory of the tensor-core kernel");

constexpr uint32_t kInfoSweepMask = 0xFFFFFFu;
constexpr uint32_t kInfoResB = 1u << 24;
constexpr uint32_t kInfoWiped = 1u << 25;
__device__ __forceinline__ uint32_t info_status_bits(int st) { return uint32_t(st + 8) << 27; }
__device__ __forceinline__ int info_status(uint32_t v) { return int((v >> 27) & 31u) - 8; }
constexpr int kConsumersBar = 1;

// ------------------------------ tcgen05 helpers ------------------------------
// Shared-memory matrix descriptor: K-major, no swizzle; LBO = 128 B between
// the two 16-byte K halves of a row group, SBO = 256 B between 8-row groups
// (bits 46-47 hold the descriptor version of this architecture).
__device__ __forceinline__ uint64_t umma_desc(const void *tile) {
  uint64_t d = uint64_t((smem_u32(tile) >> 4) & 0x3FFFu);
  d |= uint64_t(128u >> 4) << 16;
  d |= uint64_t(256u >> 4) << 32;
  d |= uint64_t(1) << 46;
  return d;
}
// D[tmem] (+)= A[tmem] x B[smem]
__device__ __forceinline__ void umma_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t db,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Arrive on an mbarrier for `count` threads at once.
__device__ __forceinline__ void mbar_arrive_n(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 32 consecutive columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(addr));
}
// 8 consecutive columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_st8(uint32_t addr, const uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(addr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

struct TcView {
  const uint32_t *C;
  uint32_t *T;
};
__device__ __forceinline__ int64_t tc_state_offset(const LaunchParams &P, int s) {
  return P.contiguous ? int64_t(s) * P.net.n : P.state_off[s];
}
__device__ __forceinline__ TcView tc_view(const LaunchParams &P, int s, int k) {
  const int64_t off = tc_state_offset(P, s);
  uint32_t *A = P.dom_out + off;
  uint32_t *B = P.bufB + int64_t(s) * P.net.n;
  TcView v;
  if (k == 1) {
    v.C = P.dom_in + off;
    v.T = B;
  } else if (k & 1) {
    v.C = A;
    v.T = B;
  } else {
    v.C = B;
    v.T = A;
  }
  return v;
}

// A removal: D_k[v] &= keep (keep a strict subset of D_{k-1}[v]).  Only with
// RAC_STOP_ON_WIPEOUT does the state end in the sweep that empties a domain,
// so only there does the atomic return the old word; otherwise the next
// sweep's owner step finds an emptied domain and no removal waits for its
// atomic's round trip.
__device__ __forceinline__ void tc_remove(TcSmem &S, const LaunchParams &P, int s, int slot_w,
                                          uint32_t *T, uint32_t v, uint32_t keep) {
  if (P.flags & RAC_STOP_ON_WIPEOUT) {
    const uint32_t old = atomicAnd(T + v, keep);
    if (old != 0u && (old & keep) == 0u) S.wipe_loc[s] = 1;
  } else {
    atomicAnd(T + v, keep);
  }
  S.any_loc[s] = 1;
  const int nb = P.net.nb;
  const uint32_t bit = 1u << (v & 31u);
  atomicOr(P.chg + (int64_t(slot_w) * P.flag_stride + s) * nb + (v >> 5), bit);
  if (P.flags & RAC_INCREMENTAL) atomicOr(P.chgU + int64_t(slot_w) * nb + (v >> 5), bit);
}

// Relation row `a` (a < 32; rows >= 4q are zero) of the t-th relation of slab
// row r, in the network's store layout: whole-word rows chunk-major, or
// packed rows (4q bits each) word-major.
__device__ __forceinline__ uint32_t rel_row(const uint32_t *hdr, const uint32_t *relw,
                                            uint32_t nrows, const NetDev &N, int r, uint32_t t,
                                            int a) {
  const int q = N.q;
  if (a >= 4 * q) return 0u;
  const uint32_t pm = hdr[r], cnt = __popc(pm);
  if (N.packed) {
    const uint32_t *mine = relw + hdr[nrows + r] * uint32_t(N.rw) + t;
    const int bits = 4 * q, off = a * bits, wd = off >> 5, sh = off & 31;
    const uint32_t lo = mine[uint32_t(wd) * cnt];
    const uint32_t hi = sh + bits > 32 ? mine[uint32_t(wd + 1) * cnt] : 0u;
    return __funnelshift_r(lo, hi, uint32_t(sh)) & ((1u << bits) - 1u);
  }
  const uint32_t base_chunk = hdr[nrows + r] * uint32_t(q);
  return relw[(base_chunk + uint32_t(a >> 2) * cnt + t) * 4u + uint32_t(a & 3)];
}

// The operand store, one warp per (slab, row, column) relation slot: lane a
// writes the forward word (row a of R_xy, bits over b) and, after a ballot
// per b, lane b the reverse word (column b of R_xy, bits over a), and the
// relation's presence bit.  Unit (tile, dir, mt) holds words [g][q][lane] of
// its 32 groups g (the other block's variables) and 4 relations q.
__global__ void __launch_bounds__(256) rac_tc_store_kernel(const NetDev N,
                                                           const int32_t *slab_tile,
                                                           uint32_t *ops, uint32_t *pmt) {
  const int lane = threadIdx.x & 31;
  const int64_t total = int64_t(N.n_slabs) * 1024;
  const int64_t stride = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t w = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); w < total;
       w += stride) {
    const int sl = int(w >> 10), r = int((w >> 5) & 31), j = int(w & 31);
    const SlabDesc sd = N.slabs[sl];
    const uint32_t nrows = sd.rows >> 8, row0 = sd.rows & 0xFFu;
    if (uint32_t(r) >= nrows) continue;
    const uint32_t *hdr = reinterpret_cast<const uint32_t *>(N.rel + sd.rel_off16);
    if (!((hdr[r] >> j) & 1u)) continue;  // warp-uniform
    const uint32_t *relw = hdr + 2 * nrows;
    const uint32_t t_rank = __popc(hdr[r] & ((1u << j) - 1u));
    const uint32_t row = rel_row(hdr, relw, nrows, N, r, t_rank, lane);
    uint32_t col = 0u;
#pragma unroll 8
    for (int b = 0; b < 32; ++b) {
      const uint32_t bal = __ballot_sync(kFull, (row >> b) & 1u);
      if (lane == b) col = bal;
    }
    const int64_t t = slab_tile[sl];
    const int xl = int(row0) + r, yl = j;
    uint32_t *fw = ops + ((t * 2 + 0) * 8 + xl / 4) * kUnitWords;
    uint32_t *rv = ops + ((t * 2 + 1) * 8 + yl / 4) * kUnitWords;
    fw[yl * 128 + (xl & 3) * 32 + lane] = row;
    rv[xl * 128 + (yl & 3) * 32 + lane] = col;
    if (lane == 0) atomicOr(pmt + t * 32 + xl, 1u << yl);
  }
}

// The CTA's abort flag, set by any role whose wait ran out (read through
// volatile: another warp may set it while this one loops).
__device__ __forceinline__ bool aborted(const TcSmem &S) {
  return *reinterpret_cast<const volatile uint32_t *>(&S.abort) != 0u;
}

// One lane waits (bounded) on an mbarrier phase for its warp; the warp
// follows the outcome.  A wait that runs out aborts the CTA's launch.
__device__ __forceinline__ bool warp_wait(TcSmem &S, const LaunchParams &P, uint64_t *bar,
                                          uint32_t parity, int lane) {
  uint32_t ok = 1u;
  if (lane == 0) {
    if (aborted(S) || !mbar_wait(bar, parity, &P.sync->err, P.wait_limit_ns)) {
      ok = 0u;
      S.abort = 1u;
    }
  }
  return __shfl_sync(kFull, ok, 0) != 0u;
}
__device__ __forceinline__ bool lane_wait(TcSmem &S, const LaunchParams &P, uint64_t *bar,
                                          uint32_t parity) {
  if (aborted(S) || !mbar_wait(bar, parity, &P.sync->err, P.wait_limit_ns)) {
    S.abort = 1u;
    return false;
  }
  return true;
}

// The B operands of an item: tile v holds, in row c, the domain word of
// variable vbase + v in the state of slot c, expanded to E5M2 bytes (zero
// rows for slots without a running state).
__device__ void build_bset(TcSmem &S, const LaunchParams &P, int k, int vbase, int ct) {
  const int n = P.net.n, R = S.n_slots, ncols = S.ncols;
  // the words, coalesced over the 32 variables, into dstage[slot][v]
  const int total = 32 * ncols;
  constexpr int kPer = (32 * kNMax + kTcCT - 1) / kTcCT;
  uint32_t w[kPer];
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const int t = ct + r * kTcCT;
    const int v = t & 31, i = t >> 5;
    w[r] = (t < total && i < R && vbase + v < n)
               ? ld_dom(tc_view(P, S.slot_state[i], k).C + vbase + v)
               : 0u;
  }
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const int t = ct + r * kTcCT;
    if (t < total) S.dstage[t >> 5][t & 31] = w[r];
  }
  named_bar(kConsumersBar, kTcCT);
  // rows of the B tiles, 16-byte chunks of consecutive rows per thread group
  for (int t = ct; t < total; t += kTcCT) {
    const int c = t % ncols, v = t / ncols;
    const uint32_t word = S.dstage[c][v];
    uint32_t e[8];
#pragma unroll
    for (int h = 0; h < 8; ++h) e[h] = spread4((word >> (4 * h)) & 0xFu, kOneBit);
    uint8_t *row = S.bset + v * kBTileBytes + (c >> 3) * 256 + (c & 7) * 16;
    *reinterpret_cast<uint4 *>(row) = make_uint4(e[0], e[1], e[2], e[3]);
    *reinterpret_cast<uint4 *>(row + 128) = make_uint4(e[4], e[5], e[6], e[7]);
  }
}

// One item (a direction of a tile) through the A / MMA / epilogue pipeline.
// gc counts the CTA's groups so far and rc its ring stages (the same in
// every role: slots and phases).
__device__ void tc_item(TcSmem &S, const LaunchParams &P, int item, int k, int slot_w, int warp,
                        int lane, uint32_t gc, uint32_t rc) {
  const NetDev &N = P.net;
  const int tile = item >> 1, dir = item & 1;
  const uint32_t ij = N.tc_ij[tile];
  const int I = int(ij & 0xFFFFu), J = int(ij >> 16);
  const uint32_t active = S.active;
  const int R = S.n_slots, ncols = S.ncols;

  if (warp < kTcAWarps) {
    // A tiles: lane a writes row a of relation q = warp of each group
    const int q = warp;
    const uint32_t arow = S.tmem_base + (uint32_t(q * 32) << 16) + kACol0;
    bool ok = true;
    for (int mt = 0; mt < 8; ++mt) {
      if (!((active >> mt) & 1u)) continue;
      const int r = int(rc % kRing);
      if (ok) ok = warp_wait(S, P, &S.ring_full[r], (rc / kRing) & 1u, lane);
      const uint32_t *U = S.ring[r];
      for (int g0 = 0; g0 < kGroups; g0 += kBatch, gc += kBatch) {
        // a batch's A tiles: slots gc .. gc + kBatch - 1, one barrier each way
        if (ok) ok = warp_wait(S, P, &S.a_empty[gc % kASlots], ((gc / kASlots) & 1u) ^ 1u, lane);
        if (!ok) continue;
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
          const uint32_t wrd = U[(g0 + b) * 128 + q * 32 + lane];
          uint32_t e[8];
#pragma unroll
          for (int h = 0; h < 8; ++h) e[h] = spread4((wrd >> (4 * h)) & 0xFu, kOneBit);
          tmem_st8(arow + ((gc + b) % kASlots) * kACols, e);
        }
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.a_full[gc % kASlots]);
      }
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&S.ring_empty[r]);
      ++rc;
    }
  } else if (warp == kTcMmaWarp) {
    if (lane == 0) {
      const uint32_t idesc = idesc_for(ncols);
      const uint64_t bdesc0 = umma_desc(S.bset);
      bool ok = true;
      for (int mt = 0; mt < 8 && ok; ++mt) {
        if (!((active >> mt) & 1u)) continue;
        for (int g0 = 0; g0 < kGroups && ok; g0 += kBatch) {
          const uint32_t sa = gc % kASlots;
          if (!(ok = lane_wait(S, P, &S.a_full[sa], (gc / kASlots) & 1u))) break;
          for (int b = 0; b < kBatch; ++b, ++gc) {
            const uint32_t sc = gc % kAccSlots;
            if (!(ok = lane_wait(S, P, &S.acc_empty[sc], ((gc / kAccSlots) & 1u) ^ 1u))) break;
            tc_fence_after();
            umma_ts(S.tmem_base + sc * kAccCols, S.tmem_base + kACol0 + (gc % kASlots) * kACols,
                    bdesc0 + uint64_t(((g0 + b) * kBTileBytes) >> 4), idesc, 0u);
            umma_commit(&S.acc_full[sc]);
            S.mma_issued = gc + 1u;
          }
          if (ok) umma_commit(&S.a_empty[sa]);
        }
      }
    }
    __syncwarp();
  } else if (warp < kTcEpiWarp0 + kTcEpiWarps) {
    const int q = warp & 3, part = (warp - kTcEpiWarp0) >> 2;
    const int col0 = 32 * part;             // this warp's state columns
    const bool cols = col0 < ncols;         // warp-uniform
    // parts without state columns sit the item out; part 0 of each quarter
    // releases the accumulators for them
    const uint32_t idle_parts = uint32_t(kTcEpiParts - (ncols + 31) / 32);
    const uint32_t tq = S.tmem_base + (uint32_t(q * 32) << 16) + uint32_t(col0);
    bool ok = cols;
    for (int mt = 0; mt < 8 && cols; ++mt) {
      if (!((active >> mt) & 1u)) continue;
      // constraints of this unit's relation q: presence over the groups g
      const uint32_t pres =
          dir == 0 ? S.pm[4 * mt + q] : __ballot_sync(kFull, (S.pm[lane] >> (4 * mt + q)) & 1u);
      const int var_m = dir == 0 ? 32 * I + 4 * mt + q : 32 * J + 4 * mt + q;
      // D_{k-1}[var_m] of this lane's slot col0 + lane, in flight during the unit
      const int slot = col0 + lane;
      const uint32_t dprev = (cols && pres != 0u && slot < R)
                                 ? ld_dom(tc_view(P, S.slot_state[slot], k).C + var_m)
                                 : 0u;
      uint32_t mn[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) mn[c] = kFull;
      for (int g = 0; g < kGroups; ++g, ++gc) {
        const uint32_t sc = gc % kAccSlots;
        if (ok) ok = warp_wait(S, P, &S.acc_full[sc], (gc / kAccSlots) & 1u, lane);
        if (!ok) continue;
        tc_fence_after();
        const bool here = cols && ((pres >> g) & 1u);  // warp-uniform
        uint32_t v[32];
        if (here) {
          tmem_ld32(tq + sc * kAccCols, v);
          tmem_wait_ld();
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_n(&S.acc_empty[sc], part == 0 ? 1u + idle_parts : 1u);
        if (here) {
#pragma unroll
          for (int c = 0; c < 32; ++c) mn[c] = min(mn[c], v[c]);
        }
      }
      if (!ok || !cols || pres == 0u || var_m >= N.n) continue;
      // row a = lane keeps value a in slot col0 + c iff mn[c] != 0; a ballot
      // per column gives the slot's kept word
      uint32_t mine = 0u;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (col0 + c < R) {
          const uint32_t bal = __ballot_sync(kFull, mn[c] != 0u);
          if (lane == c) mine = bal;
        }
      }
      if (slot < R) {
        const uint32_t keep = mine & dprev;
        if (keep != dprev) {
          const int s = S.slot_state[slot];
          tc_remove(S, P, s, slot_w, tc_view(P, s, k).T, uint32_t(var_m), keep);
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kTcThreads, 1) rac_tc_kernel(const LaunchParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw);
  const NetDev &N = P.net;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, cta = blockIdx.x;
  const int B = P.n_states;
  const int n = N.n;
  const bool is_producer = warp == kTcConsumerWarps;
  const int n_items = 2 * N.tc_tiles;
  const int64_t gtid = int64_t(cta) * blockDim.x + tid;
  const int64_t gstride = int64_t(G) * blockDim.x;
  const int64_t cgtid = int64_t(cta) * kTcCT + tid;
  const int64_t cgstride = int64_t(G) * kTcCT;

  if (warp == 0) {  // 512 tensor-memory columns: accumulators and A tiles
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kRing; ++i) {
      mbar_init(&S.ring_full[i], 1);
      mbar_init(&S.ring_empty[i], kTcAWarps);
    }
    for (int i = 0; i < kASlots; ++i) {  // used by the first slot of each batch
      mbar_init(&S.a_full[i], kTcAWarps);
      mbar_init(&S.a_empty[i], 1);
    }
    for (int i = 0; i < kAccSlots; ++i) {
      mbar_init(&S.acc_full[i], 1);
      mbar_init(&S.acc_empty[i], kTcEpiWarps);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.item_full[i], 1);
      mbar_init(&S.item_empty[i], 1);
    }
    fence_mbar_init();
    S.mma_issued = 0;
    S.ring_issued = 0;
    S.abort = 0;
    S.failed = 0;
    S.all_done = 0;
    S.base = ld_acquire(&P.sync->base);
    S.poisoned = ld_acquire(&P.sync->err) != 0u ? 1u : 0u;
  }
  for (int s = tid; s < B; s += blockDim.x) {
    S.st_info[s] = 0;
    S.any_loc[s] = 0;
    S.wipe_loc[s] = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t base = S.base;
  uint32_t gc = 0, rc = 0, iq = 0;  // groups, ring stages, queued items (consumers)
  uint32_t prc = 0, piq = 0;        // ring stages, queued items (producer)
  int k = 0;
  if (S.poisoned) {
    S.failed = 1;
  } else {
    // A := dom_in, B (all ones between launches) &= dom_in, empty input domains
    for (int64_t i = gtid; i < int64_t(B) * n; i += gstride) {
      const int s = int(i / n), x = int(i % n);
      const int64_t off = tc_state_offset(P, s);
      const uint32_t v = P.dom_in[off + x];
      atomicAnd(P.bufB + i, v);
      if (P.dom_out != P.dom_in) P.dom_out[off + x] = v;
      if (v == 0u) S.wipe_loc[s] = 1;
    }
    __syncthreads();
    for (;;) {
      ++k;
      const int slot_w = int((base + k) % 3), slot_r = int((base + k + 2) % 3);
      const int slot_c = int((base + k + 1) % 3);
      if (tid == 0) {  // the running states, in slots 0 .. R-1
        int R = 0;
        for (int s = 0; s < B; ++s)
          if (!(S.st_info[s] & kInfoSweepMask)) S.slot_state[R++] = uint8_t(s);
        S.n_slots = R;
        S.ncols = 16 * ((R + 15) / 16);
      }
      __syncthreads();
      if (is_producer) {
        if (lane == 0 && cta == 0) {  // the slot of the next sweep
          P.sync->bar[slot_c] = 0ull;
          P.sync->claim[slot_c] = 0u;
        }
        const bool incr = (P.flags & RAC_INCREMENTAL) && k >= 2;
        const uint32_t *cu = P.chgU + int64_t(slot_r) * N.nb;
        bool ok = true;
        for (;;) {
          int item = -1;
          if (lane == 0) {
            for (;;) {  // claim the next item that needs evaluating
              const int c = int(atomicAdd(&P.sync->claim[slot_w], 1u));
              if (c >= n_items) break;
              if (incr) {  // Prop. 2: neither block changed in sweep k-1
                const uint32_t tij = N.tc_ij[c >> 1];
                if (ld_dom(cu + (tij & 0xFFFFu)) == 0u && ld_dom(cu + (tij >> 16)) == 0u)
                  continue;
              }
              item = c;
              break;
            }
            const int s = int(piq & 1u);
            if (!lane_wait(S, P, &S.item_empty[s], ((piq >> 1) & 1u) ^ 1u)) {
              ok = false;
            } else {
              S.item_q[s] = item;
              mbar_arrive(&S.item_full[s]);
            }
          }
          ++piq;
          ok = __shfl_sync(kFull, ok ? 1u : 0u, 0) != 0u;
          item = __shfl_sync(kFull, item, 0);
          if (!ok || item < 0) break;
          // the item's units with a constraint, as the consumers compute them
          const uint32_t pmw = N.tc_pm[int64_t(item >> 1) * 32 + lane];
          uint32_t act = 0u;
          if ((item & 1) == 0) {
            const uint32_t b = __ballot_sync(kFull, pmw != 0u);
#pragma unroll
            for (int mt = 0; mt < 8; ++mt) act |= ((b >> (4 * mt)) & 0xFu) ? (1u << mt) : 0u;
          } else {
            uint32_t cols = pmw;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cols |= __shfl_xor_sync(kFull, cols, o);
#pragma unroll
            for (int mt = 0; mt < 8; ++mt) act |= ((cols >> (4 * mt)) & 0xFu) ? (1u << mt) : 0u;
          }
          if (lane == 0) {
            const uint32_t *ops =
                N.tc_ops + (int64_t(item) * 8) * kUnitWords;  // (tile * 2 + dir) * 8 units
            for (int mt = 0; mt < 8 && ok; ++mt) {
              if (!((act >> mt) & 1u)) continue;
              const int r = int(prc % kRing);
              if (!lane_wait(S, P, &S.ring_empty[r], ((prc / kRing) & 1u) ^ 1u)) {
                ok = false;
                break;
              }
              mbar_arrive_expect_tx(&S.ring_full[r], kUnitBytes);
              bulk_copy_g2s(S.ring[r], ops + int64_t(mt) * kUnitWords, kUnitBytes,
                            &S.ring_full[r]);
              ++prc;
              S.ring_issued = prc;
            }
          }
          prc = __shfl_sync(kFull, prc, 0);
          ok = __shfl_sync(kFull, ok ? 1u : 0u, 0) != 0u;
          if (!ok) break;
        }
        if (!ok && lane == 0) S.abort = 1;
      } else {
        const int ct = tid;
        const int64_t stride = P.flag_stride;
        for (int64_t i = cgtid; i < stride; i += cgstride) {
          P.any[slot_c * stride + i] = 0u;
          P.wipe[slot_c * stride + i] = 0u;
        }
        for (int64_t i = cgtid; i < stride * N.nb; i += cgstride)
          P.chg[slot_c * stride * N.nb + i] = 0u;
        for (int64_t i = cgtid; i < N.nb; i += cgstride) P.chgU[int64_t(slot_c) * N.nb + i] = 0u;
        if (k >= 2) {  // owner step, as in kernel (a)
          for (int64_t i = cgtid; i < int64_t(B) * N.nb; i += cgstride) {
            const int s = int(i / N.nb), blk = int(i % N.nb);
            if (S.st_info[s] & kInfoSweepMask) continue;
            uint32_t w = ld_dom(P.chg + (int64_t(slot_r) * stride + s) * N.nb + blk);
            if (w == 0u) continue;
            const TcView V = tc_view(P, s, k);
            while (w) {
              const int b = __ffs(w) - 1;
              w &= w - 1u;
              const int x = blk * 32 + b;
              const uint32_t c = ld_dom(V.C + x);
              atomicAnd(V.T + x, c);
              if (c == 0u) S.wipe_loc[s] = 1;  // emptied in sweep k-1
            }
          }
        }
        for (;;) {
          // the next item from the producer's queue, and its tile's presence
          if (warp == 0) {
            int item = -1;
            if (lane == 0) {
              const int s = int(iq & 1u);
              if (lane_wait(S, P, &S.item_full[s], (iq >> 1) & 1u)) {
                item = S.item_q[s];
                mbar_arrive(&S.item_empty[s]);
              }
            }
            item = __shfl_sync(kFull, item, 0);
            if (item >= 0) {
              const uint32_t pmw = N.tc_pm[int64_t(item >> 1) * 32 + lane];
              S.pm[lane] = pmw;
              uint32_t act = 0u;
              if ((item & 1) == 0) {
                const uint32_t b = __ballot_sync(kFull, pmw != 0u);
#pragma unroll
                for (int mt = 0; mt < 8; ++mt) act |= ((b >> (4 * mt)) & 0xFu) ? (1u << mt) : 0u;
              } else {
                uint32_t cols = pmw;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cols |= __shfl_xor_sync(kFull, cols, o);
#pragma unroll
                for (int mt = 0; mt < 8; ++mt)
                  act |= ((cols >> (4 * mt)) & 0xFu) ? (1u << mt) : 0u;
              }
              if (lane == 0) S.active = act;
            }
            if (lane == 0) S.cur_item = aborted(S) ? -1 : item;
          }
          ++iq;
          named_bar(kConsumersBar, kTcCT);
          const int item = S.cur_item;
          if (item < 0) break;
          const uint32_t ij = N.tc_ij[item >> 1];
          build_bset(S, P, k, (item & 1) == 0 ? 32 * int(ij >> 16) : 32 * int(ij & 0xFFFFu), ct);
          fence_async_smem();
          named_bar(kConsumersBar, kTcCT);
          tc_item(S, P, item, k, slot_w, warp, lane, gc, rc);
          const uint32_t units = __popc(S.active);
          gc += units * kGroups;
          rc += units;
          __syncwarp();
          named_bar(kConsumersBar, kTcCT);  // B tiles and staged words free
        }
      }
      __syncthreads();
      if (tid == 0) {
        S.cta_any = 0;
        S.cta_wipe = 0;
      }
      __syncthreads();
      for (int s = tid; s < B; s += blockDim.x) {
        if (S.any_loc[s]) {
          if (B > 1) atomicOr(P.any + slot_w * P.flag_stride + s, 1u);
          S.cta_any = 1;
          S.any_loc[s] = 0;
        }
        if (S.wipe_loc[s]) {
          if (B > 1) atomicOr(P.wipe + slot_w * P.flag_stride + s, 1u);
          S.cta_wipe = 1;
          S.wipe_loc[s] = 0;
        }
      }
      if (S.abort) S.failed = 1;
      __syncthreads();
      if (tid == 0) {  // grid barrier carrying the sweep's counts
        unsigned long long *w = &P.sync->bar[slot_w];
        constexpr unsigned long long kMask = (1ull << kBarCountBits) - 1ull;
        const unsigned long long mine = 1ull |
                                        (uint64_t(S.cta_any ? 1u : 0u) << kBarCountBits) |
                                        (uint64_t(S.cta_wipe ? 1u : 0u) << (2 * kBarCountBits)) |
                                        (uint64_t(S.failed ? 1u : 0u) << (3 * kBarCountBits));
        __threadfence();
        // test hook: CTA 0 withholds its arrivals, so every wait runs out
        const bool withhold = (P.flags & RAC_TEST_WITHHOLD_ARRIVAL) && cta == 0;
        unsigned long long v = withhold ? 0ull : atomicAdd(w, mine) + mine;
        const uint64_t t0 = global_timer();
        while ((v & kMask) < uint64_t(G)) {
          if (ld_acquire(&P.sync->err) != 0u) {
            S.failed = 1;
            break;
          }
          if (global_timer() - t0 > P.wait_limit_ns) {
            atomicOr(&P.sync->err, kErrGridWait);
            S.failed = 1;
            break;
          }
          __nanosleep(20);
          asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(w) : "memory");
        }
        __threadfence();
        S.any_total = uint32_t((v >> kBarCountBits) & kMask);
        S.wipe_total = uint32_t((v >> (2 * kBarCountBits)) & kMask);
        if ((v >> (3 * kBarCountBits)) & kMask) S.failed = 1;
      }
      __syncthreads();
      if (S.failed) break;
      const bool stop = (P.flags & RAC_STOP_ON_WIPEOUT) != 0;
      const bool any_at_all = S.any_total != 0u, wipe_at_all = S.wipe_total != 0u;
      for (int s = tid; s < B; s += blockDim.x) {
        uint32_t info = S.st_info[s];
        if (info & kInfoSweepMask) continue;
        bool any = any_at_all, wp = wipe_at_all;
        if (B > 1) {
          any = any && ld_dom(P.any + slot_w * P.flag_stride + s) != 0u;
          wp = wp && ld_dom(P.wipe + slot_w * P.flag_stride + s) != 0u;
        }
        if (wp) info |= kInfoWiped;
        const uint32_t t_is_b = (k & 1) ? kInfoResB : 0u;
        const uint32_t c_is_b = (k >= 2 && !(k & 1)) ? kInfoResB : 0u;
        if (stop && wp) {
          info |= uint32_t(k) | t_is_b | info_status_bits(RAC_WIPEOUT);
        } else if (!any) {
          info |= uint32_t(k) | c_is_b | info_status_bits((info & kInfoWiped) ? RAC_WIPEOUT : RAC_OK);
        } else if ((P.max_sweeps > 0 && k >= P.max_sweeps) || k >= P.sweep_bound) {
          info |= uint32_t(k) | t_is_b | info_status_bits(RAC_ETIMEOUT);
        }
        S.st_info[s] = info;
      }
      if (tid == 0) S.all_done = 1;
      __syncthreads();
      for (int s = tid; s < B; s += blockDim.x)
        if (!(S.st_info[s] & kInfoSweepMask)) S.all_done = 0;
      __syncthreads();
      if (S.all_done) break;
    }
  }

  if (S.abort) S.failed = 1;
  __syncthreads();
  const bool failed = S.failed != 0u;
  if (!S.poisoned) {
    for (int64_t i = gtid; i < int64_t(B) * n; i += gstride) {
      const int s = int(i / n), x = int(i % n);
      if (!failed && (S.st_info[s] & kInfoResB))
        P.dom_out[tc_state_offset(P, s) + x] = ld_dom(P.bufB + i);
      P.bufB[i] = kFull;
    }
  }
  if (cta == 0) {
    if (tid == 0 && !failed) P.sync->base = (base + uint32_t(k)) % 3u;
    for (int s = tid; s < B; s += blockDim.x) {
      const uint32_t info = S.st_info[s];
      const int idx = P.contiguous ? s : P.res_idx[s];
      P.iterations[idx] = int32_t(info & kInfoSweepMask) ? int32_t(info & kInfoSweepMask) : k;
      P.status[idx] = failed ? RAC_EBARRIER : info_status(info);
    }
  }
  if (failed && tid == 0) atomicOr(&P.sync->err, kErrCopyWait);
  // no MMA may still write tensor memory, and no relation copy may still be
  // in flight, when the CTA releases them: wait for the last ones issued (a
  // normal run has completed them already)
  if (tid == 0) {
    const uint32_t mi = S.mma_issued, ri = S.ring_issued;
    if (mi > 0) {
      const uint32_t c = mi - 1u;
      mbar_wait(&S.acc_full[c % kAccSlots], (c / kAccSlots) & 1u, &P.sync->err,
                P.wait_limit_ns);
    }
    const uint32_t first = ri > uint32_t(kRing) ? ri - kRing : 0u;
    for (uint32_t c = first; c < ri; ++c)
      mbar_wait(&S.ring_full[c % kRing], (c / kRing) & 1u, &P.sync->err, P.wait_limit_ns);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base),
                 "r"(kTmemCols)
                 : "memory");
}

}  // namespace

rac_status launch_tc(const LaunchParams &P, cudaStream_t stream) {
  static LaunchCache cache;
  const size_t smem = sizeof(TcSmem);
  if (P.n_states > kTcMaxStates) {
    set_error("the tensor-core kernel takes at most 128 states per launch");
    return RAC_EINVAL;
  }
  if (!P.net.tc_ops) {
    set_error("the network's tensor-core operand store is missing");
    return RAC_EINVAL;
  }
  int per_sm = 0, sms = 0;
  rac_status rc = persistent_shape(cache, reinterpret_cast<const void *>(rac_tc_kernel),
                                   kTcThreads, smem, "tensor-core kernel set-up", &per_sm, &sms);
  if (rc != RAC_OK) return rc;
  if (per_sm != 1) {  // one CTA per SM: it owns all 512 tensor-memory columns
    set_error("the tensor-core kernel must run one CTA per SM");
    return RAC_ECUDA;
  }
  const int grid = sms;
  cudaError_t e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(kTcThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, rac_tc_kernel, P);
  if (e != cudaSuccess) return cuda_fail(e, "launch of the tensor-core kernel");
  return RAC_OK;
}

rac_status ensure_tc_store(const rac_network *net, cudaStream_t stream) {
  std::lock_guard<std::mutex> lock(net->mu);
  if (net->d_tc) return RAC_OK;
  // the tiles holding a constraint, in slab order
  std::vector<SlabDesc> slabs(size_t(net->n_slabs));
  cudaError_t e = cudaSuccess;
  if (!slabs.empty())
    e = cudaMemcpy(slabs.data(), net->d_slabs, slabs.size() * sizeof(SlabDesc),
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "reading the slab table");
  std::unordered_map<uint32_t, int32_t> tile_of;
  std::vector<uint32_t> tile_ij;
  std::vector<int32_t> slab_tile(slabs.size());
  for (size_t i = 0; i < slabs.size(); ++i) {
    auto it = tile_of.find(slabs[i].ij);
    if (it == tile_of.end()) {
      it = tile_of.emplace(slabs[i].ij, int32_t(tile_ij.size())).first;
      tile_ij.push_back(slabs[i].ij);
    }
    slab_tile[i] = it->second;
  }
  const size_t tiles = tile_ij.size();
  const size_t ops_words = tiles * size_t(kTcStoreWordsPerTile);
  const size_t words = ops_words + tiles * 32 + tiles;
  const size_t bytes = words * 4;
  if (bytes > (size_t(64) << 30)) {
    set_error("the tensor-core operand store of this network would take " +
              std::to_string(bytes >> 30) + " GiB (at most 64)");
    return RAC_ENOTSUP;
  }
  void *p = nullptr;
  e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("out of device memory for the tensor-core operand store (" +
              std::to_string(bytes) + " bytes)");
    return RAC_ENOMEM;
  }
  uint32_t *ops = static_cast<uint32_t *>(p);
  uint32_t *pmt = ops + ops_words, *ijt = pmt + tiles * 32;
  int32_t *d_slab_tile = nullptr;
  auto fail = [&](cudaError_t err, const char *what) {
    cudaFree(d_slab_tile);
    cudaFree(p);
    return cuda_fail(err, what);
  };
  if (tiles > 0) {
    if ((e = cudaMalloc(&d_slab_tile, slab_tile.size() * sizeof(int32_t))) != cudaSuccess)
      return fail(e, "building the tensor-core operand store");
    if ((e = cudaMemcpy(d_slab_tile, slab_tile.data(), slab_tile.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(ijt, tile_ij.data(), tiles * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemsetAsync(ops, 0, (ops_words + tiles * 32) * 4, stream)) != cudaSuccess)
      return fail(e, "building the tensor-core operand store");
    NetDev N = net_dev(net);
    const int64_t warps = int64_t(net->n_slabs) * 1024;
    const int64_t blocks = std::min<int64_t>((warps + 7) / 8, int64_t(1) << 20);
    rac_tc_store_kernel<<<unsigned(blocks), 256, 0, stream>>>(N, d_slab_tile, ops, pmt);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(e, "building the tensor-core operand store");
    cudaFree(d_slab_tile);
  }
  net->d_tc = ops;
  net->tc_bytes = bytes;
  net->tc_tiles = int32_t(tiles);
  return RAC_OK;
}

}  // namespace rac
