// Kernel (a): the bit-packed support step of Eq. 1, swept to its fixpoint
// inside one persistent cooperative launch.
//
// One sweep evaluates, for every constraint c_xy stored as R_xy (x < y):
//   forward  (x,a) keeps a support on c_xy  iff  R_xy[a] & D[y] != 0
//            (Fig. 1: Sup_xy[a] = sum_b R_xy[a][b] D[y][b] > 0; the listing
//            clamps the count to 1, so only its being non-zero matters);
//   reverse  (y,b) keeps a support on c_yx  iff  bit b of OR_{a in D[x]} R_xy[a],
// so one read of each relation serves both arcs.  A value survives the sweep
// iff it keeps a support on every constraint of C_x (Algorithm 1
// `tensorRevise`: the sum over the constraints must equal their number).
//
// Mapping: a CTA owns every G-th relation slab (in a plain sweep of one to
// three states only its first kStaticSlabs of them; the rest go to whichever
// CTA claims them first from a grid-wide counter).  A producer warp streams
// slabs into a shared-memory ring with bulk copies (cp.async.bulk, completion
// on mbarriers); three consumer groups of four warps (five in the many-state
// variant) take alternate stages.  A lane holds one relation (the pair (x,
// y = 32 J + lane)); the AND over C_x of the forward masks is a warp
// AND-reduction (redux.sync) for the row's x, and the reverse masks are
// AND-accumulated per lane over the rows for y.  With few states a state's
// rows are split over a group's warps; with many, the group's warps take the
// slab's states by rank, two per pass.  Partial results reach the
// next-domain buffer through atomicAnd only when they remove something; an
// emptied domain is found by the next sweep's owner step (with
// RAC_STOP_ON_WIPEOUT, by the value the atomic returns).
//
// Sweeps are synchronous (Jacobi) as Eq. 1 requires: sweep k reads D_{k-1}
// from one buffer and ANDs into the other, which still holds D_{k-2} (a
// superset); the owner of each variable that changed in sweep k-1 first ANDs
// D_{k-1} into it.  A grid barrier with a bounded wait separates sweeps; the
// per-state decisions (fixpoint, wipe-out, sweep cap) are taken by every CTA
// from the same flags.  With RAC_INCREMENTAL, sweep k >= 2 skips slabs whose
// rows and columns all kept their domains in sweep k-1 (Proposition 2).
#include <cooperative_groups.h>

#include <cstdio>

#include <algorithm>

#include "rac_device.cuh"
#include "rac_internal.h"
#include "rac_mlp.cuh"

namespace rac {

// The instances for packed relation rows (rac_bits_packed.cu): variant var
// (kVar below), with the completion word when done.
rac_status launch_bits_packed(const LaunchParams &P, cudaStream_t stream, int var, bool done);

namespace {

using namespace dev;

struct StageInfo {
  int32_t sl;  // slab index, -1 = end of the sweep's slabs
  uint32_t ij, rows, pad;
};

// kernel variants (see rac_bits_kernel)
constexpr int kVarFew = 0, kVarMany = 1, kVarGated1 = 2, kVarGated2 = 3;
// warps of a consumer group: five in the many-state variant (16 warps with
// the producer: one more warp per SM sub-partition to hide the support
// test's latencies), four in the others
constexpr int group_warps(int var) { return var == kVarMany ? kGroupWarps + 1 : kGroupWarps; }
constexpr int consumer_warps(int var) { return group_warps(var) * kGroups; }
constexpr int kMaxConsumerWarps = (kGroupWarps + 1) * kGroups;
// the gated variants add one scorer warp per consumer group (16 warps: at most
// 4 per SM sub-partition, so the 128 registers per thread still fit)
constexpr int kScorerWarps = kGroups;
constexpr int threads_for(int var) {
  return (consumer_warps(var) + 1 + (var >= kVarGated1 ? kScorerWarps : 0)) * 32;
}
constexpr int kChgULocal = 64;  // variables <= 2048: the union is collected in shared memory

struct Smem {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t issued[kStages];  // gated variants: the stage's slab is known (scorer may start)
  StageInfo stage[kStages];
  uint32_t stage_ok[kStages];
  uint32_t base;        // barrier k uses slot (base + k) % 3
  uint32_t poisoned;    // an earlier launch on this workspace failed
  uint32_t all_done;
  uint32_t abort;
  uint32_t dom_cached;
  uint32_t chg_off;     // chg_cached: the words start at dom + chg_off
  uint32_t chg_cached;  // sweep k >= 2 keeps the changed-variable words of sweep k-1 in dom
  uint32_t chgu_local;  // RAC_INCREMENTAL with nb <= kChgULocal: chgu_loc collects the union
  // this CTA's share of the sweep's changed-variable union (over the states),
  // merged into P.chgU once per sweep instead of one global atomic per removal
  uint32_t chgu_loc[kChgULocal];
  uint32_t any_total;   // CTAs that removed a value in the last sweep
  uint32_t wipe_total;  // CTAs that emptied a domain in the last sweep
  uint32_t failed;      // a wait of this CTA gave up, or another CTA reported one
  uint32_t cta_any;
  uint32_t cta_wipe;
  uint32_t load_all;    // learned gating: some running state is in its full phase
  uint32_t red[2][kMaxConsumerWarps][32];
  uint32_t remw[2][kMaxConsumerWarps];  // per-warp "removed a value" of a state group
  uint32_t st_info[kMaxStatesPerLaunch];  // see kInfo* below
  uint8_t any_loc[kMaxStatesPerLaunch];
  uint8_t wipe_loc[kMaxStatesPerLaunch];
  SlabDesc desc[kDescCache];
  // D_{k-1} of every running state, when it fits; the gated variant keeps the
  // predictor's packed weights in the last kMlpSmemWords words instead
  alignas(16) uint32_t dom[kDomWords];
};
constexpr int kMlpSmemWords = kPackVec4 * 4;
// gated variants: per ring stage, the producer's decisions for the slab in it
// -- ev[32] (states to evaluate), need[32] (states with a trace record),
// rec_lo[32], rec_hi[32] (first record index of each 32-state chunk)
constexpr int kDecWords = 128;
constexpr int kDecBase = kDomWords - kMlpSmemWords - kStages * kDecWords;
static_assert(kDecBase > 0 && kDecBase % 4 == 0 && (kDomWords - kMlpSmemWords) % 4 == 0,
              "weights and stage decisions fit 16-byte aligned at the end of the domain cache");
static_assert(kMaxStatesPerLaunch <= 32 * 32, "one decision word per 32 states");
__device__ __forceinline__ const uint4 *smem_mlp(const Smem &S) {
  return reinterpret_cast<const uint4 *>(S.dom + (kDomWords - kMlpSmemWords));
}
__device__ __forceinline__ uint32_t *stage_dec(Smem &S, int stg) {
  return S.dom + kDecBase + stg * kDecWords;
}
// domain words the cache holds in the given variant
template <int kGate>
constexpr int dom_cache_words() { return kGate > 0 ? kDecBase : kDomWords; }
static_assert(kStages % kGroups == 0, "each ring stage belongs to one consumer group");
static_assert(size_t(kStages) * kStageBytes + sizeof(Smem) <= 232448,
              "shared memory of the bit-packed kernel exceeds 227 KB");
// st_info: bits 0..23 sweep at which the state finished (0 = running),
// bit 24 result in buffer B, bit 25 some domain emptied so far,
// bit 26 gated phase (learned gating), bits 27..31 status code + 8.
constexpr uint32_t kInfoSweepMask = 0xFFFFFFu;
constexpr uint32_t kInfoResB = 1u << 24;
constexpr uint32_t kInfoWiped = 1u << 25;
constexpr uint32_t kInfoGated = 1u << 26;  // learned gating: the state is in its gated phase

__device__ __forceinline__ uint32_t info_status_bits(int st) { return uint32_t(st + 8) << 27; }
__device__ __forceinline__ int info_status(uint32_t v) { return int((v >> 27) & 31u) - 8; }

// named barriers: 1 = all consumer warps, 2 + cg = the warps of consumer group
// cg, 2 + kGroups + 2 cg + g = the warps of state group g (g < 2) inside
// consumer group cg (only needed when a state group has several warps)
constexpr int kAllConsumersBar = 1;
__device__ __forceinline__ int group_bar(int cg) { return 2 + cg; }
__device__ __forceinline__ int state_group_bar(int cg, int g) { return 2 + kGroups + 2 * cg + g; }
static_assert(2 + kGroups + 2 * kGroups <= 16, "named barrier ids");

// The input domain word of variable x as sweep 1 sees it (the search's
// assignment, if any, applied).
__device__ __forceinline__ uint32_t input_word(const LaunchParams &P, int x, uint32_t v) {
  return x == P.seed_var ? (v & P.seed_keep) : v;
}

// Does a slab of rows [row0, row0 + nrows) of block I and columns of block J
// hold a constraint on the seeded variable (sweep 1 of an assignment)?
__device__ __forceinline__ bool slab_touches_seed(const LaunchParams &P, uint32_t I, uint32_t J,
                                                  uint32_t row0, uint32_t nrows) {
  const uint32_t sv = uint32_t(P.seed_var);
  if ((sv >> 5) == J) return true;
  return (sv >> 5) == I && (sv & 31u) >= row0 && (sv & 31u) < row0 + nrows;
}

struct StateView {
  const uint32_t *C;  // D_{k-1}
  uint32_t *T;        // becomes D_k
};

__device__ __forceinline__ int64_t state_offset(const LaunchParams &P, int s) {
  return P.contiguous ? int64_t(s) * P.net.n : P.state_off[s];
}

// Buffers: A = dom_out, B = bufB.  Sweep 1 reads dom_in and writes B; even
// sweeps read B and write A; odd sweeps >= 3 read A and write B.
__device__ __forceinline__ StateView state_view(const LaunchParams &P, int s, int k) {
  const int64_t off = state_offset(P, s);
  uint32_t *A = P.dom_out + off;
  uint32_t *B = P.bufB + int64_t(s) * P.net.n;
  StateView v;
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

// Word blk of the variables state s changed in sweep k-1 (sweep k >= 2): from
// the copy the consumers made at the start of the sweep when it fits, else
// from L2.
__device__ __forceinline__ uint32_t chg_word(const Smem &S, const LaunchParams &P, int slot_r,
                                             int s, uint32_t blk) {
  if (S.chg_cached) return S.dom[S.chg_off + uint32_t(s) * uint32_t(P.net.nb) + blk];
  return ld_dom(P.chg + (int64_t(slot_r) * P.flag_stride + s) * P.net.nb + blk);
}

// Apply a removal: D_k[v] &= keep, where keep is a strict subset of D_{k-1}[v].
// Whether it empties the domain matters at once only with RAC_STOP_ON_WIPEOUT
// (the state ends after this sweep): there the atomic returns the old word.
// Otherwise an emptied domain only decides the final status, and the next
// sweep's owner step finds it (it reads D_k of every variable that changed),
// so the removal does not wait for the atomic's round trip.
__device__ __forceinline__ void remove_value(Smem &S, const LaunchParams &P, int s, uint32_t *T,
                                             uint32_t v, uint32_t keep) {
  if (P.flags & RAC_STOP_ON_WIPEOUT) {
    const uint32_t old = atomicAnd(T + v, keep);
    if (old != 0u && (old & keep) == 0u) S.wipe_loc[s] = 1;
  } else {
    atomicAnd(T + v, keep);
  }
}

// Record the variables one evaluation of state s removed values from: xbits
// in 32-variable block I (the slab's rows), ybits in block J (its columns).
// One atomic per block and evaluation instead of one per removal; the union
// over the states (Proposition 2) goes to the CTA's shared copy when it has
// one.
__device__ __forceinline__ void mark_changed(Smem &S, const LaunchParams &P, int s, int slot_w,
                                             uint32_t I, uint32_t xbits, uint32_t J,
                                             uint32_t ybits) {
  S.any_loc[s] = 1;
  const int nb = P.net.nb;
  uint32_t *ch = P.chg + (int64_t(slot_w) * P.flag_stride + s) * nb;
  uint32_t *cu = P.chgU + int64_t(slot_w) * nb;
  const bool incr = (P.flags & RAC_INCREMENTAL) != 0u;
  if (xbits) {
    atomicOr(ch + I, xbits);
    if (S.chgu_local)
      atomicOr(&S.chgu_loc[I], xbits);
    else if (incr)
      atomicOr(cu + I, xbits);
  }
  if (ybits) {
    atomicOr(ch + J, ybits);
    if (S.chgu_local)
      atomicOr(&S.chgu_loc[J], ybits);
    else if (incr)
      atomicOr(cu + J, ybits);
  }
}

// Bounded grid barrier over all CTAs (co-resident: cooperative launch).  The
// arrival also counts the CTAs that removed values, emptied a domain or failed
// a wait in the sweep; the totals land in S.any_total, S.wipe_total and
// S.failed, so no flag needs a separate load after the barrier.
__device__ void grid_barrier(Smem &S, const LaunchParams &P, int slot) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long *w = &P.sync->bar[slot];
    constexpr unsigned long long kMask = (1ull << kBarCountBits) - 1ull;
    const unsigned long long mine = 1ull |
                                    (uint64_t(S.cta_any ? 1u : 0u) << kBarCountBits) |
                                    (uint64_t(S.cta_wipe ? 1u : 0u) << (2 * kBarCountBits)) |
                                    (uint64_t(S.failed ? 1u : 0u) << (3 * kBarCountBits));
    // test hook: CTA 0 withholds its first arrival, so every wait runs out
    const bool withhold = (P.flags & RAC_TEST_WITHHOLD_ARRIVAL) && blockIdx.x == 0;
    // the arrival releases this CTA's removals; the last arrival acquires all
    unsigned long long v = withhold ? 0ull : atom_add_acq_rel_u64(w, mine) + mine;
    const uint64_t t0 = global_timer();
    uint32_t spins = 0;
    // poll the barrier word alone; the error word and the time limit are
    // looked at every 64 polls (one L2 round trip each)
    while ((v & kMask) < gridDim.x) {
      if ((++spins & 63u) == 0u) {
        if (ld_acquire(&P.sync->err) != 0u) {
          S.failed = 1;
          break;
        }
        if (global_timer() - t0 > P.wait_limit_ns) {
          atomicOr(&P.sync->err, kErrGridWait);
          S.failed = 1;
          break;
        }
      }
      v = ld_acquire_u64(w);
    }
    S.any_total = uint32_t((v >> kBarCountBits) & kMask);
    S.wipe_total = uint32_t((v >> (2 * kBarCountBits)) & kMask);
    if ((v >> (3 * kBarCountBits)) & kMask) S.failed = 1;
  }
  __syncthreads();
}

// D_{k-1} words of state s a slab's evaluation needs: the column word of
// this lane (Dy) and the row word of this lane (Dxl, lane < slab rows), read
// in two coalesced loads (sweep 1: the input domains, with a search
// assignment applied).
__device__ __forceinline__ void load_words(const Smem &S, const LaunchParams &P, int s, int k,
                                           bool cached, int y, bool y_ok, int x_l, bool x_ok,
                                           uint32_t &Dy, uint32_t &Dxl) {
  const int n = P.net.n;
  const uint32_t *Dc = cached ? S.dom + s * n : state_view(P, s, k).C;
  Dy = y_ok ? (cached ? Dc[y] : ld_dom(Dc + y)) : 0u;
  Dxl = x_ok ? (cached ? Dc[x_l] : ld_dom(Dc + x_l)) : 0u;
  if (k == 1 && !cached) {  // the cached copy has the assignment applied already
    Dy = input_word(P, y, Dy);
    Dxl = input_word(P, x_l, Dxl);
  }
}

// The states of a 32-state chunk (bit i: state c0 + i) that warp g of a
// consumer group with `groups` warps evaluates: those of rank g, g + groups,
// ... among the chunk's states to evaluate, so that the group's warps get
// equal shares however the evaluated states fall.
__device__ __forceinline__ uint32_t warp_share(uint32_t m, int g, int groups, int lane) {
  const int rank = __popc(m & lanemask_lt());
  return __ballot_sync(kFull, ((m >> lane) & 1u) && rank % groups == g);
}

// Evaluate one state on one slab: the support step of Eq. 1 restricted to the
// slab's constraints, with its removals applied to D_k.  With kPre, Dy / Dxl
// are the state's words from load_words and a row's word is taken from lane
// r; without, every row reads its word when it gets to it (the shorter path
// when a state's rows are split over several warps).  With kLabel, the state
// group's first warp (sub == 0) gets back whether the evaluation removed a
// value.
template <int L, bool kLabel, bool kPre>
__device__ __forceinline__ bool eval_state(Smem &S, const LaunchParams &P, int s, int k,
                                           int slot_w, const uint32_t *hdr, const uint4 *rel,
                                           uint32_t I, uint32_t row0, uint32_t nrows, int y,
                                           bool y_ok, bool cached, uint32_t Dy, uint32_t Dxl,
                                           int warp, int lane, int cg, int g, int sub, int wps,
                                           uint32_t &red_iter) {
  const NetDev &N = P.net;
  const uint32_t dfull = N.d >= 32 ? kFull : ((1u << N.d) - 1u);
  const StateView V = state_view(P, s, k);
  const uint32_t *Dc = cached ? S.dom + s * N.n : V.C;
  if (!kPre) {
    Dy = y_ok ? (cached ? Dc[y] : ld_dom(Dc + y)) : 0u;
    if (k == 1 && !cached) Dy = input_word(P, y, Dy);
  }
  uint32_t racc = kFull;
  uint32_t xbits = 0u;  // rows of this warp whose domain lost a value
  for (int r = sub; r < int(nrows); r += wps) {
    const uint32_t pm = hdr[r];
    if (pm == 0u) continue;
    const int x = int(I) * 32 + int(row0) + r;
    uint32_t Dx;
    if (kPre) {
      Dx = __shfl_sync(kFull, Dxl, r);
    } else {
      Dx = cached ? Dc[x] : ld_dom(Dc + x);
      if (k == 1 && !cached) Dx = input_word(P, x, Dx);
    }
    uint32_t fwd = kFull, rev = kFull;
    if ((pm >> lane) & 1u) {
      // this lane's relation: rank t in the row, chunk c at c * cnt + t
      const uint32_t t = __popc(pm & lanemask_lt());
      if (Dx == dfull)
        support_at<L, true>(rel, hdr[nrows + r], t, __popc(pm), Dx, Dy, fwd, rev);
      else
        support_at<L, false>(rel, hdr[nrows + r], t, __popc(pm), Dx, Dy, fwd, rev);
    }
    const uint32_t keep_x = __reduce_and_sync(kFull, fwd) & Dx;  // warp-uniform
    if (keep_x != Dx) {
      if (lane == 0) remove_value(S, P, s, V.T, uint32_t(x), keep_x);
      xbits |= 1u << (row0 + uint32_t(r));
    }
    racc &= rev;
  }
  bool rem = xbits != 0u;
  if (wps > 1) {
    const int buf = red_iter & 1;
    S.red[buf][warp][lane] = racc;
    if (kLabel && lane == 0) S.remw[buf][warp] = rem ? 1u : 0u;
    named_bar(state_group_bar(cg, g), wps * 32);
    if (sub == 0) {
      for (int j = 1; j < wps; ++j) {
        racc &= S.red[buf][warp + j][lane];
        if (kLabel) rem = rem || S.remw[buf][warp + j] != 0u;
      }
    }
    ++red_iter;
  }
  bool rem_y = false;
  if (sub == 0 && y_ok) {
    const uint32_t keep_y = racc & Dy;
    if (keep_y != Dy) {
      remove_value(S, P, s, V.T, uint32_t(y), keep_y);
      rem_y = true;
    }
  }
  const uint32_t ybits = __ballot_sync(kFull, rem_y);
  if (lane == 0 && (xbits | ybits) != 0u)
    mark_changed(S, P, s, slot_w, I, xbits, uint32_t(y) >> 5, ybits);
  if (kLabel) rem = rem || ybits != 0u;
  return rem;
}

// Evaluate two states s1, s2 on one slab in one pass (a warp that owns whole
// states): each relation chunk is read from shared memory once for both, and
// the two support tests give the warp independent work.  Dy*, Dx*l as in
// eval_state with kPre.  Returns, in rem1 / rem2, whether each removed a
// value.
template <int L>
__device__ __forceinline__ void eval_pair(Smem &S, const LaunchParams &P, int s1, int s2, int k,
                                          int slot_w, const uint32_t *hdr, const uint4 *rel,
                                          uint32_t I, uint32_t row0, uint32_t nrows, int y,
                                          bool y_ok, uint32_t Dy1, uint32_t Dx1l, uint32_t Dy2,
                                          uint32_t Dx2l, int lane, bool &rem1, bool &rem2) {
  const NetDev &N = P.net;
  const uint32_t dfull = N.d >= 32 ? kFull : ((1u << N.d) - 1u);
  uint32_t *T1 = state_view(P, s1, k).T;
  uint32_t *T2 = state_view(P, s2, k).T;
  uint32_t racc1 = kFull, racc2 = kFull, xb1 = 0u, xb2 = 0u;
  for (int r = 0; r < int(nrows); ++r) {
    const uint32_t pm = hdr[r];
    if (pm == 0u) continue;
    const uint32_t Dx1 = __shfl_sync(kFull, Dx1l, r);
    const uint32_t Dx2 = __shfl_sync(kFull, Dx2l, r);
    uint32_t f1 = kFull, v1 = kFull, f2 = kFull, v2 = kFull;
    if ((pm >> lane) & 1u) {
      const uint32_t t = __popc(pm & lanemask_lt());
      if (Dx1 == dfull && Dx2 == dfull)
        support_pair_at<L, true>(rel, hdr[nrows + r], t, __popc(pm), Dx1, Dy1, Dx2, Dy2, f1, v1,
                                 f2, v2);
      else
        support_pair_at<L, false>(rel, hdr[nrows + r], t, __popc(pm), Dx1, Dy1, Dx2, Dy2, f1,
                                  v1, f2, v2);
    }
    const uint32_t keep1 = __reduce_and_sync(kFull, f1) & Dx1;  // warp-uniform
    const uint32_t keep2 = __reduce_and_sync(kFull, f2) & Dx2;
    const uint32_t x = I * 32u + row0 + uint32_t(r);
    if (keep1 != Dx1) {
      if (lane == 0) remove_value(S, P, s1, T1, x, keep1);
      xb1 |= 1u << (row0 + uint32_t(r));
    }
    if (keep2 != Dx2) {
      if (lane == 0) remove_value(S, P, s2, T2, x, keep2);
      xb2 |= 1u << (row0 + uint32_t(r));
    }
    racc1 &= v1;
    racc2 &= v2;
  }
  bool ry1 = false, ry2 = false;
  if (y_ok) {
    const uint32_t keep1 = racc1 & Dy1, keep2 = racc2 & Dy2;
    if (keep1 != Dy1) {
      remove_value(S, P, s1, T1, uint32_t(y), keep1);
      ry1 = true;
    }
    if (keep2 != Dy2) {
      remove_value(S, P, s2, T2, uint32_t(y), keep2);
      ry2 = true;
    }
  }
  const uint32_t yb1 = __ballot_sync(kFull, ry1), yb2 = __ballot_sync(kFull, ry2);
  const uint32_t J = uint32_t(y) >> 5;
  if (lane == 0 && (xb1 | yb1) != 0u) mark_changed(S, P, s1, slot_w, I, xb1, J, yb1);
  if (lane == 0 && (xb2 | yb2) != 0u) mark_changed(S, P, s2, slot_w, I, xb2, J, yb2);
  rem1 = (xb1 | yb1) != 0u;
  rem2 = (xb2 | yb2) != 0u;
}

// Next state of a mask (bit i: state c0 + i), or -1.
__device__ __forceinline__ int pop_state(uint32_t &m) {
  const int i = m ? __ffs(m) - 1 : -1;
  m &= m - 1u;
  return i;
}

// The decisions of rac_enforce_learned for the slab in ring stage `stg`,
// taken by the producer warp right after it issued the slab's copy, so that
// they run ahead of the consumers (every sweep; the first one counts a
// variable as changed when its input domain is not full).  Lane i stands for
// state c0 + i of each 32-state chunk: the Proposition-2 test (a variable of
// the slab's rows or columns changed in sweep k-1), the predictor's features
// (D_{k-1} read from global memory: the shared-memory copy of the consumers
// is still being filled), for states in their gated phase the logit (one
// tensor-core MLP pass per chunk), the decision, the pending flag and the
// optional trace record.  The decision words land in stage_dec(S, stg).
template <int kMT>
__device__ void score_stage(Smem &S, const LaunchParams &P, int stg, int sl, uint32_t ij,
                            uint32_t rows, int k, int slot_r, int lane) {
  const NetDev &N = P.net;
  const int n = N.n, B = P.n_states;
  const uint32_t I = ij & 0xFFFFu, J = ij >> 16;
  const uint32_t row0 = rows & 0xFFu, nrows = rows >> 8;
  const uint32_t rowmask = (nrows >= 32 ? kFull : ((1u << nrows) - 1u)) << row0;
  const uint32_t dfull = N.d >= 32 ? kFull : ((1u << N.d) - 1u);
  const int ncols = min(32, n - int(J) * 32);
  const int xrows = min(int(nrows), n - int(I) * 32 - int(row0));
  const float2 sf = N.slab_feat[sl];
  const bool learned = P.mlp != nullptr;
  const bool recording = P.tr_count != nullptr;
  const bool pending_on = P.pend != nullptr;
  uint32_t *dec = stage_dec(S, stg);
  for (int c0 = 0; c0 < B; c0 += 32) {
    const int s_l = c0 + lane;
    const uint32_t info = s_l < B ? S.st_info[s_l] : 1u;  // lanes past the end look finished
    const bool valid = (info & kInfoSweepMask) == 0u;
    const bool gated = learned && (info & kInfoGated);
    uint32_t cI = 0u, cJ = 0u;
    bool p2 = valid;  // sweep 1: every pair is a candidate
    if (valid && k >= 2) {
      const uint32_t *ch = P.chg + (int64_t(slot_r) * P.flag_stride + s_l) * N.nb;
      cJ = ld_dom(ch + J);
      cI = ld_dom(ch + I) & rowmask;
      p2 = (cI | cJ) != 0u;
    }
    // a chunk with fewer than min_scored gated candidates is evaluated
    // without scoring: the predictor's fixed cost per slab would exceed the
    // few evaluations it could save
    const bool scored = learned &&
                        __popc(__ballot_sync(kFull, valid && p2 && gated)) >= P.mlp_min_scored;
    const bool need = valid && p2 && ((gated && scored) || recording);
    const uint32_t need_mask = __ballot_sync(kFull, need);
    float f[kMlpIn];
    f[0] = float(min(k, 16)) * (1.0f / 16.0f);
    f[3] = sf.x;
    f[4] = sf.y;
    if (need) {
      // this lane's state: its column and row words, 16 loads in flight at a time
      const uint32_t *C = state_view(P, s_l, k).C;
      const uint32_t *Cy = C + int(J) * 32;
      const uint32_t *Cx = C + int(I) * 32 + int(row0);
      uint32_t cmin = 32u, csum = 0u, rmin = 32u, nfc = 0u, nfr = 0u;
#pragma unroll
      for (int h = 0; h < 32; h += 16) {
        uint32_t w[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) w[j] = h + j < ncols ? ld_dom(Cy + h + j) : dfull;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (h + j < ncols) {
            const uint32_t c = uint32_t(__popc(w[j]));
            cmin = min(cmin, c);
            csum += c;
            nfc += w[j] != dfull ? 1u : 0u;
          }
        }
      }
#pragma unroll
      for (int h = 0; h < 32; h += 16) {
        if (h >= xrows) break;
        uint32_t w[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) w[j] = h + j < xrows ? ld_dom(Cx + h + j) : dfull;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (h + j < xrows) {
            rmin = min(rmin, uint32_t(__popc(w[j])));
            nfr += w[j] != dfull ? 1u : 0u;
          }
        }
      }
      // sweep 1: a variable counts as changed when its input domain is not full
      f[1] = float(k == 1 ? nfr : uint32_t(__popc(cI))) / float(nrows);
      f[2] = float(k == 1 ? nfc : uint32_t(__popc(cJ))) * (1.0f / 32.0f);
      f[5] = float(cmin) / float(N.d);
      f[6] = float(csum) / float(ncols * N.d);
      f[7] = float(rmin) / float(N.d);
    } else {
      f[1] = f[2] = f[5] = f[6] = f[7] = 0.0f;
    }
    float z = __int_as_float(0x7FC00000);  // NaN: not scored
    if (scored && need_mask != 0u) z = mlp_warp_logits_mt<kMT>(smem_mlp(S), f);
    uint8_t *pd_ptr = pending_on ? P.pend + int64_t(sl) * P.flag_stride + s_l : nullptr;
    const bool pd = pending_on && valid && *pd_ptr != 0;
    bool ev;
    if (!valid)
      ev = false;
    else if (!learned)
      ev = p2;                   // Proposition 2 (sweep 1: everything)
    else if (gated && !scored)
      ev = p2;                   // too few candidates to score: evaluate them all
    else if (gated)
      ev = p2 && z > P.mlp_thr;  // the predictor's choice among the candidates
    else if (pending_on)
      ev = p2 || pd;             // verification: candidates and pending pairs
    else
      ev = true;                 // RAC_VERIFY_FULL: every slab
    const uint32_t ev_mask = __ballot_sync(kFull, ev);
    if (pending_on && valid) {
      // a skipped candidate becomes pending; an evaluated pair is no longer
      const bool npd = !ev && (pd || (gated && p2));
      if (npd != pd) {
        *pd_ptr = npd ? 1 : 0;
        const int delta = npd ? 1 : -1;
        atomicAdd(P.pend_slab + sl, delta);
        atomicAdd(P.pcount + s_l, delta);
      }
    }
    unsigned long long base = 0ull;
    if (recording) {
      if (lane == 0 && need_mask != 0u) base = atomicAdd(P.tr_count, (unsigned long long)__popc(need_mask));
      base = __shfl_sync(kFull, base, 0);
      const int64_t r = int64_t(base) + __popc(need_mask & lanemask_lt());
      if (need && r < P.tr_cap) {
#pragma unroll
        for (int j = 0; j < kMlpIn; ++j) P.tr_x[r * kMlpIn + j] = f[j];
        P.tr_y[r] = ev ? 0.0f : -1.0f;  // an evaluated record gets its label from the consumer
        if (P.tr_z) P.tr_z[r] = z;
        int32_t *w = P.tr_w + r * 4;
        w[0] = k | (gated ? (1 << 30) : 0);
        w[1] = P.tr_state_base + s_l;
        w[2] = int32_t(ij);
        w[3] = int32_t(rows);
      }
    }
    if (lane == 0) {
      if (P.tr_evals && ev_mask != 0u) atomicAdd(P.tr_evals, (unsigned long long)__popc(ev_mask));
      const int ch = c0 >> 5;
      dec[ch] = ev_mask;
      dec[32 + ch] = need_mask;
      dec[64 + ch] = uint32_t(base);
      dec[96 + ch] = uint32_t(base >> 32);
    }
  }
  __syncwarp();
}

// The consumers' side of rac_enforce_learned: the states the producer decided
// to evaluate (stage_dec), each warp its own states as in the plain kernel,
// the next state's words loaded during the current evaluation; evaluated
// records get their label.
template <int L>
__device__ void consume_slab_scored(Smem &S, const LaunchParams &P, const uint32_t *hdr,
                                    const uint4 *rel, const StageInfo &si, int stg, int k,
                                    int slot_w, int warp, int lane, int cg, int g, int sub,
                                    int wps, int groups, uint32_t &red_iter) {
  const NetDev &N = P.net;
  const int n = N.n, B = P.n_states;
  const uint32_t I = si.ij & 0xFFFFu, J = si.ij >> 16;
  const uint32_t row0 = si.rows & 0xFFu, nrows = si.rows >> 8;
  const int y = int(J) * 32 + lane;
  const bool y_ok = y < n;
  const int x_l = int(I) * 32 + int(row0) + lane;
  const bool x_ok = lane < int(nrows) && x_l < n;
  const bool cached = S.dom_cached != 0;
  const bool recording = P.tr_count != nullptr;
  const uint32_t *dec = stage_dec(S, stg);
  for (int c0 = 0; c0 < B; c0 += 32) {
    const uint32_t ev_all = dec[c0 >> 5];  // states past B are never set
    if (ev_all == 0u) continue;
    uint32_t m = warp_share(ev_all, g, groups, lane);
    // an evaluated record gets its label, from the warp that holds the whole
    // result (the first of the state's warps)
    auto label = [&](int s, bool removed, bool writer) {
      if (recording && writer && lane == 0) {
        const uint32_t need = dec[32 + (s >> 5)];
        if ((need >> (s & 31)) & 1u) {
          const int64_t r = int64_t(dec[64 + (s >> 5)] | (uint64_t(dec[96 + (s >> 5)]) << 32)) +
                            __popc(need & ((1u << (s & 31)) - 1u));
          if (r < P.tr_cap) P.tr_y[r] = removed ? 1.0f : 0.0f;
        }
      }
    };
    if (wps > 1) {  // fewer than four states: a state's rows over several warps
      for (int i = pop_state(m); i >= 0; i = pop_state(m)) {
        uint32_t Dy, Dxl;
        load_words(S, P, c0 + i, k, cached, y, y_ok, x_l, x_ok, Dy, Dxl);
        label(c0 + i,
              eval_state<L, true, true>(S, P, c0 + i, k, slot_w, hdr, rel, I, row0, nrows, y, y_ok,
                                        cached, Dy, Dxl, warp, lane, cg, g, sub, wps, red_iter),
              sub == 0);
      }
      continue;
    }
    if (__popc(ev_all) <= 2) {
      // one or two states to evaluate on this slab: the group's warps split
      // their rows, four or two warps per state (after meeting, as in
      // consume_slab)
      named_bar(group_bar(cg), kGroupWarps * 32);
      const int wps2 = __popc(ev_all) == 1 ? kGroupWarps : kGroupWarps / 2;
      const int g2 = (warp % kGroupWarps) / wps2, sub2 = (warp % kGroupWarps) % wps2;
      const int s2 = c0 + __fns(ev_all, 0, g2 + 1);  // the state of rank g2
      uint32_t Dy, Dxl;
      load_words(S, P, s2, k, cached, y, y_ok, x_l, x_ok, Dy, Dxl);
      label(s2,
            eval_state<L, true, true>(S, P, s2, k, slot_w, hdr, rel, I, row0, nrows, y, y_ok,
                                      cached, Dy, Dxl, warp, lane, cg, g2, sub2, wps2, red_iter),
            sub2 == 0);
      continue;
    }
    if (m == 0u) continue;
    // two states per pass; the next pair's words load during this one
    int i1 = pop_state(m), i2 = pop_state(m);
    uint32_t Dy1, Dx1, Dy2 = 0u, Dx2 = 0u;
    load_words(S, P, c0 + i1, k, cached, y, y_ok, x_l, x_ok, Dy1, Dx1);
    if (i2 >= 0) load_words(S, P, c0 + i2, k, cached, y, y_ok, x_l, x_ok, Dy2, Dx2);
    for (;;) {
      const int n1 = pop_state(m), n2 = pop_state(m);
      uint32_t Ny1 = 0u, Nx1 = 0u, Ny2 = 0u, Nx2 = 0u;
      if (n1 >= 0) load_words(S, P, c0 + n1, k, cached, y, y_ok, x_l, x_ok, Ny1, Nx1);
      if (n2 >= 0) load_words(S, P, c0 + n2, k, cached, y, y_ok, x_l, x_ok, Ny2, Nx2);
      if (i2 >= 0) {
        bool r1, r2;
        eval_pair<L>(S, P, c0 + i1, c0 + i2, k, slot_w, hdr, rel, I, row0, nrows, y, y_ok, Dy1,
                     Dx1, Dy2, Dx2, lane, r1, r2);
        label(c0 + i1, r1, true);
        label(c0 + i2, r2, true);
      } else {
        label(c0 + i1,
              eval_state<L, true, true>(S, P, c0 + i1, k, slot_w, hdr, rel, I, row0, nrows, y,
                                        y_ok, cached, Dy1, Dx1, warp, lane, cg, g, sub, wps,
                                        red_iter),
              true);
      }
      if (n1 < 0) break;
      i1 = n1;
      i2 = n2;
      Dy1 = Ny1;
      Dx1 = Nx1;
      Dy2 = Ny2;
      Dx2 = Nx2;
    }
  }
}

// Is slab sl (descriptor sd) streamed in a Proposition-2 sweep?  When a
// variable of its rows or columns changed in the previous sweep in some state
// (cu: the union over the states), or a pair of it is pending.
__device__ __forceinline__ bool slab_streamed(const LaunchParams &P, const SlabDesc &sd, int sl,
                                              const uint32_t *cu) {
  const uint32_t I = sd.ij & 0xFFFFu, J = sd.ij >> 16;
  const uint32_t row0 = sd.rows & 0xFFu, nrows = sd.rows >> 8;
  const uint32_t rowmask = (nrows >= 32 ? kFull : ((1u << nrows) - 1u)) << row0;
  return ld_dom(cu + J) != 0u || (ld_dom(cu + I) & rowmask) != 0u ||
         (P.pend_slab && ld_dom(reinterpret_cast<const uint32_t *>(P.pend_slab) + sl) != 0u);
}

// The producer warp's slab stream for sweep k: lane 0 issues a bulk copy for
// every slab this CTA streams (slab_streamed), then one end marker per
// consumer group.  Proposition-2 sweeps test 32 slabs at a time, a lane
// each, so that the tests' L2 reads overlap; the other sweeps stream every
// slab (sweep 1 of a search assignment: those on the assigned variable) from
// lane 0 alone.  kGate: the learned variants, where the producer also
// arrives on the stage's `issued` barrier once the slab is set (the stage's
// scorer warp gives the full barrier's second arrival).
template <int kGate, bool kDyn>
__device__ void produce_sweep(Smem &S, const LaunchParams &P, unsigned char *ring, int k,
                              int slot_r, int slot_c, int cta, int G, int my_slabs,
                              uint32_t &prod_it, int lane) {
  const NetDev &N = P.net;
  if (cta == 0 && lane == 0) {  // last used two sweeps (or a launch) ago
    P.sync->bar[slot_c] = 0ull;
    P.sync->claim[slot_c] = 0u;
  }
  // (learned gating: every slab while some state is in its full phase)
  const bool incr = (P.flags & RAC_INCREMENTAL) && k >= 2 && !(P.mlp && S.load_all);
  const uint32_t *cu = P.chgU + int64_t(slot_r) * N.nb;
  bool ok = true;  // lane 0's wait outcomes
  // lane 0: the copy of slab sl (descriptor sd) into the next ring stage
  auto issue_sd = [&](int sl, const SlabDesc &sd) {
    const int stg = prod_it % kStages;
    const uint32_t par = (prod_it / kStages) & 1u;
    if (!mbar_wait(&S.empty[stg], par ^ 1u, &P.sync->err, P.wait_limit_ns)) return false;
    S.stage[stg].sl = sl;
    S.stage[stg].ij = sd.ij;
    S.stage[stg].rows = sd.rows;
    if (kGate > 0) mbar_arrive(&S.issued[stg]);
    mbar_arrive_expect_tx(&S.full[stg], sd.nbytes);
    bulk_copy_g2s(ring + size_t(stg) * kStageBytes, N.rel + size_t(sd.rel_off16), sd.nbytes,
                  &S.full[stg]);
    ++prod_it;
    return true;
  };
  // lane 0: this CTA's slab j (slab cta + j G)
  auto issue = [&](int j) {
    const int sl = cta + j * G;
    return issue_sd(sl, j < kDescCache ? S.desc[j] : N.slabs[sl]);
  };
  // a plain sweep of the one-to-three-state variant claims the slabs beyond
  // each CTA's first kStaticSlabs dynamically.  The gated variants and the
  // seeded first sweep keep the static split (pending flags and the seed
  // filter are per owner), and so does the many-state variant: there the
  // two slabs of a claimed batch (neighbours in one tile, the same column
  // block) sent their removals and change marks to the same words from two
  // consumer groups at once, and the launch got slower (595 -> 674 us for
  // n=1000, d=24 with 32 states)
  const bool dyn = kDyn && kGate == 0 && !(k == 1 && P.seed_var >= 0);
  if (!incr) {
    if (lane != 0) return;
    const int n_static = dyn ? (my_slabs < kStaticSlabs ? my_slabs : kStaticSlabs) : my_slabs;
    // in sweep 1 the first slab may already be on its way
    for (int j = (k == 1 && prod_it == 1) ? 1 : 0; j < n_static; ++j) {
      if (k == 1 && P.seed_var >= 0) {
        const SlabDesc sd = j < kDescCache ? S.desc[j] : N.slabs[cta + j * G];
        if (!slab_touches_seed(P, sd.ij & 0xFFFFu, sd.ij >> 16, sd.rows & 0xFFu, sd.rows >> 8))
          continue;  // sweep 1 of an assignment: only constraints on the assigned variable
      }
      if (!(ok = issue(j))) break;
    }
    if (dyn && ok && int64_t(kStaticSlabs) * G < int64_t(N.n_slabs)) {
      // slabs [kStaticSlabs G, n_slabs), kClaimBatch at a time; the next
      // batch is claimed before this one's copies wait for free stages
      uint32_t *ctr = &P.sync->claim[(slot_r + 1) % 3];  // this sweep's slot
      const int first_dyn = kStaticSlabs * G;
      int lo = first_dyn + int(atomicAdd(ctr, uint32_t(kClaimBatch)));
      while (ok && lo < N.n_slabs) {
        SlabDesc sd[kClaimBatch];
#pragma unroll
        for (int i = 0; i < kClaimBatch; ++i)
          if (lo + i < N.n_slabs) sd[i] = N.slabs[lo + i];
        const int next = first_dyn + int(atomicAdd(ctr, uint32_t(kClaimBatch)));
#pragma unroll
        for (int i = 0; i < kClaimBatch; ++i)
          if (ok && lo + i < N.n_slabs) ok = issue_sd(lo + i, sd[i]);
        lo = next;
      }
    }
  } else {
    for (int j0 = 0; j0 < my_slabs; j0 += 32) {
      const int jl = j0 + lane;
      bool act = false;
      if (jl < my_slabs) {
        const int sl = cta + jl * G;
        act = slab_streamed(P, jl < kDescCache ? S.desc[jl] : N.slabs[sl], sl, cu);
      }
      uint32_t am = __ballot_sync(kFull, act);
      if (lane == 0) {
        while (am != 0u && ok) {
          ok = issue(j0 + __ffs(am) - 1);
          am &= am - 1u;
        }
      }
      if (__shfl_sync(kFull, ok ? 1 : 0, 0) == 0) break;
    }
    if (lane != 0) return;
  }
  // end of this sweep's slabs: one marker for each consumer group
  for (int e = 0; e < kGroups && ok; ++e) {
    const int stg = prod_it % kStages;
    const uint32_t par = (prod_it / kStages) & 1u;
    if (!mbar_wait(&S.empty[stg], par ^ 1u, &P.sync->err, P.wait_limit_ns)) {
      ok = false;
      break;
    }
    S.stage[stg].sl = -1;
    if (kGate > 0) mbar_arrive(&S.issued[stg]);
    mbar_arrive(&S.full[stg]);
    ++prod_it;
  }
  if (!ok) S.abort = 1;
}

// Scorer warp sc of rac_enforce_learned: the stages of consumer group sc
// (ring positions sc, sc + 3, ...), in order; for each, waits until the
// producer has set the slab, takes the decisions (score_stage) and gives the
// stage's second full-barrier arrival.  Ends the sweep at the group's marker.
template <int kMT>
__device__ void score_sweep(Smem &S, const LaunchParams &P, int k, int slot_r, int sc,
                            uint32_t &sc_it, int lane) {
  for (;;) {
    const uint32_t pos = sc_it * kGroups + sc;
    const int stg = pos % kStages;
    const uint32_t par = (pos / kStages) & 1u;
    uint32_t ok = 1u;
    if (lane == 0) ok = mbar_wait(&S.issued[stg], par, &P.sync->err, P.wait_limit_ns) ? 1u : 0u;
    ok = __shfl_sync(kFull, ok, 0);
    if (!ok) {
      if (lane == 0) S.abort = 1;
      return;
    }
    const StageInfo si = S.stage[stg];
    if (si.sl >= 0) score_stage<kMT>(S, P, stg, si.sl, si.ij, si.rows, k, slot_r, lane);
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.full[stg]);
    ++sc_it;
    if (si.sl < 0) return;
  }
}

template <int L, int kVar>
__device__ void consume_slab(Smem &S, const LaunchParams &P, const unsigned char *stage,
                             const StageInfo &si, int stg, int k, int slot_r, int slot_w,
                             int warp, int lane, uint32_t &red_iter) {
  constexpr int kGW = group_warps(kVar);
  const int cg = warp / kGW, lw = warp % kGW;
  const NetDev &N = P.net;
  const int n = N.n;
  const uint32_t I = si.ij & 0xFFFFu, J = si.ij >> 16;
  const uint32_t row0 = si.rows & 0xFFu, nrows = si.rows >> 8;
  const uint32_t *hdr = reinterpret_cast<const uint32_t *>(stage);
  const uint4 *rel = reinterpret_cast<const uint4 *>(stage) + (2 * nrows) / 4;
  const int y = int(J) * 32 + lane;
  const bool y_ok = y < n;
  // states are split over warp groups, rows over the warps of a group
  static_assert(kGroupWarps == 4, "state grouping below assumes 4 warps per consumer group");
  const int wps = P.n_states >= 4 ? 1 : (P.n_states >= 2 ? 2 : 4);
  const int groups = kGW / wps;
  const int g = lw / wps, sub = lw % wps;
  const bool incr = (P.flags & RAC_INCREMENTAL) && k >= 2;
  const uint32_t rowmask = (nrows >= 32 ? kFull : ((1u << nrows) - 1u)) << row0;
  const bool cached = S.dom_cached != 0;
  if (k == 1 && P.seed_var >= 0 && !slab_touches_seed(P, I, J, row0, nrows)) return;
  if constexpr (kVar >= kVarGated1) {
    consume_slab_scored<L>(S, P, hdr, rel, si, stg, k, slot_w, warp, lane, cg, g, sub, wps,
                           groups, red_iter);
  } else if constexpr (kVar == kVarFew) {
    // one to three states, each split over several warps: a short loop
    for (int s = g; s < P.n_states; s += groups) {
      if (S.st_info[s] & kInfoSweepMask) continue;  // finished state
      if (incr && chg_word(S, P, slot_r, s, J) == 0u &&
          (chg_word(S, P, slot_r, s, I) & rowmask) == 0u)
        continue;
      eval_state<L, false, false>(S, P, s, k, slot_w, hdr, rel, I, row0, nrows, y, y_ok, cached,
                                  0u, 0u, warp, lane, cg, g, sub, wps, red_iter);
    }
  } else {
    const int x_l = int(I) * 32 + int(row0) + lane;
    const bool x_ok = lane < int(nrows) && x_l < n;
    // one warp per state (four or more states): 32 states at a time, lane i
    // checking state c0 + i (running, and with RAC_INCREMENTAL a
    // Proposition-2 candidate), the warp taking its share of them; the words
    // of the next state are loaded while the current one is evaluated
    for (int c0 = 0; c0 < P.n_states; c0 += 32) {
      const int s_l = c0 + lane;
      bool act = s_l < P.n_states && !(S.st_info[s_l] & kInfoSweepMask);
      if (act && incr)
        act = chg_word(S, P, slot_r, s_l, J) != 0u ||
              (chg_word(S, P, slot_r, s_l, I) & rowmask) != 0u;
      uint32_t am = __ballot_sync(kFull, act);  // the same in every warp of the group
      if (am == 0u) continue;
      if (__popc(am) <= 2) {
        // one or two states on this slab (late sweeps): the group's warps
        // split their rows, five (all) or two warps per state, as with few states.
        // The group meets first: which warps share a state barrier depends
        // on the chunk, and a warp still in an earlier chunk's split must not
        // meet one of this chunk's on the same barrier.
        named_bar(group_bar(cg), kGW * 32);
        const int na = __popc(am);
        const int wps2 = na == 1 ? kGW : kGW / 2;  // a fifth warp of a group sits out two states
        const int g2 = lw / wps2, sub2 = lw % wps2;
        if (g2 < na) {
          const int s2 = c0 + __fns(am, 0, g2 + 1);  // the state of rank g2
          uint32_t Dy, Dxl;
          load_words(S, P, s2, k, cached, y, y_ok, x_l, x_ok, Dy, Dxl);
          eval_state<L, false, true>(S, P, s2, k, slot_w, hdr, rel, I, row0, nrows, y, y_ok,
                                     cached, Dy, Dxl, warp, lane, cg, g2, sub2, wps2, red_iter);
        } else {
          ++red_iter;  // every warp of the group keeps the same reduction-buffer parity
        }
        continue;
      }
      am = warp_share(am, g, groups, lane);
      if (am == 0u) continue;
      // two states per pass (eval_pair); the next pair's words load during
      // this one
      int i1 = pop_state(am), i2 = pop_state(am);
      uint32_t Dy1, Dx1, Dy2 = 0u, Dx2 = 0u;
      load_words(S, P, c0 + i1, k, cached, y, y_ok, x_l, x_ok, Dy1, Dx1);
      if (i2 >= 0) load_words(S, P, c0 + i2, k, cached, y, y_ok, x_l, x_ok, Dy2, Dx2);
      for (;;) {
        const int n1 = pop_state(am), n2 = pop_state(am);
        uint32_t Ny1 = 0u, Nx1 = 0u, Ny2 = 0u, Nx2 = 0u;
        if (n1 >= 0) load_words(S, P, c0 + n1, k, cached, y, y_ok, x_l, x_ok, Ny1, Nx1);
        if (n2 >= 0) load_words(S, P, c0 + n2, k, cached, y, y_ok, x_l, x_ok, Ny2, Nx2);
        if (i2 >= 0) {
          bool r1, r2;
          eval_pair<L>(S, P, c0 + i1, c0 + i2, k, slot_w, hdr, rel, I, row0, nrows, y, y_ok, Dy1,
                       Dx1, Dy2, Dx2, lane, r1, r2);
        } else {
          eval_state<L, false, true>(S, P, c0 + i1, k, slot_w, hdr, rel, I, row0, nrows, y, y_ok,
                                     cached, Dy1, Dx1, warp, lane, cg, g, sub, wps, red_iter);
        }
        if (n1 < 0) break;
        i1 = n1;
        i2 = n2;
        Dy1 = Ny1;
        Dx1 = Nx1;
        Dy2 = Ny2;
        Dx2 = Nx2;
      }
    }
  }
}

// L: the relation layout (whole-word rows of 4L bits for L = 1..8, packed
// rows of 4q bits for L = 16 + q), fixed per network.
// kVar: the plain variants for one to three states (kVarFew: a state's rows
// split over several warps) and for four or more (kVarMany: a warp per
// state, words prefetched), and the variants of rac_enforce_learned (learned
// gating and/or trace records) whose producer warp scores up to 16 or up to
// 32 states at a time (one or two MMA M tiles).  Separate kernels keep each
// one's instruction footprint small: a launch after an L2 flush fetches its
// code from HBM.  kDone: the instance the host entry point launches, which
// publishes a completion number to host memory at its end (P.host_done); a
// separate instance keeps that code out of every other launch, where it had
// cost 1-5% of the time.
template <int L, int kVar, bool kDone>
__global__ void __launch_bounds__(threads_for(kVar), 1) rac_bits_kernel(const LaunchParams P) {
  constexpr int kGate = kVar >= kVarGated1 ? 1 : 0;
  constexpr int kGW = group_warps(kVar), kCW = consumer_warps(kVar);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *ring = smem_raw;
  Smem &S = *reinterpret_cast<Smem *>(smem_raw + size_t(kStages) * kStageBytes);
  const NetDev &N = P.net;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, cta = blockIdx.x;
  const int B = P.n_states;
  const int n = N.n;
  const int64_t gtid = int64_t(cta) * blockDim.x + tid;
  const int64_t gstride = int64_t(G) * blockDim.x;
  const int my_slabs = cta < N.n_slabs ? (N.n_slabs - cta + G - 1) / G : 0;
  const bool is_producer = warp == kCW;
  const bool is_scorer = warp > kCW;  // gated variants only
  // consumer thread index and grid-wide consumer stride
  const int ctid = tid;
  const int64_t cgtid = int64_t(cta) * (kCW * 32) + ctid;
  const int64_t cgstride = int64_t(G) * (kCW * 32);

  // Loads the first sweep waits on, issued before the set-up so that their
  // latency (a cold miss after an idle spell) overlaps it: this CTA's first
  // slab descriptors (producer lanes) and the workspace's barrier base and
  // error word (thread 0; plain loads: the previous launch on this
  // workspace ran on the same stream and has finished).
  SlabDesc desc0 = {};
  if (is_producer && lane < my_slabs) desc0 = N.slabs[cta + lane * G];
  uint32_t base0 = 0u, err0 = 0u;
  if (tid == 0) {
    base0 = ld_dom(&P.sync->base);
    err0 = ld_dom(&P.sync->err);
  }

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&S.full[i], kGate > 0 ? 2 : 1);  // gated: the copy, then the decisions
      mbar_init(&S.empty[i], kGW);
      mbar_init(&S.issued[i], 1);
    }
    fence_mbar_init();
    S.all_done = 0;
    S.load_all = 1;
    S.abort = 0;
    S.failed = 0;
    S.dom_cached = int64_t(B) * n <= dom_cache_words<kGate>() ? 1u : 0u;
    // the changed-variable words of every state go after the cached domains
    S.chg_off = S.dom_cached ? uint32_t((int64_t(B) * n + 3) & ~int64_t(3)) : 0u;
    S.chg_cached =
        int64_t(S.chg_off) + int64_t(B) * N.nb <= dom_cache_words<kGate>() ? 1u : 0u;
    S.chgu_local = (P.flags & RAC_INCREMENTAL) && N.nb <= kChgULocal ? 1u : 0u;
  }
  if constexpr (kGate > 0) {
    if (P.mlp) {
      uint4 *dst = reinterpret_cast<uint4 *>(S.dom + (kDomWords - kMlpSmemWords));
      for (int i = tid; i < kPackVec4; i += blockDim.x) dst[i] = P.mlp[i];
    }
    if (P.pend) {
      // no pair of this CTA's slabs is pending yet (the per-state counts were
      // zeroed before the launch)
      for (int64_t i = tid; i < int64_t(my_slabs) * B; i += blockDim.x) {
        const int sl = cta + int(i / B) * G;
        P.pend[int64_t(sl) * P.flag_stride + (i % B)] = 0;
      }
      for (int j = tid; j < my_slabs; j += blockDim.x) P.pend_slab[cta + j * G] = 0;
    }
  }
  for (int w = tid; w < kChgULocal; w += blockDim.x) S.chgu_loc[w] = 0u;
  for (int s = tid; s < B; s += blockDim.x) {
    S.st_info[s] = P.mlp ? kInfoGated : 0u;  // learned gating starts with a gated sweep
    S.any_loc[s] = 0;
    S.wipe_loc[s] = 0;
  }
  __syncthreads();

  uint32_t ring_it = 0;   // consumer-side position in the ring (per consumer group)
  uint32_t prod_it = 0;   // producer-side position in the ring
  uint32_t sc_it = 0;     // scorer-side position in its consumer group's stages
  uint32_t red_iter = 0;  // parity of the cross-warp reduction buffer
  if (is_producer) {
    if (lane == 0 && my_slabs > 0 && cta < P.n_first &&
        (P.seed_var < 0 || slab_touches_seed(P, P.first[cta].ij & 0xFFFFu, P.first[cta].ij >> 16,
                                             P.first[cta].rows & 0xFFu, P.first[cta].rows >> 8))) {
      // the first slab's descriptor came with the launch: no load before it
      const SlabDesc sd = P.first[cta];
      S.stage[0].sl = cta;
      S.stage[0].ij = sd.ij;
      S.stage[0].rows = sd.rows;
      if (kGate > 0) mbar_arrive(&S.issued[0]);
      mbar_arrive_expect_tx(&S.full[0], sd.nbytes);
      bulk_copy_g2s(ring, N.rel + size_t(sd.rel_off16), sd.nbytes, &S.full[0]);
      prod_it = 1;
    }
    prod_it = __shfl_sync(kFull, prod_it, 0);
    // this CTA's slab descriptors (slabs cta, cta + G, ...)
    for (int j = lane; j < my_slabs && j < kDescCache; j += 32)
      S.desc[j] = j < 32 ? desc0 : N.slabs[cta + j * G];
    __syncwarp();
  } else if (ctid == 0) {
    S.base = base0;
    S.poisoned = err0 != 0u ? 1u : 0u;
  }
  __syncthreads();
  const uint32_t base = S.base;

  int k = 0;
  if (S.poisoned) {
    S.failed = 1;
  } else {
    for (;;) {
      ++k;
      const int slot_w = int((base + k) % 3), slot_r = int((base + k + 2) % 3);
      const int slot_c = int((base + k + 1) % 3);

      if (is_scorer) {
        if constexpr (kGate > 0)
          score_sweep<kVar - kVarGated1 + 1>(S, P, k, slot_r, warp - kCW - 1, sc_it,
                                             lane);
      } else if (is_producer) {
        produce_sweep<kGate, kVar == kVarFew>(S, P, ring, k, slot_r, slot_c, cta, G, my_slabs,
                                              prod_it, lane);
      } else {
        const int64_t stride = P.flag_stride;
        // this sweep's domains D_{k-1} into shared memory
        // (eight independent loads per thread before any store, so that a
        // thread waits about one round trip, not one per word)
        if (S.dom_cached) {
          constexpr int kU = 8;
          const int total = B * n;
          for (int i0 = ctid; i0 < total; i0 += kU * kCW * 32) {
            uint32_t v[kU];
#pragma unroll
            for (int j = 0; j < kU; ++j) {
              const int i = i0 + j * kCW * 32, s = i / n;
              v[j] = i < total && !(S.st_info[s] & kInfoSweepMask)
                         ? ld_dom(state_view(P, s, k).C + (i - s * n))
                         : 0u;
            }
#pragma unroll
            for (int j = 0; j < kU; ++j) {
              const int i = i0 + j * kCW * 32, s = i / n;
              if (i < total && !(S.st_info[s] & kInfoSweepMask))
                S.dom[i] = k == 1 ? input_word(P, i - s * n, v[j]) : v[j];
            }
          }
        }
        // clear the slot written next sweep (last read two sweeps ago)
        for (int64_t i = cgtid; i < stride; i += cgstride) {
          P.any[slot_c * stride + i] = 0u;
          P.wipe[slot_c * stride + i] = 0u;
        }
        for (int64_t i = cgtid; i < stride * N.nb; i += cgstride)
          P.chg[slot_c * stride * N.nb + i] = 0u;
        for (int64_t i = cgtid; i < N.nb; i += cgstride) P.chgU[int64_t(slot_c) * N.nb + i] = 0u;
        // the variables every state changed in sweep k-1, read once here
        // instead of once per slab
        if (k >= 2 && S.chg_cached) {
          const uint32_t *src = P.chg + int64_t(slot_r) * stride * N.nb;
          for (int i = ctid; i < B * N.nb; i += kCW * 32)
            S.dom[S.chg_off + i] = ld_dom(src + i);
        }
        named_bar(kAllConsumersBar, kCW * 32);
        if (k == 1) {
          // A := dom_in; B (all ones between launches) &= dom_in -- an AND,
          // so it needs no ordering against this sweep's removals; note
          // empty input domains.
          for (int64_t i = cgtid; i < int64_t(B) * n; i += cgstride) {
            const int s = int(i / n), x = int(i % n);
            const int64_t off = state_offset(P, s);
            const uint32_t v = S.dom_cached ? S.dom[i] : input_word(P, x, P.dom_in[off + x]);
            atomicAnd(P.bufB + i, v);
            if (P.dom_out != P.dom_in) P.dom_out[off + x] = v;
            if (v == 0u) S.wipe_loc[s] = 1;  // D_1 will hold this empty domain
          }
        } else {
          // owner step: T still holds D_{k-2}; AND D_{k-1} into it where it
          // differs (a warp per 32-variable block of a state, lane = variable);
          // a domain that sweep k-1 emptied is found here (see remove_value)
          const int64_t cw = int64_t(cta) * kCW + warp;
          for (int64_t i = cw; i < int64_t(B) * N.nb; i += int64_t(G) * kCW) {
            const int s = int(i / N.nb), blk = int(i % N.nb);
            if (S.st_info[s] & kInfoSweepMask) continue;
            const int x = blk * 32 + lane;
            if (!((chg_word(S, P, slot_r, s, uint32_t(blk)) >> lane) & 1u)) continue;
            const StateView V = state_view(P, s, k);
            const uint32_t c = S.dom_cached ? S.dom[s * n + x] : ld_dom(V.C + x);
            atomicAnd(V.T + x, c);
            if (c == 0u) S.wipe_loc[s] = 1;
          }
        }
        // consumer group cg takes ring positions cg, cg + kGroups, ...
        const int cg = warp / kGW;
        const bool group_leader = (warp % kGW) == 0 && lane == 0;
        for (;;) {
          const uint32_t pos = ring_it * kGroups + cg;
          const int stg = pos % kStages;
          const uint32_t par = (pos / kStages) & 1u;
          // One thread takes the bounded wait and every warp of the group
          // follows its outcome, so a wait that gives up never leaves a peer
          // warp blocked on a named barrier inside the slab evaluation.
          if (group_leader) S.stage_ok[stg] = mbar_wait(&S.full[stg], par, &P.sync->err, P.wait_limit_ns) ? 1u : 0u;
          named_bar(group_bar(cg), kGW * 32);
          if (!S.stage_ok[stg]) {
            if (group_leader) S.abort = 1;
            break;
          }
          if (lane == 0) mbar_try_wait(&S.full[stg], par);  // completed: acquire the copy
          __syncwarp();
          const StageInfo si = S.stage[stg];
          if (si.sl >= 0)
            consume_slab<L, kVar>(S, P, ring + size_t(stg) * kStageBytes, si, stg, k, slot_r, slot_w, warp,
                            lane, red_iter);
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.empty[stg]);
          ++ring_it;
          if (si.sl < 0) break;
        }
      }
      __syncthreads();

      // this CTA's flags for sweep k (per state only when there are several)
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
      if (S.chgu_local) {
        for (int w = tid; w < N.nb; w += blockDim.x) {
          const uint32_t u = S.chgu_loc[w];
          if (u != 0u) {
            atomicOr(P.chgU + int64_t(slot_w) * N.nb + w, u);
            S.chgu_loc[w] = 0u;
          }
        }
      }
      if (S.abort) S.failed = 1;
      grid_barrier(S, P, slot_w);
      if (S.failed) break;

      // decisions (every CTA reads the same flags and takes the same ones)
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
        const uint32_t t_is_b = (k & 1) ? kInfoResB : 0u;               // T of sweep k
        const uint32_t c_is_b = (k >= 2 && !(k & 1)) ? kInfoResB : 0u;  // C of sweep k
        const bool gated = (info & kInfoGated) != 0u;
        // a sweep that removed nothing ends the state if it proves the
        // fixpoint: any sweep of the plain and Proposition-2 recurrences; with
        // pending pairs, one that left no pair pending; with RAC_VERIFY_FULL,
        // a full sweep
        const bool proves = !P.mlp ? true
                            : P.pend ? ld_dom(reinterpret_cast<const uint32_t *>(P.pcount) + s) == 0u
                                     : !gated;
        if (stop && wp) {
          info |= uint32_t(k) | t_is_b | info_status_bits(RAC_WIPEOUT);
        } else if (!any && proves) {
          info |= uint32_t(k) | c_is_b |
                  info_status_bits((info & kInfoWiped) ? RAC_WIPEOUT : RAC_OK);
        } else if ((P.max_sweeps > 0 && k >= P.max_sweeps) || k >= P.sweep_bound) {
          info |= uint32_t(k) | t_is_b | info_status_bits(RAC_ETIMEOUT);
        } else if (P.mlp) {
          info = any ? (info | kInfoGated) : (info & ~kInfoGated);
        }
        S.st_info[s] = info;
      }
      if (tid == 0) {
        S.all_done = 1;
        S.load_all = 0;
      }
      __syncthreads();
      for (int s = tid; s < B; s += blockDim.x) {
        const uint32_t info = S.st_info[s];
        if (!(info & kInfoSweepMask)) {
          S.all_done = 0;
          if (!(info & kInfoGated) && (P.flags & RAC_VERIFY_FULL)) S.load_all = 1;
        }
      }
      __syncthreads();
      if (S.all_done) break;
    }
  }

  // Epilogue: results that ended in buffer B move to dom_out and B goes back
  // to all ones; with P.host_out the results are also written there (host
  // memory: the caller's copy out).  The next launch on this workspace starts
  // at the barrier slot after this launch's last one (see Sync).
  if (S.abort) S.failed = 1;
  __syncthreads();
  const bool failed = S.failed != 0u;
  if (!S.poisoned) {
    for (int64_t i = gtid; i < int64_t(B) * n; i += gstride) {
      const int s = int(i / n), x = int(i % n);
      const int64_t o = state_offset(P, s) + x;
      if (!failed && (S.st_info[s] & kInfoResB)) {
        const uint32_t v = ld_dom(P.bufB + i);
        P.dom_out[o] = v;
        if (P.host_out) P.host_out[o] = v;
      } else if (P.host_out) {
        P.host_out[o] = ld_dom(P.dom_out + o);
      }
      P.bufB[i] = kFull;
    }
  }
  if (cta == 0) {
    if (tid == 0 && !failed) P.sync->base = (base + uint32_t(k)) % 3u;
    for (int s = tid; s < B; s += blockDim.x) {
      const uint32_t info = S.st_info[s];
      const int idx = P.contiguous ? s : P.res_idx[s];
      const int32_t its = int32_t(info & kInfoSweepMask) ? int32_t(info & kInfoSweepMask) : k;
      const int32_t st = failed ? RAC_EBARRIER : info_status(info);
      P.iterations[idx] = its;
      P.status[idx] = st;
      if (P.host_out) {
        int32_t *res = reinterpret_cast<int32_t *>(P.host_out + int64_t(B) * n);
        res[idx] = its;
        res[B + idx] = st;
      }
    }
  }
  if constexpr (kDone) {
    // the last CTA to finish its host writes publishes the completion
    // number: the caller reads the results once it sees it
    __syncthreads();
    if (tid == 0) {
      __threadfence_system();
      if (atomicAdd(&P.sync->done_cta, 1u) == uint32_t(G) - 1u) {
        P.sync->done_cta = 0u;
        const uint32_t seq = P.sync->done_seq + 1u;
        P.sync->done_seq = seq;
        __threadfence_system();
        *reinterpret_cast<volatile uint32_t *>(P.host_done) = seq;
      }
    }
  }
  if (failed && tid == 0) atomicOr(&P.sync->err, kErrCopyWait);  // poison (idempotent)
  // Drain copies still in flight (only after a failed wait or on a poisoned
  // workspace) before the CTA's shared memory goes away.
  if (is_producer && lane == 0) {
    const uint32_t first = prod_it > uint32_t(kStages) ? prod_it - kStages : 0u;
    for (uint32_t j = first; j < prod_it; ++j)
      mbar_wait(&S.full[j % kStages], (j / kStages) & 1u, &P.sync->err, P.wait_limit_ns);
  }
}

template <int L, int kVar, bool kDone>
rac_status launch_q(const LaunchParams &P, cudaStream_t stream) {
  static LaunchCache cache;
  const size_t smem = size_t(kStages) * kStageBytes + sizeof(Smem);
  int per_sm = 0, sms = 0;
  rac_status rc = persistent_shape(cache,
                                   reinterpret_cast<const void *>(rac_bits_kernel<L, kVar, kDone>),
                                   threads_for(kVar), smem, "bit-packed kernel set-up", &per_sm,
                                   &sms);
  if (rc != RAC_OK) return rc;
  // every resident CTA, but no more than the tiles (a CTA without a tile
  // would only join the sweep barriers) nor the network's cap
  int grid = per_sm * sms;
  grid = std::min(grid, std::max(1, P.net.n_slabs));
  if (P.net.max_ctas > 0) grid = std::min(grid, P.net.max_ctas);
  cudaError_t e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(threads_for(kVar));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, rac_bits_kernel<L, kVar, kDone>, P);
  if (e != cudaSuccess) return cuda_fail(e, "launch of the bit-packed kernel");
  return RAC_OK;
}

// The instance for the network's relation layout: whole-word rows of width
// q = dp / 4 here; packed rows (layout code 16 + q) in the packed unit, which
// compiles this file once more with RAC_BITS_PACKED_UNIT defined so that the
// two halves of the instances build in parallel.
template <int kVar, bool kDone>
rac_status launch_width(const LaunchParams &P, cudaStream_t stream) {
#ifndef RAC_BITS_PACKED_UNIT
  if (P.net.packed) return launch_bits_packed(P, stream, kVar, kDone);
  switch (P.net.q) {
    case 1: return launch_q<1, kVar, kDone>(P, stream);
    case 2: return launch_q<2, kVar, kDone>(P, stream);
    case 3: return launch_q<3, kVar, kDone>(P, stream);
    case 4: return launch_q<4, kVar, kDone>(P, stream);
    case 5: return launch_q<5, kVar, kDone>(P, stream);
    case 6: return launch_q<6, kVar, kDone>(P, stream);
    case 7: return launch_q<7, kVar, kDone>(P, stream);
    case 8: return launch_q<8, kVar, kDone>(P, stream);
    default: break;
  }
#else
  switch (P.net.q) {
    case 1: return launch_q<17, kVar, kDone>(P, stream);
    case 2: return launch_q<18, kVar, kDone>(P, stream);
    case 3: return launch_q<19, kVar, kDone>(P, stream);
    case 4: return launch_q<20, kVar, kDone>(P, stream);
    case 5: return launch_q<21, kVar, kDone>(P, stream);
    case 6: return launch_q<22, kVar, kDone>(P, stream);
    case 7: return launch_q<23, kVar, kDone>(P, stream);
    default: break;
  }
#endif
  set_error("unsupported relation width");
  return RAC_EINVAL;
}

}  // namespace

#ifdef RAC_BITS_PACKED_UNIT
rac_status launch_bits_packed(const LaunchParams &P, cudaStream_t stream, int var, bool done) {
  if (done) return launch_width<kVarFew, true>(P, stream);
  switch (var) {
    case kVarFew: return launch_width<kVarFew, false>(P, stream);
    case kVarMany: return launch_width<kVarMany, false>(P, stream);
    case kVarGated1: return launch_width<kVarGated1, false>(P, stream);
    default: return launch_width<kVarGated2, false>(P, stream);
  }
}
#else
rac_status launch_bits(const LaunchParams &P, cudaStream_t stream) {
  const bool gate = P.mlp != nullptr || P.tr_count != nullptr || P.tr_evals != nullptr;
  if (P.host_done) {  // the host entry point's one-to-three-state launch
    if (gate || P.n_states >= 4) {
      set_error("a completion word is published by the one-to-three-state launch only");
      return RAC_EINVAL;
    }
    return launch_width<kVarFew, true>(P, stream);
  }
  if (!gate) return P.n_states < 4 ? launch_width<kVarFew, false>(P, stream)
                                   : launch_width<kVarMany, false>(P, stream);
  // the producer warp scores 32 states at a time (lane = state): one MMA M
  // tile covers them while there are at most 16
  return P.n_states <= 16 ? launch_width<kVarGated1, false>(P, stream)
                          : launch_width<kVarGated2, false>(P, stream);
}
#endif

}  // namespace rac
