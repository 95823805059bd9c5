// Batched enforcement: many networks (of any n and d), each with its own
// domain states, swept to their fixpoints in ONE persistent cooperative
// launch.  The support test is the one of the single-network kernel (Eq. 1,
// Fig. 1: per relation, fwd bit a = (R[a] & D_y) != 0, rev = OR of the rows
// in D_x, both directions from one read), applied to every running state of
// the relation's network while the slab sits in shared memory, so a slab is
// read once per sweep for all of its network's states.
//
// Work: global slab g of job (network) j; CTA c streams slabs c, c+G, ...
// through a 6-stage bulk-copy ring (a producer warp).  Three groups of four
// consumer warps take alternate stages; the warps of a group take the slab's
// job states by rank and evaluate them two per pass (one or two states: the
// group splits their rows), loading a state's column and row words straight
// into registers (the next pair's while the current one is evaluated).  The
// relation width is dispatched once per slab.
//
// Per sweep: one barrier after the removals (its word counts the CTAs that
// removed values), then the owners of the states (state t belongs to CTA
// t mod G) take the per-state decisions of Algorithm 1 and a second barrier
// publishes them and the number of states still running.  A sweep in which no
// CTA removed anything ends every running state at once.
#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {
namespace {

using namespace dev;

constexpr int kBGroupWarps = 4;
constexpr int kBGroups = 3;
constexpr int kBConsumerWarps = kBGroupWarps * kBGroups;
constexpr int kBThreads = (kBConsumerWarps + 1) * 32;
constexpr int kBStages = 6;
static_assert(kBStages % kBGroups == 0, "each ring stage belongs to one consumer group");

struct BStage {
  int32_t job;   // -1: end of the sweep's slabs
  int32_t slab;  // slab index inside the job
  uint32_t ij, rows;
};

struct BSmem {
  uint64_t full[kBStages];
  uint64_t empty[kBStages];
  BStage stage[kBStages];
  uint32_t base, poisoned, abort, failed;
  uint32_t any_total, wipe_total, running_total;
  uint32_t cta_any, cta_wipe, cta_running;
  uint32_t stage_ok[kBStages];
  uint32_t red[kBConsumerWarps][32];  // reverse masks of a state's rows split over warps
};
static_assert(size_t(kBStages) * kStageBytes + sizeof(BSmem) <= 232448,
              "shared memory of the batched kernel exceeds 227 KB");

constexpr uint32_t kInfoSweepMask = 0xFFFFFFu;
constexpr uint32_t kInfoResB = 1u << 24;
constexpr uint32_t kInfoWiped = 1u << 25;
__device__ __forceinline__ uint32_t info_status_bits(int st) { return uint32_t(st + 8) << 27; }
__device__ __forceinline__ int info_status(uint32_t v) { return int((v >> 27) & 31u) - 8; }


__device__ __forceinline__ int group_bar(int cg) { return 1 + cg; }
// the warps of state group g (< 2) of consumer group cg when a slab's rows
// are split over them
__device__ __forceinline__ int split_bar(int cg, int g) { return 1 + kBGroups + 2 * cg + g; }
static_assert(1 + kBGroups + 2 * kBGroups <= 16, "named barrier ids");

struct BView {
  const uint32_t *C;
  uint32_t *T;
};

// Buffers as in the single-network kernel: A = dom_out, B = bufB.
__device__ __forceinline__ BView bview(const BatchParams &P, int t, int k) {
  uint32_t *A = P.dom_out + P.state_off[t];
  uint32_t *B = P.bufB + P.scratch_off[t];
  BView v;
  if (k == 1) {
    v.C = P.dom_in + P.state_off[t];
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

__device__ void batch_barrier(const BatchParams &P, unsigned long long *w,
                              unsigned long long mine, unsigned long long target_mask,
                              uint32_t G, unsigned long long &out, uint32_t &failed) {
  // thread 0 only: the arrival releases this CTA's writes (the last arrival
  // acquires everyone's); poll the barrier word alone and look at the error
  // word and the time limit every 64 polls
  unsigned long long v = atom_add_acq_rel_u64(w, mine) + mine;
  const uint64_t t0 = global_timer();
  uint32_t spins = 0;
  while ((v & target_mask) < G) {
    if ((++spins & 63u) == 0u) {
      if (ld_acquire(&P.sync->err) != 0u) {
        failed = 1;
        break;
      }
      if (global_timer() - t0 > P.wait_limit_ns) {
        atomicOr(&P.sync->err, kErrGridWait);
        failed = 1;
        break;
      }
    }
    v = ld_acquire_u64(w);
  }
  out = v;
}

// The support test of relation t of a slab row (first relation roff, cnt
// relations) in relation layout L (rac_device.cuh: whole-word or packed rows).
template <int L>
__device__ __forceinline__ void support_dispatch_q(const uint4 *rel, uint32_t roff, uint32_t t,
                                                   uint32_t cnt, uint32_t Dx, uint32_t Dy,
                                                   uint32_t dfull, uint32_t &fwd, uint32_t &rev) {
  if (Dx == dfull)
    support_at<L, true>(rel, roff, t, cnt, Dx, Dy, fwd, rev);
  else
    support_at<L, false>(rel, roff, t, cnt, Dx, Dy, fwd, rev);
}

// Apply a removal to state t: D_k[v] &= keep.  As in kernel (a), only
// RAC_STOP_ON_WIPEOUT needs to know at once whether it emptied the domain;
// otherwise the next sweep's owner step finds emptied domains.
__device__ __forceinline__ void batch_remove(BSmem &S, const BatchParams &P, int t, int slot_w,
                                             uint32_t *T, uint32_t v, uint32_t keep) {
  if (P.flags & RAC_STOP_ON_WIPEOUT) {
    const uint32_t old = atomicAnd(T + v, keep);
    if (old != 0u && (old & keep) == 0u) {
      S.cta_wipe = 1;
      atomicOr(P.wipe + int64_t(slot_w) * P.total_states + t, 1u);
    }
  } else {
    atomicAnd(T + v, keep);
  }
}

// The variables one evaluation of state t removed values from (xbits in
// block I, ybits in block Jb): one flag and at most four atomics per
// evaluation instead of one per removal.
__device__ __forceinline__ void batch_mark(BSmem &S, const BatchParams &P, const BatchJob &J,
                                           int t, int64_t chgoff, int slot_w, uint32_t I,
                                           uint32_t xbits, uint32_t Jb, uint32_t ybits) {
  S.cta_any = 1;
  atomicOr(P.any + int64_t(slot_w) * P.total_states + t, 1u);
  uint32_t *ch = P.chg + int64_t(slot_w) * P.chg_slot_words + chgoff;
  uint32_t *cu = P.chgU + int64_t(slot_w) * P.u_slot_words + J.u_off;
  const bool incr = (P.flags & RAC_INCREMENTAL) != 0u;
  if (xbits) {
    atomicOr(ch + I, xbits);
    if (incr) atomicOr(cu + I, xbits);
  }
  if (ybits) {
    atomicOr(ch + Jb, ybits);
    if (incr) atomicOr(cu + Jb, ybits);
  }
}

// One or two states (kTwo) of job J on one slab in one pass: each relation
// chunk is read once for both, and the two support tests give the warp
// independent work.  State u: index t_u, D_k buffer T_u, chg offset co_u,
// column word Dy_u and row words Dx_ul (lane r: row r).
template <int L, bool kTwo>
__device__ __forceinline__ void batch_eval(BSmem &S, const BatchParams &P, const BatchJob &J,
                                           int slot_w, const uint32_t *hdr, const uint4 *rel,
                                           uint32_t I, uint32_t Jb, uint32_t row0, uint32_t nrows,
                                           int y, bool y_ok, int lane, int t1, uint32_t *T1,
                                           int64_t co1, uint32_t Dy1, uint32_t Dx1l, int t2,
                                           uint32_t *T2, int64_t co2, uint32_t Dy2,
                                           uint32_t Dx2l) {
  const uint32_t dfull = J.d >= 32 ? kFull : ((1u << J.d) - 1u);
  uint32_t racc1 = kFull, racc2 = kFull, xb1 = 0u, xb2 = 0u;
  for (int r = 0; r < int(nrows); ++r) {
    const uint32_t pm = hdr[r];
    if (pm == 0u) continue;
    const uint32_t Dx1 = __shfl_sync(kFull, Dx1l, r);
    const uint32_t Dx2 = kTwo ? __shfl_sync(kFull, Dx2l, r) : 0u;
    uint32_t f1 = kFull, v1 = kFull, f2 = kFull, v2 = kFull;
    if ((pm >> lane) & 1u) {
      const uint32_t tt = __popc(pm & lanemask_lt());
      const uint32_t roff = hdr[nrows + r], cnt = __popc(pm);
      if (!kTwo)
        support_dispatch_q<L>(rel, roff, tt, cnt, Dx1, Dy1, dfull, f1, v1);
      else if (Dx1 == dfull && Dx2 == dfull)
        support_pair_at<L, true>(rel, roff, tt, cnt, Dx1, Dy1, Dx2, Dy2, f1, v1, f2, v2);
      else
        support_pair_at<L, false>(rel, roff, tt, cnt, Dx1, Dy1, Dx2, Dy2, f1, v1, f2, v2);
    }
    const uint32_t x = I * 32u + row0 + uint32_t(r);
    const uint32_t keep1 = __reduce_and_sync(kFull, f1) & Dx1;
    if (keep1 != Dx1) {
      if (lane == 0) batch_remove(S, P, t1, slot_w, T1, x, keep1);
      xb1 |= 1u << (row0 + uint32_t(r));
    }
    racc1 &= v1;
    if (kTwo) {
      const uint32_t keep2 = __reduce_and_sync(kFull, f2) & Dx2;
      if (keep2 != Dx2) {
        if (lane == 0) batch_remove(S, P, t2, slot_w, T2, x, keep2);
        xb2 |= 1u << (row0 + uint32_t(r));
      }
      racc2 &= v2;
    }
  }
  bool ry1 = false, ry2 = false;
  if (y_ok) {
    const uint32_t keep1 = racc1 & Dy1;
    if (keep1 != Dy1) {
      batch_remove(S, P, t1, slot_w, T1, uint32_t(y), keep1);
      ry1 = true;
    }
    if (kTwo) {
      const uint32_t keep2 = racc2 & Dy2;
      if (keep2 != Dy2) {
        batch_remove(S, P, t2, slot_w, T2, uint32_t(y), keep2);
        ry2 = true;
      }
    }
  }
  const uint32_t yb1 = __ballot_sync(kFull, ry1);
  if (lane == 0 && (xb1 | yb1) != 0u) batch_mark(S, P, J, t1, co1, slot_w, I, xb1, Jb, yb1);
  if (kTwo) {
    const uint32_t yb2 = __ballot_sync(kFull, ry2);
    if (lane == 0 && (xb2 | yb2) != 0u) batch_mark(S, P, J, t2, co2, slot_w, I, xb2, Jb, yb2);
  }
}

// One state of job J on one slab with its rows split over the wps warps of
// state group g2 (sub = this warp's place): each warp takes rows sub, sub +
// wps, ...; the reverse masks meet in shared memory, and the group's first
// warp applies the column removals.  The caller has the consumer group meet
// before the call, which also frees the reduction slots of the previous one.
template <int L>
__device__ __forceinline__ void batch_eval_split(BSmem &S, const BatchParams &P, const BatchJob &J,
                                                 int slot_w, const uint32_t *hdr,
                                                 const uint4 *rel, uint32_t I, uint32_t Jb,
                                                 uint32_t row0, uint32_t nrows, int y, bool y_ok,
                                                 int lane, int warp, int cg, int g2, int sub,
                                                 int wps, int t, uint32_t *T, int64_t co,
                                                 uint32_t Dy, uint32_t Dxl) {
  const uint32_t dfull = J.d >= 32 ? kFull : ((1u << J.d) - 1u);
  uint32_t racc = kFull, xb = 0u;
  for (int r = sub; r < int(nrows); r += wps) {
    const uint32_t pm = hdr[r];
    if (pm == 0u) continue;
    const uint32_t Dx = __shfl_sync(kFull, Dxl, r);
    uint32_t f = kFull, v = kFull;
    if ((pm >> lane) & 1u) {
      const uint32_t tt = __popc(pm & lanemask_lt());
      support_dispatch_q<L>(rel, hdr[nrows + r], tt, __popc(pm), Dx, Dy, dfull, f,
                            v);
    }
    const uint32_t keep = __reduce_and_sync(kFull, f) & Dx;
    if (keep != Dx) {
      if (lane == 0) batch_remove(S, P, t, slot_w, T, I * 32u + row0 + uint32_t(r), keep);
      xb |= 1u << (row0 + uint32_t(r));
    }
    racc &= v;
  }
  S.red[warp][lane] = racc;
  named_bar(split_bar(cg, g2), wps * 32);
  bool ry = false;
  if (sub == 0) {
    for (int j = 1; j < wps; ++j) racc &= S.red[warp + j][lane];
    if (y_ok) {
      const uint32_t keep = racc & Dy;
      if (keep != Dy) {
        batch_remove(S, P, t, slot_w, T, uint32_t(y), keep);
        ry = true;
      }
    }
  }
  const uint32_t yb = __ballot_sync(kFull, ry);
  if (lane == 0 && (xb | yb) != 0u) batch_mark(S, P, J, t, co, slot_w, I, xb, Jb, yb);
}

// One slab of job J for every running state of J, by one consumer group.  The
// job's states go 32 at a time (lane i checks state base + i: running, and
// with RAC_INCREMENTAL a Proposition-2 candidate); warp lw of the group takes
// those of rank lw, lw + 4, ... among the ones to evaluate, so the group's
// warps get equal shares, and evaluates them two per pass (batch_eval): each
// state's column words (lane = column) and row words (lane = row) come in two
// coalesced loads, issued for the next pair while the current one is
// evaluated.
template <int L>
__device__ void batch_consume_q(BSmem &S, const BatchParams &P, const BatchJob &J,
                                const unsigned char *stage, const BStage &si, int k, int slot_r,
                                int slot_w, int cg, int lw, int lane) {
  const int n = J.n;
  const uint32_t I = si.ij & 0xFFFFu, Jb = si.ij >> 16;
  const uint32_t row0 = si.rows & 0xFFu, nrows = si.rows >> 8;
  const uint32_t *hdr = reinterpret_cast<const uint32_t *>(stage);
  const uint4 *rel = reinterpret_cast<const uint4 *>(stage) + (2 * nrows) / 4;
  const int y = int(Jb) * 32 + lane;
  const bool y_ok = y < n;
  const int x_l = int(I) * 32 + int(row0) + lane;
  const bool x_ok = lane < int(nrows) && x_l < n;
  const bool incr = (P.flags & RAC_INCREMENTAL) && k >= 2;
  const uint32_t rowmask = (nrows >= 32 ? kFull : ((1u << nrows) - 1u)) << row0;
  const uint32_t *Cbase = k == 1 ? P.dom_in : ((k & 1) ? P.dom_out : P.bufB);
  uint32_t *Tbase = (k == 1 || (k & 1)) ? P.bufB : P.dom_out;
  for (int base = 0; base < J.n_states; base += 32) {
    // lane i: state t = state_base + base + i
    const int q = base + lane;
    const int t = J.state_base + q;
    bool act = false;
    int64_t c_off = 0, t_off = 0, chgoff = 0;
    if (q < J.n_states) {
      act = (ld_dom(P.st_info + t) & kInfoSweepMask) == 0u;
      chgoff = P.chg_off[t];
      if (act && incr) {
        const uint32_t *ch = P.chg + int64_t(slot_r) * P.chg_slot_words + chgoff;
        act = ld_dom(ch + Jb) != 0u || (ld_dom(ch + I) & rowmask) != 0u;
      }
      if (act) {
        // the buffers of sweep k (as bview): C = D_{k-1}, T receives D_k
        const int64_t a = P.state_off[t], b = P.scratch_off[t];
        c_off = k == 1 ? a : ((k & 1) ? a : b);
        t_off = (k == 1 || (k & 1)) ? b : a;
      }
    }
    uint32_t am = __ballot_sync(kFull, act);  // the same in every warp of the group
    if (am == 0u) continue;
    if (__popc(am) <= 2) {
      // one or two states on this slab: the group's warps split their rows,
      // four or two warps per state.  The group meets first: which warps
      // share a split barrier depends on the chunk, and a warp still in an
      // earlier chunk's split must not meet one of this chunk's on the same
      // barrier.
      named_bar(group_bar(cg), kBGroupWarps * 32);
      const int wps = __popc(am) == 1 ? kBGroupWarps : kBGroupWarps / 2;
      const int g2 = lw / wps, sub = lw % wps;
      const int i = __fns(am, 0, g2 + 1);  // lane of the state of rank g2
      const int ts = __shfl_sync(kFull, t, i);
      const int64_t to = __shfl_sync(kFull, t_off, i);
      const int64_t co = __shfl_sync(kFull, chgoff, i);
      const int64_t cc = __shfl_sync(kFull, c_off, i);
      const uint32_t *C = Cbase + cc;
      const uint32_t Dy = y_ok ? ld_dom(C + y) : 0u;
      const uint32_t Dxl = x_ok ? ld_dom(C + x_l) : 0u;
      batch_eval_split<L>(S, P, J, slot_w, hdr, rel, I, Jb, row0, nrows, y, y_ok, lane,
                          cg * kBGroupWarps + lw, cg, g2, sub, wps, ts, Tbase + to, co, Dy, Dxl);
      continue;
    }
    // this warp's share: the states of rank lw, lw + 4, ... among them
    am = __ballot_sync(kFull, act && __popc(am & lanemask_lt()) % kBGroupWarps == lw);
    if (am == 0u) continue;
    auto pop = [&]() {
      const int i = am ? __ffs(am) - 1 : -1;
      am &= am - 1u;
      return i;
    };
    // the words of the state in lane ii (every lane must call this)
    auto fetch = [&](int ii, uint32_t &dy, uint32_t &dx) {
      const int64_t co = __shfl_sync(kFull, c_off, ii < 0 ? 0 : ii);
      dy = dx = 0u;
      if (ii < 0) return;
      const uint32_t *C = Cbase + co;
      dy = y_ok ? ld_dom(C + y) : 0u;
      dx = x_ok ? ld_dom(C + x_l) : 0u;
    };
    int i1 = pop(), i2 = pop();
    uint32_t Dy1, Dx1, Dy2, Dx2;
    fetch(i1, Dy1, Dx1);
    fetch(i2, Dy2, Dx2);
    for (;;) {
      const int n1 = pop(), n2 = pop();
      uint32_t Ny1, Nx1, Ny2, Nx2;
      fetch(n1, Ny1, Nx1);  // in flight during this evaluation
      fetch(n2, Ny2, Nx2);
      const int t1 = __shfl_sync(kFull, t, i1);
      const int64_t to1 = __shfl_sync(kFull, t_off, i1);
      const int64_t co1 = __shfl_sync(kFull, chgoff, i1);
      const int j2 = i2 < 0 ? i1 : i2;
      const int t2 = __shfl_sync(kFull, t, j2);
      const int64_t to2 = __shfl_sync(kFull, t_off, j2);
      const int64_t co2 = __shfl_sync(kFull, chgoff, j2);
      if (i2 >= 0)
        batch_eval<L, true>(S, P, J, slot_w, hdr, rel, I, Jb, row0, nrows, y, y_ok, lane, t1,
                            Tbase + to1, co1, Dy1, Dx1, t2, Tbase + to2, co2, Dy2, Dx2);
      else
        batch_eval<L, false>(S, P, J, slot_w, hdr, rel, I, Jb, row0, nrows, y, y_ok, lane, t1,
                             Tbase + to1, co1, Dy1, Dx1, -1, nullptr, 0, 0u, 0u);
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

// kPk: the instance for plans with a packed network, which also dispatches
// the packed layout codes; plans of whole-word networks only run the other,
// whose code is that of a kernel without packed rows.
template <bool kPk>
__device__ void batch_consume(BSmem &S, const BatchParams &P, const unsigned char *stage,
                              const BStage &si, int k, int slot_r, int slot_w, int cg, int lw,
                              int lane) {
  const BatchJob J = P.jobs[si.job];
  if constexpr (kPk) {
    switch (J.lcode) {
      case 17: batch_consume_q<17>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); return;
      case 18: batch_consume_q<18>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); return;
      case 19: batch_consume_q<19>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); return;
      case 20: batch_consume_q<20>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); return;
      case 21: batch_consume_q<21>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); return;
      case 22: batch_consume_q<22>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); return;
      case 23: batch_consume_q<23>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); return;
      default: break;
    }
  }
  switch (J.q) {
    case 1: batch_consume_q<1>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); break;
    case 2: batch_consume_q<2>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); break;
    case 3: batch_consume_q<3>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); break;
    case 4: batch_consume_q<4>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); break;
    case 5: batch_consume_q<5>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); break;
    case 6: batch_consume_q<6>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); break;
    case 7: batch_consume_q<7>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); break;
    default: batch_consume_q<8>(S, P, J, stage, si, k, slot_r, slot_w, cg, lw, lane); break;
  }
}

template <bool kPk>
__global__ void __launch_bounds__(kBThreads, 1) rac_batch_kernel(const BatchParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *ring = smem_raw;
  BSmem &S = *reinterpret_cast<BSmem *>(smem_raw + size_t(kBStages) * kStageBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, cta = blockIdx.x;
  const bool is_producer = warp == kBConsumerWarps;
  const int T_total = P.total_states;

  if (tid == 0) {
    for (int i = 0; i < kBStages; ++i) {
      mbar_init(&S.full[i], 1);
      mbar_init(&S.empty[i], kBGroupWarps);
    }
    fence_mbar_init();
    S.abort = 0;
    S.failed = 0;
    S.base = ld_acquire(&P.sync->base);
    S.poisoned = ld_acquire(&P.sync->err) != 0u ? 1u : 0u;
    S.cta_any = 0;
    S.cta_wipe = 0;
  }
  __syncthreads();
  const uint32_t base = S.base;
  uint32_t ring_it = 0, prod_it = 0;
  int k = 0;
  bool ended_quiet = false;  // the last sweep removed nothing anywhere
  if (S.poisoned) {
    S.failed = 1;
  } else {
    // Phase 0 (owners): A := dom_in, B &= dom_in, note empty input domains.
    const int slot1 = int((base + 1) % 3);
    for (int t = cta; t < T_total; t += G) {
      const int n = P.jobs[P.state_job[t]].n;
      const int64_t off = P.state_off[t], so = P.scratch_off[t];
      for (int x = tid; x < n; x += blockDim.x) {
        const uint32_t v = P.dom_in[off + x];
        atomicAnd(P.bufB + so + x, v);
        if (P.dom_out != P.dom_in) P.dom_out[off + x] = v;
        if (v == 0u) {
          atomicOr(P.wipe + int64_t(slot1) * T_total + t, 1u);
          S.cta_wipe = 1;
        }
      }
    }
    __syncthreads();
    for (;;) {
      ++k;
      const int slot_w = int((base + k) % 3), slot_r = int((base + k + 2) % 3);
      const int slot_c = int((base + k + 1) % 3);
      if (is_producer) {
        {
          if (cta == 0 && lane == 0) {  // barrier words last used two sweeps (or a launch) ago
            P.sync->bar[slot_c] = 0ull;
            P.sync->bar2[slot_c] = 0ull;
          }
          const bool incr = (P.flags & RAC_INCREMENTAL) && k >= 2;
          bool ok = true;  // lane 0's wait outcomes
          // the jobs 32 at a time (lane = job): alive ones in order; for each,
          // this CTA's slabs of it (global slab g = cta + i G) 32 at a time
          // (lane = slab): the Proposition-2 test, then lane 0 issues the
          // copies of the slabs that pass
          for (int j0 = 0; j0 < P.n_jobs && ok; j0 += 32) {
            const int jl = j0 + lane;
            bool alive = jl < P.n_jobs;
            if (alive && k >= 2) alive = ld_dom(P.job_alive + int64_t(slot_r) * P.n_jobs + jl) != 0u;
            for (uint32_t am = __ballot_sync(kFull, alive); am != 0u && ok; am &= am - 1u) {
              const int j = j0 + __ffs(am) - 1;
              const BatchJob &J = P.jobs[j];
              const int sb = J.slab_base, se = J.slab_base + J.n_slabs;
              const int first = sb + ((cta - sb) % G + G) % G;  // first g >= sb with g = cta (mod G)
              for (int g0 = first; g0 < se && ok; g0 += 32 * G) {
                const int g = g0 + lane * G;
                bool act = g < se;
                SlabDesc sd = {};
                if (act) {
                  sd = J.slabs[g - sb];
                  if (incr) {
                    const uint32_t I = sd.ij & 0xFFFFu, Jb = sd.ij >> 16;
                    const uint32_t row0 = sd.rows & 0xFFu, nrows = sd.rows >> 8;
                    const uint32_t rowmask = (nrows >= 32 ? kFull : ((1u << nrows) - 1u)) << row0;
                    const uint32_t *cu = P.chgU + int64_t(slot_r) * P.u_slot_words + J.u_off;
                    act = ld_dom(cu + Jb) != 0u || (ld_dom(cu + I) & rowmask) != 0u;
                  }
                }
                for (uint32_t sm = __ballot_sync(kFull, act); sm != 0u; sm &= sm - 1u) {
                  const int src = __ffs(sm) - 1;
                  const uint32_t off16 = __shfl_sync(kFull, sd.rel_off16, src);
                  const uint32_t nbytes = __shfl_sync(kFull, sd.nbytes, src);
                  const uint32_t ij = __shfl_sync(kFull, sd.ij, src);
                  const uint32_t rows = __shfl_sync(kFull, sd.rows, src);
                  uint32_t got = 1u;
                  if (lane == 0) {
                    const int stg = prod_it % kBStages;
                    const uint32_t par = (prod_it / kBStages) & 1u;
                    if (mbar_wait(&S.empty[stg], par ^ 1u, &P.sync->err, P.wait_limit_ns)) {
                      S.stage[stg].job = j;
                      S.stage[stg].slab = g0 + src * G - sb;
                      S.stage[stg].ij = ij;
                      S.stage[stg].rows = rows;
                      mbar_arrive_expect_tx(&S.full[stg], nbytes);
                      if (P.rel_evict_first)
                        bulk_copy_g2s_hint(ring + size_t(stg) * kStageBytes, J.rel + size_t(off16),
                                           nbytes, &S.full[stg], policy_evict_first());
                      else
                        bulk_copy_g2s(ring + size_t(stg) * kStageBytes, J.rel + size_t(off16),
                                      nbytes, &S.full[stg]);
                      ++prod_it;
                    } else {
                      got = 0u;
                    }
                  }
                  if (__shfl_sync(kFull, got, 0) == 0u) {
                    ok = false;
                    break;
                  }
                }
              }
            }
          }
          // end of this sweep's slabs: one marker for each consumer group
          for (int e = 0; e < kBGroups && ok && lane == 0; ++e) {
            const int stg = prod_it % kBStages;
            const uint32_t par = (prod_it / kBStages) & 1u;
            if (!mbar_wait(&S.empty[stg], par ^ 1u, &P.sync->err,
                           P.wait_limit_ns)) {
              ok = false;
              break;
            }
            S.stage[stg].job = -1;
            mbar_arrive(&S.full[stg]);
            ++prod_it;
          }
          if (lane == 0 && !ok) S.abort = 1;
        }
      } else {
        // clear the slots written next sweep (last read two sweeps ago)
        const int64_t cgtid = int64_t(cta) * (kBConsumerWarps * 32) + tid;
        const int64_t cgstride = int64_t(G) * (kBConsumerWarps * 32);
        for (int64_t i = cgtid; i < T_total; i += cgstride) {
          P.any[int64_t(slot_c) * T_total + i] = 0u;
          P.wipe[int64_t(slot_c) * T_total + i] = 0u;
        }
        for (int64_t i = cgtid; i < P.chg_slot_words; i += cgstride)
          P.chg[int64_t(slot_c) * P.chg_slot_words + i] = 0u;
        for (int64_t i = cgtid; i < P.u_slot_words; i += cgstride)
          P.chgU[int64_t(slot_c) * P.u_slot_words + i] = 0u;
        for (int64_t i = cgtid; i < P.n_jobs; i += cgstride)
          P.job_alive[int64_t(slot_c) * P.n_jobs + i] = 0u;
        if (k >= 2) {
          // owner step: T still holds D_{k-2}; AND D_{k-1} into it where it
          // differs.  A thread per word of the chg slot (32 variables of one
          // state), over the whole grid; a domain sweep k-1 emptied is found
          // here (see batch_remove).
          const uint32_t *chs = P.chg + int64_t(slot_r) * P.chg_slot_words;
          for (int64_t i = cgtid; i < P.chg_slot_words; i += cgstride) {
            const uint32_t w = ld_dom(chs + i);
            const int t = P.chg_state[i];
            if (w == 0u) continue;
            if (ld_dom(P.st_info + t) & kInfoSweepMask) continue;  // finished state
            const int blk = int(i - P.chg_off[t]);
            const BView V = bview(P, t, k);
            const uint32_t *Cb = V.C + blk * 32;
            uint32_t *Tb = V.T + blk * 32;
            bool emptied = false;
#pragma unroll
            for (int h = 0; h < 32; h += 16) {  // sixteen loads in flight
              uint32_t c[16];
#pragma unroll
              for (int b = 0; b < 16; ++b) c[b] = ((w >> (h + b)) & 1u) ? ld_dom(Cb + h + b) : kFull;
#pragma unroll
              for (int b = 0; b < 16; ++b) {
                if ((w >> (h + b)) & 1u) {
                  atomicAnd(Tb + h + b, c[b]);
                  emptied = emptied || c[b] == 0u;
                }
              }
            }
            if (emptied) {
              S.cta_wipe = 1;
              atomicOr(P.wipe + int64_t(slot_w) * T_total + t, 1u);
            }
          }
        }
        const int cg = warp / kBGroupWarps, lw = warp % kBGroupWarps;
        const bool leader = lw == 0 && lane == 0;
        for (;;) {
          const uint32_t pos = ring_it * kBGroups + cg;
          const int stg = pos % kBStages;
          const uint32_t par = (pos / kBStages) & 1u;
          if (leader)
            S.stage_ok[stg] = mbar_wait(&S.full[stg], par, &P.sync->err,
                                        P.wait_limit_ns) ? 1u : 0u;
          named_bar(group_bar(cg), kBGroupWarps * 32);
          if (!S.stage_ok[stg]) {
            if (leader) S.abort = 1;
            break;
          }
          if (lane == 0) mbar_try_wait(&S.full[stg], par);
          __syncwarp();
          const BStage si = S.stage[stg];
          if (si.job >= 0)
            batch_consume<kPk>(S, P, ring + size_t(stg) * kStageBytes, si, k, slot_r, slot_w, cg, lw,
                          lane);
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.empty[stg]);
          ++ring_it;
          if (si.job < 0) break;
        }
      }
      __syncthreads();
      if (S.abort) S.failed = 1;
      // barrier 1: removals of sweep k done everywhere
      if (tid == 0) {
        constexpr unsigned long long kMask = (1ull << kBarCountBits) - 1ull;
        const unsigned long long mine = 1ull |
                                        (uint64_t(S.cta_any ? 1u : 0u) << kBarCountBits) |
                                        (uint64_t(S.cta_wipe ? 1u : 0u) << (2 * kBarCountBits)) |
                                        (uint64_t(S.failed ? 1u : 0u) << (3 * kBarCountBits));
        unsigned long long v = 0;
        uint32_t f = S.failed;
        batch_barrier(P, &P.sync->bar[slot_w], mine, kMask, uint32_t(G), v, f);
        S.any_total = uint32_t((v >> kBarCountBits) & kMask);
        S.wipe_total = uint32_t((v >> (2 * kBarCountBits)) & kMask);
        if (((v >> (3 * kBarCountBits)) & kMask) || f) S.failed = 1;
        S.cta_any = 0;
        S.cta_wipe = 0;
        S.cta_running = 0;
      }
      __syncthreads();
      if (S.failed) break;
      if (S.any_total == 0u && S.wipe_total == 0u) {
        ended_quiet = true;  // D_k = D_{k-1} for every running state
        break;
      }
      // decisions of the states this CTA owns
      const bool stop = (P.flags & RAC_STOP_ON_WIPEOUT) != 0;
      for (int t = cta + G * tid; t < T_total; t += G * int(blockDim.x)) {
        uint32_t info = ld_dom(P.st_info + t);
        if (info & kInfoSweepMask) continue;
        const bool any = ld_dom(P.any + int64_t(slot_w) * T_total + t) != 0u;
        const bool wp = ld_dom(P.wipe + int64_t(slot_w) * T_total + t) != 0u;
        if (wp) info |= kInfoWiped;
        const uint32_t t_is_b = (k & 1) ? kInfoResB : 0u;
        const uint32_t c_is_b = (k >= 2 && !(k & 1)) ? kInfoResB : 0u;
        if (stop && wp) {
          info |= uint32_t(k) | t_is_b | info_status_bits(RAC_WIPEOUT);
        } else if (!any) {
          info |= uint32_t(k) | c_is_b | info_status_bits((info & kInfoWiped) ? RAC_WIPEOUT : RAC_OK);
        } else if ((P.max_sweeps > 0 && k >= P.max_sweeps) || k >= 0xFFFFF0) {
          info |= uint32_t(k) | t_is_b | info_status_bits(RAC_ETIMEOUT);
        } else {
          atomicAdd(&S.cta_running, 1u);
          atomicOr(P.job_alive + int64_t(slot_w) * P.n_jobs + P.state_job[t], 1u);
        }
        P.st_info[t] = info;
      }
      __syncthreads();
      // barrier 2: decisions published; how many states still run
      if (tid == 0) {
        constexpr unsigned long long kMask = (1ull << kBarCountBits) - 1ull;
        const unsigned long long mine = 1ull | (uint64_t(S.cta_running) << 32);
        unsigned long long v = 0;
        uint32_t f = S.failed;
        batch_barrier(P, &P.sync->bar2[slot_w], mine, kMask, uint32_t(G), v, f);
        S.running_total = uint32_t(v >> 32);
        if (f) S.failed = 1;
      }
      __syncthreads();
      if (S.failed || S.running_total == 0u) break;
    }
  }

  // Epilogue (owners): final status and sweep count of every state, results
  // that ended in B copied to dom_out, B back to all ones, decisions reset.
  __syncthreads();
  const bool failed = S.failed != 0u;
  if (!S.poisoned) {
    for (int t = cta; t < T_total; t += G) {
      const uint32_t info = ld_dom(P.st_info + t);
      const bool done = (info & kInfoSweepMask) != 0u;
      bool res_b;
      int sweeps, st;
      if (done) {
        res_b = (info & kInfoResB) != 0u;
        sweeps = int(info & kInfoSweepMask);
        st = info_status(info);
      } else {  // still running when the loop ended: a quiet last sweep
        res_b = ended_quiet && k >= 2 && !(k & 1);
        sweeps = k;
        st = ended_quiet ? ((info & kInfoWiped) ? RAC_WIPEOUT : RAC_OK) : RAC_EBARRIER;
      }
      const int n = P.jobs[P.state_job[t]].n;
      const int64_t off = P.state_off[t], so = P.scratch_off[t];
      for (int x = tid; x < n; x += blockDim.x) {
        if (!failed && res_b) P.dom_out[off + x] = ld_dom(P.bufB + so + x);
        P.bufB[so + x] = kFull;
      }
      if (tid == 0) {
        P.iterations[P.res_idx[t]] = sweeps;
        P.status[P.res_idx[t]] = failed ? RAC_EBARRIER : st;
        P.st_info[t] = 0u;
      }
    }
  }
  if (cta == 0 && tid == 0 && !failed) P.sync->base = (base + uint32_t(k)) % 3u;
  if (failed && tid == 0) atomicOr(&P.sync->err, kErrCopyWait);
  if (is_producer && lane == 0) {
    const uint32_t first = prod_it > uint32_t(kBStages) ? prod_it - kBStages : 0u;
    for (uint32_t j = first; j < prod_it; ++j)
      mbar_wait(&S.full[j % kBStages], (j / kBStages) & 1u,
                &P.sync->err, P.wait_limit_ns);
  }
}

}  // namespace

template <bool kPk>
rac_status launch_batch_instance(const BatchParams &P, cudaStream_t stream) {
  static LaunchCache cache;
  const size_t smem = size_t(kBStages) * kStageBytes + sizeof(BSmem);
  int per_sm = 0, sms = 0;
  rac_status rc = persistent_shape(cache, reinterpret_cast<const void *>(rac_batch_kernel<kPk>),
                                   kBThreads, smem, "batched kernel set-up", &per_sm, &sms);
  if (rc != RAC_OK) return rc;
  const int grid = per_sm * sms;
  cudaError_t e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(kBThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, rac_batch_kernel<kPk>, P);
  if (e != cudaSuccess) return cuda_fail(e, "launch of the batched kernel");
  return RAC_OK;
}

rac_status launch_batch(const BatchParams &P, cudaStream_t stream) {
  return P.any_packed ? launch_batch_instance<true>(P, stream)
                      : launch_batch_instance<false>(P, stream);
}

}  // namespace rac
