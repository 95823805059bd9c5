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
// Mapping: a CTA owns every G-th relation slab.  One producer thread streams
// slabs into a shared-memory ring with bulk copies (cp.async.bulk, completion
// on mbarriers); 8 consumer warps evaluate them.  A lane holds one relation
// (the pair (x, y = 32 J + lane)); the AND over C_x of the forward masks is a
// warp AND-reduction (redux.sync) for the row's x, and the reverse masks are
// AND-accumulated per lane over the rows for y.  Partial results reach the
// next-domain buffer through atomicAnd only when they remove something; the
// value returned by the atomic tells the writer whether it emptied a domain.
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

#include "rac_internal.h"

namespace rac {
namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s for any device-side wait
constexpr uint32_t kFull = 0xFFFFFFFFu;

// ------------------------------- PTX helpers -------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false (and sets the error bit) after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, Sync *sy) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_timer() - t0 > kWaitLimitNs) {
      atomicOr(&sy->err, kErrCopyWait);
      return false;
    }
  }
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ void named_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Domain words change between sweeps through L2 atomics: read them at L2.
__device__ __forceinline__ uint32_t ld_dom(const uint32_t *p) { return __ldcg(p); }

// ------------------------- bank-conflict-free order -------------------------
// Relation r of a stage starts at r * 16 Q bytes.  A quarter warp reading one
// 16-byte chunk per lane is conflict-free when the 8 chunks fall in distinct
// 16-byte bank groups; starting lane r's walk at chunk rot(r) makes that hold
// for any 8 consecutive relations (found by exhaustive search over Q <= 8).
template <int Q>
__device__ __forceinline__ int chunk_rot(uint32_t r) {
  if constexpr (Q == 2 || Q == 6) return (r >> 2) & 1;
  if constexpr (Q == 4) return (r >> 1) & 3;
  if constexpr (Q == 8) return r & 7;
  return 0;
}

// Rotate the low NBITS bits of v right / left by s (0 < s < NBITS).
template <int NBITS>
__device__ __forceinline__ uint32_t rotr_field(uint32_t v, int s) {
  if constexpr (NBITS == 32) {
    return __funnelshift_r(v, v, s);
  } else {
    const uint32_t mask = (1u << NBITS) - 1u;
    return ((v >> s) | (v << (NBITS - s))) & mask;
  }
}
template <int NBITS>
__device__ __forceinline__ uint32_t rotl_field(uint32_t v, int s) {
  if constexpr (NBITS == 32) {
    return __funnelshift_l(v, v, s);
  } else {
    const uint32_t mask = (1u << NBITS) - 1u;
    return ((v << s) | (v >> (NBITS - s))) & mask;
  }
}

// The support test of one relation (rows a = 0..4Q-1, padding rows are 0):
//   fwd bit a  = (R[a] & Dy) != 0
//   rev        = OR over a in Dx of R[a]
template <int Q>
__device__ __forceinline__ void support_relation(const uint4 *rel, int rot, uint32_t Dx,
                                                 uint32_t Dy, uint32_t &fwd, uint32_t &rev) {
  constexpr int NBITS = 4 * Q;
  const uint32_t dx = rot ? rotr_field<NBITS>(Dx, 4 * rot) : Dx;
  uint32_t f = 0, r = 0;
#pragma unroll
  for (int c = 0; c < Q; ++c) {
    int cc = c + rot;
    if (cc >= Q) cc -= Q;
    const uint4 w = rel[cc];
    f |= ((w.x & Dy) != 0u ? 1u : 0u) << (4 * c + 0);
    f |= ((w.y & Dy) != 0u ? 1u : 0u) << (4 * c + 1);
    f |= ((w.z & Dy) != 0u ? 1u : 0u) << (4 * c + 2);
    f |= ((w.w & Dy) != 0u ? 1u : 0u) << (4 * c + 3);
    if (dx & (1u << (4 * c + 0))) r |= w.x;
    if (dx & (1u << (4 * c + 1))) r |= w.y;
    if (dx & (1u << (4 * c + 2))) r |= w.z;
    if (dx & (1u << (4 * c + 3))) r |= w.w;
  }
  fwd = rot ? rotl_field<NBITS>(f, 4 * rot) : f;
  rev = r;
}

struct Smem {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  int32_t stage_slab[kStages];
  uint32_t bar0_ok;
  uint32_t all_done;
  uint32_t abort;
  uint32_t red[2][kConsumerWarps][32];
  uint32_t st_info[kMaxStatesPerLaunch];  // see kInfo* below
  uint8_t any_loc[kMaxStatesPerLaunch];
  uint8_t wipe_loc[kMaxStatesPerLaunch];
};
// st_info: bits 0..23 sweep at which the state finished (0 = running),
// bit 24 result in buffer B, bit 25 some domain emptied so far,
// bits 28..30 status code + 4.
constexpr uint32_t kInfoSweepMask = 0xFFFFFFu;
constexpr uint32_t kInfoResB = 1u << 24;
constexpr uint32_t kInfoWiped = 1u << 25;
__device__ __forceinline__ uint32_t info_status_bits(int st) { return uint32_t(st + 8) << 27; }
__device__ __forceinline__ int info_status(uint32_t v) { return int((v >> 27) & 31u) - 8; }

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

__device__ __forceinline__ void wait_bar0(Smem &S, const LaunchParams &P) {
  if (S.bar0_ok) return;
  const uint64_t t0 = global_timer();
  while (ld_acquire(&P.sync->bar0) < gridDim.x) {
    if (global_timer() - t0 > kWaitLimitNs) {
      atomicOr(&P.sync->err, kErrGridWait);
      break;
    }
    __nanosleep(32);
  }
  S.bar0_ok = 1;
}

// Apply a removal: D_k[v] &= keep, where keep is a strict subset of D_{k-1}[v].
__device__ __forceinline__ void remove_values(Smem &S, const LaunchParams &P, int s, int k,
                                              uint32_t *T, uint32_t v, uint32_t keep) {
  if (k == 1) wait_bar0(S, P);
  const uint32_t old = atomicAnd(T + v, keep);
  S.any_loc[s] = 1;
  if (old != 0u && (old & keep) == 0u) S.wipe_loc[s] = 1;
  const int slot = k % 3;
  const int nb = P.net.nb;
  const uint32_t bit = 1u << (v & 31u);
  atomicOr(P.chg + (int64_t(slot) * P.n_states + s) * nb + (v >> 5), bit);
  if (P.flags & RAC_INCREMENTAL) atomicOr(P.chgU + int64_t(slot) * nb + (v >> 5), bit);
}

// Bounded grid barrier over all CTAs (co-resident: cooperative launch).
__device__ void grid_barrier(const LaunchParams &P, uint32_t target) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&P.sync->bar_main, 1u);
    const uint64_t t0 = global_timer();
    for (;;) {
      if (ld_acquire(&P.sync->bar_main) >= target) break;
      if (ld_acquire(&P.sync->err) != 0u) break;
      if (global_timer() - t0 > kWaitLimitNs) {
        atomicOr(&P.sync->err, kErrGridWait);
        break;
      }
      __nanosleep(20);
    }
    __threadfence();
  }
  __syncthreads();
}

template <int Q>
__device__ void consume_slab(Smem &S, const LaunchParams &P, const uint4 *stage, int sl, int k,
                             int warp, int lane, uint32_t &red_iter) {
  const NetDev &N = P.net;
  const SlabDesc sd = N.slabs[sl];
  const int n = N.n;
  const int y = int(sd.J) * 32 + lane;
  const bool y_ok = y < n;
  // states are split over warp groups, rows over the warps of a group
  const int wps = P.n_states >= 8 ? 1 : (P.n_states >= 4 ? 2 : (P.n_states >= 2 ? 4 : 8));
  const int groups = kConsumerWarps / wps;
  const int g = warp / wps, sub = warp % wps;
  const bool incr = (P.flags & RAC_INCREMENTAL) && k >= 2;
  const uint32_t rowmask =
      (sd.nrows >= 32 ? kFull : ((1u << sd.nrows) - 1u)) << sd.row0;
  const int slot_r = (k + 2) % 3;
  for (int s = g; s < P.n_states; s += groups) {
    if (S.st_info[s] & kInfoSweepMask) continue;  // finished state
    if (incr) {
      const uint32_t *ch = P.chg + (int64_t(slot_r) * P.n_states + s) * N.nb;
      if (ld_dom(ch + sd.J) == 0u && (ld_dom(ch + sd.I) & rowmask) == 0u) continue;
    }
    const StateView V = state_view(P, s, k);
    const uint32_t Dy = y_ok ? ld_dom(V.C + y) : 0u;
    uint32_t racc = kFull;
    for (int r = sub; r < int(sd.nrows); r += wps) {
      const uint32_t pm = __ldg(N.pmask + sd.meta_off + r);
      if (pm == 0u) continue;
      const int x = int(sd.I) * 32 + int(sd.row0) + r;
      const uint32_t Dx = ld_dom(V.C + x);
      uint32_t fwd = kFull, rev = kFull;
      if ((pm >> lane) & 1u) {
        const uint32_t ridx = __ldg(N.roff + sd.meta_off + r) + __popc(pm & lanemask_lt());
        support_relation<Q>(stage + ridx * Q, chunk_rot<Q>(ridx), Dx, Dy, fwd, rev);
      }
      const uint32_t keep_x = __reduce_and_sync(kFull, fwd) & Dx;
      if (keep_x != Dx && lane == 0) remove_values(S, P, s, k, V.T, uint32_t(x), keep_x);
      racc &= rev;
    }
    if (wps > 1) {
      const int buf = red_iter & 1;
      S.red[buf][warp][lane] = racc;
      named_bar(1 + g, wps * 32);
      if (sub == 0) {
        for (int j = 1; j < wps; ++j) racc &= S.red[buf][warp + j][lane];
      }
      ++red_iter;
    }
    if (sub == 0 && y_ok) {
      const uint32_t keep_y = racc & Dy;
      if (keep_y != Dy) remove_values(S, P, s, k, V.T, uint32_t(y), keep_y);
    }
  }
}

template <int Q>
__global__ void __launch_bounds__(kThreads, 1) rac_bits_kernel(const LaunchParams P) {
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

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&S.full[i], 1);
      mbar_init(&S.empty[i], kConsumerWarps);
    }
    fence_mbar_init();
    S.bar0_ok = 0;
    S.all_done = 0;
    S.abort = 0;
  }
  for (int s = tid; s < B; s += blockDim.x) {
    S.st_info[s] = 0;
    S.any_loc[s] = 0;
    S.wipe_loc[s] = 0;
  }
  __syncthreads();

  // Phase 0: B := dom_in, A := dom_in, note empty input domains, clear the
  // flag slots written by sweeps 1 and 2.  Removals of sweep 1 wait for all
  // CTAs to pass this point (bar0).
  for (int64_t i = gtid; i < int64_t(B) * n; i += gstride) {
    const int s = int(i / n), x = int(i % n);
    const int64_t off = state_offset(P, s);
    const uint32_t v = P.dom_in[off + x];
    P.bufB[int64_t(s) * n + x] = v;
    if (P.dom_out != P.dom_in) P.dom_out[off + x] = v;
    if (v == 0u) S.wipe_loc[s] = 1;  // D_1 will hold this empty domain
  }
  {
    const int64_t per_slot = int64_t(B) * N.nb;
    for (int slot = 1; slot <= 2; ++slot) {
      for (int64_t i = gtid; i < B; i += gstride) {
        P.any[slot * B + i] = 0u;
        P.wipe[slot * B + i] = 0u;
      }
      for (int64_t i = gtid; i < per_slot; i += gstride) P.chg[slot * per_slot + i] = 0u;
      for (int64_t i = gtid; i < N.nb; i += gstride) P.chgU[int64_t(slot) * N.nb + i] = 0u;
    }
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    atomicAdd(&P.sync->bar0, 1u);
  }

  uint32_t ring_it = 0;   // consumer-side position in the ring
  uint32_t prod_it = 0;   // producer-side position in the ring
  uint32_t red_iter = 0;  // parity of the cross-warp reduction buffer
  int k = 0;
  for (;;) {
    ++k;
    const int slot_w = k % 3, slot_r = (k + 2) % 3, slot_c = (k + 1) % 3;
    if (k >= 2) {
      // clear the slot written next sweep (last read in sweep k-1)
      const int64_t per_slot = int64_t(B) * N.nb;
      for (int64_t i = gtid; i < B; i += gstride) {
        P.any[slot_c * B + i] = 0u;
        P.wipe[slot_c * B + i] = 0u;
      }
      for (int64_t i = gtid; i < per_slot; i += gstride) P.chg[slot_c * per_slot + i] = 0u;
      for (int64_t i = gtid; i < N.nb; i += gstride) P.chgU[int64_t(slot_c) * N.nb + i] = 0u;
      // owner step: T still holds D_{k-2}; AND D_{k-1} into it where it differs
      for (int64_t i = gtid; i < per_slot; i += gstride) {
        const int s = int(i / N.nb), blk = int(i % N.nb);
        if (S.st_info[s] & kInfoSweepMask) continue;
        uint32_t w = ld_dom(P.chg + slot_r * per_slot + i);
        if (w == 0u) continue;
        const StateView V = state_view(P, s, k);
        while (w) {
          const int b = __ffs(w) - 1;
          w &= w - 1u;
          const int x = blk * 32 + b;
          atomicAnd(V.T + x, ld_dom(V.C + x));
        }
      }
    }

    if (warp == kConsumerWarps) {
      // producer: stream this CTA's active slabs through the ring
      if (lane == 0) {
        const bool incr = (P.flags & RAC_INCREMENTAL) && k >= 2;
        const uint32_t *cu = P.chgU + int64_t(slot_r) * N.nb;
        bool ok = true;
        for (int sl = cta; sl < N.n_slabs && ok; sl += G) {
          const SlabDesc sd = N.slabs[sl];
          if (incr) {
            const uint32_t rowmask =
                (sd.nrows >= 32 ? kFull : ((1u << sd.nrows) - 1u)) << sd.row0;
            if (ld_dom(cu + sd.J) == 0u && (ld_dom(cu + sd.I) & rowmask) == 0u) continue;
          }
          const int stg = prod_it % kStages;
          const uint32_t par = (prod_it / kStages) & 1u;
          if (!mbar_wait(&S.empty[stg], par ^ 1u, P.sync)) {
            ok = false;
            break;
          }
          S.stage_slab[stg] = sl;
          mbar_arrive_expect_tx(&S.full[stg], sd.nbytes);
          bulk_copy_g2s(ring + size_t(stg) * kStageBytes, N.rel + size_t(sd.rel_off16),
                        sd.nbytes, &S.full[stg]);
          ++prod_it;
        }
        const int stg = prod_it % kStages;
        const uint32_t par = (prod_it / kStages) & 1u;
        if (ok && mbar_wait(&S.empty[stg], par ^ 1u, P.sync)) {
          S.stage_slab[stg] = -1;  // end of this sweep's slabs
          mbar_arrive(&S.full[stg]);
          ++prod_it;
        } else {
          S.abort = 1;
        }
      }
    } else {
      for (;;) {
        const int stg = ring_it % kStages;
        const uint32_t par = (ring_it / kStages) & 1u;
        bool ok = true;
        if (lane == 0) ok = mbar_wait(&S.full[stg], par, P.sync);
        ok = __shfl_sync(kFull, ok ? 1 : 0, 0) != 0;
        if (!ok || S.abort) break;
        const int sl = S.stage_slab[stg];
        if (sl >= 0) {
          consume_slab<Q>(S, P, reinterpret_cast<const uint4 *>(ring + size_t(stg) * kStageBytes),
                          sl, k, warp, lane, red_iter);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[stg]);
        ++ring_it;
        if (sl < 0) break;
      }
    }
    __syncthreads();

    // publish this CTA's per-state flags for sweep k
    if (k == 1 && tid == 0) wait_bar0(S, P);
    __syncthreads();
    for (int s = tid; s < B; s += blockDim.x) {
      if (S.any_loc[s]) {
        atomicOr(P.any + slot_w * B + s, 1u);
        S.any_loc[s] = 0;
      }
      if (S.wipe_loc[s]) {
        atomicOr(P.wipe + slot_w * B + s, 1u);
        S.wipe_loc[s] = 0;
      }
    }
    grid_barrier(P, uint32_t(k) * uint32_t(G));
    if (ld_acquire(&P.sync->err) != 0u || S.abort) break;

    // decisions (every CTA reads the same flags and takes the same ones)
    const bool stop = (P.flags & RAC_STOP_ON_WIPEOUT) != 0;
    for (int s = tid; s < B; s += blockDim.x) {
      uint32_t info = S.st_info[s];
      if (info & kInfoSweepMask) continue;
      const bool any = ld_dom(P.any + slot_w * B + s) != 0u;
      const bool wp = ld_dom(P.wipe + slot_w * B + s) != 0u;
      if (wp) info |= kInfoWiped;
      const uint32_t t_is_b = (k & 1) ? kInfoResB : 0u;           // T of sweep k
      const uint32_t c_is_b = (k >= 2 && !(k & 1)) ? kInfoResB : 0u;  // C of sweep k
      if (stop && wp) {
        info |= uint32_t(k) | t_is_b | info_status_bits(RAC_WIPEOUT);
      } else if (!any) {
        info |= uint32_t(k) | c_is_b |
                info_status_bits((info & kInfoWiped) ? RAC_WIPEOUT : RAC_OK);
      } else if ((P.max_sweeps > 0 && k >= P.max_sweeps) || k >= P.sweep_bound) {
        info |= uint32_t(k) | t_is_b | info_status_bits(RAC_ETIMEOUT);
        if (k >= P.sweep_bound && !(P.max_sweeps > 0 && k >= P.max_sweeps) && cta == 0)
          atomicOr(&P.sync->err, kErrSweepBound);
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

  // Epilogue: results that ended in buffer B move to dom_out.
  const bool failed = ld_acquire(&P.sync->err) != 0u || S.abort;
  if (!failed) {
    for (int64_t i = gtid; i < int64_t(B) * n; i += gstride) {
      const int s = int(i / n), x = int(i % n);
      if (S.st_info[s] & kInfoResB) P.dom_out[state_offset(P, s) + x] = ld_dom(P.bufB + i);
    }
  }
  if (cta == 0) {
    for (int s = tid; s < B; s += blockDim.x) {
      const uint32_t info = S.st_info[s];
      const int idx = P.contiguous ? s : P.res_idx[s];
      P.iterations[idx] = int32_t(info & kInfoSweepMask) ? int32_t(info & kInfoSweepMask) : k;
      P.status[idx] = failed ? RAC_EBARRIER : info_status(info);
    }
  }
  // Drain copies still in flight (only after a failed wait), then leave; the
  // last CTA out resets the sync words for the next launch on this workspace.
  if (warp == kConsumerWarps && lane == 0) {
    const uint32_t first = prod_it > uint32_t(kStages) ? prod_it - kStages : 0u;
    for (uint32_t j = first; j < prod_it; ++j)
      mbar_wait(&S.full[j % kStages], (j / kStages) & 1u, P.sync);
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(&P.sync->exit_count, 1u);
    if (prev == uint32_t(G) - 1u) {
      P.sync->bar0 = 0u;
      P.sync->bar_main = 0u;
      P.sync->err = 0u;
      __threadfence();
      P.sync->exit_count = 0u;
    }
  }
}

template <int Q>
rac_status launch_q(const LaunchParams &P, cudaStream_t stream) {
  static int grid = 0;
  static int dev_cached = -1;
  const size_t smem = size_t(kStages) * kStageBytes + sizeof(Smem);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (grid == 0 || dev_cached != dev) {
    e = cudaFuncSetAttribute(rac_bits_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(smem));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rac_bits_kernel<Q>, kThreads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    if (per_sm < 1) {
      set_error("bit-packed kernel does not fit on an SM");
      return RAC_ECUDA;
    }
    grid = per_sm * sms;
    dev_cached = dev;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, rac_bits_kernel<Q>, P);
  if (e != cudaSuccess) return cuda_fail(e, "launch of the bit-packed kernel");
  return RAC_OK;
}

}  // namespace

rac_status launch_bits(const LaunchParams &P, cudaStream_t stream) {
  switch (P.net.q) {
    case 1: return launch_q<1>(P, stream);
    case 2: return launch_q<2>(P, stream);
    case 3: return launch_q<3>(P, stream);
    case 4: return launch_q<4>(P, stream);
    case 5: return launch_q<5>(P, stream);
    case 6: return launch_q<6>(P, stream);
    case 7: return launch_q<7>(P, stream);
    case 8: return launch_q<8>(P, stream);
    default: set_error("unsupported relation width"); return RAC_EINVAL;
  }
}

}  // namespace rac
