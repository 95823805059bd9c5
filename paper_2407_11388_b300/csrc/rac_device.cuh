// Device helpers shared by the bit-packed kernels: PTX wrappers for
// mbarriers and bulk copies, bounded waits, and the support test of one
// bit-packed relation.
#pragma once

#include "rac_internal.h"

namespace rac {
namespace dev {

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
// try_wait that may suspend the thread until the phase completes, for at
// most about `hint_ns`: a waiting warp then takes no issue slots from the
// warps that work on its sub-partition.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t *bar, uint32_t parity,
                                                      uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false (and sets the error bit) after `limit_ns`.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t *err,
                                          uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer();
  for (;;) {
    if (mbar_try_wait_suspend(bar, parity, 100000u)) return true;
    if (global_timer() - t0 > limit_ns) {
      atomicOr(err, kErrCopyWait);
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
// L2 policy for data streamed once per sweep with no reuse before it would be
// evicted anyway (a relation store larger than L2): evict it first, so the
// small, reused domain and flag words stay resident.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void bulk_copy_g2s_hint(void *dst, const void *src, uint32_t bytes,
                                                   uint64_t *bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], "
      "%2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Add with release and acquire semantics at GPU scope: the writes that happen
// before it (this thread's, and the CTA's before a __syncthreads) are visible
// to whoever acquires the result, and the caller sees everything released
// before the value it reads.
__device__ __forceinline__ unsigned long long atom_add_acq_rel_u64(unsigned long long *p,
                                                                    unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
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

// r |= w when (m & bit) != 0, as a test into a predicate and a predicated OR:
// both the forward test ((R[a] & D_y) != 0 sets bit a) and the masked reverse
// OR take this form, with fewer integer instructions than comparing and
// selecting or forming a mask
__device__ __forceinline__ void or_if_bit(uint32_t &r, uint32_t w, uint32_t m, uint32_t bit) {
  asm("{\n .reg .pred p;\n .reg .b32 t;\n and.b32 t, %1, %2;\n setp.ne.u32 p, t, 0;\n"
      " @p or.b32 %0, %0, %3;\n}\n"
      : "+r"(r)
      : "r"(m), "r"(bit), "r"(w));
}

// The support test of one relation, rows a = 0..4Q-1 (padding rows are 0),
// read as Q 16-byte chunks `stride` chunks apart:
//   fwd bit a  = (R[a] & Dy) != 0        (Sup_xy[a] > 0, Fig. 1)
//   rev        = OR over a in Dx of R[a] (bit b: (y,b) has a support in Dx)
// Two independent accumulators per result keep the OR chains short.
template <int Q, bool kDxFull>
__device__ __forceinline__ void support_relation(const uint4 *rel, uint32_t stride, uint32_t Dx,
                                                 uint32_t Dy, uint32_t &fwd, uint32_t &rev) {
  uint32_t f0 = 0, f1 = 0, r0 = 0, r1 = 0;
#pragma unroll
  for (int c = 0; c < Q; ++c) {
    const uint4 w = rel[c * stride];
    or_if_bit(f0, 1u << (4 * c + 0), w.x, Dy);
    or_if_bit(f1, 1u << (4 * c + 1), w.y, Dy);
    or_if_bit(f0, 1u << (4 * c + 2), w.z, Dy);
    or_if_bit(f1, 1u << (4 * c + 3), w.w, Dy);
    if (kDxFull) {  // every row of R is in Dx (rows >= d are zero)
      r0 |= w.x | w.z;
      r1 |= w.y | w.w;
    } else {
      or_if_bit(r0, w.x, Dx, 1u << (4 * c + 0));
      or_if_bit(r1, w.y, Dx, 1u << (4 * c + 1));
      or_if_bit(r0, w.z, Dx, 1u << (4 * c + 2));
      or_if_bit(r1, w.w, Dx, 1u << (4 * c + 3));
    }
  }
  fwd = f0 | f1;
  rev = r0 | r1;
}

// The support test of one relation for two domain states at once (Dx1, Dy1)
// and (Dx2, Dy2): each 16-byte chunk is read once and serves both.  Same
// results as support_relation for each state.
template <int Q, bool kDxFull>
__device__ __forceinline__ void support_relation_pair(const uint4 *rel, uint32_t stride,
                                                      uint32_t Dx1, uint32_t Dy1, uint32_t Dx2,
                                                      uint32_t Dy2, uint32_t &fwd1, uint32_t &rev1,
                                                      uint32_t &fwd2, uint32_t &rev2) {
  uint32_t f1 = 0, g1 = 0, f2 = 0, g2 = 0, r1 = 0, q1 = 0, r2 = 0, q2 = 0;
#pragma unroll
  for (int c = 0; c < Q; ++c) {
    const uint4 w = rel[c * stride];
    or_if_bit(f1, 1u << (4 * c + 0), w.x, Dy1);
    or_if_bit(g1, 1u << (4 * c + 1), w.y, Dy1);
    or_if_bit(f1, 1u << (4 * c + 2), w.z, Dy1);
    or_if_bit(g1, 1u << (4 * c + 3), w.w, Dy1);
    or_if_bit(f2, 1u << (4 * c + 0), w.x, Dy2);
    or_if_bit(g2, 1u << (4 * c + 1), w.y, Dy2);
    or_if_bit(f2, 1u << (4 * c + 2), w.z, Dy2);
    or_if_bit(g2, 1u << (4 * c + 3), w.w, Dy2);
    if (kDxFull) {  // both row domains full: every row of R counts for both
      r1 |= w.x | w.z;
      q1 |= w.y | w.w;
    } else {
      or_if_bit(r1, w.x, Dx1, 1u << (4 * c + 0));
      or_if_bit(q1, w.y, Dx1, 1u << (4 * c + 1));
      or_if_bit(r1, w.z, Dx1, 1u << (4 * c + 2));
      or_if_bit(q1, w.w, Dx1, 1u << (4 * c + 3));
      or_if_bit(r2, w.x, Dx2, 1u << (4 * c + 0));
      or_if_bit(q2, w.y, Dx2, 1u << (4 * c + 1));
      or_if_bit(r2, w.z, Dx2, 1u << (4 * c + 2));
      or_if_bit(q2, w.w, Dx2, 1u << (4 * c + 3));
    }
  }
  fwd1 = f1 | g1;
  fwd2 = f2 | g2;
  rev1 = r1 | q1;
  rev2 = kDxFull ? rev1 : (r2 | q2);
}

// ---------------------------------------------------------------------------
// Packed relation rows (RAC_LAYOUT_PACKED): the relation's rows a = 0..4Q-1
// lie back to back, 4Q bits each, in packed_words(Q) words read `stride`
// words apart.  Row a is bits [4Q a, 4Q a + 4Q): one shift of its word, or a
// funnel shift of two words when it straddles them.  The bits above a row's
// 4Q belong to the next rows: the forward test ANDs them with Dy (no bits >=
// d), and the reverse mask is cut to 4Q bits at the end.  Same results as
// support_relation on the whole-word rows.
template <int Q, int A>
__device__ __forceinline__ uint32_t packed_row(const uint32_t (&w)[packed_words(Q)]) {
  constexpr int kBits = 4 * Q, kOff = A * kBits, kWord = kOff >> 5, kShift = kOff & 31;
  constexpr int kNext = kWord + 1 < packed_words(Q) ? kWord + 1 : kWord;
  if constexpr (kShift == 0) return w[kWord];
  else if constexpr (kShift + kBits <= 32) return w[kWord] >> kShift;
  else return __funnelshift_r(w[kWord], w[kNext], kShift);
}

template <int Q, bool kDxFull, int A = 0>
__device__ __forceinline__ void packed_rows(const uint32_t (&w)[packed_words(Q)], uint32_t Dx,
                                            uint32_t Dy, uint32_t &f0, uint32_t &f1,
                                            uint32_t &r0, uint32_t &r1) {
  if constexpr (A < 4 * Q) {
    const uint32_t row = packed_row<Q, A>(w);
    if constexpr (A % 2 == 0) {
      or_if_bit(f0, 1u << A, row, Dy);
      if (kDxFull) r0 |= row;
      else or_if_bit(r0, row, Dx, 1u << A);
    } else {
      or_if_bit(f1, 1u << A, row, Dy);
      if (kDxFull) r1 |= row;
      else or_if_bit(r1, row, Dx, 1u << A);
    }
    packed_rows<Q, kDxFull, A + 1>(w, Dx, Dy, f0, f1, r0, r1);
  }
}

template <int Q, bool kDxFull>
__device__ __forceinline__ void support_relation_packed(const uint32_t *rel, uint32_t stride,
                                                        uint32_t Dx, uint32_t Dy, uint32_t &fwd,
                                                        uint32_t &rev) {
  uint32_t w[packed_words(Q)];
#pragma unroll
  for (int j = 0; j < packed_words(Q); ++j) w[j] = rel[j * stride];
  uint32_t f0 = 0, f1 = 0, r0 = 0, r1 = 0;
  packed_rows<Q, kDxFull>(w, Dx, Dy, f0, f1, r0, r1);
  fwd = f0 | f1;
  rev = (r0 | r1) & ((1u << (4 * Q)) - 1u);
}

// Two domain states on one packed relation: each row is taken out of its
// words once and tested for both (as support_relation_pair).
template <int Q, bool kDxFull, int A = 0>
__device__ __forceinline__ void packed_rows_pair(const uint32_t (&w)[packed_words(Q)],
                                                 uint32_t Dx1, uint32_t Dy1, uint32_t Dx2,
                                                 uint32_t Dy2, uint32_t (&f)[4],
                                                 uint32_t (&r)[4]) {
  if constexpr (A < 4 * Q) {
    constexpr int h = A % 2;
    const uint32_t row = packed_row<Q, A>(w);
    or_if_bit(f[h], 1u << A, row, Dy1);
    or_if_bit(f[2 + h], 1u << A, row, Dy2);
    if (kDxFull) {
      r[h] |= row;
    } else {
      or_if_bit(r[h], row, Dx1, 1u << A);
      or_if_bit(r[2 + h], row, Dx2, 1u << A);
    }
    packed_rows_pair<Q, kDxFull, A + 1>(w, Dx1, Dy1, Dx2, Dy2, f, r);
  }
}

template <int Q, bool kDxFull>
__device__ __forceinline__ void support_relation_pair_packed(
    const uint32_t *rel, uint32_t stride, uint32_t Dx1, uint32_t Dy1, uint32_t Dx2, uint32_t Dy2,
    uint32_t &fwd1, uint32_t &rev1, uint32_t &fwd2, uint32_t &rev2) {
  uint32_t w[packed_words(Q)];
#pragma unroll
  for (int j = 0; j < packed_words(Q); ++j) w[j] = rel[j * stride];
  uint32_t f[4] = {0u, 0u, 0u, 0u}, r[4] = {0u, 0u, 0u, 0u};
  packed_rows_pair<Q, kDxFull>(w, Dx1, Dy1, Dx2, Dy2, f, r);
  constexpr uint32_t kRow = (1u << (4 * Q)) - 1u;
  fwd1 = f[0] | f[1];
  fwd2 = f[2] | f[3];
  rev1 = (r[0] | r[1]) & kRow;
  rev2 = kDxFull ? rev1 : ((r[2] | r[3]) & kRow);
}

// ---------------------------------------------------------------------------
// A kernel's relation layout code L: L = Q (1..8) for whole-word rows, L = 16
// + Q (Q = 1..7) for packed rows.  The support test of the t-th relation of a
// slab row whose first relation has index roff (the header's roff[r]) and
// which holds cnt relations; rel points at the slab's first relation.
template <int L>
struct RelLayout {
  static constexpr bool kPacked = L >= 16;
  static constexpr int kQ = kPacked ? L - 16 : L;
  static_assert(kQ >= 1 && kQ <= (kPacked ? 7 : 8), "relation layout code");
};

template <int L, bool kDxFull>
__device__ __forceinline__ void support_at(const uint4 *rel, uint32_t roff, uint32_t t,
                                           uint32_t cnt, uint32_t Dx, uint32_t Dy, uint32_t &fwd,
                                           uint32_t &rev) {
  constexpr int Q = RelLayout<L>::kQ;
  if constexpr (RelLayout<L>::kPacked)
    support_relation_packed<Q, kDxFull>(
        reinterpret_cast<const uint32_t *>(rel) + roff * uint32_t(packed_words(Q)) + t, cnt, Dx,
        Dy, fwd, rev);
  else
    support_relation<Q, kDxFull>(rel + roff * uint32_t(Q) + t, cnt, Dx, Dy, fwd, rev);
}

template <int L, bool kDxFull>
__device__ __forceinline__ void support_pair_at(const uint4 *rel, uint32_t roff, uint32_t t,
                                                uint32_t cnt, uint32_t Dx1, uint32_t Dy1,
                                                uint32_t Dx2, uint32_t Dy2, uint32_t &fwd1,
                                                uint32_t &rev1, uint32_t &fwd2, uint32_t &rev2) {
  constexpr int Q = RelLayout<L>::kQ;
  if constexpr (RelLayout<L>::kPacked)
    support_relation_pair_packed<Q, kDxFull>(
        reinterpret_cast<const uint32_t *>(rel) + roff * uint32_t(packed_words(Q)) + t, cnt, Dx1,
        Dy1, Dx2, Dy2, fwd1, rev1, fwd2, rev2);
  else
    support_relation_pair<Q, kDxFull>(rel + roff * uint32_t(Q) + t, cnt, Dx1, Dy1, Dx2, Dy2,
                                      fwd1, rev1, fwd2, rev2);
}

}  // namespace dev
}  // namespace rac
