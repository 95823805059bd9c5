// Kernel (b): the support counts of Eq. 1 on the 5th-generation tensor cores
// (tcgen05.mma, FP8 E4M3 0/1 operands, FP32 accumulation in tensor memory),
// for up to 128 domain states of one network, swept to the fixpoint in one
// persistent cooperative launch.
//
// For every relation R_xy of a slab and every state s the counts are
//   forward  Sup_xy[a](s) = sum_b R[a][b] D_s[y][b]     (Fig. 1)
//   reverse  Sup_yx[b](s) = sum_a R[a][b] D_s[x][a]
// computed as MMAs with M = 128 states, K = 32 values and N = 256 = 8
// relations x 32 rows: a forward job per (group of 8 rows, column y) takes
// D_s[y] as A and the 8 relations R_{x,y} as B; a reverse job per (row x,
// group of 8 columns) takes D_s[x] as A and the 8 transposed relations as B.
// Counts are exact in FP32 (at most 32).  The epilogue reads the accumulator
// lanes (one state per lane), clamps every count to {0,1} (only Sup > 0
// matters, as in the paper's listing), packs the 32 values of a relation row
// into one word and ANDs it over the row's or column's constraints; the
// removals then follow kernel (a) (atomicAnd into the next domain buffer).
//
// The B operands are the network's FP8 operand store (RAC_LAYOUT_FP8: every
// job's tile expanded once, on the device, in the MMA's shared-memory layout),
// brought in by bulk copies.  A slab's jobs run through a pipeline of warps
// that wait on mbarriers only (no CTA-wide barrier per MMA):
//   warps 0-15   epilogue: TMEM lane quarter warp % 4 (32 states), a
//                quarter of each job's 8 relations (warp / 4); they keep a
//                slab's AND masks in registers and make its removals;
//   warps 16-19  A tiles: the states' domain word of the job's column (or
//                row) expanded to E4M3 bytes, 32 states each;
//   warp 20      B tiles: one bulk copy of 8 KiB per job;
//   warp 21      MMA issuer: waits for the job's A and B tiles and a free
//                accumulator, issues the MMA, and commits its completion to
//                the A and B stages it frees and to the accumulator's full
//                barrier;
//   warp 22      helps stage the slab's domain words;
//   warp 23      streams the bit-packed slabs (their headers name the
//                relations present) into a small ring, as in kernel (a).
// Four epilogue warps per quarter keep several tensor-memory loads in
// flight on each SM sub-partition.
// An A ring of four stages, a B ring of eight (64 KiB of copies in flight)
// and two accumulators of 256 columns let the roles run apart by several
// jobs.
#include <algorithm>
#include <mutex>
#include <string>

#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {
namespace {

using namespace dev;

// warp roles (see the file comment)
constexpr int kTcEpiParts = 4;                   // epilogue warps per TMEM lane quarter
constexpr int kTcEpiWarps = 4 * kTcEpiParts;      // warps 0-15
constexpr int kRelPerPart = 8 / kTcEpiParts;      // a job's relations per epilogue warp
constexpr int kTcAWarp0 = kTcEpiWarps, kTcAWarps = 4;  // warps 16-19
constexpr int kTcBWarp = kTcAWarp0 + kTcAWarps;        // warp 20
constexpr int kTcMmaWarp = kTcBWarp + 1;               // warp 21
constexpr int kTcConsumerWarps = kTcMmaWarp + 2;  // warps 0-22 (22 helps stage the domains);
                                                  // warp 23 streams the bit-packed slabs
constexpr int kTcThreads = (kTcConsumerWarps + 1) * 32;
constexpr int kTcStages = 2;   // bit-packed slab ring
constexpr int kTcAStages = 4;  // A operand ring (built on chip)
constexpr int kTcBStages = 8;  // B operand ring (8 KiB copies in flight from HBM)
constexpr int kTcMaxStates = 128;  // M of the MMA
constexpr int kTcN = 256;          // N of the MMA: 8 relations x 32 rows
constexpr uint32_t kTmemCols = 512;  // two accumulators of 256 columns
constexpr int kATileBytes = kTcMaxStates * 32;  // 4 KB
constexpr int kBTileBytes = kFp8TileBytes;      // 8 KB
static_assert(kBTileBytes == kTcN * 32, "a B tile is N rows of 32 bytes");
constexpr int kTcDomWords = 64;  // per state: 32 columns + up to 32 rows

struct TcStage {
  int32_t sl;
  uint32_t ij, rows, pad;
};

struct TcSmem {
  uint8_t a_tile[kTcAStages][kATileBytes];
  uint8_t b_tile[kTcBStages][kBTileBytes];
  uint32_t dom[kTcMaxStates][kTcDomWords];  // staged D_{k-1} words of the slab
  uint64_t full[kTcStages];
  uint64_t empty[kTcStages];
  uint64_t a_full[kTcAStages], a_empty[kTcAStages];
  uint64_t b_full[kTcBStages], b_empty[kTcBStages];
  uint64_t acc_full[2], acc_empty[2];
  TcStage stage[kTcStages];
  uint32_t stage_ok[kTcStages];
  uint32_t tmem_base;
  uint32_t mma_issued, b_issued;
  uint32_t base, poisoned, abort, failed, all_done;
  uint32_t any_total, wipe_total, cta_any, cta_wipe;
  uint32_t st_info[kTcMaxStates];
  uint8_t any_loc[kTcMaxStates], wipe_loc[kTcMaxStates];
};
static_assert(size_t(kTcStages) * kStageBytes + sizeof(TcSmem) + 1024 <= 232448,
              "shared memory of the tensor-core kernel exceeds 227 KB");
static_assert((size_t(kTcStages) * kStageBytes) % 128 == 0, "operand tiles 128-byte aligned");

constexpr uint32_t kInfoSweepMask = 0xFFFFFFu;
constexpr uint32_t kInfoResB = 1u << 24;
constexpr uint32_t kInfoWiped = 1u << 25;
__device__ __forceinline__ uint32_t info_status_bits(int st) { return uint32_t(st + 8) << 27; }
__device__ __forceinline__ int info_status(uint32_t v) { return int((v >> 27) & 31u) - 8; }
constexpr int kConsumersBar = 1;

// ------------------------------ tcgen05 helpers ------------------------------
// Shared-memory matrix descriptor: K-major, no swizzle; LBO = 128 B between
// core matrices along K, SBO = 256 B between 8-row groups (bits 46-47 hold the
// descriptor version of this architecture).
__device__ __forceinline__ uint64_t umma_desc(const void *tile) {
  uint64_t d = uint64_t((smem_u32(tile) >> 4) & 0x3FFFu);
  d |= uint64_t(128u >> 4) << 16;
  d |= uint64_t(256u >> 4) << 32;
  d |= uint64_t(1) << 46;
  return d;
}
// Instruction descriptor: FP32 accumulator, E4M3 A and B, both K-major,
// N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (uint32_t(kTcN >> 3) << 17) | (uint32_t(128 >> 4) << 24);

__device__ __forceinline__ void umma_f8(uint32_t tmem_d, uint64_t da, uint64_t db) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(kIdesc), "r"(0)
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
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 32 consecutive accumulator columns of this warp's 32 lanes.
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
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Byte offset of element (row, k) in a K-major 32-byte-K tile.
__device__ __forceinline__ uint32_t tile_off(uint32_t row, uint32_t k) {
  return (row >> 3) * 256u + (k >> 4) * 128u + (row & 7u) * 16u + (k & 15u);
}
// Four bits (bit i of nib) -> four bytes, 0x38 (E4M3 1.0) or 0.
__device__ __forceinline__ uint32_t expand4(uint32_t nib) {
  return ((nib * 0x00204081u) & 0x01010101u) * 0x38u;
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

__device__ __forceinline__ void tc_remove(TcSmem &S, const LaunchParams &P, int s, int slot_w,
                                          uint32_t *T, uint32_t v, uint32_t keep) {
  const uint32_t old = atomicAnd(T + v, keep);
  S.any_loc[s] = 1;
  if (old != 0u && (old & keep) == 0u) S.wipe_loc[s] = 1;
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

// The FP8 operand store: word w of tile (slab sl, job idx), job order as in
// tc_consume (forward jobs g * 32 + j, then reverse jobs 32 rg + g nrows + r).
__global__ void __launch_bounds__(256) rac_fp8_build_kernel(const NetDev N, uint8_t *out) {
  const int64_t total = int64_t(N.n_slabs) * N.fp8_jobs * (kFp8TileBytes / 4);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t t = i / (kFp8TileBytes / 4);
    const int w = int(i % (kFp8TileBytes / 4));
    const int sl = int(t / N.fp8_jobs), idx = int(t % N.fp8_jobs);
    const SlabDesc sd = N.slabs[sl];
    const uint32_t *hdr = reinterpret_cast<const uint32_t *>(N.rel + sd.rel_off16);
    const uint32_t nrows = sd.rows >> 8;
    const uint32_t *relw = hdr + 2 * nrows;
    const int rg = int(nrows + 7) / 8;
    const int row = w >> 3, qq = w & 7;
    uint32_t nib = 0u;
    if (idx < 32 * rg) {  // forward: rows (r, a) of R_{x_r, y_j}, K = b
      const int j = idx & 31, g = idx >> 5;
      const int r = 8 * g + (row >> 5), a = row & 31;
      if (r < int(nrows) && ((hdr[r] >> j) & 1u)) {
        const uint32_t t_rank = __popc(hdr[r] & ((1u << j) - 1u));
        nib = (rel_row(hdr, relw, nrows, N, r, t_rank, a) >> (4 * qq)) & 0xFu;
      }
    } else {  // reverse: rows (j, b) of R_{x_r, y_j} transposed, K = a
      const int ridx = idx - 32 * rg;
      const int r = ridx % int(nrows), g = ridx / int(nrows);
      const int j = 8 * g + (row >> 5), b = row & 31;
      if ((hdr[r] >> j) & 1u) {
        const uint32_t t_rank = __popc(hdr[r] & ((1u << j) - 1u));
#pragma unroll
        for (int i2 = 0; i2 < 4; ++i2)
          nib |= ((rel_row(hdr, relw, nrows, N, r, t_rank, 4 * qq + i2) >> b) & 1u) << i2;
      }
    }
    *reinterpret_cast<uint32_t *>(out + t * kFp8TileBytes + tile_off(uint32_t(row), 4u * qq)) =
        expand4(nib);
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

// Packs the 32 counts of one relation row (one state per lane) into a word:
// bit a set iff count a > 0 (the listing's clamp).  FP32 counts are >= 0, so
// a count is positive iff its bits are not all zero.
__device__ __forceinline__ uint32_t pack_positive(const uint32_t (&v)[32]) {
  uint32_t m = 0u;
#pragma unroll
  for (int a = 0; a < 32; ++a) m |= (v[a] != 0u ? 1u : 0u) << a;
  return m;
}

// The whole slab for every running state: 32 rg forward jobs and 4 nrows
// reverse jobs, each through the A / B / MMA / epilogue pipeline.  jc counts
// the CTA's jobs so far (the same in every role: ring stages and phases).
__device__ void tc_consume(TcSmem &S, const LaunchParams &P, const unsigned char *stage,
                           const TcStage &si, int k, int slot_w, int warp, int lane,
                           uint32_t &jc) {
  const NetDev &N = P.net;
  const int n = N.n, B = P.n_states;
  const uint32_t I = si.ij & 0xFFFFu, J = si.ij >> 16;
  const uint32_t row0 = si.rows & 0xFFu, nrows = si.rows >> 8;
  const uint32_t *hdr = reinterpret_cast<const uint32_t *>(stage);
  const int ct = warp * 32 + lane;  // consumer thread
  constexpr int nct = kTcConsumerWarps * 32;

  // stage this slab's domain words of every state: [0,32) columns, [32,..) rows
  for (int i = ct; i < B * kTcDomWords; i += nct) {
    const int st = i / kTcDomWords, w = i % kTcDomWords;
    const TcView V = tc_view(P, st, k);
    uint32_t val = 0u;
    if (w < 32) {
      const int yy = int(J) * 32 + w;
      if (yy < n) val = ld_dom(V.C + yy);
    } else if (uint32_t(w - 32) < nrows) {
      const int xx = int(I) * 32 + int(row0) + (w - 32);
      if (xx < n) val = ld_dom(V.C + xx);
    }
    S.dom[st][w] = val;
  }
  named_bar(kConsumersBar, nct);

  const int rg = int(nrows + 7) / 8;
  const int n_jobs = 32 * rg + 4 * int(nrows);
  if (warp >= kTcAWarp0 && warp < kTcAWarp0 + kTcAWarps) {
    // A tiles: state s's word of the job's column (forward) or row (reverse)
    const int s = (warp - kTcAWarp0) * 32 + lane;
    for (int idx = 0; idx < n_jobs; ++idx) {
      const uint32_t c = jc + uint32_t(idx);
      const int st = int(c % kTcAStages);
      if (!warp_wait(S, P, &S.a_empty[st], ((c / kTcAStages) & 1u) ^ 1u, lane)) break;
      const int word = idx < 32 * rg ? (idx & 31) : 32 + (idx - 32 * rg) % int(nrows);
      const uint32_t w = s < B ? S.dom[s][word] : 0u;
      uint8_t *At = S.a_tile[st];
#pragma unroll
      for (int qq = 0; qq < 8; ++qq)
        *reinterpret_cast<uint32_t *>(At + tile_off(uint32_t(s), 4u * qq)) =
            expand4((w >> (4 * qq)) & 0xFu);
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.a_full[st]);
    }
  } else if (warp == kTcBWarp) {
    // B tiles: the job's 8 KiB of the FP8 operand store
    if (lane == 0) {
      const uint8_t *tiles = N.fp8 + size_t(si.sl) * size_t(N.fp8_jobs) * kFp8TileBytes;
      for (int idx = 0; idx < n_jobs; ++idx) {
        const uint32_t c = jc + uint32_t(idx);
        const int st = int(c % kTcBStages);
        if (aborted(S) || !mbar_wait(&S.b_empty[st], ((c / kTcBStages) & 1u) ^ 1u,
                                     &P.sync->err, P.wait_limit_ns)) {
          S.abort = 1u;
          break;
        }
        mbar_arrive_expect_tx(&S.b_full[st], kBTileBytes);
        bulk_copy_g2s(S.b_tile[st], tiles + size_t(idx) * kFp8TileBytes, kBTileBytes,
                      &S.b_full[st]);
        S.b_issued = c + 1u;
      }
    }
  } else if (warp == kTcMmaWarp) {
    if (lane == 0) {
      for (int idx = 0; idx < n_jobs; ++idx) {
        const uint32_t c = jc + uint32_t(idx);
        const int sa = int(c % kTcAStages), sb = int(c % kTcBStages);
        const int ab = int(c & 1u);
        if (aborted(S) ||
            !mbar_wait(&S.a_full[sa], (c / kTcAStages) & 1u, &P.sync->err, P.wait_limit_ns) ||
            !mbar_wait(&S.b_full[sb], (c / kTcBStages) & 1u, &P.sync->err, P.wait_limit_ns) ||
            !mbar_wait(&S.acc_empty[ab], ((c >> 1) & 1u) ^ 1u, &P.sync->err, P.wait_limit_ns)) {
          S.abort = 1u;
          break;
        }
        tc_fence_after();
        umma_f8(S.tmem_base + uint32_t(ab) * 256u, umma_desc(S.a_tile[sa]),
                umma_desc(S.b_tile[sb]));
        umma_commit(&S.a_empty[sa]);
        umma_commit(&S.b_empty[sb]);
        umma_commit(&S.acc_full[ab]);
        S.mma_issued = c + 1u;
      }
    }
  } else if (warp < kTcEpiWarps) {
    const int quarter = warp & 3, part = warp >> 2;
    const int s = quarter * 32 + lane;  // this thread's state
    const bool s_ok = s < B && !(S.st_info[s] & kInfoSweepMask);
    // a quarter without running states only keeps the accumulators moving
    const bool live = __any_sync(kFull, s_ok);
    const uint32_t tq = S.tmem_base + (uint32_t(quarter * 32) << 16);
    // AND masks of this part's rows (forward) and columns (reverse): with
    // R = kRelPerPart, facc[R g + i] for row 8 g + R part + i and racc[R g + i]
    // for column 8 g + R part + i
    constexpr int R = kRelPerPart;
    uint32_t facc[4 * R], racc[4 * R];
#pragma unroll
    for (int i = 0; i < 4 * R; ++i) {
      facc[i] = kFull;
      racc[i] = kFull;
    }
    bool ok = true;
    int idx = 0;
#pragma unroll
    for (int g = 0; g < 4; ++g) {  // forward jobs g * 32 + j
      if (g >= rg) break;
      for (int j = 0; j < 32; ++j, ++idx) {
        const uint32_t c = jc + uint32_t(idx);
        const int ab = int(c & 1u);
        if (!ok || !(ok = warp_wait(S, P, &S.acc_full[ab], (c >> 1) & 1u, lane))) continue;
        tc_fence_after();
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const int rr = R * part + i, r = 8 * g + rr;
          if (live && r < int(nrows) && ((hdr[r] >> j) & 1u)) {  // warp-uniform
            uint32_t v[32];
            tmem_ld32(tq + uint32_t(ab) * 256u + uint32_t(rr * 32), v);
            facc[R * g + i] &= pack_positive(v);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.acc_empty[ab]);
      }
    }
    idx = 32 * rg;
#pragma unroll
    for (int g = 0; g < 4; ++g) {  // reverse jobs 32 rg + g nrows + r
      for (int r = 0; r < int(nrows); ++r, ++idx) {
        const uint32_t c = jc + uint32_t(idx);
        const int ab = int(c & 1u);
        if (!ok || !(ok = warp_wait(S, P, &S.acc_full[ab], (c >> 1) & 1u, lane))) continue;
        tc_fence_after();
        const uint32_t pm = hdr[r];
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const int jj = R * part + i, j = 8 * g + jj;
          if (live && ((pm >> j) & 1u)) {  // warp-uniform
            uint32_t v[32];
            tmem_ld32(tq + uint32_t(ab) * 256u + uint32_t(jj * 32), v);
            racc[R * g + i] &= pack_positive(v);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.acc_empty[ab]);
      }
    }
    // removals of this thread's state: this part's rows and columns
    if (ok && s_ok) {
      uint32_t *T = tc_view(P, s, k).T;
      uint32_t colmask = 0u;  // columns with at least one constraint in the slab
      for (int r = 0; r < int(nrows); ++r) colmask |= hdr[r];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const int r = 8 * g + R * part + i;
          if (r < int(nrows) && hdr[r] != 0u) {
            const uint32_t Dx = S.dom[s][32 + r];
            const uint32_t keep = facc[R * g + i] & Dx;
            if (keep != Dx)
              tc_remove(S, P, s, slot_w, T, uint32_t(int(I) * 32 + int(row0) + r), keep);
          }
          const int j = 8 * g + R * part + i;
          if ((colmask >> j) & 1u) {
            const uint32_t Dy = S.dom[s][j];
            const uint32_t keep = racc[R * g + i] & Dy;
            if (keep != Dy) tc_remove(S, P, s, slot_w, T, uint32_t(int(J) * 32 + j), keep);
          }
        }
      }
    }
  }
  jc += uint32_t(n_jobs);
  __syncwarp();                   // the single-lane roles rejoin their warps
  named_bar(kConsumersBar, nct);  // S.dom free for the next slab
}

__global__ void __launch_bounds__(kTcThreads, 1) rac_tc_kernel(const LaunchParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *ring = smem_raw;
  TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw + size_t(kTcStages) * kStageBytes);
  const NetDev &N = P.net;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, cta = blockIdx.x;
  const int B = P.n_states;
  const int n = N.n;
  const bool is_producer = warp == kTcConsumerWarps;
  const int my_slabs = cta < N.n_slabs ? (N.n_slabs - cta + G - 1) / G : 0;
  const int64_t gtid = int64_t(cta) * blockDim.x + tid;
  const int64_t gstride = int64_t(G) * blockDim.x;
  const int64_t cgtid = int64_t(cta) * (kTcConsumerWarps * 32) + tid;
  const int64_t cgstride = int64_t(G) * (kTcConsumerWarps * 32);

  if (warp == 0) {  // the accumulators: 512 tensor-memory columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      mbar_init(&S.full[i], 1);
      mbar_init(&S.empty[i], kTcConsumerWarps);
    }
    for (int i = 0; i < kTcAStages; ++i) {
      mbar_init(&S.a_full[i], kTcAWarps);
      mbar_init(&S.a_empty[i], 1);
    }
    for (int i = 0; i < kTcBStages; ++i) {
      mbar_init(&S.b_full[i], 1);
      mbar_init(&S.b_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.acc_full[i], 1);
      mbar_init(&S.acc_empty[i], kTcEpiWarps);
    }
    fence_mbar_init();
    S.mma_issued = 0;
    S.b_issued = 0;
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
  uint32_t ring_it = 0, prod_it = 0, jc = 0;
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
      if (is_producer) {
        if (lane == 0) {
          if (cta == 0) {  // the slot of the next sweep (the bit-packed kernel's claims too)
            P.sync->bar[slot_c] = 0ull;
            P.sync->claim[slot_c] = 0u;
          }
          const bool incr = (P.flags & RAC_INCREMENTAL) && k >= 2;
          const uint32_t *cu = P.chgU + int64_t(slot_r) * N.nb;
          bool ok = true;
          for (int j = 0; j < my_slabs; ++j) {
            const int sl = cta + j * G;
            const SlabDesc sd = N.slabs[sl];
            if (incr) {
              const uint32_t I = sd.ij & 0xFFFFu, J = sd.ij >> 16;
              const uint32_t row0 = sd.rows & 0xFFu, nrows = sd.rows >> 8;
              const uint32_t rowmask = (nrows >= 32 ? kFull : ((1u << nrows) - 1u)) << row0;
              if (ld_dom(cu + J) == 0u && (ld_dom(cu + I) & rowmask) == 0u) continue;
            }
            const int stg = prod_it % kTcStages;
            const uint32_t par = (prod_it / kTcStages) & 1u;
            if (!mbar_wait(&S.empty[stg], par ^ 1u, &P.sync->err, P.wait_limit_ns)) {
              ok = false;
              break;
            }
            S.stage[stg].sl = sl;
            S.stage[stg].ij = sd.ij;
            S.stage[stg].rows = sd.rows;
            mbar_arrive_expect_tx(&S.full[stg], sd.nbytes);
            bulk_copy_g2s(ring + size_t(stg) * kStageBytes, N.rel + size_t(sd.rel_off16),
                          sd.nbytes, &S.full[stg]);
            ++prod_it;
          }
          if (ok) {
            const int stg = prod_it % kTcStages;
            const uint32_t par = (prod_it / kTcStages) & 1u;
            if (mbar_wait(&S.empty[stg], par ^ 1u, &P.sync->err, P.wait_limit_ns)) {
              S.stage[stg].sl = -1;
              mbar_arrive(&S.full[stg]);
              ++prod_it;
            } else {
              ok = false;
            }
          }
          if (!ok) S.abort = 1;
        }
      } else {
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
              atomicAnd(V.T + x, ld_dom(V.C + x));
            }
          }
        }
        for (;;) {
          const int stg = ring_it % kTcStages;
          const uint32_t par = (ring_it / kTcStages) & 1u;
          // one thread takes the bounded wait; every consumer warp follows its
          // outcome (and only it), so no warp is left at a named barrier
          if (tid == 0)
            S.stage_ok[stg] = mbar_wait(&S.full[stg], par, &P.sync->err, P.wait_limit_ns) ? 1u : 0u;
          named_bar(kConsumersBar, kTcConsumerWarps * 32);
          if (!S.stage_ok[stg]) {
            if (tid == 0) S.abort = 1;
            break;
          }
          if (lane == 0) mbar_try_wait(&S.full[stg], par);
          __syncwarp();
          const TcStage si = S.stage[stg];
          if (si.sl >= 0)
            tc_consume(S, P, ring + size_t(stg) * kStageBytes, si, k, slot_w, warp, lane, jc);
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.empty[stg]);
          ++ring_it;
          if (si.sl < 0) break;
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
  if (is_producer && lane == 0) {
    const uint32_t first = prod_it > uint32_t(kTcStages) ? prod_it - kTcStages : 0u;
    for (uint32_t j = first; j < prod_it; ++j)
      mbar_wait(&S.full[j % kTcStages], (j / kTcStages) & 1u, &P.sync->err, P.wait_limit_ns);
  }
  // no MMA may still write the accumulators, and no operand copy may still
  // be in flight, when they are released: wait for the last ones issued (the
  // phases of a normal run are complete already)
  if (tid == 0) {
    const uint32_t mi = S.mma_issued, bi = S.b_issued;
    if (mi > 0) {
      const uint32_t c = mi - 1u;
      mbar_wait(&S.acc_full[c & 1u], (c >> 1) & 1u, &P.sync->err, P.wait_limit_ns);
    }
    const uint32_t first = bi > uint32_t(kTcBStages) ? bi - kTcBStages : 0u;
    for (uint32_t c = first; c < bi; ++c)
      mbar_wait(&S.b_full[c % kTcBStages], (c / kTcBStages) & 1u, &P.sync->err,
                P.wait_limit_ns);
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
  const size_t smem = size_t(kTcStages) * kStageBytes + sizeof(TcSmem);
  if (P.n_states > kTcMaxStates) {
    set_error("the tensor-core kernel takes at most 128 states per launch");
    return RAC_EINVAL;
  }
  if (!P.net.fp8 || P.net.fp8_jobs != fp8_jobs_for(P.net.rows_per_slab)) {
    set_error("the network's FP8 operand store is missing");
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

rac_status ensure_fp8(const rac_network *net, cudaStream_t stream) {
  std::lock_guard<std::mutex> lock(net->mu);
  if (net->d_fp8) return RAC_OK;
  const size_t tiles = size_t(net->n_slabs) * size_t(net->fp8_jobs);
  const size_t bytes = tiles * size_t(kFp8TileBytes);
  if (bytes > (size_t(64) << 30)) {
    set_error("the FP8 operand store of this network would take " +
              std::to_string(bytes >> 30) + " GiB (at most 64)");
    return RAC_ENOTSUP;
  }
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("out of device memory for the FP8 operand store (" + std::to_string(bytes) +
              " bytes)");
    return RAC_ENOMEM;
  }
  if (tiles > 0) {
    NetDev N = net_dev(net);
    const int64_t words = int64_t(tiles) * (kFp8TileBytes / 4);
    const int64_t blocks = std::min<int64_t>((words + 255) / 256, int64_t(1) << 20);
    rac_fp8_build_kernel<<<unsigned(blocks), 256, 0, stream>>>(N, static_cast<uint8_t *>(p));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
      cudaFree(p);
      return cuda_fail(e, "building the FP8 operand store");
    }
  }
  net->d_fp8 = static_cast<uint8_t *>(p);
  net->fp8_bytes = bytes;
  return RAC_OK;
}

}  // namespace rac
