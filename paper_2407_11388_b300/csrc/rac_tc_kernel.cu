// Kernel (b): the support counts of Eq. 1 on the 5th-generation tensor cores
// (tcgen05.mma, FP8 E4M3 0/1 operands, FP32 accumulation in tensor memory),
// for up to 128 domain states of one network, swept to the fixpoint in one
// persistent cooperative launch.
//
// For every relation R_xy of a slab and every state s the counts are
//   forward  Sup_xy[a](s) = sum_b R[a][b] D_s[y][b]     (Fig. 1)
//   reverse  Sup_yx[b](s) = sum_a R[a][b] D_s[x][a]
// computed as GEMMs with M = 128 states, K = 32 values and N = 256 =
// 8 relations x 32 rows: a forward MMA per (column y, group of 8 rows) takes
// D_s[y] as A and the 8 relations R_{x,y} as B; a reverse MMA per (row x,
// group of 8 columns) takes D_s[x] as A and the 8 transposed relations as B.
// Counts are exact in FP32 (at most 32).  The epilogue reads the accumulator
// lanes (one state per lane), clamps every count to {0,1} (only Sup > 0
// matters, as in the paper's listing), packs the 32 values of a relation row
// into one word and ANDs it over the row's or column's constraints; the
// removals then follow kernel (a) (atomicAnd into the next domain buffer).
//
// Operand tiles are built in shared memory from the bit-packed slab (the
// reverse direction transposes each relation with 32 warp ballots) in the
// canonical K-major layout without swizzle (8-row x 16-byte core matrices,
// 128 B apart along K, 256 B apart along M/N).  Operand buffers and
// accumulators are double-buffered: while MMA i runs, the warps build the
// operands of MMA i+1 and run the epilogue of MMA i-1.
#include "rac_device.cuh"
#include "rac_internal.h"

namespace rac {
namespace {

using namespace dev;

constexpr int kTcConsumerWarps = 12;  // 3 per TMEM lane quarter
constexpr int kTcThreads = (kTcConsumerWarps + 1) * 32;
constexpr int kTcStages = 4;
constexpr int kTcMaxStates = 128;     // M of the MMA
constexpr int kTcN = 256;             // N of the MMA: 8 relations x 32 rows
constexpr uint32_t kTmemCols = 512;   // two accumulators of 256 columns
constexpr int kATileBytes = kTcMaxStates * 32;  // 4 KB
constexpr int kBTileBytes = kTcN * 32;          // 8 KB
constexpr int kTcDomWords = 64;                 // per state: 32 columns + up to 32 rows

struct TcStage {
  int32_t sl;
  uint32_t ij, rows, pad;
};

struct TcSmem {
  uint8_t a_tile[2][kATileBytes];
  uint8_t b_tile[2][kBTileBytes];
  uint32_t dom[kTcMaxStates][kTcDomWords];  // staged D_{k-1} words of the slab
  uint64_t full[kTcStages];
  uint64_t empty[kTcStages];
  uint64_t mma_done[2];
  TcStage stage[kTcStages];
  uint32_t stage_ok[kTcStages];
  uint32_t tmem_base;
  uint32_t base, poisoned, abort, failed, all_done;
  uint32_t any_total, wipe_total, cta_any, cta_wipe;
  uint32_t st_info[kTcMaxStates];
  uint8_t any_loc[kTcMaxStates], wipe_loc[kTcMaxStates];
};
static_assert(size_t(kTcStages) * kStageBytes + sizeof(TcSmem) + 1024 <= 232448,
              "shared memory of the tensor-core kernel exceeds 227 KB");

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
// Row word w (bit k = 1) -> the 32 bytes of one tile row.
__device__ __forceinline__ void put_row(uint8_t *tile, uint32_t row, uint32_t w) {
#pragma unroll
  for (int q = 0; q < 8; ++q)
    *reinterpret_cast<uint32_t *>(tile + tile_off(row, 4u * q)) = expand4((w >> (4 * q)) & 0xFu);
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

// Relation row `a` (a < 32; rows >= 4Q are zero) of the t-th relation of slab
// row r, in the chunk-major stage layout.
__device__ __forceinline__ uint32_t rel_row(const uint32_t *hdr, const uint32_t *relw,
                                            uint32_t nrows, int q, int r, uint32_t t, int a) {
  if (a >= 4 * q) return 0u;
  const uint32_t pm = hdr[r], cnt = __popc(pm);
  const uint32_t base_chunk = hdr[nrows + r] * uint32_t(q);
  return relw[(base_chunk + uint32_t(a >> 2) * cnt + t) * 4u + uint32_t(a & 3)];
}

// The whole slab for every running state: 2 * ceil(nrows/8) * 32 MMAs.
__device__ void tc_consume(TcSmem &S, const LaunchParams &P, const unsigned char *stage,
                           const TcStage &si, int k, int slot_w, int warp, int lane,
                           uint32_t &mma_count) {
  const NetDev &N = P.net;
  const int n = N.n, q = N.q, B = P.n_states;
  const uint32_t I = si.ij & 0xFFFFu, J = si.ij >> 16;
  const uint32_t row0 = si.rows & 0xFFu, nrows = si.rows >> 8;
  const uint32_t *hdr = reinterpret_cast<const uint32_t *>(stage);
  const uint32_t *relw = hdr + 2 * nrows;
  const int ct = warp * 32 + lane;  // consumer thread
  const int nct = kTcConsumerWarps * 32;
  const int quarter = warp & 3, part = warp >> 2;  // TMEM lanes 32*quarter.., column part
  const int s = quarter * 32 + lane;               // this thread's state in the epilogue
  const bool s_ok = s < B && !(S.st_info[s] & kInfoSweepMask);

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

  const int rgroups = int(nrows + 7) / 8;
  const int n_mma = 32 * rgroups + int(nrows) * 4;  // forward (column, row group), reverse (row, column group)
  // this thread's AND accumulators: rows r with (r % 8) % 3 == part, columns j
  // with (j % 8) % 3 == part (12 of each at most)
  uint32_t facc[12], racc[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    facc[i] = kFull;
    racc[i] = kFull;
  }

  auto build = [&](int idx, int buf) {
    uint8_t *At = S.a_tile[buf];
    uint8_t *Bt = S.b_tile[buf];
    if (idx < 32 * rgroups) {  // forward: column j, rows 8g..8g+7
      const int j = idx / rgroups, g = idx % rgroups;
      for (int i = ct; i < kTcMaxStates * 8; i += nct) {  // A: D_s[y_j] bits
        const int st = i >> 3, qq = i & 7;
        const uint32_t w = st < B ? S.dom[st][j] : 0u;
        *reinterpret_cast<uint32_t *>(At + tile_off(st, 4 * qq)) = expand4((w >> (4 * qq)) & 0xFu);
      }
      for (int i = ct; i < kTcN * 8; i += nct) {  // B: rows (r, a) of R_{x_r, y_j}
        const int row = i >> 3, qq = i & 7;
        const int r = 8 * g + (row >> 5), a = row & 31;
        uint32_t w = 0u;
        if (r < int(nrows)) {
          const uint32_t pm = hdr[r];
          if ((pm >> j) & 1u) w = rel_row(hdr, relw, nrows, q, r, __popc(pm & ((1u << j) - 1u)), a);
        }
        *reinterpret_cast<uint32_t *>(Bt + tile_off(row, 4 * qq)) = expand4((w >> (4 * qq)) & 0xFu);
      }
    } else {  // reverse: row r, columns 8g..8g+7
      const int ridx = idx - 32 * rgroups;
      const int r = ridx / 4, g = ridx % 4;
      for (int i = ct; i < kTcMaxStates * 8; i += nct) {  // A: D_s[x_r] bits
        const int st = i >> 3, qq = i & 7;
        const uint32_t w = st < B ? S.dom[st][32 + r] : 0u;
        *reinterpret_cast<uint32_t *>(At + tile_off(st, 4 * qq)) = expand4((w >> (4 * qq)) & 0xFu);
      }
      // B: rows (j, b) = column b of R_{x_r, y_j}: one warp transposes one relation
      const uint32_t pm = hdr[r];
      for (int jj = warp; jj < 8; jj += kTcConsumerWarps) {
        const int j = 8 * g + jj;
        const bool present = (pm >> j) & 1u;
        const uint32_t t = __popc(pm & ((1u << j) - 1u));
        const uint32_t mine = present ? rel_row(hdr, relw, nrows, q, r, t, lane) : 0u;
        uint32_t col = 0u;
#pragma unroll 8
        for (int b = 0; b < 32; ++b) {
          const uint32_t m = __ballot_sync(kFull, (mine >> b) & 1u);
          if (lane == b) col = m;
        }
        put_row(Bt, uint32_t(jj * 32 + lane), col);
      }
    }
  };

  auto epilogue = [&](int idx, int buf) {
    const uint32_t acc = S.tmem_base + uint32_t(buf) * 256u + (uint32_t(quarter * 32) << 16);
    if (idx < 32 * rgroups) {
      const int j = idx / rgroups, g = idx % rgroups;
      for (int rr = part; rr < 8; rr += 3) {
        const int r = 8 * g + rr;
        uint32_t v[32];
        tmem_ld32(acc + uint32_t(rr * 32), v);  // all lanes of the warp, even idle states
        if (r >= int(nrows) || !s_ok || !((hdr[r] >> j) & 1u)) continue;
        uint32_t m = 0u;
#pragma unroll
        for (int a = 0; a < 32; ++a) m |= (__uint_as_float(v[a]) > 0.5f ? 1u : 0u) << a;
        facc[(r / 8) * 3 + (r % 8) / 3] &= m;
      }
    } else {
      const int ridx = idx - 32 * rgroups;
      const int r = ridx / 4, g = ridx % 4;
      for (int jj = part; jj < 8; jj += 3) {
        const int j = 8 * g + jj;
        uint32_t v[32];
        tmem_ld32(acc + uint32_t(jj * 32), v);
        if (!s_ok || !((hdr[r] >> j) & 1u)) continue;
        uint32_t m = 0u;
#pragma unroll
        for (int b = 0; b < 32; ++b) m |= (__uint_as_float(v[b]) > 0.5f ? 1u : 0u) << b;
        racc[(j / 8) * 3 + (j % 8) / 3] &= m;
      }
    }
  };

  // MMA number g (counted over the whole launch) uses operand buffer and
  // accumulator g & 1; it is the (g >> 1)-th use of that buffer, so its
  // completion is the phase of parity (g >> 1) & 1 of mma_done[g & 1].
  const bool leader = ct == 0;
  for (int idx = 0; idx <= n_mma; ++idx) {
    const uint32_t g = mma_count + uint32_t(idx);
    const int buf = int(g & 1u);
    if (idx < n_mma) {
      build(idx, buf);  // buffer last read by MMA g-2, whose completion was awaited
      fence_async_smem();
      tc_fence_before();
      named_bar(kConsumersBar, nct);
      tc_fence_after();
      if (leader) {
        umma_f8(S.tmem_base + uint32_t(buf) * 256u, umma_desc(S.a_tile[buf]),
                umma_desc(S.b_tile[buf]));
        umma_commit(&S.mma_done[buf]);
      }
    }
    if (idx >= 1) {
      const uint32_t gp = g - 1u;
      const int pb = int(gp & 1u);
      const bool ok = mbar_wait(&S.mma_done[pb], (gp >> 1) & 1u, &P.sync->err, P.wait_limit_ns);
      if (!ok) S.abort = 1;
      tc_fence_after();
      epilogue(idx - 1, pb);
      tc_fence_before();
      named_bar(kConsumersBar, nct);  // accumulator pb free for MMA g+1
    }
  }
  mma_count += uint32_t(n_mma);

  // removals of this thread's state, rows and columns
  if (s_ok) {
    uint32_t *T = tc_view(P, s, k).T;
    for (int r = 0; r < int(nrows); ++r) {
      if ((r % 8) % 3 != part || hdr[r] == 0u) continue;
      const uint32_t Dx = S.dom[s][32 + r];
      const uint32_t keep = facc[(r / 8) * 3 + (r % 8) / 3] & Dx;
      if (keep != Dx) tc_remove(S, P, s, slot_w, T, uint32_t(int(I) * 32 + int(row0) + r), keep);
    }
    uint32_t colmask = 0u;  // columns with at least one constraint in the slab
    for (int r = 0; r < int(nrows); ++r) colmask |= hdr[r];
    for (int j = 0; j < 32; ++j) {
      if ((j % 8) % 3 != part || !((colmask >> j) & 1u)) continue;
      const uint32_t Dy = S.dom[s][j];
      const uint32_t keep = racc[(j / 8) * 3 + (j % 8) / 3] & Dy;
      if (keep != Dy) tc_remove(S, P, s, slot_w, T, uint32_t(int(J) * 32 + j), keep);
    }
  }
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
    mbar_init(&S.mma_done[0], 1);
    mbar_init(&S.mma_done[1], 1);
    fence_mbar_init();
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
  uint32_t ring_it = 0, prod_it = 0, mma_count = 0;
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
            tc_consume(S, P, ring + size_t(stg) * kStageBytes, si, k, slot_w, warp, lane,
                       mma_count);
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
        unsigned long long v = atomicAdd(w, mine) + mine;
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
  // no MMA may still write the accumulators when they are released
  if (tid == 0 && mma_count > 0) {
    for (uint32_t b = 0; b < 2; ++b) {
      const uint32_t uses = (mma_count + 1u - b) / 2u;  // MMAs issued on buffer b
      if (uses) mbar_wait(&S.mma_done[b], (uses - 1u) & 1u, &P.sync->err, P.wait_limit_ns);
    }
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

}  // namespace rac
