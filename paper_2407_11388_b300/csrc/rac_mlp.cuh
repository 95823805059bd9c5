// The active-block predictor: an MLP 8 -> 64 -> 64 -> 1 (ReLU, logit out)
// with BF16 weights and FP32 accumulation.  It scores a (relation slab,
// domain state) pair before sweep k >= 2 evaluates it: a high logit means
// the evaluation is likely to remove a value.  Exactness never depends on
// it (a skipped pair is caught by the full verification sweep; Lemma 1 makes
// every removal made on the way sound).
//
// Features (all in [0, 1]), from D_{k-1} and the variables changed by
// sweep k-1:
//   f0  min(k, 16) / 16                                sweep index
//   f1  slab rows (x) that lost a value in sweep k-1 / slab rows
//   f2  column-block variables (y) that lost a value in sweep k-1 / 32
//   f3  disallowed fraction of the slab's relation bits (tightness)
//   f4  constraints in the slab / (slab rows * 32)     (density)
//   f5  min over the column variables of |D_{k-1}(y)| / d
//   f6  mean over the column variables of |D_{k-1}(y)| / d
//   f7  min over the slab's row variables of |D_{k-1}(x)| / d
//
// Forward pass (both in training and in the sweep kernel): the features and
// the first hidden layer are rounded to BF16 before they enter a product
// (they are the BF16 operands of the tensor-core MMA in the sweep kernel);
// every product is accumulated in FP32.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace rac {

constexpr int kMlpIn = 8;
constexpr int kMlpHidden = 64;
// parameter layout (elements): W1[64][8] b1[64] W2[64][64] b2[64] w3[64] b3
constexpr int kMlpW1 = 0;
constexpr int kMlpB1 = kMlpW1 + kMlpHidden * kMlpIn;
constexpr int kMlpW2 = kMlpB1 + kMlpHidden;
constexpr int kMlpB2 = kMlpW2 + kMlpHidden * kMlpHidden;
constexpr int kMlpW3 = kMlpB2 + kMlpHidden;
constexpr int kMlpB3 = kMlpW3 + kMlpHidden;
constexpr int kMlpParams = kMlpB3 + 1;  // 4,801
static_assert(kMlpB1 % 2 == 0 && kMlpW2 % 2 == 0 && kMlpB2 % 2 == 0 && kMlpW3 % 2 == 0,
              "pairs of BF16 parameters are read as 32-bit words");

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16(v)); }

__device__ __forceinline__ float mlp_w(const __nv_bfloat16 *w, int i) {
  return __bfloat162float(w[i]);
}

// Scalar forward pass for one sample (training).  xr receives the rounded
// inputs, h1 the rounded first hidden layer, h2 the second.
__device__ __forceinline__ float mlp_forward(const __nv_bfloat16 *w, const float *x, float *xr,
                                             float *h1, float *h2) {
#pragma unroll
  for (int j = 0; j < kMlpIn; ++j) xr[j] = bf16r(x[j]);
  for (int i = 0; i < kMlpHidden; ++i) {
    float acc = mlp_w(w, kMlpB1 + i);
#pragma unroll
    for (int j = 0; j < kMlpIn; ++j) acc = fmaf(mlp_w(w, kMlpW1 + i * kMlpIn + j), xr[j], acc);
    h1[i] = bf16r(fmaxf(acc, 0.0f));
  }
  float z = mlp_w(w, kMlpB3);
  for (int i = 0; i < kMlpHidden; ++i) {
    float acc = mlp_w(w, kMlpB2 + i);
    for (int j = 0; j < kMlpHidden; ++j) acc = fmaf(mlp_w(w, kMlpW2 + i * kMlpHidden + j), h1[j], acc);
    h2[i] = fmaxf(acc, 0.0f);
    z = fmaf(mlp_w(w, kMlpW3 + i), h2[i], z);
  }
  return z;
}

// ---------------------------------------------------------------------------
// Warp-wide inference on the tensor cores: lane i holds the 8 features of
// sample i (32 samples); returns sample i's logit in lane i.  The samples are
// the 16-row M tiles of mma.m16n8k16 (BF16 in, FP32 accumulate); layer 1 is
// K = 16 (features padded with zeros), layer 2 is K = 64, and the 64 -> 1
// output layer is folded into the layer-2 epilogue.  The accumulator
// fragment of two adjacent n8 tiles is exactly the A fragment of one k16
// slice of the next layer, so the hidden activations never leave registers.
//
// The weights come fragment-packed (mlp_pack_word): lane l's B fragments,
// biases and output weights are 24 consecutive-by-lane 16-byte chunks, so
// every weight load of the warp is one coalesced 512-byte read (the sweep
// kernel keeps the packed copy in shared memory).
// ---------------------------------------------------------------------------
constexpr int kPackChunks = 24;                       // uint4 per lane
constexpr int kPackWords = kPackChunks * 32 * 4 + 4;  // + b3 (as a float) and padding
constexpr int kPackVec4 = kPackWords / 4;             // the same in 16-byte units
// chunks: 0-1 W1 fragments, 2-3 b1 pairs, 4-19 W2 fragments (n tile nt: chunks
// 4 + 2 nt, 5 + 2 nt = k slices 0,1 | 2,3, each b0 b1), 20-21 b2 pairs,
// 22-23 w3 pairs; word j of lane l is word j % 4 of chunk j / 4.

// Word j (0..95) of lane l = 4 g + t: two BF16 parameters, the first in the
// low half.  Returns the parameter indices.
__host__ __device__ inline void mlp_pack_word(int lane, int j, int &i0, int &i1) {
  const int g = lane >> 2, t = lane & 3;
  if (j < 8) {
    i0 = kMlpW1 + (8 * j + g) * kMlpIn + 2 * t;
  } else if (j < 16) {
    i0 = kMlpB1 + 8 * (j - 8) + 2 * t;
  } else if (j < 80) {
    const int q = j - 16, nt = q >> 3, ks = (q & 7) >> 1, half = q & 1;
    i0 = kMlpW2 + (8 * nt + g) * kMlpHidden + 16 * ks + 2 * t + 8 * half;
  } else if (j < 88) {
    i0 = kMlpB2 + 8 * (j - 80) + 2 * t;
  } else {
    i0 = kMlpW3 + 8 * (j - 88) + 2 * t;
  }
  i1 = i0 + 1;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float2 unpack_bf16(uint32_t v) {
  const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&v);
  return __bfloat1622float2(b);
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], uint32_t a0, uint32_t a1,
                                               uint32_t a2, uint32_t a3, uint32_t b0,
                                               uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// MT = 1: only samples 0..15 are scored (the other lanes get garbage).
template <int MT>
__device__ __forceinline__ float mlp_warp_logits_mt(const uint4 *wp, const float (&f)[kMlpIn]) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const uint4 *L = wp + lane;
  // each lane's features as four BF16 pairs (f0 f1 | f2 f3 | f4 f5 | f6 f7)
  const uint32_t p0 = pack_bf16(f[0], f[1]), p1 = pack_bf16(f[2], f[3]);
  const uint32_t p2 = pack_bf16(f[4], f[5]), p3 = pack_bf16(f[6], f[7]);
  // word j of this lane (chunk j / 4, component j % 4)
  const uint32_t *Lw = reinterpret_cast<const uint32_t *>(L);
  auto word = [&](int j) { return Lw[(j >> 2) * 128 + (j & 3)]; };
  uint32_t h[MT][4][4];  // layer-2 A fragments: [m tile][k slice][reg]
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
    // A fragment of layer 1: rows r0 = 16 mt + g and r0 + 8, columns 2t, 2t+1
    // (columns 8..15 are the zero padding)
    const int r0 = 16 * mt + g;
    uint32_t q0 = __shfl_sync(0xFFFFFFFFu, p0, r0), q1 = __shfl_sync(0xFFFFFFFFu, p1, r0);
    uint32_t q2 = __shfl_sync(0xFFFFFFFFu, p2, r0), q3 = __shfl_sync(0xFFFFFFFFu, p3, r0);
    const uint32_t a0 = t == 0 ? q0 : t == 1 ? q1 : t == 2 ? q2 : q3;
    q0 = __shfl_sync(0xFFFFFFFFu, p0, r0 + 8);
    q1 = __shfl_sync(0xFFFFFFFFu, p1, r0 + 8);
    q2 = __shfl_sync(0xFFFFFFFFu, p2, r0 + 8);
    q3 = __shfl_sync(0xFFFFFFFFu, p3, r0 + 8);
    const uint32_t a1 = t == 0 ? q0 : t == 1 ? q1 : t == 2 ? q2 : q3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16_16816(c, a0, a1, 0u, 0u, word(nt), 0u);
      const float2 b = unpack_bf16(word(8 + nt));
      const uint32_t lo = pack_bf16(fmaxf(c[0] + b.x, 0.f), fmaxf(c[1] + b.y, 0.f));  // row g
      const uint32_t hi = pack_bf16(fmaxf(c[2] + b.x, 0.f), fmaxf(c[3] + b.y, 0.f));  // row g+8
      h[mt][nt >> 1][(nt & 1) ? 2 : 0] = lo;
      h[mt][nt >> 1][(nt & 1) ? 3 : 1] = hi;
    }
  }
  // layer 2 by n tile, both M tiles per weight load, with ReLU and the output
  // layer in the epilogue
  float sl[MT], sh[MT];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) sl[mt] = sh[mt] = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const uint4 wq0 = L[(4 + 2 * nt) * 32], wq1 = L[(5 + 2 * nt) * 32];
    const float2 b = unpack_bf16(word(80 + nt));
    const float2 o = unpack_bf16(word(88 + nt));
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16_16816(c, h[mt][0][0], h[mt][0][1], h[mt][0][2], h[mt][0][3], wq0.x, wq0.y);
      mma_bf16_16816(c, h[mt][1][0], h[mt][1][1], h[mt][1][2], h[mt][1][3], wq0.z, wq0.w);
      mma_bf16_16816(c, h[mt][2][0], h[mt][2][1], h[mt][2][2], h[mt][2][3], wq1.x, wq1.y);
      mma_bf16_16816(c, h[mt][3][0], h[mt][3][1], h[mt][3][2], h[mt][3][3], wq1.z, wq1.w);
      sl[mt] = fmaf(o.x, fmaxf(c[0] + b.x, 0.f), fmaf(o.y, fmaxf(c[1] + b.y, 0.f), sl[mt]));
      sh[mt] = fmaf(o.x, fmaxf(c[2] + b.x, 0.f), fmaf(o.y, fmaxf(c[3] + b.y, 0.f), sh[mt]));
    }
  }
  // the four lanes of a quad hold disjoint columns: sum them
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
    sl[mt] += __shfl_xor_sync(0xFFFFFFFFu, sl[mt], 1);
    sl[mt] += __shfl_xor_sync(0xFFFFFFFFu, sl[mt], 2);
    sh[mt] += __shfl_xor_sync(0xFFFFFFFFu, sh[mt], 1);
    sh[mt] += __shfl_xor_sync(0xFFFFFFFFu, sh[mt], 2);
  }
  // sample i = 16 mt + 8 h + r sits in lane 4 r of the (mt, h) value
  const int src = 4 * (lane & 7);
  const int sel = lane >> 3;
  const float v0 = __shfl_sync(0xFFFFFFFFu, sl[0], src), v1 = __shfl_sync(0xFFFFFFFFu, sh[0], src);
  float z = sel == 0 ? v0 : v1;
  if (MT == 2) {
    const float v2 = __shfl_sync(0xFFFFFFFFu, sl[MT - 1], src);
    const float v3 = __shfl_sync(0xFFFFFFFFu, sh[MT - 1], src);
    z = sel == 0 ? v0 : sel == 1 ? v1 : sel == 2 ? v2 : v3;
  }
  const float b3 = *reinterpret_cast<const float *>(wp + kPackChunks * 32);
  return z + b3;
}

// Every lane must call this (warp-synchronous); `upper` says whether any of
// samples 16..31 is needed.
__device__ __forceinline__ float mlp_warp_logits(const uint4 *wp, const float (&f)[kMlpIn],
                                                 bool upper) {
  return upper ? mlp_warp_logits_mt<2>(wp, f) : mlp_warp_logits_mt<1>(wp, f);
}


}  // namespace rac
