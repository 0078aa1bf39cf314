// The FP16 x 3 operand format of the tensor-core product (gemm_tc.cu), shared with the Krylov kernels that
// write the next basis vector straight into it.
//
// A value v (already scaled into |v| <= 1) is stored as hi = fp16(v) and lo = fp16(2^11 (v - hi)).  The
// right-hand-side block is the K-major operand Bt of 128 rows: for system s, row s holds the pairs
// (Re x_s[k], -Im x_s[k]) and row 64 + s the pairs (Im x_s[k], Re x_s[k]), at FP16 columns 2k and 2k + 1.
#pragma once

#include <cuda_fp16.h>

namespace bem {

constexpr float kTcLoScale = 2048.f;   // lo parts are stored times 2^11

// Stream-K partial tiles of the product D = A Bt^T (gemm_tc.cu): CTA c of G owns K-steps [total c / G,
// total (c + 1) / G) of the (row tile, K-step) sequence (kpt K-steps per tile of kTcM rows) and writes one partial
// tile per row tile it touches, at partial + (2 c + slot) kTcM kTcN, slot 0 for the first row tile of its range
// and 1 for the second.  A partial tile is column-major: (row rr, column col) at col kTcM + rr, column s holding
// Re y_s and column 64 + s Im y_s of the scaled product; y = (sum of the partials) / (rsc[row] tsc[s]).
constexpr int kTcM = 128;
constexpr int kTcN = 128;
constexpr int kTcMaxCover = 64;   // partial tiles of one row tile at most (about 24 at worst for n >= 128)

// The CTAs whose ranges meet row tile t, in CTA order, as 2 c + slot; at most maxc are written, the count is
// returned.  32-bit unsigned divisions where total G fits (every practical size): 64-bit divisions are long
// instruction sequences.
__device__ __forceinline__ int tc_cover(int t, int kpt, long long total, int G, int* out, int maxc) {
  int m = 0;
  if ((unsigned long long)total * (unsigned long long)G < (1ull << 32)) {
    const unsigned tot = (unsigned)total, g = (unsigned)G, lo = (unsigned)t * (unsigned)kpt, hi = lo + (unsigned)kpt;
    unsigned c0 = (lo * g) / tot;
    while (c0 > 0 && tot * c0 / g > lo) --c0;
    while (tot * (c0 + 1) / g <= lo) ++c0;
    for (unsigned c = c0; c < g && m < maxc; ++c) {
      const unsigned beg = tot * c / g;
      if (beg >= hi) break;
      out[m++] = (int)(2 * c + ((beg / (unsigned)kpt == (unsigned)t) ? 0 : 1));
    }
  } else {
    const long long lo = (long long)t * kpt, hi = lo + kpt;
    int c0 = (int)((lo * G) / total);
    while (c0 > 0 && total * c0 / G > lo) --c0;
    while (total * (c0 + 1) / G <= lo) ++c0;
    for (int c = c0; c < G && total * c / G < hi && m < maxc; ++c)
      out[m++] = 2 * c + (((total * c / G) / kpt == t) ? 0 : 1);
  }
  return m;
}

__device__ __forceinline__ void tc_split16(float v, __half& h, __half& l) {
  h = __float2half_rn(v);
  l = __float2half_rn((v - __half2float(h)) * kTcLoScale);
}

// Two values at once with the packed conversions (two FP32 -> FP16 in one instruction).
__device__ __forceinline__ void tc_split16x2(float v0, float v1, __half2& h, __half2& l) {
  h = __floats2half2_rn(v0, v1);
  const float2 hf = __half22float2(h);
  l = __floats2half2_rn((v0 - hf.x) * kTcLoScale, (v1 - hf.y) * kTcLoScale);
}

// Column k of system s of Bt (hi rows at bhi, lo rows at blo, row stride ldb FP16 elements).
__device__ __forceinline__ void tc_write_b(__half* bhi, __half* blo, size_t ldb, int s, int k, float re, float im) {
  __half2 h, l;
  size_t o = (size_t)s * ldb + 2 * (size_t)k;
  tc_split16x2(re, -im, h, l);
  *reinterpret_cast<__half2*>(bhi + o) = h;
  *reinterpret_cast<__half2*>(blo + o) = l;
  o = (size_t)(64 + s) * ldb + 2 * (size_t)k;
  tc_split16x2(im, re, h, l);
  *reinterpret_cast<__half2*>(bhi + o) = h;
  *reinterpret_cast<__half2*>(blo + o) = l;
}

}  // namespace bem
