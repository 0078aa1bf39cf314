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
