// Small dense steps of GMRES (Sec. 3.2, no restart): the Givens rotations that triangularise each new
// Hessenberg column, and the back substitution for the least-squares coefficients.  Shared by the
// single-problem solver (krylov.cu) and the batched engine (batch.cu).  The rotations run in FP64, or in
// FP32 for the inner solves on an FP32 basis (complex type C = double2 or float2); the back substitution
// is FP64.
#pragma once

#include "internal.cuh"

namespace bem {

__device__ __forceinline__ double2 shfl_up2(double2 v, int off) {
  return make_double2(__shfl_up_sync(0xffffffffu, v.x, off), __shfl_up_sync(0xffffffffu, v.y, off));
}
__device__ __forceinline__ double2 shfl2(double2 v, int lane) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, lane), __shfl_sync(0xffffffffu, v.y, lane));
}
__device__ __forceinline__ float2 shfl_up2(float2 v, int off) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, off), __shfl_up_sync(0xffffffffu, v.y, off));
}
__device__ __forceinline__ float2 shfl2(float2 v, int lane) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, lane), __shfl_sync(0xffffffffu, v.y, lane));
}
template <typename C> __device__ __forceinline__ C cx(double x, double y);
template <> __device__ __forceinline__ double2 cx<double2>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 cx<float2>(double x, double y) { return make_float2((float)x, (float)y); }

// Apply rotations 0..j-1 to the Hessenberg column h[0..j] (shared memory; rotation i acts on rows (i, i+1)
// as [[conj c_i, conj s_i], [-s_i, c_i]]).  Called by all 32 lanes of one warp.
//
// Row i+1 of the running column obeys the first-order recurrence a_{i+1} = -s_i a_i + c_i h_{i+1}
// (a_0 = h_0), and the rotated entry is conj(c_i) a_i + conj(s_i) h_{i+1}.  The recurrence is a chain of
// affine maps a -> p a + q, whose composition is associative, so the warp evaluates it as a scan: each lane
// composes the maps of a contiguous run of ceil(j/32) rotations, an inclusive shuffle scan combines the
// runs, and each lane then walks its own run from its entry value.  That is ceil(j/32) + 5 + ceil(j/32)
// dependent steps instead of j (|s_i| <= 1, so the composed maps stay bounded).
// On return h[0..j-1] hold the rotated entries and every lane has the rotated row j (the new pivot).
template <typename C>
__device__ __forceinline__ C warp_rotate_column(C* h, const C* c, const C* s, int j) {
  const int lane = threadIdx.x & 31;
  const C h0 = h[0];
  if (j == 0) return h0;
  const int seg = (j + 31) >> 5;
  const int lo = min(lane * seg, j), hi = min(lo + seg, j);
  const C hb = h[hi];     // first entry of the next run: the next lane overwrites it during its walk
  C P = cx<C>(1.0, 0.0), Q = cx<C>(0.0, 0.0);
  for (int i = lo; i < hi; ++i) {
    const C p = cx<C>(-s[i].x, -s[i].y);
    Q = cadd(cmul(p, Q), cmul(c[i], h[i + 1]));
    P = cmul(p, P);
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const C Pp = shfl_up2(P, off), Qp = shfl_up2(Q, off);
    if (lane >= off) {
      Q = cadd(cmul(P, Qp), Q);
      P = cmul(P, Pp);
    }
  }
  C Pe = shfl_up2(P, 1), Qe = shfl_up2(Q, 1);
  if (lane == 0) {
    Pe = cx<C>(1.0, 0.0);
    Qe = cx<C>(0.0, 0.0);
  }
  C a = cadd(cmul(Pe, h0), Qe);
  __syncwarp();
  for (int i = lo; i < hi; ++i) {
    const C b = (i + 1 < hi) ? h[i + 1] : hb;
    h[i] = cadd(cdotc(c[i], a), cdotc(s[i], b));
    a = csub(cmul(c[i], b), cmul(s[i], a));
  }
  __syncwarp();
  return shfl2(a, (j - 1) / seg);
}

// den = sqrt(|a|^2 + hn^2) and inv = 1 / den for a new Givens rotation, by one reciprocal square root
// (FP64 division and hypot are long instruction sequences on GB300's narrow FP64 pipe, and this runs once
// per system and iteration on the critical path); hypot only where the sum of squares would leave the
// normal range.  inv = 0 when den = 0.
__device__ __forceinline__ void givens_norm(double2 a, double hn, double& den, double& inv) {
  const double q = fma(a.x, a.x, fma(a.y, a.y, hn * hn));
  if (q > 1e-280 && q < 1e280) {
    inv = rsqrt(q);
    den = q * inv;
  } else {
    den = hypot(hypot(a.x, a.y), hn);
    inv = den > 0.0 ? 1.0 / den : 0.0;
  }
}
__device__ __forceinline__ void givens_norm(float2 a, float hn, float& den, float& inv) {
  const float q = fmaf(a.x, a.x, fmaf(a.y, a.y, hn * hn));
  if (q > 1e-30f && q < 1e30f) {
    inv = rsqrtf(q);
    den = q * inv;
  } else {
    den = hypotf(hypotf(a.x, a.y), hn);
    inv = den > 0.f ? 1.f / den : 0.f;
  }
}

// Back substitution R y = g for the mm x mm upper-triangular R (column i at R + i*ld, rows 0..i), by a whole
// CTA of kBsThreads threads: column-oriented, y_i = g_i / R_ii and then g_k -= R_ki y_i for every k < i in
// parallel, with the next column prefetched into registers while the current one is applied.
// sg and sinv are shared arrays of at least mm entries.  mm <= kBsThreads * kBsPer.
constexpr int kBsThreads = 256;
constexpr int kBsPer = 4;
__device__ __forceinline__ void block_back_substitute(const double2* R, size_t ld, const double2* g, double2* y,
                                                      int mm, double2* sg, double2* sinv, double2* sy) {
  const int tid = threadIdx.x;
  for (int k = tid; k < mm; k += kBsThreads) {
    sg[k] = g[k];
    const double2 d = R[(size_t)k * ld + k];
    const double q = d.x * d.x + d.y * d.y;
    sinv[k] = q > 0.0 ? make_double2(d.x / q, -d.y / q) : make_double2(0.0, 0.0);
  }
  double2 rn[kBsPer];
#pragma unroll
  for (int t = 0; t < kBsPer; ++t) {
    const int k = tid + t * kBsThreads;
    rn[t] = (mm > 0 && k < mm - 1) ? R[(size_t)(mm - 1) * ld + k] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int i = mm - 1; i >= 0; --i) {
    double2 r[kBsPer];
#pragma unroll
    for (int t = 0; t < kBsPer; ++t) {
      r[t] = rn[t];
      const int k = tid + t * kBsThreads;
      rn[t] = (i > 0 && k < i - 1) ? R[(size_t)(i - 1) * ld + k] : make_double2(0.0, 0.0);
    }
    if (tid == 0) {
      *sy = cmul(sg[i], sinv[i]);
      y[i] = *sy;
    }
    __syncthreads();
    const double2 yi = *sy;
#pragma unroll
    for (int t = 0; t < kBsPer; ++t) {
      const int k = tid + t * kBsThreads;
      if (k < i) sg[k] = csub(sg[k], cmul(r[t], yi));
    }
    __syncthreads();
  }
}

}  // namespace bem
