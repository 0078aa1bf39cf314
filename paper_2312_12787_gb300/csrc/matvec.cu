// Dense complex matrix-vector and matrix-block products of the GMRES solve (steps a6, a9, a11).
//
// A is the 2N x 2N collocation matrix, row-major.  Right-hand-side blocks are stored column after
// column (column s of X at X + s*n), so both A and X are contiguous along the summation index.
//
//  * k_gemv_f64   - y = A x, one warp per row, FP64 arithmetic (FP64 path; on GB300 the FP64 pipe,
//                   not HBM, bounds it); with RESID it forms the FP64 path's residual b - A x.
//  * k_gemv_c32   - y = A x with complex FP32 storage and products (mixed inner solve): each lane streams
//                   16-byte float4 loads (two complex entries), so a warp moves 512 contiguous bytes per
//                   step; partial sums are folded into FP64 every 16 steps.  HBM-bound.
//  * k_gemm_f64   - Y = A X for several columns, SIMT tile 64 rows x 64 columns, FP64 arithmetic.
//  * k_gemm_c32   - the same in complex FP32 with two-level FP32 accumulation.
//  * k_resid_df_* - refinement residual b - (hi + lo) x in double-float arithmetic (see below).
#include <algorithm>
#include <atomic>

#include "internal.cuh"

namespace bem {

namespace {

struct LoadC64 {
  const double2* A;
  __device__ __forceinline__ double2 operator()(size_t idx) const { return __ldg(A + idx); }
};

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// y[s][r] = (RESID ? b[s][r] - : ) sum_c A[r][c] x[s][c]; grid.y = s
template <class ALoad, bool RESID>
__global__ void __launch_bounds__(256) k_gemv_f64(ALoad A, size_t lda, int n, const double2* x, const double2* b,
                                                   double2* y, const int* gate) {
  if (gate && *gate == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * 8 + warp;
  const int s = blockIdx.y;
  if (r >= n) return;
  const double2* xs = x + (size_t)s * n;
  const size_t row = (size_t)r * lda;
  double2 acc0 = make_double2(0, 0), acc1 = make_double2(0, 0);
  int c = lane;
  for (; c + 32 < n; c += 64) {
    const double2 a0 = A(row + c), a1 = A(row + c + 32);
    const double2 x0 = __ldg(xs + c), x1 = __ldg(xs + c + 32);
    acc0.x = fma(a0.x, x0.x, fma(-a0.y, x0.y, acc0.x));
    acc0.y = fma(a0.x, x0.y, fma(a0.y, x0.x, acc0.y));
    acc1.x = fma(a1.x, x1.x, fma(-a1.y, x1.y, acc1.x));
    acc1.y = fma(a1.x, x1.y, fma(a1.y, x1.x, acc1.y));
  }
  for (; c < n; c += 32) {
    const double2 a0 = A(row + c);
    const double2 x0 = __ldg(xs + c);
    acc0.x = fma(a0.x, x0.x, fma(-a0.y, x0.y, acc0.x));
    acc0.y = fma(a0.x, x0.y, fma(a0.y, x0.x, acc0.y));
  }
  double2 acc = warp_sum(cadd(acc0, acc1));
  if (lane == 0) {
    if (RESID) {
      const double2 bb = b[(size_t)s * n + r];
      acc = csub(bb, acc);
    }
    y[(size_t)s * n + r] = acc;
  }
}

// complex FP32, up to NR right-hand sides per read of A.  One CTA per row at a time: its 256 threads split
// the row into 16-byte pieces (two complex entries, columns 2c and 2c+1 for c = tid, tid + 256, ...), so a
// row is 4 KB per step and a CTA finishes a row quickly.  CTAs stride over the rows (the grid fills every SM
// exactly once), which leaves no partial second wave: with one warp per row, the 8192 rows of a 0.5 GB
// matrix needed 1.12 waves and the tail cost a third of the bandwidth.  Products are FP32, folded into
// FP64 every 16 steps; the warp sums go to shared memory and are combined in a fixed order (deterministic)
// once per group of kGvGroup rows.  n must be even (it is: n = 2N); inactive columns are skipped.
constexpr int kGvGroup = 16;
// rows (<= n) rows of A from A onwards, written to y at rows yoff .. yoff + rows - 1 (the whole matrix: rows = n,
// yoff = 0; a stored part of a partly recomputed matrix otherwise).
template <int NR>
__global__ void __launch_bounds__(256) k_gemv_c32(const float2* __restrict__ A, size_t lda, int n, int rows, int yoff,
                                                   const float2* __restrict__ x, float2* __restrict__ y,
                                                   const int* __restrict__ active) {
  __shared__ double2 part[kGvGroup][8][NR];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  bool act[NR];
  bool any = false;
#pragma unroll
  for (int s = 0; s < NR; ++s) {
    act[s] = !active || active[s];
    any = any || act[s];
  }
  if (!any) return;
  const int n2 = n >> 1;   // float4 per row
  const int G = gridDim.x;
  for (int base = blockIdx.x; base < rows; base += kGvGroup * G) {
    int k = 0;
    for (; k < kGvGroup && base + k * G < rows; ++k) {
      const int r = base + k * G;
      const float4* row = reinterpret_cast<const float4*>(A + (size_t)r * lda);
      double ax[NR], ay[NR];
#pragma unroll
      for (int s = 0; s < NR; ++s) ax[s] = ay[s] = 0.0;
      int c = tid;
      while (c < n2) {
        float px[NR], py[NR];
#pragma unroll
        for (int s = 0; s < NR; ++s) px[s] = py[s] = 0.f;
#pragma unroll 4
        for (int t = 0; t < 16 && c < n2; ++t, c += 256) {
          const float4 a = __ldcs(row + c);
#pragma unroll
          for (int s = 0; s < NR; ++s) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(x + (size_t)s * n) + c);
            px[s] = fmaf(a.x, v.x, px[s]); px[s] = fmaf(-a.y, v.y, px[s]);
            py[s] = fmaf(a.x, v.y, py[s]); py[s] = fmaf(a.y, v.x, py[s]);
            px[s] = fmaf(a.z, v.z, px[s]); px[s] = fmaf(-a.w, v.w, px[s]);
            py[s] = fmaf(a.z, v.w, py[s]); py[s] = fmaf(a.w, v.z, py[s]);
          }
        }
#pragma unroll
        for (int s = 0; s < NR; ++s) {
          ax[s] += (double)px[s];
          ay[s] += (double)py[s];
        }
      }
#pragma unroll
      for (int s = 0; s < NR; ++s) {
        const double2 w = warp_sum(make_double2(ax[s], ay[s]));
        if (lane == 0) part[k][warp][s] = w;
      }
    }
    __syncthreads();
    if (tid < k * NR) {
      const int kk = tid / NR, s = tid % NR;
      if (act[s]) {
        double2 acc = part[kk][0][s];
#pragma unroll
        for (int w = 1; w < 8; ++w) acc = cadd(acc, part[kk][w][s]);
        y[(size_t)s * n + yoff + base + kk * G] = make_float2((float)acc.x, (float)acc.y);
      }
    }
    __syncthreads();
  }
}

// SIMT tiled GEMM, FP64: Y[s][r] = sum_c A[r][c] X[s][c].  Tile 64 rows x 64 columns x 8, 256 threads,
// each thread 4 rows x 4 columns (rows ty + 16 i, columns tx + 16 j).
template <class ALoad, bool RESID>
__global__ void __launch_bounds__(256) k_gemm_f64(ALoad A, size_t lda, int n, int nrhs, const double2* X,
                                                   const double2* B, double2* Y, const int* gate) {
  if (gate && *gate == 0) return;
  constexpr int BR = 64, BS = 64, BK = 8;
  __shared__ double2 As[BK][BR + 1];
  __shared__ double2 Xs[BK][BS + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.x * BR, s0 = blockIdx.y * BS;
  double2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_double2(0, 0);
  for (int k0 = 0; k0 < n; k0 += BK) {
    // 512 A values and 512 X values per tile, two each per thread
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int e = tid + t * 256;
      const int rr = e >> 3, kk = e & 7;
      const int gr = r0 + rr, gk = k0 + kk;
      As[kk][rr] = (gr < n && gk < n) ? A((size_t)gr * lda + gk) : make_double2(0, 0);
      const int gs = s0 + rr;
      Xs[kk][rr] = (gs < nrhs && gk < n) ? X[(size_t)gs * n + gk] : make_double2(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double2 av[4], xv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) xv[b] = Xs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc[a][b].x = fma(av[a].x, xv[b].x, fma(-av[a].y, xv[b].y, acc[a][b].x));
          acc[a][b].y = fma(av[a].x, xv[b].y, fma(av[a].y, xv[b].x, acc[a][b].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gr = r0 + ty + 16 * a, gs = s0 + tx + 16 * b;
      if (gr < n && gs < nrhs) {
        double2 v = acc[a][b];
        if (RESID) v = csub(B[(size_t)gs * n + gr], v);
        Y[(size_t)gs * n + gr] = v;
      }
    }
}

// SIMT tiled GEMM in complex FP32, same tiling; the inner FP32 accumulator is folded into a second FP32
// accumulator every 64 columns to keep the summation error near FP32 rounding of short sums.
__global__ void __launch_bounds__(256) k_gemm_c32(const float2* __restrict__ A, size_t lda, int n, int nrhs,
                                                   const float2* __restrict__ X, float2* __restrict__ Y,
                                                   const int* gate) {
  if (gate && *gate == 0) return;
  constexpr int BR = 64, BS = 64, BK = 8;
  __shared__ float2 As[BK][BR + 1];
  __shared__ float2 Xs[BK][BS + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.x * BR, s0 = blockIdx.y * BS;
  float2 acc[4][4], tot[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b] = make_float2(0, 0); tot[a][b] = make_float2(0, 0); }
  int tiles = 0;
  for (int k0 = 0; k0 < n; k0 += BK) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int e = tid + t * 256;
      const int rr = e >> 3, kk = e & 7;
      const int gr = r0 + rr, gk = k0 + kk;
      As[kk][rr] = (gr < n && gk < n) ? A[(size_t)gr * lda + gk] : make_float2(0, 0);
      const int gs = s0 + rr;
      Xs[kk][rr] = (gs < nrhs && gk < n) ? X[(size_t)gs * n + gk] : make_float2(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 av[4], xv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) xv[b] = Xs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc[a][b].x = fmaf(av[a].x, xv[b].x, fmaf(-av[a].y, xv[b].y, acc[a][b].x));
          acc[a][b].y = fmaf(av[a].x, xv[b].y, fmaf(av[a].y, xv[b].x, acc[a][b].y));
        }
    }
    __syncthreads();
    if (++tiles == 8) {
      tiles = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          tot[a][b].x += acc[a][b].x; tot[a][b].y += acc[a][b].y;
          acc[a][b] = make_float2(0, 0);
        }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gr = r0 + ty + 16 * a, gs = s0 + tx + 16 * b;
      if (gr < n && gs < nrhs)
        Y[(size_t)gs * n + gr] = make_float2(tot[a][b].x + acc[a][b].x, tot[a][b].y + acc[a][b].y);
    }
}

__global__ void k_c64_to_c32(const double2* in, float2* out, size_t count) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x)
    out[t] = make_float2((float)in[t].x, (float)in[t].y);
}
__global__ void k_c32_to_c64(const float2* in, double2* out, size_t count) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x)
    out[t] = make_double2(in[t].x, in[t].y);
}
// one block per column, FP64 sum of squares
__global__ void __launch_bounds__(256) k_column_norms(const double2* v, int n, double* out) {
  __shared__ double red[8];
  const double2* vs = v + (size_t)blockIdx.x * n;
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) acc += vs[k].x * vs[k].x + vs[k].y * vs[k].y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    out[blockIdx.x] = sqrt(t);
  }
}

// ---- refinement residual r = b - (hi + lo) x in double-float arithmetic on the FP32 pipes ----------
// x (FP64) is first split into x_hi + x_lo (FP32).  The leading products hi * x_hi are formed exactly
// (p = a b, e = fma(a, b, -p)) and summed with error-free two-sum steps into a running sum s and a
// compensation c (the accurate dot-product scheme of Ogita, Rump and Oishi; the one-column kernel) or with
// an offset accumulator (the tiled kernel, below); the small terms hi * x_lo + lo * x_hi join c directly.
// The result s + c carries about twice FP32 precision, enough for the residual of the FP64 refinement, at
// FP32-pipe speed instead of GB300's scarce FP64 rate.

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  const float t = a + b;
  const float bp = t - a;
  e = (a - (t - bp)) + (b - bp);
  s = t;
}

__device__ __forceinline__ void dot2_acc(float a, float b, float& s, float& c) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  const float t = s + p;
  const float bp = t - s;
  c += ((s - (t - bp)) + (p - bp)) + e;
  s = t;
}

__global__ void k_split_x(const double2* __restrict__ x, float2* __restrict__ xh, float2* __restrict__ xl,
                          size_t count) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) {
    const double2 v = x[t];
    const float hx = (float)v.x, hy = (float)v.y;
    xh[t] = make_float2(hx, hy);
    xl[t] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
  }
}

// one complex multiply-accumulate y += (ah + al)(xh + xl) into (sr, cr), (si, ci)
__device__ __forceinline__ void cmac_df(float2 ah, float2 al, float2 xh, float2 xl, float& sr, float& cr, float& si,
                                        float& ci) {
  dot2_acc(ah.x, xh.x, sr, cr);
  dot2_acc(-ah.y, xh.y, sr, cr);
  dot2_acc(ah.x, xh.y, si, ci);
  dot2_acc(ah.y, xh.x, si, ci);
  cr = fmaf(ah.x, xl.x, cr); cr = fmaf(-ah.y, xl.y, cr); cr = fmaf(al.x, xh.x, cr); cr = fmaf(-al.y, xh.y, cr);
  ci = fmaf(ah.x, xl.y, ci); ci = fmaf(ah.y, xl.x, ci); ci = fmaf(al.x, xh.y, ci); ci = fmaf(al.y, xh.x, ci);
}

// r[s][row] = b[s][row] - sum_c (hi + lo)[row][c] x[s][c]; one warp per row, grid.y = column.
__global__ void __launch_bounds__(256) k_resid_df_gemv(const float2* __restrict__ Ah, const float2* __restrict__ Al,
                                                        size_t lda, int n, const float2* __restrict__ xh,
                                                        const float2* __restrict__ xl, const double2* __restrict__ b,
                                                        double2* __restrict__ r) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + warp;
  const int s = blockIdx.y;
  if (row >= n) return;
  const float2* ah = Ah + (size_t)row * lda;
  const float2* al = Al + (size_t)row * lda;
  const float2* vh = xh + (size_t)s * n;
  const float2* vl = xl + (size_t)s * n;
  float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
#pragma unroll 4
  for (int c = lane; c < n; c += 32) cmac_df(__ldcs(ah + c), __ldcs(al + c), __ldg(vh + c), __ldg(vl + c), sr, cr, si, ci);
  double re = (double)sr + (double)cr, im = (double)si + (double)ci;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    const double2 bb = b[(size_t)s * n + row];
    r[(size_t)s * n + row] = make_double2(bb.x - re, bb.y - im);
  }
}

// Tiled version for many columns: tile 32 rows x 64 columns x 16, 256 threads, each 2 rows x 4 columns.
// K may be split over blockIdx.z in ranges of kchunk columns: then each CTA writes its partial product
// (rounded to FP64) to part[z][s][row] and k_resid_combine forms r; with part == nullptr the CTA covers all
// of K and writes r directly.
//
// The leading products hi * x_hi are summed with an offset accumulator instead of two-sum steps.  For a run
// of kResSub columns, let M bound every |hi_re/im| * |x_hi re/im| of the run (from the run's maxima) and
// let sigma be a power of two with sigma >= 64 M.  The accumulator starts at sigma; each product enters as
//     t = fma(a, b, acc),  d = t - acc,  c += fma(a, b, -d),  acc = t.
// acc stays within sigma +- 17 M, so t and acc lie within a factor two of each other and d is exact
// (Sterbenz); d + (a b - d) is the exact product, and fma(a, b, -d) rounds a quantity below ulp(sigma).  At
// the end of the run acc - sigma (again exact) joins a double-float total (S, L) by one two-sum step, and
// c joins L.  Four FP32 operations per product instead of ten; the price is that the rounding of c is
// relative to sigma instead of the running sum, a few times the error of the two-sum scheme and far below
// what the refinement needs.
constexpr int kResBR = 32, kResBS = 64, kResBK = 16, kResSub = 8, kResMargin = 6;
static_assert(kResBK % kResSub == 0 && kResSub == 8, "the maxima of a run are reduced over 8 lanes");
static_assert((1 << kResMargin) >= 2 * (2 * kResSub + 1) + 2, "offset too small for exact differences");

// max(|v.x|, |v.y|) over the 8 lanes that hold one run of one row (or column) of the staged tile
__device__ __forceinline__ float run_max8(float2 v) {
  float m = fmaxf(fabsf(v.x), fabsf(v.y));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
  return m;
}

// power of two sigma >= 2^kResMargin * M (M < 2^e  ->  sigma = 2^(e + kResMargin)), capped at 2^127
__device__ __forceinline__ float offset_of(float m) {
  const unsigned e = __float_as_uint(m) & 0x7f800000u;
  return __uint_as_float(min(e + ((unsigned)(kResMargin + 1) << 23), 0x7f000000u));
}

__device__ __forceinline__ void offset_acc(float a, float b, float& acc, float& c) {
  const float t = fmaf(a, b, acc);
  const float d = t - acc;
  c += fmaf(a, b, -d);
  acc = t;
}

//
// kCross = false: the small terms hi * x_lo + lo * x_hi are not formed here; they arrive as the FP32 block
// cross (nrhs x n, a tensor-core product: they carry 2^-24 of the sum, so its FP32 accumulation is ample)
// and join the sum in FP64 (in k_resid_combine when K is split).
template <bool kCross>
__global__ void __launch_bounds__(256) k_resid_df_gemm(const float2* __restrict__ Ah, const float2* __restrict__ Al,
                                                        size_t lda, int n, int nrhs, const float2* __restrict__ xh,
                                                        const float2* __restrict__ xl, const double2* __restrict__ b,
                                                        double2* __restrict__ r, int kchunk,
                                                        double2* __restrict__ part, const float2* __restrict__ cross) {
  constexpr int BR = kResBR, BS = kResBS, BK = kResBK, NSUB = kResBK / kResSub;
  const int kbeg = blockIdx.z * kchunk, kend = min(n, kbeg + kchunk);
  __shared__ float2 Ash[BK][BR + 1], Asl[BK][BR + 1];
  __shared__ float2 Xsh[BK][BS + 1], Xsl[BK][BS + 1];
  __shared__ float Amax[NSUB][BR], Xmax[NSUB][BS];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.x * BR, s0 = blockIdx.y * BS;
  // double-float totals (S, L) of the real and imaginary parts
  float Sr[2][4], Lr[2][4], Si[2][4], Li[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) Sr[a][q] = Lr[a][q] = Si[a][q] = Li[a][q] = 0.f;
  const float2 z = make_float2(0.f, 0.f);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    // A: 32 x 16 = 512 entries (2 per thread); X: 64 x 16 = 1024 entries (4 per thread).  The 16 lanes
    // of a half-warp hold one row (column) of the tile; each run of 8 lanes is one offset run.
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int e = tid + t * 256;
      const int rr = e >> 4, kk = e & 15;
      const int gr = r0 + rr, gk = k0 + kk;
      const bool in = gr < n && gk < kend;
      const float2 vh = in ? __ldcs(Ah + (size_t)gr * lda + gk) : z;
      Ash[kk][rr] = vh;
      if (kCross) Asl[kk][rr] = in ? __ldcs(Al + (size_t)gr * lda + gk) : z;
      const float m = run_max8(vh);
      if ((kk & (kResSub - 1)) == 0) Amax[kk / kResSub][rr] = m;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + t * 256;
      const int ss = e >> 4, kk = e & 15;
      const int gs = s0 + ss, gk = k0 + kk;
      const bool in = gs < nrhs && gk < kend;
      const float2 vh = in ? xh[(size_t)gs * n + gk] : z;
      Xsh[kk][ss] = vh;
      if (kCross) Xsl[kk][ss] = in ? xl[(size_t)gs * n + gk] : z;
      const float m = run_max8(vh);
      if ((kk & (kResSub - 1)) == 0) Xmax[kk / kResSub][ss] = m;
    }
    __syncthreads();
#pragma unroll
    for (int sub = 0; sub < NSUB; ++sub) {
      float sg[2][4], ar[2][4], ai[2][4], cr[2][4], ci[2][4];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          sg[a][q] = offset_of(Amax[sub][ty + 16 * a] * Xmax[sub][tx + 16 * q]);
          ar[a][q] = ai[a][q] = sg[a][q];
          cr[a][q] = ci[a][q] = 0.f;
        }
#pragma unroll 2
      for (int kk = sub * kResSub; kk < (sub + 1) * kResSub; ++kk) {
        float2 ah[2], al[2], vh[4], vl[4];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          ah[a] = Ash[kk][ty + 16 * a];
          if (kCross) al[a] = Asl[kk][ty + 16 * a];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          vh[q] = Xsh[kk][tx + 16 * q];
          if (kCross) vl[q] = Xsl[kk][tx + 16 * q];
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            offset_acc(ah[a].x, vh[q].x, ar[a][q], cr[a][q]);
            offset_acc(-ah[a].y, vh[q].y, ar[a][q], cr[a][q]);
            offset_acc(ah[a].x, vh[q].y, ai[a][q], ci[a][q]);
            offset_acc(ah[a].y, vh[q].x, ai[a][q], ci[a][q]);
            if (kCross) {
              float& c1 = cr[a][q];
              float& c2 = ci[a][q];
              c1 = fmaf(ah[a].x, vl[q].x, c1); c1 = fmaf(-ah[a].y, vl[q].y, c1);
              c1 = fmaf(al[a].x, vh[q].x, c1); c1 = fmaf(-al[a].y, vh[q].y, c1);
              c2 = fmaf(ah[a].x, vl[q].y, c2); c2 = fmaf(ah[a].y, vl[q].x, c2);
              c2 = fmaf(al[a].x, vh[q].y, c2); c2 = fmaf(al[a].y, vh[q].x, c2);
            }
          }
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float e;
          two_sum(Sr[a][q], ar[a][q] - sg[a][q], Sr[a][q], e);
          Lr[a][q] += e + cr[a][q];
          two_sum(Si[a][q], ai[a][q] - sg[a][q], Si[a][q], e);
          Li[a][q] += e + ci[a][q];
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gr = r0 + ty + 16 * a, gs = s0 + tx + 16 * q;
      if (gr < n && gs < nrhs) {
        double2 ax = make_double2((double)Sr[a][q] + (double)Lr[a][q], (double)Si[a][q] + (double)Li[a][q]);
        if (part) {
          part[((size_t)blockIdx.z * nrhs + gs) * n + gr] = ax;
        } else {
          if (!kCross) {
            const float2 cv = cross[(size_t)gs * n + gr];
            ax.x += (double)cv.x;
            ax.y += (double)cv.y;
          }
          const double2 bb = b[(size_t)gs * n + gr];
          r[(size_t)gs * n + gr] = make_double2(bb.x - ax.x, bb.y - ax.y);
        }
      }
    }
}

// r = b - sum over the K splits of the partial products (FP64, in split order) - cross (if given).
__global__ void k_resid_combine(const double2* __restrict__ part, int nsplit, size_t count,
                                const double2* __restrict__ b, double2* __restrict__ r,
                                const float2* __restrict__ cross) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) {
    double ax = 0.0, ay = 0.0;
    for (int z = 0; z < nsplit; ++z) {
      const double2 v = part[(size_t)z * count + t];
      ax += v.x;
      ay += v.y;
    }
    if (cross) {
      ax += (double)cross[t].x;
      ay += (double)cross[t].y;
    }
    const double2 bb = b[t];
    r[t] = make_double2(bb.x - ax, bb.y - ay);
  }
}

__global__ void k_add_c32(float2* __restrict__ a, const float2* __restrict__ b, size_t count) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) {
    const float2 u = a[t], v = b[t];
    a[t] = make_float2(u.x + v.x, u.y + v.y);
  }
}

__global__ void k_sub_c32(double2* r, const float2* y, size_t count) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) {
    const float2 v = y[t];
    r[t] = make_double2(r[t].x - (double)v.x, r[t].y - (double)v.y);
  }
}

__global__ void k_b_minus(const double2* b, double2* r, size_t count) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x)
    r[t] = csub(b[t], r[t]);
}

}  // namespace

// CTAs that fill every SM of the current device once (cached per device and width).
static int gemv_c32_grid(int nrhs) {
  constexpr int kGvMaxDevices = 64;
  static std::atomic<int> cache[kGvMaxDevices][2];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kGvMaxDevices) return 0;
  const int w = nrhs == 1 ? 0 : 1;
  int g = cache[dev][w].load(std::memory_order_relaxed);
  if (g > 0) return g;
  int sms = 0, per = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const cudaError_t e = w == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gemv_c32<1>, 256, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gemv_c32<2>, 256, 0);
  if (e != cudaSuccess || per <= 0) return 0;
  g = sms * per;
  cache[dev][w].store(g, std::memory_order_relaxed);
  return g;
}

cudaError_t launch_axpby_neg(const double2* b, double2* r, size_t count, cudaStream_t s) {
  k_b_minus<<<1024, 256, 0, s>>>(b, r, count);
  return cudaGetLastError();
}

cudaError_t launch_sub_c32(double2* r, const float2* y, size_t count, cudaStream_t s) {
  k_sub_c32<<<1024, 256, 0, s>>>(r, y, count);
  return cudaGetLastError();
}

cudaError_t launch_convert_c64_c32(const double2* in, float2* out, size_t count, cudaStream_t s) {
  k_c64_to_c32<<<1024, 256, 0, s>>>(in, out, count);
  return cudaGetLastError();
}
cudaError_t launch_convert_c32_c64(const float2* in, double2* out, size_t count, cudaStream_t s) {
  k_c32_to_c64<<<1024, 256, 0, s>>>(in, out, count);
  return cudaGetLastError();
}
cudaError_t launch_column_norms(const double2* v, int n, int ncol, double* out, cudaStream_t s) {
  k_column_norms<<<ncol, 256, 0, s>>>(v, n, out);
  return cudaGetLastError();
}

cudaError_t launch_matvec_c64(const double2* A, size_t lda, int n, int nrhs, const double2* x, double2* y,
                              cudaStream_t s, const int* gate) {
  LoadC64 ld{A};
  if (nrhs == 1) {
    dim3 grd((n + 7) / 8, 1);
    k_gemv_f64<LoadC64, false><<<grd, 256, 0, s>>>(ld, lda, n, x, nullptr, y, gate);
  } else {
    dim3 grd((n + 63) / 64, (nrhs + 63) / 64);
    k_gemm_f64<LoadC64, false><<<grd, 256, 0, s>>>(ld, lda, n, nrhs, x, nullptr, y, gate);
  }
  return cudaGetLastError();
}

cudaError_t launch_matvec_c32(const float2* A, size_t lda, int n, int nrhs, const float2* x, float2* y,
                              const int* active, cudaStream_t s, const int* gate) {
  if (nrhs <= 2) {
    const int grd = std::min(n, gemv_c32_grid(nrhs));
    if (grd <= 0) return cudaErrorInvalidValue;
    if (nrhs == 1)
      k_gemv_c32<1><<<grd, 256, 0, s>>>(A, lda, n, n, 0, x, y, active);
    else
      k_gemv_c32<2><<<grd, 256, 0, s>>>(A, lda, n, n, 0, x, y, active);
  } else {
    dim3 grd((n + 63) / 64, (nrhs + 63) / 64);
    k_gemm_c32<<<grd, 256, 0, s>>>(A, lda, n, nrhs, x, y, gate);
  }
  return cudaGetLastError();
}

cudaError_t launch_matvec_c32_rows(const float2* A, size_t lda, int n, int rows, int yoff, int nrhs, const float2* x,
                                   float2* y, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  if (nrhs < 1 || nrhs > 2 || rows > n || yoff < 0 || yoff + rows > n) return cudaErrorInvalidValue;
  const int grd = std::min(rows, gemv_c32_grid(nrhs));
  if (grd <= 0) return cudaErrorInvalidValue;
  if (nrhs == 1) k_gemv_c32<1><<<grd, 256, 0, s>>>(A, lda, n, rows, yoff, x, y, nullptr);
  else k_gemv_c32<2><<<grd, 256, 0, s>>>(A, lda, n, rows, yoff, x, y, nullptr);
  return cudaGetLastError();
}

// Number of K splits for the tiled residual: the CTA count tiles x S should fill whole waves of the SMs
// (tiles alone, e.g. 256 for 8192 unknowns x 64 columns, leave a partial second wave), with at least 512
// columns of K per split and the partials within the workspace.
static int resid_splits(int n, int nrhs, size_t part_room, bool cross_terms) {
  static std::atomic<int> slots_cache[2];
  int slots = slots_cache[cross_terms].load(std::memory_order_relaxed);
  if (slots <= 0) {
    int dev = 0, sms = 0, per = 0;
    const cudaError_t e =
        cross_terms ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_resid_df_gemm<true>, 256, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_resid_df_gemm<false>, 256, 0);
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || e != cudaSuccess ||
        per <= 0)
      return 1;
    slots = sms * per;
    slots_cache[cross_terms].store(slots, std::memory_order_relaxed);
  }
  const long long tiles = (long long)((n + kResBR - 1) / kResBR) * ((nrhs + kResBS - 1) / kResBS);
  int best = 1;
  double best_eff = 0.0;
  for (int S = 1; S <= 32; ++S) {
    if (S > 1 && (n / S < 512 || (size_t)S * nrhs * n * sizeof(double2) > part_room)) break;
    const long long ctas = tiles * S;
    const double eff = (double)ctas / ((double)slots * (double)((ctas + slots - 1) / slots));
    if (eff > best_eff + 1e-3) {
      best_eff = eff;
      best = S;
    }
  }
  return best;
}

cudaError_t launch_residual_split(const float2* Ahi, const float2* Alo, size_t lda, int n, int nrhs,
                                  const double2* x, const double2* b, double2* r, void* ws, cudaStream_t s,
                                  size_t ws_bytes, int* nlaunch) {
  // ws holds x split into two complex FP32 blocks (2 * nrhs * n float2), then the K-split partials
  float2* xh = static_cast<float2*>(ws);
  float2* xl = xh + (size_t)nrhs * n;
  k_split_x<<<512, 256, 0, s>>>(x, xh, xl, (size_t)nrhs * n);
  if (nrhs < 4) {
    dim3 grd((n + 7) / 8, nrhs);
    k_resid_df_gemv<<<grd, 256, 0, s>>>(Ahi, Alo, lda, n, xh, xl, b, r);
    if (nlaunch) *nlaunch = 2;
  } else {
    const size_t xbytes = ((2 * (size_t)nrhs * n * sizeof(float2)) + 255) & ~(size_t)255;
    const int S = ws_bytes > xbytes ? resid_splits(n, nrhs, ws_bytes - xbytes, true) : 1;
    const int kchunk = ((n + S - 1) / S + kResBK - 1) / kResBK * kResBK;
    double2* part = S > 1 ? reinterpret_cast<double2*>(static_cast<char*>(ws) + xbytes) : nullptr;
    dim3 grd((n + kResBR - 1) / kResBR, (nrhs + kResBS - 1) / kResBS, S);
    k_resid_df_gemm<true><<<grd, 256, 0, s>>>(Ahi, Alo, lda, n, nrhs, xh, xl, b, r, S > 1 ? kchunk : n, part, nullptr);
    if (S > 1) k_resid_combine<<<1024, 256, 0, s>>>(part, S, (size_t)nrhs * n, b, r, nullptr);
    if (nlaunch) *nlaunch = S > 1 ? 3 : 2;
  }
  return cudaGetLastError();
}

cudaError_t residual_split_preload() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, k_split_x);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_resid_df_gemv);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_resid_df_gemm<true>);
  return e;
}

size_t residual_tc_ws_bytes(int n, int nrhs) {
  return ((4 * (size_t)nrhs * n * sizeof(float2)) + 255) & ~(size_t)255;
}

cudaError_t launch_residual_split_tc(const float2* Ahi, const float2* Alo, size_t lda, const void* a16,
                                     const void* alo16, int n, int nrhs, const double2* x, const double2* b,
                                     double2* r, void* ws, size_t ws_bytes, void* tcws, size_t tcws_bytes,
                                     cudaStream_t s, int* nlaunch) {
  const size_t xbytes = residual_tc_ws_bytes(n, nrhs);
  if (ws_bytes < xbytes || nrhs < 2) return cudaErrorInvalidValue;
  // ws: x_hi | x_lo | hi x_lo | lo x_hi (each nrhs x n complex FP32), then the K-split partials
  float2* xh = static_cast<float2*>(ws);
  float2* xl = xh + (size_t)nrhs * n;
  float2* c1 = xl + (size_t)nrhs * n;
  float2* c2 = c1 + (size_t)nrhs * n;
  k_split_x<<<512, 256, 0, s>>>(x, xh, xl, (size_t)nrhs * n);
  cudaError_t e = launch_matvec_tc(a16, n, nrhs, xl, c1, tcws, tcws_bytes, s);
  if (e != cudaSuccess) return e;
  e = launch_matvec_tc(alo16, n, nrhs, xh, c2, tcws, tcws_bytes, s);
  if (e != cudaSuccess) return e;
  k_add_c32<<<512, 256, 0, s>>>(c1, c2, (size_t)nrhs * n);
  const int S = resid_splits(n, nrhs, ws_bytes - xbytes, false);
  const int kchunk = ((n + S - 1) / S + kResBK - 1) / kResBK * kResBK;
  double2* part = S > 1 ? reinterpret_cast<double2*>(static_cast<char*>(ws) + xbytes) : nullptr;
  dim3 grd((n + kResBR - 1) / kResBR, (nrhs + kResBS - 1) / kResBS, S);
  k_resid_df_gemm<false><<<grd, 256, 0, s>>>(Ahi, Alo, lda, n, nrhs, xh, xl, b, r, S > 1 ? kchunk : n, part, c1);
  if (S > 1) k_resid_combine<<<1024, 256, 0, s>>>(part, S, (size_t)nrhs * n, b, r, c1);
  // kernels: split, 2 x (column maxima, operand, product, reduction), sum, residual [, combine]
  if (nlaunch) *nlaunch = 11 + (S > 1 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_residual_c64(const double2* A, size_t lda, int n, int nrhs, const double2* x, const double2* b,
                                double2* r, cudaStream_t s) {
  LoadC64 ld{A};
  if (nrhs == 1) {
    dim3 grd((n + 7) / 8, 1);
    k_gemv_f64<LoadC64, true><<<grd, 256, 0, s>>>(ld, lda, n, x, b, r, nullptr);
  } else {
    dim3 grd((n + 63) / 64, (nrhs + 63) / 64);
    k_gemm_f64<LoadC64, true><<<grd, 256, 0, s>>>(ld, lda, n, nrhs, x, b, r, nullptr);
  }
  return cudaGetLastError();
}

}  // namespace bem
