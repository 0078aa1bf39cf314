// Element geometry (step a1), collocation-matrix assembly (steps a3-a5), plane-wave right-hand side
// (step a2) and far field (step a10).
//
// Assembly follows the paper: operators S, D, D*, N of Sec. 3.3 (eqs. stmp-ddtmp) with
// G = (i/4) H0^(1)(k r) (eq. fundamental_sol); constant elements collocated at their centres and
// Gauss-Legendre quadrature off the diagonal, exact self-element integrals on it (Sec. 7 opening
// paragraph); rows placed by the Sec. 6 recipe (eq. calderon_bieb with beta = -alpha, eq.
// 3dom_calderon_bie with gamma = alpha/eps) or one of the comparison forms.
//
// One thread owns one element pair (i, j) and writes its four entries A[i, j], A[i, N+j],
// A[N+i, j], A[N+i, N+j] (pair.cuh); a warp spans 32 consecutive columns, so every store is a coalesced
// 32-entry row segment.  The node geometry and the phase k r are FP64, the rest double-float on the FP32
// pipe; the mixed path stores the double-float entry as complex FP32 (hi) plus its FP32 remainder (lo).
#include <algorithm>
#include <mutex>

#include "internal.cuh"
#include "bessel.cuh"
#include "pair.cuh"

namespace bem {

// The Bessel table of the Taylor branch (bessel.cuh) lives in this translation unit's device memory; it is
// copied in once per device, before the first launch of a kernel that evaluates Hankel functions.
static cudaError_t ensure_bessel_table() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  e = cudaMemcpyToSymbol(g_bessel_tab, bessel_tab_host(), sizeof(BesselTabEntry) * kTabN);
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

namespace {

__global__ void k_elements(ElemDev e, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double dx = e.bx[i] - e.ax[i], dy = e.by[i] - e.ay[i];
  const double h = sqrt(dx * dx + dy * dy);
  e.h[i] = h;
  e.tx[i] = dx / h;
  e.ty[i] = dy / h;
  e.mx[i] = 0.5 * (e.ax[i] + e.bx[i]);
  e.my[i] = 0.5 * (e.ay[i] + e.by[i]);
  const F2 tx = f2_from(dx / h), ty = f2_from(dy / h), hh = f2_from(0.5 * h);
  e.txh[i] = tx.h; e.txl[i] = tx.l;
  e.tyh[i] = ty.h; e.tyl[i] = ty.l;
  e.hhh[i] = hh.h; e.hhl[i] = hh.l;
}

// Mixed store: the double-float entry (hi, lo) is already the complex FP32 rounding of the entry and the
// FP32 rounding of its remainder; the FP64 store adds the two parts.
// lower: the row of the Burton-Miller half of element i is lower + i (n for the whole matrix; the number of
// stored element rows for a compact block).  With Aloout null the remainder is not stored.
template <int MIXED>
__device__ __forceinline__ void store_pair(int n, int i, int j, const C2 (&out)[2][2], void* Aout, void* Aloout,
                                           size_t lda, int lower) {
  const size_t r0 = (size_t)i * lda, r1 = (size_t)(lower + i) * lda;
  const size_t idx[4] = {r0 + j, r0 + n + j, r1 + j, r1 + n + j};
  const C2 v[4] = {out[0][0], out[0][1], out[1][0], out[1][1]};
  if (MIXED) {
    float2* A = static_cast<float2*>(Aout);
    float2* L = static_cast<float2*>(Aloout);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      A[idx[t]] = make_float2(v[t].x.h, v[t].y.h);
      if (L) L[idx[t]] = make_float2(v[t].x.l, v[t].y.l);
    }
  } else {
    double2* A = static_cast<double2*>(Aout);
#pragma unroll
    for (int t = 0; t < 4; ++t) A[idx[t]] = c2_to(v[t]);
  }
}

// Resident CTAs per SM of the assembly and matrix-free kernels: two (128 registers, no spills) measured
// 5.34 ms per launch on the 4096-element star against 5.48 ms with three and 5.52 ms with four (per-pair FP64
// geometry and Bessel arguments); the kernels are latency-bound, so this is a register-versus-occupancy choice.
#ifndef BEM_ASM_CTAS_PER_SM
#define BEM_ASM_CTAS_PER_SM 2
#endif
// Element rows i < rows (rows = n: the whole matrix; fewer: the stored part of a partly recomputed matrix, rows
// i and lower + i).
// ASYM = false: no Bessel argument of the launch reaches Hankel's expansion (decided on the host from the
// geometry's extent and the largest wavenumber), so the reduction of the arguments by pi/2 is left out.
template <int MIXED, bool ASYM>
__global__ void __launch_bounds__(256, BEM_ASM_CTAS_PER_SM) k_assemble(ElemDev e, int n, DomTab dom, Quad q, int form, void* Aout,
                                                   void* Aloout, size_t lda, int rows, int lower) {
  const int j = blockIdx.x * 32 + threadIdx.x;
  const int i = blockIdx.y * 8 + threadIdx.y;
  if (i >= rows || j >= n) return;
  C2 out[2][2];
  assemble_pair_f2<ASYM>(e, dom, q, form, i, j, out);
  store_pair<MIXED>(n, i, j, out, Aout, Aloout, lda, lower);
}

// Matrix-free product y = A x (no stored matrix): each block owns 8 element rows (16 matrix rows i and
// N + i); the 32 lanes of a warp stride over the element columns j, evaluate the four entries of (i, j) with
// the assembly's own code and accumulate; a warp reduction gives the two row sums (FP64 products and sums).
// Resident CTAs per SM as for k_assemble.
template <typename T> __device__ __forceinline__ double2 ld_c(const T* p);
template <> __device__ __forceinline__ double2 ld_c<double2>(const double2* p) { return *p; }
template <> __device__ __forceinline__ double2 ld_c<float2>(const float2* p) {
  const float2 v = *p;
  return make_double2(v.x, v.y);
}
__device__ __forceinline__ void st_c(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void st_c(float2* p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }

// Element rows i0 .. n-1 (all of them for i0 = 0).  ASYM as for k_assemble.
template <typename T, bool ASYM>
__global__ void __launch_bounds__(256, BEM_ASM_CTAS_PER_SM) k_matvec_free(ElemDev e, int n, DomTab dom, Quad q, int form, int i0,
                                                      const T* __restrict__ x, T* __restrict__ y, const int* gate) {
  if (gate && *gate == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = i0 + blockIdx.x * 8 + warp;
  if (i >= n) return;
  double2 up = make_double2(0, 0), lo = make_double2(0, 0);
  for (int j = lane; j < n; j += 32) {
    C2 o2[2][2];
    assemble_pair_f2<ASYM>(e, dom, q, form, i, j, o2);
    const double2 xu = ld_c(x + j), xw = ld_c(x + n + j);
    up = cadd(up, cadd(cmul(c2_to(o2[0][0]), xu), cmul(c2_to(o2[0][1]), xw)));
    lo = cadd(lo, cadd(cmul(c2_to(o2[1][0]), xu), cmul(c2_to(o2[1][1]), xw)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    up.x += __shfl_xor_sync(0xffffffffu, up.x, o);
    up.y += __shfl_xor_sync(0xffffffffu, up.y, o);
    lo.x += __shfl_xor_sync(0xffffffffu, lo.x, o);
    lo.y += __shfl_xor_sync(0xffffffffu, lo.y, o);
  }
  if (lane == 0) {
    st_c(y + i, up);
    st_c(y + n + i, lo);
  }
}

// Many problems in one launch: blockIdx.x walks a list of 32 x TY tiles of all problems (problem found by
// binary search in the tile prefix sums); each problem keeps its own elements, domain table and matrices.
// 16 resident warps per SM (128 registers a thread), as for k_assemble: at 24 warps (85 registers) the pair code
// spills.  ASYM as for k_assemble, for the whole batch.
template <int MIXED, int TY, bool ASYM>
__global__ void __launch_bounds__(32 * TY, 512 / (32 * TY)) k_assemble_batched(const AsmJob* __restrict__ jobs, int njobs,
                                                              const long long* __restrict__ tile_prefix, Quad q,
                                                              int form) {
  const long long t = blockIdx.x;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_prefix[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const AsmJob& jb = jobs[lo];
  const long long local = t - tile_prefix[lo];
  const int tiles_x = (jb.n + 31) / 32;
  const int tx = (int)(local % tiles_x), ty = (int)(local / tiles_x);
  const int j = tx * 32 + threadIdx.x;
  const int i = ty * TY + threadIdx.y;
  if (i >= jb.n || j >= jb.n) return;
  C2 out[2][2];
  assemble_pair_f2<ASYM>(jb.e, jb.dom, q, form, i, j, out);
  store_pair<MIXED>(jb.n, i, j, out, jb.A, jb.Alo, (size_t)2 * jb.n, jb.n);
}

// b[r][half*N + i] for plane wave r (eq. naive_bie right-hand side, placed like the matrix rows).
__global__ void k_rhs_planewave(ElemDev e, int n, DomTab dom, int form, int nrhs, const double* ang, double2* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= n || r >= nrhs) return;
  const double k1 = dom.k[0];
  double st, ct;
  sincos(ang[r], &st, &ct);
  const double ph = k1 * (ct * e.mx[i] + st * e.my[i]);
  double sp, cp;
  sincos(ph, &sp, &cp);
  const double2 uin = make_double2(cp, sp);
  const double dn = ct * (-e.ty[i]) + st * e.tx[i];           // d . n_i
  // alpha q_in = (-i/k1) (i k1 dn) u_in = dn u_in
  const double2 bm_val = make_double2(uin.x * (1.0 + dn), uin.y * (1.0 + dn));
  double2* br = b + (size_t)r * 2 * n;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const RowEq eq = row_eq(form, half, e.P[i], e.M[i], k1);
    double2 v = make_double2(0.0, 0.0);
    if (eq.dom == 0) v = cmul(eq.scale, eq.bm ? bm_val : uin);
    br[half * n + i] = v;
  }
}

// u_inf(theta_a) = e^{i pi/4}/sqrt(8 pi k1) sum_j s_{1,j} sum_q W_q e^{-i k1 xh.y_q} [w_j + i k1 (xh.n_j) u_j]
// One block per (angle, rhs); threads stride over elements; FP64 block reduction.
// Far field in two steps.  The element sums depend on the angle and the element only, so they are formed
// once for all right-hand sides:
//   F[a][j] = s_j (h_j / 2) sum_m w_m exp(-i k1 xh_a . y_m),   G[a][j] = i k1 (xh_a . n_j) F[a][j],
// with s_j = +1 / -1 / 0 as the host is on the element's P side / M side / neither; then
//   u_inf(a) = e^{i pi/4} / sqrt(8 pi k1) sum_j (F[a][j] w_j + G[a][j] u_j)
// for every solution, one CTA per (angle, solution) with a fixed-order reduction.
__global__ void __launch_bounds__(256) k_ff_table(ElemDev e, int n, DomTab dom, Quad q, int nang,
                                                  const double* ang, double2* F, double2* G) {
  const double k1 = dom.k[0];
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)nang * n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / n), j = (int)(t % n);
    const int Pj = e.P[j], Mj = e.M[j];
    const double sg = (Pj == 0) ? 1.0 : ((Mj == 0) ? -1.0 : 0.0);
    double2 f = make_double2(0.0, 0.0), g = make_double2(0.0, 0.0);
    if (sg != 0.0) {
      double st, ct;
      sincos(ang[a], &st, &ct);
      const double tx = e.tx[j], ty = e.ty[j], hh = 0.5 * e.h[j];
      const double mx = e.mx[j], my = e.my[j];
      for (int m = 0; m < q.Q; ++m) {
        const double sq = hh * q.t[m];
        const double ph = -k1 * (ct * (mx + sq * tx) + st * (my + sq * ty));
        double sp, cp;
        sincos(ph, &sp, &cp);
        f.x += hh * q.w[m] * cp;
        f.y += hh * q.w[m] * sp;
      }
      f = cscale(f, sg);
      const double xn = ct * (-ty) + st * tx;   // xh . n_j
      g = make_double2(-k1 * xn * f.y, k1 * xn * f.x);
    }
    F[t] = f;
    G[t] = g;
  }
}

__global__ void __launch_bounds__(256) k_ff_apply(int n, int nang, const double2* __restrict__ F,
                                                  const double2* __restrict__ G, const double2* __restrict__ x,
                                                  double k1, double2* __restrict__ out) {
  const int a = blockIdx.x, r = blockIdx.y;
  const double2* xr = x + (size_t)r * 2 * n;
  const double2* Fa = F + (size_t)a * n;
  const double2* Ga = G + (size_t)a * n;
  double2 acc = make_double2(0.0, 0.0);
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    acc = cadd(acc, cadd(cmul(Fa[j], xr[n + j]), cmul(Ga[j], xr[j])));
  __shared__ double2 red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double c = 1.0 / sqrt(8.0 * kPi * k1);
    const double2 ph = make_double2(c * kInvSqrt2, c * kInvSqrt2);   // e^{i pi/4} / sqrt(8 pi k1)
    out[(size_t)r * nang + a] = cmul(ph, red[0]);
  }
}

// Field at points (Green's representation in the domain containing each point):
//   u(x) = [u_in(x) for the host] + sum_j sigma_{d,j} sum_q W_q [ eps_d G_d(x - y_q) w_j - dG_d/dn(y_q) u_j ]
// One warp per (point, right-hand side); lanes stride over elements; FP64 with the assembly's Hankel code.
__global__ void __launch_bounds__(256) k_near_field(ElemDev e, int n, DomTab dom, Quad q, int nrhs, const double2* x,
                                                    int npts, const double* pts, const int* pdom,
                                                    const double* angles, double2* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pt = blockIdx.x * 8 + warp;
  const int r = blockIdx.y;
  if (pt >= npts || r >= nrhs) return;
  const double px = pts[2 * pt], py = pts[2 * pt + 1];
  const int d = pdom[pt];
  const double k = dom.k[d], eps = dom.eps[d];
  const double2* xr = x + (size_t)r * 2 * n;
  double2 acc = make_double2(0, 0);
  for (int j = lane; j < n; j += 32) {
    const int Pj = e.P[j], Mj = e.M[j];
    const double sg = (Pj == d) ? 1.0 : ((Mj == d) ? -1.0 : 0.0);
    if (sg == 0.0) continue;
    const double tx = e.tx[j], ty = e.ty[j], hh = 0.5 * e.h[j], mx = e.mx[j], my = e.my[j];
    const double nxj = -ty, nyj = tx;
    double2 sS = make_double2(0, 0), sD = make_double2(0, 0);
    for (int m = 0; m < q.Q; ++m) {
      const double sq = hh * q.t[m], W = hh * q.w[m];
      const double zx = px - (mx + sq * tx), zy = py - (my + sq * ty);
      const double r2 = zx * zx + zy * zy;
      const double ir = rsqrt(r2);
      const double rr = r2 * ir;
      const double cj = (zx * nxj + zy * nyj) * ir;
      Bessel01 b;
      bessel01(k * rr, b);
      sS.x += W * b.j0; sS.y += W * b.y0;
      sD.x += W * cj * b.j1; sD.y += W * cj * b.y1;
    }
    // G = (i/4) H0 -> (i/4) sS ; dG/dn(y) = (ik/4) H1 (zh . n_y) -> (ik/4) sD
    const double2 S = make_double2(-0.25 * sS.y, 0.25 * sS.x);
    const double2 D = make_double2(-0.25 * k * sD.y, 0.25 * k * sD.x);
    const double2 u = xr[j], w = xr[n + j];
    const double2 t = csub(cscale(cmul(S, w), eps), cmul(D, u));
    acc.x += sg * t.x;
    acc.y += sg * t.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) {
    if (d == 0 && angles) {
      double st, ct;
      sincos(angles[r], &st, &ct);
      double sp, cp;
      sincos(dom.k[0] * (ct * px + st * py), &sp, &cp);
      acc.x += cp;
      acc.y += sp;
    }
    out[(size_t)r * npts + pt] = acc;
  }
}

__global__ void k_matrix_to_c64(const void* A, const void* Alo, int mixed, int which, size_t nn, double2* out) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x) {
    if (!mixed) {
      out[t] = static_cast<const double2*>(A)[t];
    } else {
      const float2 h = static_cast<const float2*>(A)[t];
      double2 v = make_double2(h.x, h.y);
      if (which == 1) {
        const float2 l = static_cast<const float2*>(Alo)[t];
        v.x += (double)l.x; v.y += (double)l.y;
      }
      out[t] = v;
    }
  }
}

}  // namespace

cudaError_t launch_elements(const ElemDev& e, int n, cudaStream_t s) {
  k_elements<<<(n + 255) / 256, 256, 0, s>>>(e, n);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const ElemDev& e, int n, const DomTab& dom, const Quad& q, int form, int store_mixed,
                            void* A, void* Alo, size_t lda, cudaStream_t s, bool asym) {
  if (const cudaError_t te = ensure_bessel_table(); te != cudaSuccess) return te;
  dim3 blk(32, 8);
  dim3 grd((n + 31) / 32, (n + 7) / 8);
  if (!store_mixed) k_assemble<0, true><<<grd, blk, 0, s>>>(e, n, dom, q, form, A, Alo, lda, n, n);
  else if (asym) k_assemble<1, true><<<grd, blk, 0, s>>>(e, n, dom, q, form, A, Alo, lda, n, n);
  else k_assemble<1, false><<<grd, blk, 0, s>>>(e, n, dom, q, form, A, Alo, lda, n, n);
  return cudaGetLastError();
}

cudaError_t launch_assemble_rows(const ElemDev& e, int n, const DomTab& dom, const Quad& q, int form, int rows,
                                 float2* H, size_t lda, cudaStream_t s, bool asym) {
  if (rows <= 0) return cudaSuccess;
  if (rows > n) return cudaErrorInvalidValue;
  if (const cudaError_t te = ensure_bessel_table(); te != cudaSuccess) return te;
  dim3 blk(32, 8);
  dim3 grd((n + 31) / 32, (rows + 7) / 8);
  if (asym) k_assemble<1, true><<<grd, blk, 0, s>>>(e, n, dom, q, form, H, nullptr, lda, rows, rows);
  else k_assemble<1, false><<<grd, blk, 0, s>>>(e, n, dom, q, form, H, nullptr, lda, rows, rows);
  return cudaGetLastError();
}

cudaError_t launch_matvec_free(const ElemDev& e, int n, const DomTab& dom, const Quad& q, int form, int nrhs,
                               const double2* x, double2* y, cudaStream_t s, const int* gate, bool asym) {
  if (const cudaError_t te = ensure_bessel_table(); te != cudaSuccess) return te;
  for (int r = 0; r < nrhs; ++r) {
    const double2* xr = x + (size_t)r * 2 * n;
    double2* yr = y + (size_t)r * 2 * n;
    if (asym) k_matvec_free<double2, true><<<(n + 7) / 8, 256, 0, s>>>(e, n, dom, q, form, 0, xr, yr, gate);
    else k_matvec_free<double2, false><<<(n + 7) / 8, 256, 0, s>>>(e, n, dom, q, form, 0, xr, yr, gate);
  }
  return cudaGetLastError();
}

cudaError_t launch_matvec_free_f32(const ElemDev& e, int n, const DomTab& dom, const Quad& q, int form, int i0,
                                   const float2* x, float2* y, cudaStream_t s, const int* gate, bool asym) {
  if (i0 >= n) return cudaSuccess;
  if (i0 < 0) return cudaErrorInvalidValue;
  if (const cudaError_t te = ensure_bessel_table(); te != cudaSuccess) return te;
  if (asym) k_matvec_free<float2, true><<<(n - i0 + 7) / 8, 256, 0, s>>>(e, n, dom, q, form, i0, x, y, gate);
  else k_matvec_free<float2, false><<<(n - i0 + 7) / 8, 256, 0, s>>>(e, n, dom, q, form, i0, x, y, gate);
  return cudaGetLastError();
}

long long assemble_batched_tiles(int n, int ty) { return (long long)((n + 31) / 32) * ((n + ty - 1) / ty); }

cudaError_t launch_assemble_batched(const AsmJob* jobs_dev, int njobs, const long long* tile_prefix_dev,
                                   long long total_tiles, const Quad& q, int form, int store_mixed, int ty,
                                   cudaStream_t s, bool asym) {
  if (total_tiles <= 0) return cudaSuccess;
  if (total_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (!store_mixed) return cudaErrorNotSupported;   // the batch engine stores the mixed form only
  if (const cudaError_t te = ensure_bessel_table(); te != cudaSuccess) return te;
  const unsigned grid = (unsigned)total_tiles;
#define BEM_ASM_CASE(TYV)                                                                                  \
  case TYV:                                                                                                \
    if (asym) k_assemble_batched<1, TYV, true><<<grid, dim3(32, TYV), 0, s>>>(jobs_dev, njobs, tile_prefix_dev, q, form); \
    else k_assemble_batched<1, TYV, false><<<grid, dim3(32, TYV), 0, s>>>(jobs_dev, njobs, tile_prefix_dev, q, form); \
    break;
  switch (ty) {
    BEM_ASM_CASE(4)
    BEM_ASM_CASE(8)
    BEM_ASM_CASE(16)
    default: return cudaErrorInvalidValue;
  }
#undef BEM_ASM_CASE
  return cudaGetLastError();
}

cudaError_t launch_rhs_planewave(const ElemDev& e, int n, const DomTab& dom, int form, int nrhs,
                                 const double* angles_dev, double2* b, cudaStream_t s) {
  dim3 grd((n + 127) / 128, nrhs);
  k_rhs_planewave<<<grd, 128, 0, s>>>(e, n, dom, form, nrhs, angles_dev, b);
  return cudaGetLastError();
}

cudaError_t launch_far_field(const ElemDev& e, int n, const DomTab& dom, const Quad& q, int nrhs, const double2* x,
                             int nang, const double* ang_dev, double2* out, double2* scratch, cudaStream_t s) {
  double2* F = scratch;
  double2* G = scratch + (size_t)nang * n;
  const size_t cnt = (size_t)nang * n;
  const int blocks = (int)std::min<size_t>((cnt + 255) / 256, 4096);
  k_ff_table<<<blocks, 256, 0, s>>>(e, n, dom, q, nang, ang_dev, F, G);
  k_ff_apply<<<dim3(nang, nrhs), 256, 0, s>>>(n, nang, F, G, x, dom.k[0], out);
  return cudaGetLastError();
}

cudaError_t launch_near_field(const ElemDev& e, int n, const DomTab& dom, const Quad& q, int nrhs, const double2* x,
                              int npts, const double* pts_dev, const int* dom_dev, const double* angles_dev,
                              double2* out, cudaStream_t s) {
  dim3 grd((npts + 7) / 8, nrhs);
  k_near_field<<<grd, 256, 0, s>>>(e, n, dom, q, nrhs, x, npts, pts_dev, dom_dev, angles_dev, out);
  return cudaGetLastError();
}

cudaError_t launch_matrix_to_c64(const void* A, const void* Alo, int mixed, int which, size_t nn, double2* out,
                                 cudaStream_t s) {
  k_matrix_to_c64<<<1024, 256, 0, s>>>(A, Alo, mixed, which, nn, out);
  return cudaGetLastError();
}

}  // namespace bem
