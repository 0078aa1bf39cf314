// GMRES without restart from x0 = 0 for a block of systems that share one matrix (paper Sec. 3.2,
// eqs. preconditioned_krylov_space / unpreconditioned_krylov_space; Sec. 7: no restart).
//
// Arnoldi uses classical Gram-Schmidt, so that each pass is two streaming sweeps over the basis (projections,
// update) instead of j dependent sweeps: twice (CGS2) for an FP64 basis, and for an FP32 basis once plus a
// second pass only for the systems whose vector the first pass shrank below a tenth of its length.  The
// basis may be complex FP64 (FP64 path) or complex FP32 (mixed inner solves); products and warp reductions
// run in the basis precision, the per-chunk partial sums are combined in FP64.  The Hessenberg column, g and
// the residual estimate are FP64; the rotations run in the basis precision.
//
// Where the device allows cooperative launches, everything after the product is one launch per iteration
// (k_arnoldi: both passes, rotations, next basis vector, index advance, with per-system barriers between the
// CTAs of a system).  Otherwise: a vector of n unknowns is cut into chunks (512, 256, 128 or 64 entries, the
// largest that still gives two CTAs per SM over all systems); one CTA owns one chunk of one system (grid =
// chunks x systems).  In the projection kernel the chunk of w is staged in shared memory and each warp owns
// every eighth basis vector; in the update kernel each thread owns a pair of entries over all basis vectors.
// One kernel ends each iteration (norm, next basis vector, rotations, iteration index).  The kernels of an
// iteration read the iteration index from the device and use programmatic dependent launch.
#include <algorithm>
#include <atomic>

#include "givens.cuh"
#include "internal.cuh"
#include "tc_operand.cuh"

namespace bem {

namespace {

constexpr int kThreads = 256;
constexpr int kCh = 64;                        // entries per chunk (one CTA of the projection kernels)

template <typename T> struct Vec;
template <> struct Vec<double2> {
  using acc_t = double;
  __device__ static __forceinline__ double2 load(const double2* p) { return *p; }
  __device__ static __forceinline__ void store(double2* p, double2 v) { *p = v; }
};
template <> struct Vec<float2> {
  using acc_t = float;
  __device__ static __forceinline__ double2 load(const float2* p) {
    const float2 v = *p;
    return make_double2(v.x, v.y);
  }
  __device__ static __forceinline__ void store(float2* p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }
};

template <typename F>
__device__ __forceinline__ F warp_sum(F v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum one double over the block; result valid in thread 0.  `red` holds 8 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (lane < kThreads / 32) ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// squared norms of 256-entry blocks (grid: blocks x columns)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_norm_part(const T* v, int n, double* npart, int nblk) {
  __shared__ double red[8];
  const int c = blockIdx.x, s = blockIdx.y;
  const int k = c * kThreads + threadIdx.x;
  double acc = 0.0;
  if (k < n) {
    const double2 a = Vec<T>::load(v + (size_t)s * n + k);
    acc = a.x * a.x + a.y * a.y;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) npart[(size_t)s * nblk + c] = acc;
}

// Start: beta = ||r0||, g = (beta, 0, ...), active = (beta > 0).
__global__ void k_start_finish(KrylovState st, int nblk) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= st.nrhs) return;
  double t = 0.0;
  for (int c = 0; c < nblk; ++c) t += st.npart[(size_t)s * nblk + c];
  const double beta = sqrt(t);
  st.beta[s] = beta;
  st.g[(size_t)s * (st.m + 1)] = make_double2(beta, 0.0);
  st.active[s] = beta > 0.0 ? 1 : 0;
  st.iters[s] = 0;
  st.resid[s] = beta > 0.0 ? 1.0 : 0.0;
  st.hnext[s] = beta;
  if (beta > 0.0) atomicAdd(st.n_active, 1);   // zeroed by the launcher
  st.relaxed[s] = beta > 0.0 ? 0 : 1;
  if (beta > 0.0) atomicAdd(st.n_unrelaxed, 1);   // zeroed by the launcher
  st.arrive[s] = 0;
  st.reo[s] = 0;
  if (s == 0) {
    *st.jdev = 0;
    *st.arrive_all = 0;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_start_scale(KrylovState st, const double2* r0) {
  const int k = blockIdx.x * kThreads + threadIdx.x, s = blockIdx.y;
  if (!st.active[s] || k >= st.n) return;
  T* v0 = static_cast<T*>(st.V) + (size_t)s * st.n;
  const double2 v = cscale(r0[(size_t)s * st.n + k], 1.0 / st.beta[s]);
  Vec<T>::store(v0 + k, v);
  if (st.b16hi)
    tc_write_b(static_cast<__half*>(st.b16hi), static_cast<__half*>(st.b16lo), st.ldb16, s, k, (float)v.x, (float)v.y);
}

// Two consecutive entries in the basis precision, moved as one 16-byte (float2) or two 16-byte (double2)
// accesses; entry indices are even and n is even, so a pair never straddles the end of a vector.
template <typename T> struct Pair;
template <> struct Pair<float2> {
  __device__ static __forceinline__ void load(const float2* p, float2& a, float2& b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
  }
  __device__ static __forceinline__ void store(float2* p, float2 a, float2 b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  }
};
template <> struct Pair<double2> {
  __device__ static __forceinline__ void load(const double2* p, double2& a, double2& b) { a = p[0]; b = p[1]; }
  __device__ static __forceinline__ void store(double2* p, double2 a, double2 b) { p[0] = a; p[1] = b; }
};

// Loads with an L2 eviction policy (createpolicy / ld.global.L2::cache_hint, PTX ISA 7.4+).
__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

template <typename T> struct PairHint;
template <> struct PairHint<float2> {
  __device__ static __forceinline__ void load(const float2* p, float2& a, float2& b, unsigned long long pol) {
    float4 v;
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
  }
};
template <> struct PairHint<double2> {
  __device__ static __forceinline__ void load(const double2* p, double2& a, double2& b, unsigned long long pol) {
    asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(a.x), "=d"(a.y) : "l"(p), "l"(pol));
    asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(b.x), "=d"(b.y) : "l"(p + 1), "l"(pol));
  }
};

// Partial projections <v_i, w> over one chunk of CH entries: warp w takes basis vectors i = w, w+8, ...;
// lane l holds the pairs k = chunk start + 2 (32 p + l), p < CH/64, so each load instruction of the warp
// moves 512 (FP32) or 1024 (FP64) contiguous bytes.  Products, lane sums and the warp reduction in the basis
// precision; chunk partials are stored for an FP64 sum over chunks.
//
// mode 0: first pass; warp 0 also records the chunk's ||w||^2 (before projection) in st.wpart.
// mode 1: conditional second pass (selective reorthogonalisation, after the norm-drop test of Daniel, Gragg,
//         Kaufman and Stewart).  A system is projected again only if the first pass shrank w below a tenth
//         of its length, ||w_after||^2 < ||w_before||^2 / 100: the cancellation then costs one classical
//         Gram-Schmidt pass in FP32 about a factor 10 of orthogonality, which the inner solves' 1e-5 tolerance
//         no longer absorbs (the textbook 1/sqrt(2) threshold re-projects most steps of smooth problems, for
//         the same iteration counts).  The first pass's update kernel records the decision in st.reo.
// mode 2: unconditional second pass.
template <typename T, int CH>
__global__ void __launch_bounds__(kThreads, sizeof(T) == sizeof(float2) ? 8 : 1)
    k_dots(KrylovState st, int nchunk, int mode) {
  pdl_enter();
  using F = typename Vec<T>::acc_t;
  constexpr int P = CH / 64;
  __shared__ __align__(16) T ws[CH];   // the chunk of w, read by every warp
  const int c = blockIdx.x, s = blockIdx.y;
  if (!st.active[s]) return;
  const int j = *st.jdev;
  if (mode == 1 && !st.reo[s]) return;   // decided by the first pass's update kernel
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t stride = (size_t)st.nrhs * st.n;
  const T* W = static_cast<const T*>(st.W) + (size_t)s * st.n;
  const T* V = static_cast<const T*>(st.V) + (size_t)s * st.n;
  for (int q = threadIdx.x; q < CH / 2; q += kThreads) {
    const int k = c * CH + 2 * q;
    T a, b;
    if (k < st.n) {
      Pair<T>::load(W + k, a, b);
    } else {
      a.x = a.y = b.x = b.y = 0;
    }
    Pair<T>::store(ws + 2 * q, a, b);
  }
  __syncthreads();
  if (mode == 0 && warp == 0) {
    F nw = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      T a, b;
      Pair<T>::load(ws + 2 * (32 * p + lane), a, b);
      nw += (F)a.x * (F)a.x + (F)a.y * (F)a.y + (F)b.x * (F)b.x + (F)b.y * (F)b.y;
    }
    nw = warp_sum(nw);
    if (lane == 0) st.wpart[(size_t)s * nchunk + c] = (double)nw;
  }
  for (int i = warp; i <= j; i += kThreads / 32) {
    const T* vi = V + (size_t)i * stride;
    F px = 0, py = 0;
    constexpr int kU = P >= 8 ? 4 : 2;   // loads in flight per lane within the register budget
#pragma unroll kU
    for (int p = 0; p < P; ++p) {
      const int q = 32 * p + lane;
      const int k = c * CH + 2 * q;
      if (k < st.n) {
        T a, b, w0, w1;
        Pair<T>::load(vi + k, a, b);
        Pair<T>::load(ws + 2 * q, w0, w1);
        px += (F)a.x * (F)w0.x + (F)a.y * (F)w0.y + (F)b.x * (F)w1.x + (F)b.y * (F)w1.y;
        py += (F)a.x * (F)w0.y - (F)a.y * (F)w0.x + (F)b.x * (F)w1.y - (F)b.y * (F)w1.x;
      }
    }
    // the warp reduction in the basis precision too: FP64 adds run at 1/64 of the FP32 rate on GB300
    const F hx = warp_sum(px), hy = warp_sum(py);
    if (lane == 0) st.part[((size_t)s * nchunk + c) * (st.m + 1) + i] = make_double2((double)hx, (double)hy);
  }
}

// h_i = sum over chunks (FP64), one warp per (system, i); accumulate into column j of H (pass 0 sets,
// later passes add).  grid = (ceil((m+1)/8), systems), 8 warps per block.
__global__ void k_dots_reduce(KrylovState st, int nchunk, int pass, int cond) {
  pdl_enter();
  const int s = blockIdx.y;
  if (!st.active[s] || (cond && !st.reo[s])) return;
  const int j = *st.jdev;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i > j) return;
  double hx = 0.0, hy = 0.0;
  for (int c = lane; c < nchunk; c += 32) {
    const double2 v = st.part[((size_t)s * nchunk + c) * (st.m + 1) + i];
    hx += v.x;
    hy += v.y;
  }
  hx = warp_sum(hx);
  hy = warp_sum(hy);
  if (lane == 0) {
    const double2 h = make_double2(hx, hy);
    st.hcol[(size_t)s * (st.m + 1) + i] = h;
    double2* Hj = st.H + ((size_t)s * st.m + j) * (st.m + 1);
    Hj[i] = pass == 0 ? h : cadd(Hj[i], h);
  }
}

// w -= sum_i h_i v_i over one chunk of CH entries: CH/2 threads, each owning one pair of entries and
// running over all i (h staged in shared memory in the basis precision), so no partial sums are combined
// across threads; also writes the chunk's ||w||^2.
constexpr int kHsMax = 1001;
// With fused != 0 every CTA also sums the chunk partials of the projections itself (FP64, chunk order) and
// CTA 0 records them in column j of H (pass 0 sets, later passes add); otherwise k_dots_reduce did that.
template <typename T, int CH>
__global__ void __launch_bounds__(CH / 2, sizeof(T) == sizeof(float2) ? 8 : 1) k_update(KrylovState st, int nchunk, int pass, int fused, int cond) {
  pdl_enter();
  using F = typename Vec<T>::acc_t;
  __shared__ F hs[2 * kHsMax];
  __shared__ double red[CH / 64];
  const int c = blockIdx.x, s = blockIdx.y;
  if (!st.active[s] || (cond && !st.reo[s])) return;   // cond: a conditional pass the system did not need
  const int j = *st.jdev;
  for (int i = threadIdx.x; i <= j; i += CH / 2) {
    double2 h;
    if (fused) {
      h = make_double2(0.0, 0.0);
#pragma unroll 4
      for (int cc = 0; cc < nchunk; ++cc) h = cadd(h, st.part[((size_t)s * nchunk + cc) * (st.m + 1) + i]);
      if (c == 0) {
        st.hcol[(size_t)s * (st.m + 1) + i] = h;
        double2* Hj = st.H + ((size_t)s * st.m + j) * (st.m + 1);
        Hj[i] = pass == 0 ? h : cadd(Hj[i], h);
      }
    } else {
      h = st.hcol[(size_t)s * (st.m + 1) + i];
    }
    hs[2 * i] = (F)h.x;
    hs[2 * i + 1] = (F)h.y;
  }
  __syncthreads();
  const int k = c * CH + 2 * threadIdx.x;
  const size_t stride = (size_t)st.nrhs * st.n;
  F nrm_f = 0;
  if (k < st.n) {
    const T* V = static_cast<const T*>(st.V) + (size_t)s * st.n + k;
    F ax = 0, ay = 0, bx = 0, by = 0;
#pragma unroll 8
    for (int i = 0; i <= j; ++i) {
      T a, b;
      Pair<T>::load(V + (size_t)i * stride, a, b);
      const F hx = hs[2 * i], hy = hs[2 * i + 1];
      ax += hx * (F)a.x - hy * (F)a.y;
      ay += hx * (F)a.y + hy * (F)a.x;
      bx += hx * (F)b.x - hy * (F)b.y;
      by += hx * (F)b.y + hy * (F)b.x;
    }
    T* W = static_cast<T*>(st.W) + (size_t)s * st.n + k;
    T w0, w1;
    Pair<T>::load(W, w0, w1);
    w0.x -= ax; w0.y -= ay;
    w1.x -= bx; w1.y -= by;
    Pair<T>::store(W, w0, w1);
    nrm_f = w0.x * w0.x + w0.y * w0.y + w1.x * w1.x + w1.y * w1.y;
  }
  nrm_f = warp_sum(nrm_f);   // basis precision within the warp, FP64 across warps and chunks
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)nrm_f;
  __syncthreads();
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < CH / 64; ++q) t += red[q];
    st.npart[(size_t)s * nchunk + c] = t;
    if (pass == 0) {
      // the last CTA of the system to finish takes the reorthogonalisation decision for the conditional pass
      // (norm-drop test, see k_dots) from all chunk sums, so that the conditional kernels only read a flag
      __threadfence();
      s_last = atomicAdd(st.arrive + s, 1) == nchunk - 1;
    }
  }
  if (pass != 0) return;
  __syncthreads();
  if (!s_last || threadIdx.x >= 32) return;
  __threadfence();
  // one warp loads the chunk sums in parallel (L2, bypassing L1) and reduces them
  double before = 0.0, after = 0.0;
  for (int cc = threadIdx.x; cc < nchunk; cc += 32) {
    before += __ldcg(st.wpart + (size_t)s * nchunk + cc);
    after += __ldcg(st.npart + (size_t)s * nchunk + cc);
  }
  before = warp_sum(before);
  after = warp_sum(after);
  if (threadIdx.x == 0) {
    st.reo[s] = st.strict[s] || after < 0.01 * before;   // ||w_after|| < ||w_before|| / 10
    st.arrive[s] = 0;
  }
}

// End of iteration j, one kernel (grid = blocks of kThreads entries x systems):
//  * every CTA forms ||w|| = h_{j+1,j} from the update kernel's chunk sums and scales its entries of w into
//    V_{j+1} (and into the FP16 x 3 operand of the next tensor-core product);
//  * the first warp of CTA 0 of each system applies the previous Givens rotations to column j of H, forms
//    the new rotation and updates g and the residual estimate |g_{j+1}| / beta (finish_column);
//  * the last CTA to finish advances the iteration index (all CTAs have read it by then).
// A system that converges at this step still gets V_{j+1}; nothing reads it.
constexpr int kFinishMaxM = 1000;

// The inputs of the rotations of column j, staged by one warp (another warp than the one that computes
// h_{j+1,j}, so the two sets of loads overlap): column j of H and the previous rotations in shared memory (complex
// type C: FP64, or FP32 for an FP32 basis), and g_j, the previous residual estimate and the tolerance.
struct FinishIn {
  double2 gj;
  double res;
  double tl;
};
// The rotations and scalars alone (the fused iteration kernel forms the column itself).
template <typename C>
__device__ __forceinline__ void stage_rotations(const KrylovState& st, int s, int j, double tol, C* sh_c, C* sh_s,
                                                FinishIn* in) {
  const int lane = threadIdx.x & 31;
  const double2* cs = st.cs + (size_t)s * st.m;
  const double2* sn = st.sn + (size_t)s * st.m;
  for (int i = lane; i < j; i += 32) {
    const double2 ci = cs[i], si = sn[i];
    sh_c[i] = cx<C>(ci.x, ci.y);
    sh_s[i] = cx<C>(si.x, si.y);
  }
  if (lane == 0) {
    in->gj = st.g[(size_t)s * (st.m + 1) + j];
    in->res = st.resid[s];
    in->tl = st.tolv ? st.tolv[s] : tol;
  }
}
template <typename C>
__device__ __forceinline__ void finish_stage(const KrylovState& st, int s, int j, double tol, C* sh_h, C* sh_c,
                                             C* sh_s, FinishIn* in) {
  const double2* Hj = st.H + ((size_t)s * st.m + j) * (st.m + 1);
  for (int i = threadIdx.x & 31; i <= j; i += 32) {
    const double2 h = Hj[i];
    sh_h[i] = cx<C>(h.x, h.y);
  }
  stage_rotations(st, s, j, tol, sh_c, sh_s, in);
}

// One warp, after finish_stage and a barrier: h_{j+1,j} = hn.  The lanes apply the previous rotations to the
// staged column as a scan (warp_rotate_column); lane 0 then forms the new rotation.  g and the residual
// estimate stay FP64.
template <typename C>
__device__ __forceinline__ void finish_column(const KrylovState& st, int s, int j, double hn, C* sh_h, C* sh_c,
                                              C* sh_s, const FinishIn* in) {
  using R = decltype(C{}.x);
  const int lane = threadIdx.x & 31;
  double2* Hj = st.H + ((size_t)s * st.m + j) * (st.m + 1);
  const C a = warp_rotate_column(sh_h, sh_c, sh_s, j);
  for (int i = lane; i < j; i += 32) Hj[i] = make_double2(sh_h[i].x, sh_h[i].y);
  if (lane != 0) return;
  R den, inv;
  givens_norm(a, (R)hn, den, inv);
  double2 c, sv;
  if (den == (R)0) { c = make_double2(1, 0); sv = make_double2(0, 0); }
  else { c = make_double2(a.x * inv, a.y * inv); sv = make_double2((R)hn * inv, 0.0); }
  st.cs[(size_t)s * st.m + j] = c;
  st.sn[(size_t)s * st.m + j] = sv;
  Hj[j] = make_double2(den, 0.0);
  Hj[j + 1] = make_double2(0.0, 0.0);
  double2* g = st.g + (size_t)s * (st.m + 1);
  const double2 gj = in->gj;
  g[j + 1] = make_double2(-(sv.x * gj.x - sv.y * gj.y), -(sv.x * gj.y + sv.y * gj.x));
  g[j] = cdotc(c, gj);
  // |g_{j+1}| = |s_j| |g_j|: the estimate shrinks by the rotation's sine (resid starts at 1)
  const double res = in->res * sv.x;
  st.resid[s] = res;
  st.iters[s] = j + 1;
  st.hnext[s] = hn;
  const bool stop = res <= in->tl || j + 1 >= st.m || hn == 0.0;
  if (!st.relaxed[s] && (stop || res <= kRelaxFactor * in->tl)) {
    st.relaxed[s] = 1;
    atomicSub(st.n_unrelaxed, 1);
  }
  if (stop) {
    st.active[s] = 0;
    atomicSub(st.n_active, 1);   // the gate of the queued iterations closes with the last system
  }
}

// dynamic shared memory: 3 (m + 1) entries of T (column and rotations for finish_column).  Each thread scales
// kStepPer entries, so that the grid of one iteration fits on the GPU in one wave.
constexpr int kStepPer = 4;
template <typename T>
__global__ void __launch_bounds__(kThreads) k_step_end(KrylovState st, int nchunk, double tol) {
  pdl_enter();
  using F = typename Vec<T>::acc_t;
  extern __shared__ __align__(16) unsigned char fin_raw[];
  T* fin_sh = reinterpret_cast<T*>(fin_raw);
  __shared__ F s_hn;
  __shared__ FinishIn s_in;
  const int c = blockIdx.x, s = blockIdx.y;
  // read once, before the arrival below: the last CTA to arrive advances the index
  const int j = *(volatile const int*)st.jdev;
  if (st.active[s]) {
    if (threadIdx.x < 32) {
      F t = 0;   // in the basis precision
      for (int cc = threadIdx.x; cc < nchunk; cc += 32) t += (F)st.npart[(size_t)s * nchunk + cc];
      t = warp_sum(t);
      if (threadIdx.x == 0) s_hn = sqrt(t);
    } else if (c == 0 && threadIdx.x < 64) {
      finish_stage(st, s, j, tol, fin_sh, fin_sh + (st.m + 1), fin_sh + 2 * (st.m + 1), &s_in);
    }
    __syncthreads();
    const F hn = s_hn;
    // the rotations are the long dependent chain of this kernel: start them before the scaling
    if (c == 0 && threadIdx.x < 32)
      finish_column(st, s, j, (double)hn, fin_sh, fin_sh + (st.m + 1), fin_sh + 2 * (st.m + 1), &s_in);
    if (hn > (F)0 && j + 1 < st.m) {
      const T* W = static_cast<const T*>(st.W) + (size_t)s * st.n;
      T* Vn = static_cast<T*>(st.V) + ((size_t)(j + 1) * st.nrhs + s) * st.n;
      const F inv = (F)1 / hn;
      const int k0 = c * (kThreads * kStepPer) + threadIdx.x;
      T w[kStepPer];
#pragma unroll
      for (int q = 0; q < kStepPer; ++q)
        if (k0 + q * kThreads < st.n) w[q] = W[k0 + q * kThreads];
#pragma unroll
      for (int q = 0; q < kStepPer; ++q) {
        const int k = k0 + q * kThreads;
        if (k < st.n) {
          w[q].x *= inv;
          w[q].y *= inv;
          Vn[k] = w[q];
          if (st.b16hi)
            tc_write_b(static_cast<__half*>(st.b16hi), static_cast<__half*>(st.b16lo), st.ldb16, s, k, (float)w[q].x,
                       (float)w[q].y);
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // with a graph loop, the last CTA reads the active count: the rotations' decrements must be visible
    if (st.cond_handle) __threadfence();
    if (atomicAdd(st.arrive + s, 1) == (int)gridDim.x - 1) {
      st.arrive[s] = 0;
      if (atomicAdd(st.arrive_all, 1) == (int)gridDim.y - 1) {
        *st.arrive_all = 0;
        *st.jdev = j + 1;
        if (st.cond_handle) {
          __threadfence();
          cudaGraphSetConditional((cudaGraphConditionalHandle)st.cond_handle, atomicAdd(st.n_active, 0) > 0 ? 1u : 0u);
        }
      }
    }
  }
}

// ---- One cooperative launch per iteration: orthogonalisation and end of iteration ----
// As separate kernels, the tail of an iteration (projections, update, a conditional second pass, end of
// iteration) pays a launch and a grid-wide drain per kernel plus a dependent chain of global round trips in each;
// at small j these fixed costs dominate (on the 64-system star: 25 us for the first pass at j = 0, where it reads
// 4 MB, 4.4 us for an empty conditional pass, 10 us for the end of iteration; the fused launch takes 19 us there).
// One persistent grid walks the (system, chunk) items in system order.  For its item a CTA stages the chunk of w
// in shared memory, where it stays for the whole iteration, and per Gram-Schmidt pass: writes the chunk's partial
// projections, waits at a per-system barrier, sums the partials of all chunks (FP64, chunk order), updates its
// chunk of w, writes the chunk's squared norm and waits at the barrier again.  Every CTA of a system then forms
// the same norm sums in the same order, so all take the same decision on the second pass (the norm-drop test of
// k_dots) with no further round trip.  After the last pass each CTA scales its chunk into v_{j+1} and its FP16
// operand, the chunk-0 CTA applies the rotations (finish_column), and the last CTA of the grid advances the
// iteration index and sets the graph loop's condition.
// Chunks are as long as one wave of the grid allows (1024 entries on the star: 512 items on 608 resident CTAs).
// The update runs over the basis newest vector first: the projections have just streamed the whole basis, and
// its last-read part is what L2 still holds (on the star, against oldest first: Arnoldi 7.7 against 8.8 ms per
// step).  Trimming the grid so that each wave's basis chunks fit in L2 was slower (every extra wave repeats the
// barrier chain with fewer loads in flight: 15.9 ms with 64 MB per wave).
// Projections: with at least as many basis vectors as warps, warp w takes vectors w, w + 8, ... over the whole
// chunk; with fewer (small j) each vector is split into NS sub-chunks so that every warp loads, and the
// sub-chunk sums are combined in shared memory (basis precision, fixed order).  Update: each thread owns
// CH / 512 pairs of entries over all basis vectors.
//
// Deadlock freedom: items are assigned statically, item q to CTA q mod G, with G >= chunks per system, so the
// chunks of one system sit on distinct CTAs, and a CTA's earlier items belong to earlier systems.  Every CTA of
// a system passes the same sequence of barriers (its decisions are uniform), so by induction on the system index
// every barrier completes.  The grid is cooperative, so every CTA is resident.  Each wait is bounded
// (wait_ns, default kCgsWaitNs): on expiry the kernel records it in st.err (the host returns BEM_ETIMEOUT) and goes on, and once
// st.err is set no later wait of the run waits at all, so no CTA can hang and a failed run ends in bounded time.
constexpr unsigned long long kCgsWaitNs = 500000000ull;   // 0.5 s (a barrier normally completes in microseconds)
std::atomic<unsigned long long> g_cgs_wait_ns{kCgsWaitNs};   // for kernels launched from now on
std::atomic<int> g_fused_on{1};

__device__ __forceinline__ unsigned long long cgs_time() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// GPU-scope release / acquire accesses of the barrier counters.  A CTA's writes made before a __syncthreads
// become visible with thread 0's release arrival after it, and a CTA whose thread 0 has read an arrival with an
// acquire load sees, after its next __syncthreads, everything the arriving CTA wrote before arriving (the
// ordering of a release pattern is cumulative over what the barrier ordered before it).  Against a full fence
// before a relaxed atomic and after the wait: 1.41 against 1.87 us per barrier of 64 systems x 8 CTAs.
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int atom_add_release_gpu(int* p, int v) {
  int old;
  asm volatile("atom.add.release.gpu.global.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ int atom_add_acq_rel_gpu(int* p, int v) {
  int old;
  asm volatile("atom.add.acq_rel.gpu.global.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// All threads of the CTA: wait until every chunk of system s has arrived.  st.sync[s] only grows (zeroed at the
// start of a run), and the CTAs of a system pass their barriers in the same order, so barrier number b of the
// iteration completes when the counter reaches a multiple of nchunk above the arrival.
// Each system's counter has a cache line of its own, and a waiting thread polls it with a short sleep between
// reads, so that the polls of one system's CTAs do not queue behind the arrivals of the others at one L2 slice.
// The data exchanged through a barrier (the chunk sums) is read with L2 loads (__ldcg).
__device__ __forceinline__ void system_barrier(const KrylovState& st, int s, int nchunk, unsigned long long wait_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int* ctr = st.sync + (size_t)s * kSyncStride;
    const int old = atom_add_release_gpu(ctr, 1);
    const int target = (old / nchunk + 1) * nchunk;
    if (ld_acquire_gpu(ctr) < target && *(volatile int*)st.err == 0) {
      const unsigned long long t0 = cgs_time();
      while (ld_acquire_gpu(ctr) < target) {
        __nanosleep(100);
        if (cgs_time() - t0 > wait_ns || *(volatile int*)st.err != 0) {
          atomicCAS(st.err, 0, 1);
          break;
        }
      }
    }
  }
  __syncthreads();
}

constexpr int kArnW = kThreads / 32;   // warps per CTA
// L2 bytes of basis chunks that the projections mark evict-last for the update's second read.  Star, 64 systems,
// per step (Arnoldi phase): no hints 7.0 ms; every load evict-first 7.4; 32 MB kept 6.94, 64 MB 6.84, 96 MB
// 6.82, 128 MB 6.98 (another box: 96 MB 6.97); leaving the older vectors or the update at normal priority
// instead of evict-first gave the same or worse (7.0, 7.2).
constexpr long long kArnKeepBytes = 96ll << 20;

// dynamic shared memory: 3 (m + 1) entries of T (the column and the rotations for finish_column)
template <typename T, int CH>
__global__ void __launch_bounds__(kThreads, sizeof(T) == sizeof(float2) ? 4 : 1)
    k_arnoldi(KrylovState st, int nchunk, int passes, double tol, unsigned long long wait_ns) {
  using F = typename Vec<T>::acc_t;
  constexpr int NS = CH >= 256 ? CH / 256 : 1;            // sub-chunks of a vector at small j
  constexpr int PP = CH / 2 > kThreads ? CH / 2 / kThreads : 1;   // update: pairs per thread
  extern __shared__ __align__(16) unsigned char fin_raw[];
  T* sh_h = reinterpret_cast<T*>(fin_raw);
  T* sh_c = sh_h + (st.m + 1);
  T* sh_s = sh_c + (st.m + 1);
  __shared__ __align__(16) T ws[CH];   // the chunk of w, for the whole iteration
  __shared__ F hs[2 * kHsMax];         // projections of the current pass, basis precision
  __shared__ F tp[2 * kArnW * NS];     // sub-chunk partials at small j
  __shared__ double red[kArnW];
  __shared__ F s_hn;
  __shared__ int s_more;
  __shared__ FinishIn s_in;
  constexpr int NT = CH >= kTcM ? CH / kTcM : 1;   // row tiles of the product per chunk
  __shared__ int cov[NT][kTcMaxCover];             // their stream-K partial tiles (when st.tc.part is set)
  __shared__ int ncov[NT];
  const int j = *(volatile const int*)st.jdev;   // read before this CTA's arrival below
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t stride = (size_t)st.nrhs * st.n;
  const size_t ldp = (size_t)st.m + 1;
  int G = gridDim.x;
  if (nchunk > G) {   // the launcher never does this: a system's chunks must sit on distinct CTAs
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(st.err, 0, 2);
    G = 0;
  }
  const int items = st.nrhs * nchunk;
  // The projections mark the newest `keep` vectors of each chunk evict-last in L2 (the update reads them first)
  // and the others evict-first, so that the update's second read finds the kept ones there; the update's own
  // loads are evict-first (nothing reads them again before the next iteration's projections).
  const unsigned long long pol_last = l2_evict_last(), pol_first = l2_evict_first();
  const int items_live = min(items, G);
  const long long keep_ll = items_live > 0 ? kArnKeepBytes / ((long long)items_live * CH * (long long)sizeof(T)) : 0;
  const int keep = (int)min(keep_ll, (long long)(j + 1));
  const int ns = j + 1 >= kArnW ? 1 : NS;   // sub-chunks per vector in this iteration
  const int ntask = (j + 1) * ns;
  const int sub_pairs = CH / 2 / ns;         // pairs of a projection task
  for (int q = blockIdx.x; (int)blockIdx.x < G && q < items; q += G) {
    const int s = q / nchunk, c = q - s * nchunk;
    if (!st.active[s]) continue;   // the same for every chunk of the system
    const int k0 = c * CH;
    const T* V = static_cast<const T*>(st.V) + (size_t)s * st.n + k0;
    const int nk = min(CH, st.n - k0);   // entries of this chunk (even)
    if (st.tc.part) {
      // w = the tensor-core product's stream-K partials of rows k0 .. k0 + nk - 1, summed in CTA order and
      // scaled by 1 / rsc (the arithmetic of k_tc_reduce, whose launch this replaces)
      if ((int)threadIdx.x < NT) {
        const int t = k0 / kTcM + threadIdx.x;
        ncov[threadIdx.x] = t * kTcM < st.n ? tc_cover(t, st.tc.kpt, st.tc.total, st.tc.G, cov[threadIdx.x],
                                                       kTcMaxCover)
                                            : 0;
      }
      __syncthreads();
      for (int qq = threadIdx.x; qq < CH / 2; qq += kThreads) {
        T a, b;
        a.x = a.y = b.x = b.y = 0;
        if (2 * qq < nk) {
          const int r = k0 + 2 * qq;   // rows r and r + 1 (one row tile: r is even)
          const int ti = r / kTcM - k0 / kTcM, rr = r % kTcM;
          float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
          for (int u = 0; u < ncov[ti]; ++u) {
            const float* P = st.tc.part + (size_t)cov[ti][u] * kTcM * kTcN + rr;
            const float2 re = *reinterpret_cast<const float2*>(P + (size_t)s * kTcM);
            const float2 im = *reinterpret_cast<const float2*>(P + (size_t)(64 + s) * kTcM);
            ax += re.x;
            bx += re.y;
            ay += im.x;
            by += im.y;
          }
          const float ia = 1.f / st.tc.rsc[r], ib = 1.f / st.tc.rsc[r + 1];   // powers of two: exact
          a.x = ax * ia;
          a.y = ay * ia;
          b.x = bx * ib;
          b.y = by * ib;
        }
        Pair<T>::store(ws + 2 * qq, a, b);
      }
    } else {
      const T* W = static_cast<const T*>(st.W) + (size_t)s * st.n + k0;
      for (int qq = threadIdx.x; qq < CH / 2; qq += kThreads) {
        T a, b;
        if (2 * qq < nk) {
          Pair<T>::load(W + 2 * qq, a, b);
        } else {
          a.x = a.y = b.x = b.y = 0;
        }
        Pair<T>::store(ws + 2 * qq, a, b);
      }
    }
    if (c == 0 && warp == kArnW - 1) stage_rotations(st, s, j, tol, sh_c, sh_s, &s_in);
    __syncthreads();
    if (passes == 0 && warp == 0) {   // ||w||^2 of the chunk before projection (norm-drop test)
      F nw = 0;
      for (int qq = lane; qq < CH / 2; qq += 32) {
        T a, b;
        Pair<T>::load(ws + 2 * qq, a, b);
        nw += (F)a.x * (F)a.x + (F)a.y * (F)a.y + (F)b.x * (F)b.x + (F)b.y * (F)b.y;
      }
      nw = warp_sum(nw);
      if (lane == 0) st.wpart[(size_t)s * nchunk + c] = (double)nw;
    }
    for (int pass = 0;; ++pass) {
      // ---- partial projections <v_i, w> over this chunk ----
      for (int t = warp; t < ntask; t += kArnW) {
        const int i = t / ns, sub = t - i * ns;
        const int p0 = sub * sub_pairs;
        const T* vi = V + (size_t)i * stride;
        F px = 0, py = 0;
#pragma unroll 4
        for (int pp = p0 + lane; pp < p0 + sub_pairs; pp += 32) {
          if (2 * pp < nk) {
            T a, b, w0, w1;
            PairHint<T>::load(vi + 2 * pp, a, b, i > j - keep ? pol_last : pol_first);
            Pair<T>::load(ws + 2 * pp, w0, w1);
            px += (F)a.x * (F)w0.x + (F)a.y * (F)w0.y + (F)b.x * (F)w1.x + (F)b.y * (F)w1.y;
            py += (F)a.x * (F)w0.y - (F)a.y * (F)w0.x + (F)b.x * (F)w1.y - (F)b.y * (F)w1.x;
          }
        }
        const F hx = warp_sum(px), hy = warp_sum(py);
        if (lane == 0) {
          if (ns == 1) {
            st.part[((size_t)s * nchunk + c) * ldp + i] = make_double2((double)hx, (double)hy);
          } else {
            tp[2 * t] = hx;
            tp[2 * t + 1] = hy;
          }
        }
      }
      if (ns > 1) {
        __syncthreads();
        if ((int)threadIdx.x <= j) {
          F hx = 0, hy = 0;
          for (int u = 0; u < ns; ++u) {
            hx += tp[2 * (threadIdx.x * ns + u)];
            hy += tp[2 * (threadIdx.x * ns + u) + 1];
          }
          st.part[((size_t)s * nchunk + c) * ldp + threadIdx.x] = make_double2((double)hx, (double)hy);
        }
      }
      system_barrier(st, s, nchunk, wait_ns);
      // ---- h_i = sum over the chunks (FP64, chunk order); chunk 0 records the column ----
      for (int i = threadIdx.x; i <= j; i += kThreads) {
        double2 h = make_double2(0.0, 0.0);
#pragma unroll 8
        for (int cc = 0; cc < nchunk; ++cc) h = cadd(h, __ldcg(st.part + ((size_t)s * nchunk + cc) * ldp + i));
        hs[2 * i] = (F)h.x;
        hs[2 * i + 1] = (F)h.y;
        if (c == 0) {
          double2* Hj = st.H + ((size_t)s * st.m + j) * ldp;
          const double2 tot = pass == 0 ? h : cadd(Hj[i], h);
          Hj[i] = tot;
          sh_h[i] = cx<T>(tot.x, tot.y);
        }
      }
      __syncthreads();
      // ---- w -= sum_i h_i v_i over this chunk; squared norm of the result ----
      F nrm = 0;
      {
        F ax[PP], ay[PP], bx[PP], by[PP];
#pragma unroll
        for (int r = 0; r < PP; ++r) ax[r] = ay[r] = bx[r] = by[r] = 0;
#pragma unroll 4
        for (int ii = 0; ii <= j; ++ii) {   // newest first: those entries are the likeliest still in L2
          const int i = j - ii;
          const F hx = hs[2 * i], hy = hs[2 * i + 1];
          const T* vi = V + (size_t)i * stride;
#pragma unroll
          for (int r = 0; r < PP; ++r) {
            const int e = 2 * (threadIdx.x + r * kThreads);
            if (e < nk) {
              T a, b;
              PairHint<T>::load(vi + e, a, b, pol_first);   // not read again this iteration
              ax[r] += hx * (F)a.x - hy * (F)a.y;
              ay[r] += hx * (F)a.y + hy * (F)a.x;
              bx[r] += hx * (F)b.x - hy * (F)b.y;
              by[r] += hx * (F)b.y + hy * (F)b.x;
            }
          }
        }
#pragma unroll
        for (int r = 0; r < PP; ++r) {
          const int e = 2 * (threadIdx.x + r * kThreads);
          if (e < nk) {
            T w0, w1;
            Pair<T>::load(ws + e, w0, w1);
            w0.x -= ax[r]; w0.y -= ay[r];
            w1.x -= bx[r]; w1.y -= by[r];
            Pair<T>::store(ws + e, w0, w1);
            nrm += w0.x * w0.x + w0.y * w0.y + w1.x * w1.x + w1.y * w1.y;
          }
        }
      }
      nrm = warp_sum(nrm);   // basis precision within the warp, FP64 across warps and chunks
      if (lane == 0) red[warp] = (double)nrm;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w8 = 0; w8 < kArnW; ++w8) t += red[w8];
        st.npart[(size_t)s * nchunk + c] = t;
      }
      system_barrier(st, s, nchunk, wait_ns);
      // ---- the system's norms: the same sums in every CTA of the system ----
      if (warp == 0) {
        F t = 0;   // ||w|| in the basis precision, as k_step_end
        double before = 0.0, after = 0.0;
        for (int cc = lane; cc < nchunk; cc += 32) {
          const double v = __ldcg(st.npart + (size_t)s * nchunk + cc);
          t += (F)v;
          after += v;
          if (passes == 0) before += __ldcg(st.wpart + (size_t)s * nchunk + cc);
        }
        t = warp_sum(t);
        after = warp_sum(after);
        before = warp_sum(before);
        if (lane == 0) {
          s_hn = sqrt(t);
          s_more = pass == 0 && (passes == 2 || (passes == 0 && (st.strict[s] || after < 0.01 * before)));
        }
      }
      __syncthreads();
      if (!s_more) break;
    }
    // ---- end of iteration: rotations (chunk 0), next basis vector ----
    const F hn = s_hn;
    if (c == 0 && warp == 0) finish_column(st, s, j, (double)hn, sh_h, sh_c, sh_s, &s_in);
    if (hn > (F)0 && j + 1 < st.m) {
      const F inv = (F)1 / hn;
      T* Vn = static_cast<T*>(st.V) + ((size_t)(j + 1) * st.nrhs + s) * st.n + k0;
      for (int qq = threadIdx.x; qq < CH / 2; qq += kThreads) {
        const int e = 2 * qq;
        if (e < nk) {
          T a, b;
          Pair<T>::load(ws + e, a, b);
          a.x *= inv; a.y *= inv;
          b.x *= inv; b.y *= inv;
          Pair<T>::store(Vn + e, a, b);
          if (st.b16hi) {
            tc_write_b(static_cast<__half*>(st.b16hi), static_cast<__half*>(st.b16lo), st.ldb16, s, k0 + e,
                       (float)a.x, (float)a.y);
            tc_write_b(static_cast<__half*>(st.b16hi), static_cast<__half*>(st.b16lo), st.ldb16, s, k0 + e + 1,
                       (float)b.x, (float)b.y);
          }
        }
      }
    }
    __syncthreads();   // ws, hs, tp and the staged rotations are reused by the next item
  }
  // every CTA arrives (those without items too, after the __syncthreads that ends the item loop); the last one
  // advances the index.  With a graph loop the last CTA reads the active count: its acquire-release arrival
  // makes the rotations' decrements, which other CTAs made before arriving, visible to it.
  if (threadIdx.x == 0) {
    if (atom_add_acq_rel_gpu(st.arrive_all, 1) == (int)gridDim.x - 1) {
      *st.arrive_all = 0;
      *st.jdev = j + 1;
      if (st.cond_handle)
        cudaGraphSetConditional((cudaGraphConditionalHandle)st.cond_handle, atomicAdd(st.n_active, 0) > 0 ? 1u : 0u);
    }
  }
}

// Least squares: back substitution of the triangularised Hessenberg system, one CTA per system.
__global__ void __launch_bounds__(kBsThreads) k_lsq(KrylovState st) {
  __shared__ double2 sg[kFinishMaxM], sinv[kFinishMaxM], sy;
  const int s = blockIdx.x;
  if (s >= st.nrhs) return;
  block_back_substitute(st.H + (size_t)s * st.m * (st.m + 1), st.m + 1, st.g + (size_t)s * (st.m + 1),
                        st.y + (size_t)s * st.m, st.iters[s], sg, sinv, &sy);
}

// x += sum_i y_i v_i: CH/2 threads per chunk, each owning one pair of entries and running over all i;
// products and sums in the basis precision (the correction only needs the inner solve's accuracy), added
// to the FP64 x.
// dout (optional): the correction sum_i y_i v_i itself, complex FP32 (the refinement's updated residual).
template <typename T, int CH>
__global__ void __launch_bounds__(CH / 2) k_xupdate(KrylovState st, double2* x, float2* dout) {
  using F = typename Vec<T>::acc_t;
  __shared__ F ys[2 * kHsMax];
  const int c = blockIdx.x, s = blockIdx.y;
  const int mm = st.iters[s];
  for (int i = threadIdx.x; i < mm; i += CH / 2) {
    const double2 y = st.y[(size_t)s * st.m + i];
    ys[2 * i] = (F)y.x;
    ys[2 * i + 1] = (F)y.y;
  }
  __syncthreads();
  const int k = c * CH + 2 * threadIdx.x;
  if (k >= st.n) return;
  if (mm == 0) {   // no correction (the system had already converged)
    if (dout) {
      float2* ds = dout + (size_t)s * st.n + k;
      ds[0] = ds[1] = make_float2(0.f, 0.f);
    }
    return;
  }
  const size_t stride = (size_t)st.nrhs * st.n;
  const T* V = static_cast<const T*>(st.V) + (size_t)s * st.n + k;
  F ax = 0, ay = 0, bx = 0, by = 0;
#pragma unroll 8
  for (int i = 0; i < mm; ++i) {
    T a, b;
    Pair<T>::load(V + (size_t)i * stride, a, b);
    const F yx = ys[2 * i], yy = ys[2 * i + 1];
    ax += yx * (F)a.x - yy * (F)a.y;
    ay += yx * (F)a.y + yy * (F)a.x;
    bx += yx * (F)b.x - yy * (F)b.y;
    by += yx * (F)b.y + yy * (F)b.x;
  }
  double2* xs = x + (size_t)s * st.n + k;
  xs[0] = make_double2(xs[0].x + (double)ax, xs[0].y + (double)ay);
  xs[1] = make_double2(xs[1].x + (double)bx, xs[1].y + (double)by);
  if (dout) {
    float2* ds = dout + (size_t)s * st.n + k;
    ds[0] = make_float2((float)ax, (float)ay);
    ds[1] = make_float2((float)bx, (float)by);
  }
}

int nchunk_of(int n) { return (n + kCh - 1) / kCh; }
int nblk_of(int n) { return (n + kThreads - 1) / kThreads; }

int sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// Chunk length of the projection and update kernels: the largest of 512, 256, 128 entries that still gives
// at least two CTAs per SM over all systems, else 64 (a single system of a few thousand unknowns).  Longer
// chunks move more bytes per warp reduction and per instruction.
int chunk_of(int n, int nrhs) {
  for (int ch : {512, 256, 128})
    if ((long long)((n + ch - 1) / ch) * nrhs >= 2LL * sm_count()) return ch;
  return kCh;
}

// mode as for k_dots (0: first pass, 1: conditional second pass, 2: second pass)
template <typename T, int CH>
void orth_pass(const KrylovState& st, int pass, int mode, cudaStream_t s) {
  const int nc = (st.n + CH - 1) / CH;
  dim3 grd(nc, st.nrhs);
  const int fused = nc <= 32;   // few chunks: each update CTA sums the partials itself (one launch less)
  const int cond = mode == 1;
  launch_pdl(k_dots<T, CH>, grd, dim3(kThreads), 0, s, st, nc, mode);
  if (!fused) launch_pdl(k_dots_reduce, dim3((st.m + 8) / 8, st.nrhs), dim3(256), 0, s, st, nc, pass, cond);
  launch_pdl(k_update<T, CH>, grd, dim3(CH / 2), 0, s, st, nc, pass, fused, cond);
}

template <typename T>
cudaError_t start_t(const KrylovState& st, const double2* r0, cudaStream_t s) {
  const int nb = nblk_of(st.n);
  dim3 grd(nb, st.nrhs);
  k_norm_part<double2><<<grd, kThreads, 0, s>>>(r0, st.n, st.npart, nb);
  cudaError_t e = cudaMemsetAsync(st.n_active, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(st.n_unrelaxed, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (st.sync) {
    e = cudaMemsetAsync(st.sync, 0, (size_t)st.nrhs * kSyncStride * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st.err, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  k_start_finish<<<(st.nrhs + 63) / 64, 64, 0, s>>>(st, nb);
  k_start_scale<T><<<grd, kThreads, 0, s>>>(st, r0);
  return cudaGetLastError();
}

// passes: 1 (classical Gram-Schmidt), 2 (twice, CGS2) or 0 (once, then again only for the systems that the
// norm-drop test flags).
// Resident CTAs of k_arnoldi<T, CH> on this device with the shared memory of the largest Krylov dimension
// (0 if its launch cannot be cooperative).
template <typename T, int CH>
int arn_grid() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  int g = cache[dev].load(std::memory_order_relaxed);
  if (g != 0) return g > 0 ? g : 0;
  const int dyn = 3 * kHsMax * (int)sizeof(T);
  int coop = 0, per = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
      cudaFuncSetAttribute(k_arnoldi<T, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_arnoldi<T, CH>, kThreads, dyn) != cudaSuccess ||
      per <= 0) {
    cudaGetLastError();
    cache[dev].store(-1, std::memory_order_relaxed);
    return 0;
  }
  g = per * sm_count();
  cache[dev].store(g, std::memory_order_relaxed);
  return g;
}

template <typename T, int CH>
int arn_fit(const KrylovState& st, int& best) {   // 1: every item in one wave; best: CH if usable at all
  const int nc = (st.n + CH - 1) / CH;
  const int G = arn_grid<T, CH>();
  if (G <= 0 || nc > G || nc > krylov_nchunk(st.n)) return 0;
  best = CH;
  return (long long)nc * st.nrhs <= G;
}

// Chunk length of the fused iteration kernel: the shortest of 64 ... 1024 entries whose items all fit in one
// wave of its grid (one pass of the per-item chain), else the longest usable one; 0 if none is usable (no
// cooperative launch, the state lacks the barrier counters, or a system's chunks exceed the grid).
template <typename T>
int arn_chunk(const KrylovState& st) {
  if (!st.sync || !st.err || st.m + 1 > kHsMax || !g_fused_on.load(std::memory_order_relaxed)) return 0;
  int best = 0;
  if (arn_fit<T, 64>(st, best)) return 64;
  if (arn_fit<T, 128>(st, best)) return 128;
  if (arn_fit<T, 256>(st, best)) return 256;
  if (arn_fit<T, 512>(st, best)) return 512;
  if (arn_fit<T, 1024>(st, best)) return 1024;
  return best;
}

template <typename T, int CH>
cudaError_t arn_launch(const KrylovState& st, int passes, double tol, cudaStream_t s) {
  const int nc = (st.n + CH - 1) / CH;
  const int G = std::min(arn_grid<T, CH>(), nc * st.nrhs);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 3 * (size_t)(st.m + 1) * sizeof(T);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_arnoldi<T, CH>, st, nc, passes, tol,
                            g_cgs_wait_ns.load(std::memory_order_relaxed));
}

template <typename T>
cudaError_t step_t(const KrylovState& st, int passes, double tol, cudaStream_t s) {
  switch (arn_chunk<T>(st)) {
    case 64: return arn_launch<T, 64>(st, passes, tol, s);
    case 128: return arn_launch<T, 128>(st, passes, tol, s);
    case 256: return arn_launch<T, 256>(st, passes, tol, s);
    case 512: return arn_launch<T, 512>(st, passes, tol, s);
    case 1024: return arn_launch<T, 1024>(st, passes, tol, s);
    default: return cudaErrorNotSupported;
  }
}

template <typename T>
cudaError_t orth_t(const KrylovState& st, int passes, cudaStream_t s) {
  const int ch = chunk_of(st.n, st.nrhs);
  const int np = passes == 1 ? 1 : 2;
  for (int p = 0; p < np; ++p) {
    const int mode = p == 0 ? 0 : (passes == 0 ? 1 : 2);
    switch (ch) {
      case 512: orth_pass<T, 512>(st, p, mode, s); break;
      case 256: orth_pass<T, 256>(st, p, mode, s); break;
      case 128: orth_pass<T, 128>(st, p, mode, s); break;
      default: orth_pass<T, 64>(st, p, mode, s); break;
    }
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t finish_t(const KrylovState& st, double tol, cudaStream_t s) {
  const int ch = chunk_of(st.n, st.nrhs);
  const int nc = (st.n + ch - 1) / ch;   // the update kernel's chunks (its squared norms)
  const int nb = (st.n + kThreads * kStepPer - 1) / (kThreads * kStepPer);
  return launch_pdl(k_step_end<T>, dim3(nb, st.nrhs), dim3(kThreads), 3 * (st.m + 1) * sizeof(T), s, st, nc, tol);
}

template <typename T>
cudaError_t xupd_t(const KrylovState& st, double2* x, float2* dout, cudaStream_t s) {
  k_lsq<<<st.nrhs, kBsThreads, 0, s>>>(st);
  const int ch = chunk_of(st.n, st.nrhs);
  const dim3 grd((st.n + ch - 1) / ch, st.nrhs);
  switch (ch) {
    case 512: k_xupdate<T, 512><<<grd, 256, 0, s>>>(st, x, dout); break;
    case 256: k_xupdate<T, 256><<<grd, 128, 0, s>>>(st, x, dout); break;
    case 128: k_xupdate<T, 128><<<grd, 64, 0, s>>>(st, x, dout); break;
    default: k_xupdate<T, 64><<<grd, 32, 0, s>>>(st, x, dout); break;
  }
  return cudaGetLastError();
}

}  // namespace

int krylov_nchunk(int n) { return std::max(nchunk_of(n), nblk_of(n)); }

cudaError_t krylov_start(const KrylovState& st, const double2* r0, double, cudaStream_t s) {
  return st.basis_fp32 ? start_t<float2>(st, r0, s) : start_t<double2>(st, r0, s);
}
cudaError_t krylov_orthogonalise(const KrylovState& st, int passes, cudaStream_t s) {
  return st.basis_fp32 ? orth_t<float2>(st, passes, s) : orth_t<double2>(st, passes, s);
}
void krylov_set_wait_ns(unsigned long long ns) { g_cgs_wait_ns.store(ns ? ns : kCgsWaitNs); }
void krylov_set_fused(int on) { g_fused_on.store(on ? 1 : 0); }
int krylov_fused(const KrylovState& st) {
  return st.basis_fp32 ? arn_chunk<float2>(st) : arn_chunk<double2>(st);
}
cudaError_t krylov_fused_step(const KrylovState& st, int passes, double tol, cudaStream_t s) {
  return st.basis_fp32 ? step_t<float2>(st, passes, tol, s) : step_t<double2>(st, passes, tol, s);
}
int krylov_orth_launches(const KrylovState& st, int passes) {
  const int ch = chunk_of(st.n, st.nrhs);
  const int nc = (st.n + ch - 1) / ch;
  return (passes == 1 ? 1 : 2) * (nc <= 32 ? 2 : 3);   // projections, [reduction,] update per pass
}
cudaError_t krylov_finish_step(const KrylovState& st, double tol, cudaStream_t s) {
  return st.basis_fp32 ? finish_t<float2>(st, tol, s) : finish_t<double2>(st, tol, s);
}
cudaError_t krylov_update_solution(const KrylovState& st, double2* x, cudaStream_t s, float2* dout) {
  return st.basis_fp32 ? xupd_t<float2>(st, x, dout, s) : xupd_t<double2>(st, x, dout, s);
}

}  // namespace bem
