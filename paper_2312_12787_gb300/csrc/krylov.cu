// GMRES without restart from x0 = 0 for a block of systems that share one matrix (paper Sec. 3.2,
// eqs. preconditioned_krylov_space / unpreconditioned_krylov_space; Sec. 7: no restart).
//
// Arnoldi uses classical Gram-Schmidt with one re-orthogonalisation pass (CGS2) so that each pass is
// two streaming sweeps over the basis instead of j dependent sweeps; the Hessenberg column, Givens
// rotations and residual estimate are kept in FP64.  The basis may be complex FP64 (FP64 path) or
// complex FP32 (mixed inner solves); in both cases partial sums of each thread are reduced across the
// block and the grid in FP64 with warp shuffles.
//
// Work split: a vector of n unknowns is cut into chunks of kChunk entries; one CTA of 256 threads owns
// one chunk of one system (grid = chunks x systems).  Every kernel reads the iteration index j from
// device memory so that one iteration can be replayed from a CUDA graph.
#include "internal.cuh"

namespace bem {

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 4;                       // entries per thread
constexpr int kChunk = kThreads * kPer;       // entries per CTA

template <typename T> struct Vec;
template <> struct Vec<double2> {
  __device__ static __forceinline__ double2 load(const double2* p) { return *p; }
  __device__ static __forceinline__ void store(double2* p, double2 v) { *p = v; }
};
template <> struct Vec<float2> {
  __device__ static __forceinline__ double2 load(const float2* p) {
    const float2 v = *p;
    return make_double2(v.x, v.y);
  }
  __device__ static __forceinline__ void store(float2* p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum one double over the block; result valid in thread 0.  `red` holds 8 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum_d(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (lane < kThreads / 32) ? red[lane] : 0.0;
    t = warp_sum_d(t);
  }
  return t;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_norm_part(const T* v, int n, double* npart, int nchunk) {
  __shared__ double red[8];
  const int c = blockIdx.x, s = blockIdx.y;
  const T* vs = v + (size_t)s * n;
  double acc = 0.0;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int k = c * kChunk + t * kThreads + threadIdx.x;
    if (k < n) {
      const double2 a = Vec<T>::load(vs + k);
      acc += a.x * a.x + a.y * a.y;
    }
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) npart[(size_t)s * nchunk + c] = acc;
}

// Start: beta = ||r0||, g = (beta, 0, ...), V_0 = r0 / beta, active = (beta > 0).
__global__ void k_start_finish(KrylovState st, int nchunk) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= st.nrhs) return;
  double t = 0.0;
  for (int c = 0; c < nchunk; ++c) t += st.npart[(size_t)s * nchunk + c];
  const double beta = sqrt(t);
  st.beta[s] = beta;
  st.g[(size_t)s * (st.m + 1)] = make_double2(beta, 0.0);
  st.active[s] = beta > 0.0 ? 1 : 0;
  st.iters[s] = 0;
  st.resid[s] = beta > 0.0 ? 1.0 : 0.0;
  st.hnext[s] = beta;
  if (s == 0) *st.jdev = 0;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_start_scale(KrylovState st, const double2* r0) {
  const int c = blockIdx.x, s = blockIdx.y;
  if (!st.active[s]) return;
  const double inv = 1.0 / st.beta[s];
  T* v0 = static_cast<T*>(st.V) + (size_t)s * st.n;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int k = c * kChunk + t * kThreads + threadIdx.x;
    if (k < st.n) Vec<T>::store(v0 + k, cscale(r0[(size_t)s * st.n + k], inv));
  }
}

// Partial projections <v_i, w> over one chunk, four basis vectors per block reduction.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dots(KrylovState st, int nchunk) {
  __shared__ double red[8 * 8];
  const int c = blockIdx.x, s = blockIdx.y;
  if (!st.active[s]) return;
  const int j = *st.jdev;
  const size_t stride = (size_t)st.nrhs * st.n;
  const T* W = static_cast<const T*>(st.W) + (size_t)s * st.n;
  const T* V = static_cast<const T*>(st.V) + (size_t)s * st.n;
  double2 w[kPer];
  int kk[kPer];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    kk[t] = c * kChunk + t * kThreads + threadIdx.x;
    w[t] = kk[t] < st.n ? Vec<T>::load(W + kk[t]) : make_double2(0, 0);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i0 = 0; i0 <= j; i0 += 4) {
    double p[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double px = 0.0, py = 0.0;
      const int i = i0 + q;
      if (i <= j) {
        const T* vi = V + (size_t)i * stride;
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
          if (kk[t] < st.n) {
            const double2 v = Vec<T>::load(vi + kk[t]);
            px += v.x * w[t].x + v.y * w[t].y;     // conj(v) w
            py += v.x * w[t].y - v.y * w[t].x;
          }
        }
      }
      p[2 * q] = warp_sum_d(px);
      p[2 * q + 1] = warp_sum_d(py);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) red[q * 8 + warp] = p[q];
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      double t = 0.0;
#pragma unroll
      for (int w8 = 0; w8 < 8; ++w8) t += red[threadIdx.x * 8 + w8];
      const int q = threadIdx.x >> 1;
      const int i = i0 + q;
      if (i <= j) {
        double* dst = reinterpret_cast<double*>(st.part + ((size_t)s * nchunk + c) * (st.m + 1) + i);
        dst[threadIdx.x & 1] = t;
      }
    }
  }
}

// h_i = sum over chunks; accumulate into column j of H (pass 0 sets, later passes add).
__global__ void k_dots_reduce(KrylovState st, int nchunk, int pass) {
  const int s = blockIdx.x;
  if (!st.active[s]) return;
  const int j = *st.jdev;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    double2 h = make_double2(0, 0);
    for (int c = 0; c < nchunk; ++c) h = cadd(h, st.part[((size_t)s * nchunk + c) * (st.m + 1) + i]);
    st.hcol[(size_t)s * (st.m + 1) + i] = h;
    double2* Hj = st.H + ((size_t)s * st.m + j) * (st.m + 1);
    Hj[i] = pass == 0 ? h : cadd(Hj[i], h);
  }
}

// w -= sum_i h_i v_i over one chunk; partial ||w||^2.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_update(KrylovState st, int nchunk) {
  __shared__ double2 hs[1024];
  __shared__ double red[8];
  const int c = blockIdx.x, s = blockIdx.y;
  if (!st.active[s]) return;
  const int j = *st.jdev;
  for (int i = threadIdx.x; i <= j; i += kThreads) hs[i] = st.hcol[(size_t)s * (st.m + 1) + i];
  __syncthreads();
  const size_t stride = (size_t)st.nrhs * st.n;
  T* W = static_cast<T*>(st.W) + (size_t)s * st.n;
  const T* V = static_cast<const T*>(st.V) + (size_t)s * st.n;
  double acc = 0.0;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int k = c * kChunk + t * kThreads + threadIdx.x;
    if (k >= st.n) continue;
    double2 w = Vec<T>::load(W + k);
    for (int i = 0; i <= j; ++i) {
      const double2 v = Vec<T>::load(V + (size_t)i * stride + k);
      const double2 h = hs[i];
      w.x -= h.x * v.x - h.y * v.y;
      w.y -= h.x * v.y + h.y * v.x;
    }
    Vec<T>::store(W + k, w);
    const double2 wr = Vec<T>::load(W + k);
    acc += wr.x * wr.x + wr.y * wr.y;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) st.npart[(size_t)s * nchunk + c] = acc;
}

// h_{j+1,j} = ||w||; apply the previous Givens rotations to column j, form the new one, update g and
// the residual estimate |g_{j+1}| / beta.  Rotation i acts on rows (i, i+1) as [[conj c, conj s], [-s, c]].
__global__ void k_finish(KrylovState st, int nchunk, double tol) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= st.nrhs || !st.active[s]) return;
  const int j = *st.jdev;
  double t = 0.0;
  for (int c = 0; c < nchunk; ++c) t += st.npart[(size_t)s * nchunk + c];
  const double hn = sqrt(t);
  double2* Hj = st.H + ((size_t)s * st.m + j) * (st.m + 1);
  Hj[j + 1] = make_double2(hn, 0.0);
  double2* cs = st.cs + (size_t)s * st.m;
  double2* sn = st.sn + (size_t)s * st.m;
  for (int i = 0; i < j; ++i) {
    const double2 a = Hj[i], b = Hj[i + 1];
    const double2 ci = cs[i], si = sn[i];
    // conj(c) a + conj(s) b ; -s a + c b
    const double2 ta = cadd(cdotc(ci, a), cdotc(si, b));
    const double2 tb = csub(cmul(ci, b), cmul(si, a));
    Hj[i] = ta;
    Hj[i + 1] = tb;
  }
  const double2 a = Hj[j], b = Hj[j + 1];
  const double den = hypot(hypot(a.x, a.y), hypot(b.x, b.y));
  double2 c, sv;
  if (den == 0.0) { c = make_double2(1, 0); sv = make_double2(0, 0); }
  else { c = cscale(a, 1.0 / den); sv = cscale(b, 1.0 / den); }
  cs[j] = c;
  sn[j] = sv;
  Hj[j] = make_double2(den, 0.0);
  Hj[j + 1] = make_double2(0.0, 0.0);
  double2* g = st.g + (size_t)s * (st.m + 1);
  const double2 gj = g[j];
  g[j + 1] = make_double2(-(sv.x * gj.x - sv.y * gj.y), -(sv.x * gj.y + sv.y * gj.x));
  g[j] = cdotc(c, gj);
  const double res = hypot(g[j + 1].x, g[j + 1].y) / st.beta[s];
  st.resid[s] = res;
  st.iters[s] = j + 1;
  st.hnext[s] = hn;
  if (res <= tol || j + 1 >= st.m || hn == 0.0) st.active[s] = 0;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_scale_next(KrylovState st) {
  const int c = blockIdx.x, s = blockIdx.y;
  if (!st.active[s]) return;
  const int j = *st.jdev;
  const double inv = 1.0 / st.hnext[s];
  const T* W = static_cast<const T*>(st.W) + (size_t)s * st.n;
  T* Vn = static_cast<T*>(st.V) + ((size_t)(j + 1) * st.nrhs + s) * st.n;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int k = c * kChunk + t * kThreads + threadIdx.x;
    if (k < st.n) Vec<T>::store(Vn + k, cscale(Vec<T>::load(W + k), inv));
  }
}

__global__ void k_advance(KrylovState st) {
  // next iteration index; count of systems still active
  if (threadIdx.x == 0) {
    *st.jdev += 1;
    int a = 0;
    for (int s = 0; s < st.nrhs; ++s) a += st.active[s];
    *st.n_active = a;
  }
}

// Least squares: back-substitution of the triangularised Hessenberg system, one thread per system.
__global__ void k_lsq(KrylovState st) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= st.nrhs) return;
  const int mm = st.iters[s];
  const double2* g = st.g + (size_t)s * (st.m + 1);
  double2* y = st.y + (size_t)s * st.m;
  for (int i = mm - 1; i >= 0; --i) {
    double2 acc = g[i];
    for (int l = i + 1; l < mm; ++l) acc = csub(acc, cmul(st.H[((size_t)s * st.m + l) * (st.m + 1) + i], y[l]));
    const double2 d = st.H[((size_t)s * st.m + i) * (st.m + 1) + i];
    const double dd = d.x * d.x + d.y * d.y;
    y[i] = make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_xupdate(KrylovState st, double2* x) {
  __shared__ double2 ys[1024];
  const int c = blockIdx.x, s = blockIdx.y;
  const int mm = st.iters[s];
  for (int i = threadIdx.x; i < mm; i += kThreads) ys[i] = st.y[(size_t)s * st.m + i];
  __syncthreads();
  const size_t stride = (size_t)st.nrhs * st.n;
  const T* V = static_cast<const T*>(st.V) + (size_t)s * st.n;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int k = c * kChunk + t * kThreads + threadIdx.x;
    if (k >= st.n) continue;
    double2 acc = x[(size_t)s * st.n + k];
    for (int i = 0; i < mm; ++i) acc = cadd(acc, cmul(ys[i], Vec<T>::load(V + (size_t)i * stride + k)));
    x[(size_t)s * st.n + k] = acc;
  }
}

template <typename T>
cudaError_t start_t(const KrylovState& st, const double2* r0, cudaStream_t s) {
  const int nc = krylov_nchunk(st.n);
  dim3 grd(nc, st.nrhs);
  k_norm_part<double2><<<grd, kThreads, 0, s>>>(r0, st.n, st.npart, nc);
  k_start_finish<<<(st.nrhs + 63) / 64, 64, 0, s>>>(st, nc);
  k_start_scale<T><<<grd, kThreads, 0, s>>>(st, r0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t orth_t(const KrylovState& st, int passes, cudaStream_t s) {
  const int nc = krylov_nchunk(st.n);
  dim3 grd(nc, st.nrhs);
  for (int p = 0; p < passes; ++p) {
    k_dots<T><<<grd, kThreads, 0, s>>>(st, nc);
    k_dots_reduce<<<st.nrhs, 128, 0, s>>>(st, nc, p);
    k_update<T><<<grd, kThreads, 0, s>>>(st, nc);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t finish_t(const KrylovState& st, double tol, cudaStream_t s) {
  const int nc = krylov_nchunk(st.n);
  dim3 grd(nc, st.nrhs);
  k_finish<<<(st.nrhs + 63) / 64, 64, 0, s>>>(st, nc, tol);
  k_scale_next<T><<<grd, kThreads, 0, s>>>(st);
  k_advance<<<1, 32, 0, s>>>(st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t xupd_t(const KrylovState& st, double2* x, cudaStream_t s) {
  const int nc = krylov_nchunk(st.n);
  k_lsq<<<(st.nrhs + 63) / 64, 64, 0, s>>>(st);
  k_xupdate<T><<<dim3(nc, st.nrhs), kThreads, 0, s>>>(st, x);
  return cudaGetLastError();
}

}  // namespace

int krylov_nchunk(int n) { return (n + kChunk - 1) / kChunk; }

cudaError_t krylov_start(const KrylovState& st, const double2* r0, double, cudaStream_t s) {
  return st.basis_fp32 ? start_t<float2>(st, r0, s) : start_t<double2>(st, r0, s);
}
cudaError_t krylov_orthogonalise(const KrylovState& st, int passes, cudaStream_t s) {
  return st.basis_fp32 ? orth_t<float2>(st, passes, s) : orth_t<double2>(st, passes, s);
}
cudaError_t krylov_finish_step(const KrylovState& st, double tol, cudaStream_t s) {
  return st.basis_fp32 ? finish_t<float2>(st, tol, s) : finish_t<double2>(st, tol, s);
}
cudaError_t krylov_update_solution(const KrylovState& st, double2* x, cudaStream_t s) {
  return st.basis_fp32 ? xupd_t<float2>(st, x, s) : xupd_t<double2>(st, x, s);
}

}  // namespace bem
