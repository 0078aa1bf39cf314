// Batched solves of many independent problems of different sizes (the random-star sweep and the
// serving stream): mixed precision only (complex FP32 matrix + remainder, FP32 Krylov basis, FP64
// refinement), one plane wave per problem.
//
// Each resident problem occupies a slot.  Slots share device pools laid out in "units" of one unknown:
// a slot with n unknowns owns units [u, u+n) of the solution / residual / right-hand-side pools (FP64) and
// of the work-vector pool, and (m+1) n entries of the basis pool.  Every kernel covers all resident slots at
// once through two work lists rebuilt when the membership changes: 64-entry chunks (Arnoldi, scaling) and
// 8-row blocks (matrix-vector products, residuals).  Each slot keeps its own iteration index, so slots
// admitted at different times iterate side by side (continuous batching); a finished inner solve is
// refined (x += V y, residual in double-float arithmetic, FP64 norm) while the others keep iterating.
// The iteration body is captured once per membership as a CUDA graph of `graph_iters` iterations and
// replayed on an internal stream that is ordered after the caller's stream by events.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "givens.cuh"
#include "internal.cuh"

namespace bem {

namespace {

constexpr int kCh = 64;            // entries per chunk
constexpr int kRb = 8;             // rows per row block
constexpr int kMaxM = 1000;

struct VDev {
  int cap, m;
  const float2* const* A;
  const float2* const* Alo;
  const int* n;
  const long long* u;
  float2* V;
  float2* W;
  double2* X;
  double2* R;
  double2* B;
  double2* H;
  double2* cs;
  double2* sn;
  double2* g;
  double2* y;
  double2* hcol;
  double* beta;
  double* hnext;
  double* resid;
  double* tol;
  double* rnorm;
  int* active;
  int* iters;
  int* j;
  int* flag;        // per-slot selector for the start / refine kernels
  const int* cbeg;
  const int* ccnt;
  const int* ch_slot;
  const int* ch_loc;
  int nchunks;
  const int* rb_slot;
  const int* rb_row;
  int nrb;
  double2* part;
  double* npart;
  double* wpart;    // per chunk: ||w||^2 before projection (selective reorthogonalisation)
  int* reo;         // per slot: 1 if the conditional second Gram-Schmidt pass runs this iteration
  int* strict;      // per slot: 1 once a refinement step stagnated (the second pass then always runs)
  int* arrive;      // per slot: first-pass update CTAs done (the last one takes the decision)
  int* n_active;
  // device-side refinement loop (bem_batch_solve_planewave): per-slot solve state kept on the device
  int* state;       // 1 iterating, 2 finished
  int* outer;       // refinement steps done
  int* itot;        // GMRES iterations over all refinement steps
  double* bnorm;    // ||b||
  double* rel;      // relative FP64 residual after the last refinement step
  int* bodies;      // loop bodies run so far (a hard stop against runaway loops)
  double otol, itol;  // outer (refinement) and inner tolerances
  int max_refine;
  int max_bodies;
};

__device__ __forceinline__ float2* vbase(const VDev& d, int s) { return d.V + d.u[s] * (long long)(d.m + 1); }

template <typename F>
__device__ __forceinline__ F wsum(F v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- iteration kernels -------------------------------------------------------------------------

// w = A_hi v_j, one warp per row, 16-byte loads, FP32 products folded into FP64 every 16 steps.
__global__ void __launch_bounds__(256) kv_gemv(VDev d) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = d.rb_slot[blockIdx.x];
  const int r = d.rb_row[blockIdx.x] + warp;
  const int n = d.n[s];
  if (!d.active[s] || r >= n) return;
  const float4* row = reinterpret_cast<const float4*>(d.A[s] + (size_t)r * n);
  const float4* xs = reinterpret_cast<const float4*>(vbase(d, s) + (size_t)d.j[s] * n);
  const int n2 = n >> 1;
  double ax = 0.0, ay = 0.0;
  int c = lane;
  while (c < n2) {
    float px = 0.f, py = 0.f;
#pragma unroll 4
    for (int t = 0; t < 16 && c < n2; ++t, c += 32) {
      const float4 a = __ldcs(row + c);
      const float4 v = xs[c];
      px = fmaf(a.x, v.x, px); px = fmaf(-a.y, v.y, px);
      py = fmaf(a.x, v.y, py); py = fmaf(a.y, v.x, py);
      px = fmaf(a.z, v.z, px); px = fmaf(-a.w, v.w, px);
      py = fmaf(a.z, v.w, py); py = fmaf(a.w, v.z, py);
    }
    ax += (double)px;
    ay += (double)py;
  }
  ax = wsum(ax);
  ay = wsum(ay);
  if (lane == 0) d.W[d.u[s] + r] = make_float2((float)ax, (float)ay);
}

// partial projections <v_i, w> of one chunk; warp w takes i = w, w+8, ...
// mode 0: first pass (warp 0 also records the chunk's ||w||^2 before projection); mode 1: conditional second
// pass, run only for slots whose first pass shrank w below a tenth of its length (the first pass's update
// kernel records the decision in d.reo); mode 2: unconditional second pass.
__global__ void __launch_bounds__(256) kv_dots(VDev d, int mode) {
  const int c = blockIdx.x;
  const int s = d.ch_slot[c];
  if (!d.active[s]) return;
  if (mode == 1 && !d.reo[s]) return;   // decided by the first pass's update kernel
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = d.n[s], j = d.j[s];
  const float2* W = d.W + d.u[s];
  const float2* V = vbase(d, s);
  const int k0 = d.ch_loc[c] * kCh + lane, k1 = k0 + 32;
  const bool in0 = k0 < n, in1 = k1 < n;
  const float2 z = make_float2(0.f, 0.f);
  const float2 w0 = in0 ? W[k0] : z, w1 = in1 ? W[k1] : z;
  if (mode == 0 && warp == 0) {
    const float nw = wsum(w0.x * w0.x + w0.y * w0.y + w1.x * w1.x + w1.y * w1.y);
    if (lane == 0) d.wpart[c] = (double)nw;
  }
  for (int i = warp; i <= j; i += 8) {
    const float2* vi = V + (size_t)i * n;
    const float2 v0 = in0 ? vi[k0] : z, v1 = in1 ? vi[k1] : z;
    float px = v0.x * w0.x + v0.y * w0.y + v1.x * w1.x + v1.y * w1.y;
    float py = v0.x * w0.y - v0.y * w0.x + v1.x * w1.y - v1.y * w1.x;
    px = wsum(px);
    py = wsum(py);
    if (lane == 0) d.part[(size_t)c * (d.m + 1) + i] = make_double2(px, py);
  }
}

__global__ void kv_dots_reduce(VDev d, int pass, int cond) {
  const int s = blockIdx.y;
  if (s >= d.cap || !d.active[s] || (cond && !d.reo[s])) return;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const int j = d.j[s];
  if (i > j) return;
  double hx = 0.0, hy = 0.0;
  const int c0 = d.cbeg[s], cn = d.ccnt[s];
  for (int c = lane; c < cn; c += 32) {
    const double2 v = d.part[(size_t)(c0 + c) * (d.m + 1) + i];
    hx += v.x;
    hy += v.y;
  }
  hx = wsum(hx);
  hy = wsum(hy);
  if (lane == 0) {
    const double2 h = make_double2(hx, hy);
    d.hcol[(size_t)s * (d.m + 1) + i] = h;
    double2* Hj = d.H + ((size_t)s * d.m + j) * (d.m + 1);
    Hj[i] = pass == 0 ? h : cadd(Hj[i], h);
  }
}

__global__ void __launch_bounds__(256) kv_update(VDev d, int pass, int cond) {
  __shared__ float2 hs[kMaxM + 1];
  __shared__ float accs[4][kCh][2];
  __shared__ double red[8];
  const int c = blockIdx.x;
  const int s = d.ch_slot[c];
  if (!d.active[s] || (cond && !d.reo[s])) return;   // cond: a conditional pass the slot did not need
  const int n = d.n[s], j = d.j[s];
  for (int i = threadIdx.x; i <= j; i += 256) {
    const double2 h = d.hcol[(size_t)s * (d.m + 1) + i];
    hs[i] = make_float2((float)h.x, (float)h.y);
  }
  __syncthreads();
  const int e = threadIdx.x & (kCh - 1), sub = threadIdx.x >> 6;
  const int k = d.ch_loc[c] * kCh + e;
  const float2* V = vbase(d, s);
  float ax = 0.f, ay = 0.f;
  if (k < n) {
#pragma unroll 4
    for (int i = sub; i <= j; i += 4) {
      const float2 v = V[(size_t)i * n + k];
      ax += hs[i].x * v.x - hs[i].y * v.y;
      ay += hs[i].x * v.y + hs[i].y * v.x;
    }
  }
  accs[sub][e][0] = ax;
  accs[sub][e][1] = ay;
  __syncthreads();
  double nrm = 0.0;
  if (sub == 0 && k < n) {
    float2* W = d.W + d.u[s];
    float2 w = W[k];
    w.x -= accs[0][e][0] + accs[1][e][0] + accs[2][e][0] + accs[3][e][0];
    w.y -= accs[0][e][1] + accs[1][e][1] + accs[2][e][1] + accs[3][e][1];
    W[k] = w;
    nrm = (double)w.x * w.x + (double)w.y * w.y;
  }
  nrm = wsum(nrm);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
  __syncthreads();
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w8 = 0; w8 < 8; ++w8) t += red[w8];
    d.npart[c] = t;
    if (pass == 0) {
      // the slot's last CTA to finish takes the decision for the conditional second pass (see kv_dots)
      __threadfence();
      s_last = atomicAdd(d.arrive + s, 1) == d.ccnt[s] - 1;
    }
  }
  if (pass != 0) return;
  __syncthreads();
  if (!s_last || threadIdx.x >= 32) return;
  __threadfence();
  // one warp loads the chunk sums in parallel (L2, bypassing L1) and reduces them
  double before = 0.0, after = 0.0;
  const int c0 = d.cbeg[s], cn = d.ccnt[s];
  for (int cc = threadIdx.x; cc < cn; cc += 32) {
    before += __ldcg(d.wpart + c0 + cc);
    after += __ldcg(d.npart + c0 + cc);
  }
  before = wsum(before);
  after = wsum(after);
  if (threadIdx.x == 0) {
    d.reo[s] = d.strict[s] || after < 0.01 * before;   // ||w_after|| < ||w_before|| / 10
    d.arrive[s] = 0;
  }
}

// Hessenberg column, Givens rotations, residual estimate (one warp per slot; see krylov.cu).
__global__ void __launch_bounds__(32) kv_finish(VDev d) {
  __shared__ double2 sh_h[kMaxM + 1], sh_c[kMaxM], sh_s[kMaxM];
  const int s = blockIdx.x, lane = threadIdx.x;
  if (!d.active[s]) return;
  const int j = d.j[s];
  double t = 0.0;
  const int c0 = d.cbeg[s], cn = d.ccnt[s];
  for (int c = lane; c < cn; c += 32) t += d.npart[c0 + c];
  t = wsum(t);
  double2* Hj = d.H + ((size_t)s * d.m + j) * (d.m + 1);
  double2* cs = d.cs + (size_t)s * d.m;
  double2* sn = d.sn + (size_t)s * d.m;
  for (int i = lane; i <= j; i += 32) {
    sh_h[i] = Hj[i];
    if (i < j) { sh_c[i] = cs[i]; sh_s[i] = sn[i]; }
  }
  __syncwarp();
  const double2 a = warp_rotate_column(sh_h, sh_c, sh_s, j);
  for (int i = lane; i < j; i += 32) Hj[i] = sh_h[i];
  if (lane != 0) return;
  const double hn = sqrt(t);
  double den, inv;
  givens_norm(a, hn, den, inv);
  double2 c, sv;
  if (den == 0.0) { c = make_double2(1, 0); sv = make_double2(0, 0); }
  else { c = cscale(a, inv); sv = make_double2(hn * inv, 0.0); }
  cs[j] = c;
  sn[j] = sv;
  Hj[j] = make_double2(den, 0.0);
  Hj[j + 1] = make_double2(0.0, 0.0);
  double2* g = d.g + (size_t)s * (d.m + 1);
  const double2 gj = g[j];
  g[j + 1] = make_double2(-(sv.x * gj.x - sv.y * gj.y), -(sv.x * gj.y + sv.y * gj.x));
  g[j] = cdotc(c, gj);
  const double res = d.resid[s] * sv.x;   // |g_{j+1}| = |s_j| |g_j| (resid starts at 1)
  d.resid[s] = res;
  d.iters[s] = j + 1;
  d.hnext[s] = hn;
  if (res <= d.tol[s] || j + 1 >= d.m || hn == 0.0) d.active[s] = 0;
}

__global__ void __launch_bounds__(kCh) kv_scale(VDev d) {
  const int c = blockIdx.x;
  const int s = d.ch_slot[c];
  if (!d.active[s]) return;
  const int n = d.n[s];
  const int k = d.ch_loc[c] * kCh + threadIdx.x;
  if (k >= n) return;
  const float inv = 1.f / (float)d.hnext[s];   // FP32: an FP64 division per entry is costly
  const float2 w = d.W[d.u[s] + k];
  vbase(d, s)[(size_t)(d.j[s] + 1) * n + k] = make_float2(w.x * inv, w.y * inv);
}

__global__ void kv_advance(VDev d) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < d.cap && d.active[s]) d.j[s] += 1;
}

// ---- start / refine kernels (slots selected by d.flag) -------------------------------------------

// FP64 2-norm of R (or B) of each flagged slot, one block per slot.
__global__ void __launch_bounds__(256) kv_norm(VDev d, int of_b) {
  __shared__ double red[8];
  const int s = blockIdx.x;
  if (!d.flag[s]) return;
  const int n = d.n[s];
  const double2* v = (of_b ? d.B : d.R) + d.u[s];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) acc += v[k].x * v[k].x + v[k].y * v[k].y;
  acc = wsum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    d.rnorm[s] = sqrt(t);
  }
}

// start an inner GMRES on R for flagged slots: beta = rnorm (computed by kv_norm), V_0 = R / beta
__global__ void kv_start_fin(VDev d) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.cap || !d.flag[s]) return;
  const double beta = d.rnorm[s];
  d.beta[s] = beta;
  d.g[(size_t)s * (d.m + 1)] = make_double2(beta, 0.0);
  d.active[s] = beta > 0.0 ? 1 : 0;
  d.iters[s] = 0;
  d.j[s] = 0;
  d.resid[s] = beta > 0.0 ? 1.0 : 0.0;
  d.arrive[s] = 0;
  d.reo[s] = 0;
}

__global__ void __launch_bounds__(kCh) kv_start_scale(VDev d) {
  const int c = blockIdx.x;
  const int s = d.ch_slot[c];
  if (!d.flag[s] || !d.active[s]) return;
  const int n = d.n[s];
  const int k = d.ch_loc[c] * kCh + threadIdx.x;
  if (k >= n) return;
  const double inv = 1.0 / d.beta[s];
  const double2 r = d.R[d.u[s] + k];
  vbase(d, s)[k] = make_float2((float)(r.x * inv), (float)(r.y * inv));
}

// y = H^-1 g (back substitution), one CTA per flagged slot
__global__ void __launch_bounds__(kBsThreads) kv_lsq(VDev d) {
  __shared__ double2 sg[kMaxM], sinv[kMaxM], sy;
  const int s = blockIdx.x;
  if (s >= d.cap || !d.flag[s]) return;
  block_back_substitute(d.H + (size_t)s * d.m * (d.m + 1), d.m + 1, d.g + (size_t)s * (d.m + 1),
                        d.y + (size_t)s * d.m, d.iters[s], sg, sinv, &sy);
}

// x += V y (FP64 x); 64 entries x 4 subsets of i per block
__global__ void __launch_bounds__(256) kv_xupdate(VDev d) {
  __shared__ double2 ys[kMaxM];
  __shared__ double2 accs[4][kCh];
  const int c = blockIdx.x;
  const int s = d.ch_slot[c];
  if (!d.flag[s]) return;
  const int n = d.n[s], mm = d.iters[s];
  for (int i = threadIdx.x; i < mm; i += 256) ys[i] = d.y[(size_t)s * d.m + i];
  __syncthreads();
  const int e = threadIdx.x & (kCh - 1), sub = threadIdx.x >> 6;
  const int k = d.ch_loc[c] * kCh + e;
  const float2* V = vbase(d, s);
  double2 acc = make_double2(0, 0);
  if (k < n)
    for (int i = sub; i < mm; i += 4) {
      const float2 v = V[(size_t)i * n + k];
      acc = cadd(acc, cmul(ys[i], make_double2(v.x, v.y)));
    }
  accs[sub][e] = acc;
  __syncthreads();
  if (sub == 0 && k < n) {
    double2 t = d.X[d.u[s] + k];
    for (int q = 0; q < 4; ++q) t = cadd(t, accs[q][e]);
    d.X[d.u[s] + k] = t;
  }
}

// x split into FP32 hi and lo, written over the (now free) basis of the slot
__global__ void __launch_bounds__(kCh) kv_split(VDev d) {
  const int c = blockIdx.x;
  const int s = d.ch_slot[c];
  if (!d.flag[s]) return;
  const int n = d.n[s];
  const int k = d.ch_loc[c] * kCh + threadIdx.x;
  if (k >= n) return;
  const double2 v = d.X[d.u[s] + k];
  const float hx = (float)v.x, hy = (float)v.y;
  float2* base = vbase(d, s);
  base[k] = make_float2(hx, hy);
  base[n + k] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
}

__device__ __forceinline__ void dot2(float a, float b, float& s, float& c) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  const float t = s + p;
  const float bp = t - s;
  c += ((s - (t - bp)) + (p - bp)) + e;
  s = t;
}

// r = b - (hi + lo) x in double-float arithmetic, one warp per row
__global__ void __launch_bounds__(256) kv_resid(VDev d) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = d.rb_slot[blockIdx.x];
  const int r = d.rb_row[blockIdx.x] + warp;
  if (!d.flag[s]) return;
  const int n = d.n[s];
  if (r >= n) return;
  const float2* ah = d.A[s] + (size_t)r * n;
  const float2* al = d.Alo[s] + (size_t)r * n;
  const float2* xh = vbase(d, s);
  const float2* xl = xh + n;
  float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
  for (int c = lane; c < n; c += 32) {
    const float2 h = __ldcs(ah + c), l = __ldcs(al + c), vh = xh[c], vl = xl[c];
    dot2(h.x, vh.x, sr, cr);
    dot2(-h.y, vh.y, sr, cr);
    dot2(h.x, vh.y, si, ci);
    dot2(h.y, vh.x, si, ci);
    cr = fmaf(h.x, vl.x, cr); cr = fmaf(-h.y, vl.y, cr); cr = fmaf(l.x, vh.x, cr); cr = fmaf(-l.y, vh.y, cr);
    ci = fmaf(h.x, vl.y, ci); ci = fmaf(h.y, vl.x, ci); ci = fmaf(l.x, vh.y, ci); ci = fmaf(l.y, vh.x, ci);
  }
  double re = (double)sr + (double)cr, im = (double)si + (double)ci;
  re = wsum(re);
  im = wsum(im);
  if (lane == 0) {
    const double2 b = d.B[d.u[s] + r];
    d.R[d.u[s] + r] = make_double2(b.x - re, b.y - im);
  }
}

// ---- device-side refinement loop ----------------------------------------------------------------
// The host-stepped engine decides on the host, after each graph replay, which inner solves stopped and
// whether their refined residual meets the tolerance.  For bem_batch_solve_planewave the same decisions run
// on the device, so that the whole solve is one graph launch: a conditional WHILE node whose body is
// graph_iters iterations followed by a refinement stage for the slots whose inner solve stopped.

// flag = the slots whose inner solve stopped (iterating, no longer active)
__global__ void kv_loop_flag(VDev d) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.cap) return;
  d.flag[s] = (d.state[s] == 1 && d.active[s] == 0) ? 1 : 0;
}

// After kv_norm: the host engine's refine_finished decisions for the flagged slots.  A slot that meets the
// tolerance (or used its refinement steps) is finished and unflagged; the others keep their flag and get the
// tolerance of their next inner solve (kv_start_fin / kv_start_scale then restart them).
__global__ void kv_loop_decide(VDev d) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.cap || !d.flag[s]) return;
  const int it = d.iters[s];
  const double rn = d.rnorm[s], bn = d.bnorm[s];
  const double prev = d.outer[s] > 0 ? d.rel[s] : 1.0;
  d.itot[s] += it;
  d.outer[s] += 1;
  const double rel = bn > 0.0 ? rn / bn : 0.0;
  // a step that used every iteration or cut the residual by less than 4x: Gram-Schmidt twice from now on
  if (it >= d.m || rel > 0.25 * prev) d.strict[s] = 1;
  d.rel[s] = rel;
  if (rel <= d.otol || d.outer[s] >= d.max_refine || !(rel == rel)) {
    d.state[s] = 2;
    d.flag[s] = 0;
  } else {
    d.tol[s] = fmax(d.itol, kRefineMargin * d.otol * bn / rn);
  }
}

// The loop condition: some slot still iterating (and the body limit not reached).
__global__ void kv_loop_cond(VDev d, unsigned long long handle) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < d.cap; s += blockDim.x)
    if (d.state[s] == 1) any = 1;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int nb = ++(*d.bodies);
  if (nb >= d.max_bodies && any) {   // cannot happen within the iteration and refinement limits
    for (int s = 0; s < d.cap; ++s)
      if (d.state[s] == 1) { d.state[s] = 2; d.active[s] = 0; }
    any = 0;
  }
  cudaGraphSetConditional((cudaGraphConditionalHandle)handle, any ? 1u : 0u);
}

}  // namespace

// ================================ host engine ====================================================

struct BatchEngine {
  bem_opts o{};
  int cap = 0, m = 0;
  long long units = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // device arrays
  const float2** dA = nullptr;
  const float2** dAlo = nullptr;
  int* dn = nullptr;
  long long* du = nullptr;
  float2* V = nullptr;
  float2* W = nullptr;
  double2 *X = nullptr, *R = nullptr, *Bv = nullptr;
  double2 *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *hcol = nullptr;
  double *beta = nullptr, *hnext = nullptr, *resid = nullptr, *tol = nullptr, *rnorm = nullptr;
  int *active = nullptr, *iters = nullptr, *jj = nullptr, *flag = nullptr, *n_active = nullptr;
  int *cbeg = nullptr, *ccnt = nullptr, *ch_slot = nullptr, *ch_loc = nullptr, *rb_slot = nullptr, *rb_row = nullptr;
  double2* part = nullptr;
  double* npart = nullptr;
  double* wpart = nullptr;
  int* reo = nullptr;
  int* strict = nullptr;
  int* h_strict = nullptr;   // pinned host copy
  int* arrive = nullptr;
  double* angles = nullptr;
  int max_chunks = 0, max_rb = 0;
  int nchunks = 0, nrb = 0;
  // pinned host mirrors
  int* h_active = nullptr;
  int* h_iters = nullptr;
  double* h_rnorm = nullptr;
  int* h_flag = nullptr;
  // graph
  cudaGraphExec_t gexec = nullptr;
  int graph_iters = 4;
  bool dirty = true;
  int asm_ty = 0;
  // device-side refinement loop
  int *state = nullptr, *outer = nullptr, *itot = nullptr, *bodies = nullptr;
  double *bnorm = nullptr, *rel = nullptr;
  cudaGraphExec_t lexec = nullptr;   // the whole-solve graph of the current membership
  bool noloop = false;               // conditional nodes unavailable: host-stepped replays instead
};

}  // namespace bem

// ================================ C interface ====================================================

using namespace bem;

struct BatchSlot {
  int state = 0;            // 0 free, 1 iterating, 2 done (result waiting to be taken)
  bem_problem* p = nullptr;
  int n2 = 0;
  long long u = 0;
  double bnorm = 0.0;
  int iters = 0;
  double resid = 0.0;
  int outer = 0;
  bool strict = false;      // a refinement step stagnated: Gram-Schmidt twice from then on
};

struct bem_batch {
  BatchEngine e;
  std::vector<BatchSlot> slot;
  std::vector<std::pair<long long, long long>> free_runs;   // [start, length) of free units
  std::vector<const float2*> hA, hAlo;
  std::vector<int> hn;
  std::vector<long long> hu;
  std::vector<double> htol;
  std::vector<int> hstrict;
};

namespace {

#define BCU(call)                                                                                      \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) {                                                                           \
      char b_[256];                                                                                    \
      snprintf(b_, sizeof(b_), "%s failed: %s", #call, cudaGetErrorString(e_));                        \
      return report_error(BEM_ECUDA, b_);                                                              \
    }                                                                                                  \
  } while (0)

VDev view(const BatchEngine& e) {
  VDev d;
  d.cap = e.cap; d.m = e.m;
  d.A = e.dA; d.Alo = e.dAlo; d.n = e.dn; d.u = e.du;
  d.V = e.V; d.W = e.W; d.X = e.X; d.R = e.R; d.B = e.Bv;
  d.H = e.H; d.cs = e.cs; d.sn = e.sn; d.g = e.g; d.y = e.y; d.hcol = e.hcol;
  d.beta = e.beta; d.hnext = e.hnext; d.resid = e.resid; d.tol = e.tol; d.rnorm = e.rnorm;
  d.active = e.active; d.iters = e.iters; d.j = e.jj; d.flag = e.flag;
  d.cbeg = e.cbeg; d.ccnt = e.ccnt; d.ch_slot = e.ch_slot; d.ch_loc = e.ch_loc; d.nchunks = e.nchunks;
  d.rb_slot = e.rb_slot; d.rb_row = e.rb_row; d.nrb = e.nrb;
  d.part = e.part; d.npart = e.npart; d.wpart = e.wpart; d.reo = e.reo; d.strict = e.strict; d.arrive = e.arrive; d.n_active = e.n_active;
  d.state = e.state; d.outer = e.outer; d.itot = e.itot; d.bnorm = e.bnorm; d.rel = e.rel; d.bodies = e.bodies;
  d.otol = e.o.tol; d.itol = e.o.inner_tol; d.max_refine = e.o.max_refine;
  // every inner solve stops within m iterations, i.e. m / graph_iters + 1 bodies, and a slot refines at most
  // max_refine times; twice that bounds the loop
  d.max_bodies = 2 * (e.o.max_refine + 1) * (e.m / std::max(1, e.graph_iters) + 2);
  return d;
}

long long take_units(bem_batch* b, long long n) {
  for (auto& r : b->free_runs) {
    if (r.second >= n) {
      const long long u = r.first;
      r.first += n;
      r.second -= n;
      return u;
    }
  }
  return -1;
}

void give_units(bem_batch* b, long long u, long long n) {
  b->free_runs.push_back({u, n});
  std::sort(b->free_runs.begin(), b->free_runs.end());
  std::vector<std::pair<long long, long long>> merged;
  for (auto& r : b->free_runs) {
    if (r.second == 0) continue;
    if (!merged.empty() && merged.back().first + merged.back().second == r.first) merged.back().second += r.second;
    else merged.push_back(r);
  }
  b->free_runs.swap(merged);
}

// Work lists for the slots that are iterating; per-slot arrays.
bem_status rebuild_tables(bem_batch* b) {
  BatchEngine& e = b->e;
  std::vector<int> cbeg(e.cap, 0), ccnt(e.cap, 0), chs, chl, rbs, rbr;
  for (int s = 0; s < e.cap; ++s) {
    const BatchSlot& sl = b->slot[s];
    if (sl.state != 1) continue;
    const int nc = (sl.n2 + kCh - 1) / kCh;
    cbeg[s] = (int)chs.size();
    ccnt[s] = nc;
    for (int c = 0; c < nc; ++c) { chs.push_back(s); chl.push_back(c); }
    for (int r = 0; r < sl.n2; r += kRb) { rbs.push_back(s); rbr.push_back(r); }
  }
  if ((int)chs.size() > e.max_chunks || (int)rbs.size() > e.max_rb) return report_error(BEM_ENOMEM, "work list overflow");
  e.nchunks = (int)chs.size();
  e.nrb = (int)rbs.size();
  BCU(cudaMemcpyAsync(e.cbeg, cbeg.data(), e.cap * sizeof(int), cudaMemcpyHostToDevice, e.st));
  BCU(cudaMemcpyAsync(e.ccnt, ccnt.data(), e.cap * sizeof(int), cudaMemcpyHostToDevice, e.st));
  if (e.nchunks) {
    BCU(cudaMemcpyAsync(e.ch_slot, chs.data(), chs.size() * sizeof(int), cudaMemcpyHostToDevice, e.st));
    BCU(cudaMemcpyAsync(e.ch_loc, chl.data(), chl.size() * sizeof(int), cudaMemcpyHostToDevice, e.st));
    BCU(cudaMemcpyAsync(e.rb_slot, rbs.data(), rbs.size() * sizeof(int), cudaMemcpyHostToDevice, e.st));
    BCU(cudaMemcpyAsync(e.rb_row, rbr.data(), rbr.size() * sizeof(int), cudaMemcpyHostToDevice, e.st));
  }
  BCU(cudaMemcpyAsync(e.dA, b->hA.data(), e.cap * sizeof(void*), cudaMemcpyHostToDevice, e.st));
  BCU(cudaMemcpyAsync(e.dAlo, b->hAlo.data(), e.cap * sizeof(void*), cudaMemcpyHostToDevice, e.st));
  BCU(cudaMemcpyAsync(e.dn, b->hn.data(), e.cap * sizeof(int), cudaMemcpyHostToDevice, e.st));
  BCU(cudaMemcpyAsync(e.du, b->hu.data(), e.cap * sizeof(long long), cudaMemcpyHostToDevice, e.st));
  BCU(cudaMemcpyAsync(e.tol, b->htol.data(), e.cap * sizeof(double), cudaMemcpyHostToDevice, e.st));
  BCU(cudaStreamSynchronize(e.st));   // host vectors are pageable and local
  if (e.gexec) {
    cudaGraphExecDestroy(e.gexec);
    e.gexec = nullptr;
  }
  if (e.lexec) {
    cudaGraphExecDestroy(e.lexec);
    e.lexec = nullptr;
  }
  e.dirty = false;
  return BEM_OK;
}

// passes: 1, 2, or 0 = one pass plus the conditional second one (selective reorthogonalisation)
void enqueue_iteration(const BatchEngine& e, const VDev& d, int passes) {
  if (e.nchunks == 0) return;
  kv_gemv<<<e.nrb, 256, 0, e.st>>>(d);
  const int np = passes == 1 ? 1 : 2;
  for (int p = 0; p < np; ++p) {
    const int mode = p == 0 ? 0 : (passes == 0 ? 1 : 2);
    kv_dots<<<e.nchunks, 256, 0, e.st>>>(d, mode);
    kv_dots_reduce<<<dim3((e.m + 8) / 8, e.cap), 256, 0, e.st>>>(d, p, mode == 1);
    kv_update<<<e.nchunks, 256, 0, e.st>>>(d, p, mode == 1);
  }
  kv_finish<<<e.cap, 32, 0, e.st>>>(d);
  kv_scale<<<e.nchunks, kCh, 0, e.st>>>(d);
  kv_advance<<<(e.cap + 255) / 256, 256, 0, e.st>>>(d);
}

bem_status run_iterations(bem_batch* b) {
  BatchEngine& e = b->e;
  if (e.dirty) {
    bem_status st = rebuild_tables(b);
    if (st != BEM_OK) return st;
  }
  if (e.nchunks == 0) return BEM_OK;
  const VDev d = view(e);
  if (!e.gexec) {
    cudaGraph_t graph;
    BCU(cudaStreamBeginCapture(e.st, cudaStreamCaptureModeThreadLocal));
    for (int it = 0; it < e.graph_iters; ++it) enqueue_iteration(e, d, e.o.orth_passes);
    BCU(cudaStreamEndCapture(e.st, &graph));
    cudaError_t ce = cudaGraphInstantiate(&e.gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return report_error(BEM_ECUDA, "cudaGraphInstantiate failed for the batch iteration");
  }
  BCU(cudaGraphLaunch(e.gexec, e.st));
  return BEM_OK;
}

// Slots flagged in h_flag: after kv_norm has put ||R|| into rnorm, start an inner solve on R.
bem_status start_flagged(bem_batch* b, const std::vector<int>& list) {
  BatchEngine& e = b->e;
  if (list.empty()) return BEM_OK;
  std::fill(e.h_flag, e.h_flag + e.cap, 0);
  for (int s : list) e.h_flag[s] = 1;
  BCU(cudaMemcpyAsync(e.flag, e.h_flag, e.cap * sizeof(int), cudaMemcpyHostToDevice, e.st));
  BCU(cudaMemcpyAsync(e.tol, b->htol.data(), e.cap * sizeof(double), cudaMemcpyHostToDevice, e.st));
  b->hstrict.resize(e.cap);
  for (int s = 0; s < e.cap; ++s) b->hstrict[s] = b->slot[s].strict ? 1 : 0;
  BCU(cudaMemcpyAsync(e.strict, b->hstrict.data(), e.cap * sizeof(int), cudaMemcpyHostToDevice, e.st));
  const VDev d = view(e);
  kv_start_fin<<<(e.cap + 127) / 128, 128, 0, e.st>>>(d);
  if (e.nchunks) kv_start_scale<<<e.nchunks, kCh, 0, e.st>>>(d);
  BCU(cudaGetLastError());
  BCU(cudaStreamSynchronize(e.st));   // htol and hstrict are pageable
  return BEM_OK;
}

// Inner solves that stopped: x += V y, r = b - (hi + lo) x, ||r||; finish or restart each.
bem_status refine_finished(bem_batch* b) {
  BatchEngine& e = b->e;
  BCU(cudaMemcpyAsync(e.h_active, e.active, e.cap * sizeof(int), cudaMemcpyDeviceToHost, e.st));
  BCU(cudaMemcpyAsync(e.h_iters, e.iters, e.cap * sizeof(int), cudaMemcpyDeviceToHost, e.st));
  BCU(cudaStreamSynchronize(e.st));
  std::vector<int> fin;
  for (int s = 0; s < e.cap; ++s)
    if (b->slot[s].state == 1 && e.h_active[s] == 0) fin.push_back(s);
  if (fin.empty()) return BEM_OK;
  std::fill(e.h_flag, e.h_flag + e.cap, 0);
  for (int s : fin) e.h_flag[s] = 1;
  BCU(cudaMemcpyAsync(e.flag, e.h_flag, e.cap * sizeof(int), cudaMemcpyHostToDevice, e.st));
  const VDev d = view(e);
  kv_lsq<<<e.cap, kBsThreads, 0, e.st>>>(d);
  kv_xupdate<<<e.nchunks, 256, 0, e.st>>>(d);
  kv_split<<<e.nchunks, kCh, 0, e.st>>>(d);
  kv_resid<<<e.nrb, 256, 0, e.st>>>(d);
  kv_norm<<<e.cap, 256, 0, e.st>>>(d, 0);
  BCU(cudaGetLastError());
  BCU(cudaMemcpyAsync(e.h_rnorm, e.rnorm, e.cap * sizeof(double), cudaMemcpyDeviceToHost, e.st));
  BCU(cudaStreamSynchronize(e.st));
  std::vector<int> restart;
  for (int s : fin) {
    BatchSlot& sl = b->slot[s];
    const double prev = sl.outer > 0 ? sl.resid : 1.0;   // relative residual before this step
    sl.iters += e.h_iters[s];
    sl.outer += 1;
    const double rel = sl.bnorm > 0 ? e.h_rnorm[s] / sl.bnorm : 0.0;
    // A step that used every iteration or cut the residual by less than 4x: the FP32 basis lost
    // orthogonality under the selective second pass, so from now on the slot runs Gram-Schmidt twice.
    if (e.h_iters[s] >= e.o.max_iter || rel > 0.25 * prev) sl.strict = true;
    sl.resid = rel;
    if (rel <= e.o.tol || sl.outer >= e.o.max_refine) {
      sl.state = 2;
      e.dirty = true;
    } else {
      b->htol[s] = std::max(e.o.inner_tol, kRefineMargin * e.o.tol * sl.bnorm / e.h_rnorm[s]);
      restart.push_back(s);
    }
  }
  return start_flagged(b, restart);
}

// The refinement stage of the device loop for the slots whose inner solve stopped (same kernels as
// refine_finished and start_flagged, with the decisions of kv_loop_decide).
void enqueue_refine_stage(const BatchEngine& e, const VDev& d) {
  const int sb = (e.cap + 127) / 128;
  kv_loop_flag<<<sb, 128, 0, e.st>>>(d);
  kv_lsq<<<e.cap, kBsThreads, 0, e.st>>>(d);
  kv_xupdate<<<e.nchunks, 256, 0, e.st>>>(d);
  kv_split<<<e.nchunks, kCh, 0, e.st>>>(d);
  kv_resid<<<e.nrb, 256, 0, e.st>>>(d);
  kv_norm<<<e.cap, 256, 0, e.st>>>(d, 0);
  kv_loop_decide<<<sb, 128, 0, e.st>>>(d);
  kv_start_fin<<<sb, 128, 0, e.st>>>(d);
  kv_start_scale<<<e.nchunks, kCh, 0, e.st>>>(d);
}

// Iterate every admitted slot to completion as one graph launch (a WHILE node over graph_iters iterations
// and a refinement stage); the slots' results (state, iterations, residual) are read back at the end.
// Returns BEM_ECUDA with e.noloop set if conditional graph nodes are not available (the caller falls back
// to host-stepped replays).
bem_status run_device_loop(bem_batch* b) {
  BatchEngine& e = b->e;
  if (e.dirty) {
    bem_status st = rebuild_tables(b);
    if (st != BEM_OK) return st;
  }
  if (e.nchunks == 0) return BEM_OK;
  // the slots' solve state on the device
  std::vector<int> state(e.cap, 0), outer(e.cap, 0), itot(e.cap, 0), strict(e.cap, 0);
  std::vector<double> bn(e.cap, 0.0), rel(e.cap, 0.0);
  for (int s = 0; s < e.cap; ++s) {
    const BatchSlot& sl = b->slot[s];
    state[s] = sl.state;
    outer[s] = sl.outer;
    itot[s] = sl.iters;
    strict[s] = sl.strict ? 1 : 0;
    bn[s] = sl.bnorm;
    rel[s] = sl.resid;
  }
  BCU(cudaMemcpyAsync(e.state, state.data(), e.cap * sizeof(int), cudaMemcpyHostToDevice, e.st));
  BCU(cudaMemcpyAsync(e.outer, outer.data(), e.cap * sizeof(int), cudaMemcpyHostToDevice, e.st));
  BCU(cudaMemcpyAsync(e.itot, itot.data(), e.cap * sizeof(int), cudaMemcpyHostToDevice, e.st));
  BCU(cudaMemcpyAsync(e.strict, strict.data(), e.cap * sizeof(int), cudaMemcpyHostToDevice, e.st));
  BCU(cudaMemcpyAsync(e.bnorm, bn.data(), e.cap * sizeof(double), cudaMemcpyHostToDevice, e.st));
  BCU(cudaMemcpyAsync(e.rel, rel.data(), e.cap * sizeof(double), cudaMemcpyHostToDevice, e.st));
  BCU(cudaMemsetAsync(e.bodies, 0, sizeof(int), e.st));
  const VDev d = view(e);
  if (!e.lexec) {
    cudaGraph_t graph = nullptr;
    cudaGraphConditionalHandle h = 0;
    cudaError_t ce = cudaGraphCreate(&graph, 0);
    if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (ce == cudaSuccess) ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    if (ce == cudaSuccess) {
      ce = cudaStreamBeginCaptureToGraph(e.st, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal);
      if (ce == cudaSuccess) {
        for (int it = 0; it < e.graph_iters; ++it) enqueue_iteration(e, d, e.o.orth_passes);
        enqueue_refine_stage(e, d);
        kv_loop_cond<<<1, 256, 0, e.st>>>(d, (unsigned long long)h);
        const cudaError_t le = cudaGetLastError();
        cudaGraph_t out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(e.st, &out);
        ce = le != cudaSuccess ? le : ee;
      }
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&e.lexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      e.lexec = nullptr;
      e.noloop = true;
      (void)cudaGetLastError();
      return report_error(BEM_ECUDA, "conditional graph nodes unavailable for the batch loop");
    }
  }
  BCU(cudaGraphLaunch(e.lexec, e.st));
  BCU(cudaMemcpyAsync(state.data(), e.state, e.cap * sizeof(int), cudaMemcpyDeviceToHost, e.st));
  BCU(cudaMemcpyAsync(outer.data(), e.outer, e.cap * sizeof(int), cudaMemcpyDeviceToHost, e.st));
  BCU(cudaMemcpyAsync(itot.data(), e.itot, e.cap * sizeof(int), cudaMemcpyDeviceToHost, e.st));
  BCU(cudaMemcpyAsync(strict.data(), e.strict, e.cap * sizeof(int), cudaMemcpyDeviceToHost, e.st));
  BCU(cudaMemcpyAsync(rel.data(), e.rel, e.cap * sizeof(double), cudaMemcpyDeviceToHost, e.st));
  BCU(cudaStreamSynchronize(e.st));
  for (int s = 0; s < e.cap; ++s) {
    BatchSlot& sl = b->slot[s];
    if (sl.state != 1) continue;
    sl.state = state[s];
    sl.outer = outer[s];
    sl.iters = itot[s];
    sl.strict = strict[s] != 0;
    sl.resid = rel[s];
  }
  e.dirty = true;   // finished slots leave the work lists
  return BEM_OK;
}

// Tile height of the batched assembly chosen by timing, per device (0 = not tuned yet).
constexpr int kTunedDevs = 64;
std::atomic<int> g_tuned_ty[kTunedDevs];

struct StreamScope {
  BatchEngine& e;
  cudaStream_t caller;
  StreamScope(BatchEngine& e_, void* s) : e(e_), caller(static_cast<cudaStream_t>(s)) {
    cudaEventRecord(e.ev_in, caller);
    cudaStreamWaitEvent(e.st, e.ev_in, 0);
  }
  ~StreamScope() {
    cudaEventRecord(e.ev_out, e.st);
    cudaStreamWaitEvent(caller, e.ev_out, 0);
  }
};

template <typename T>
bool dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(1, count) * sizeof(T)) == cudaSuccess;
}

}  // namespace

extern "C" {

BEM_API bem_status bem_batch_create(bem_batch** out, const bem_opts* opts, int max_slots, long long pool_unknowns) {
  if (!out || !opts || max_slots < 1 || max_slots > 65536 || pool_unknowns < 2)
    return report_error(BEM_EINVAL, "invalid argument");
  *out = nullptr;
  if (opts->prec == BEM_PREC_FP64) return report_error(BEM_EINVAL, "batched solves use a mixed precision");
  if (opts->max_iter < 1 || opts->max_iter > kMaxM) return report_error(BEM_EINVAL, "max_iter out of range");
  bem_batch* b = new bem_batch();
  BatchEngine& e = b->e;
  e.o = *opts;
  e.cap = max_slots;
  e.m = opts->max_iter;
  e.units = pool_unknowns;
  const size_t cap = max_slots, m = e.m, U = pool_unknowns;
  e.max_chunks = (int)(U / kCh + cap);
  e.max_rb = (int)(U / kRb + cap);
  bool ok = cudaStreamCreateWithFlags(&e.st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&e.ev_in, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&e.ev_out, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && dalloc(&e.dA, cap) && dalloc(&e.dAlo, cap) && dalloc(&e.dn, cap) && dalloc(&e.du, cap) &&
       dalloc(&e.V, U * (m + 1)) && dalloc(&e.W, U) && dalloc(&e.X, U) && dalloc(&e.R, U) && dalloc(&e.Bv, U) &&
       dalloc(&e.H, cap * m * (m + 1)) && dalloc(&e.cs, cap * m) && dalloc(&e.sn, cap * m) &&
       dalloc(&e.g, cap * (m + 1)) && dalloc(&e.y, cap * m) && dalloc(&e.hcol, cap * (m + 1)) &&
       dalloc(&e.beta, cap) && dalloc(&e.hnext, cap) && dalloc(&e.resid, cap) && dalloc(&e.tol, cap) &&
       dalloc(&e.rnorm, cap) && dalloc(&e.active, cap) && dalloc(&e.iters, cap) && dalloc(&e.jj, cap) &&
       dalloc(&e.flag, cap) && dalloc(&e.n_active, 1) && dalloc(&e.cbeg, cap) && dalloc(&e.ccnt, cap) &&
       dalloc(&e.ch_slot, e.max_chunks) && dalloc(&e.ch_loc, e.max_chunks) && dalloc(&e.rb_slot, e.max_rb) &&
       dalloc(&e.rb_row, e.max_rb) && dalloc(&e.part, (size_t)e.max_chunks * (m + 1)) &&
       dalloc(&e.npart, e.max_chunks) && dalloc(&e.wpart, e.max_chunks) && dalloc(&e.reo, cap) && dalloc(&e.strict, cap) && dalloc(&e.arrive, cap) &&
       dalloc(&e.angles, cap) && dalloc(&e.state, cap) && dalloc(&e.outer, cap) && dalloc(&e.itot, cap) &&
       dalloc(&e.bodies, 1) && dalloc(&e.bnorm, cap) && dalloc(&e.rel, cap);
  ok = ok && cudaMallocHost(&e.h_active, cap * sizeof(int)) == cudaSuccess &&
       cudaMallocHost(&e.h_iters, cap * sizeof(int)) == cudaSuccess &&
       cudaMallocHost(&e.h_rnorm, cap * sizeof(double)) == cudaSuccess &&
       cudaMallocHost(&e.h_flag, cap * sizeof(int)) == cudaSuccess;
  if (ok) ok = cudaMemset(e.active, 0, cap * sizeof(int)) == cudaSuccess && cudaMemset(e.flag, 0, cap * sizeof(int)) == cudaSuccess;
  b->slot.resize(cap);
  b->hA.assign(cap, nullptr);
  b->hAlo.assign(cap, nullptr);
  b->hn.assign(cap, 0);
  b->hu.assign(cap, 0);
  b->htol.assign(cap, opts->inner_tol);
  b->free_runs.push_back({0, pool_unknowns});
  if (!ok) {
    bem_batch_destroy(b);
    return report_error(BEM_ENOMEM, "batch engine allocation failed");
  }
  *out = b;
  return BEM_OK;
}

BEM_API void bem_batch_destroy(bem_batch* b) {
  if (!b) return;
  BatchEngine& e = b->e;
  if (e.st) cudaStreamSynchronize(e.st);
  if (e.gexec) cudaGraphExecDestroy(e.gexec);
  if (e.lexec) cudaGraphExecDestroy(e.lexec);
  void* ptrs[] = {e.dA, e.dAlo, e.dn, e.du, e.V, e.W, e.X, e.R, e.Bv, e.H, e.cs, e.sn, e.g, e.y, e.hcol, e.beta,
                  e.hnext, e.resid, e.tol, e.rnorm, e.active, e.iters, e.jj, e.flag, e.n_active, e.cbeg, e.ccnt,
                  e.ch_slot, e.ch_loc, e.rb_slot, e.rb_row, e.part, e.npart, e.wpart, e.reo, e.strict, e.arrive, e.angles,
                  e.state, e.outer, e.itot, e.bodies, e.bnorm, e.rel};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (e.h_active) cudaFreeHost(e.h_active);
  if (e.h_iters) cudaFreeHost(e.h_iters);
  if (e.h_rnorm) cudaFreeHost(e.h_rnorm);
  if (e.h_flag) cudaFreeHost(e.h_flag);
  if (e.ev_in) cudaEventDestroy(e.ev_in);
  if (e.ev_out) cudaEventDestroy(e.ev_out);
  if (e.st) cudaStreamDestroy(e.st);
  delete b;
}

BEM_API bem_status bem_batch_admit(bem_batch* b, int n, bem_problem* const* probs, const double* angles,
                                   int* slots_out, void* stream) {
  if (!b || n < 0 || (n > 0 && (!probs || !angles || !slots_out))) return report_error(BEM_EINVAL, "invalid argument");
  BatchEngine& e = b->e;
  StreamScope scope(e, stream);
  std::vector<AsmJob> jobs;
  std::vector<int> newslots;
  bool all = true;
  for (int i = 0; i < n; ++i) {
    slots_out[i] = -1;
    if (!std::isfinite(angles[i])) return report_error(BEM_EINVAL, "angle is not finite");
    int s = -1;
    for (int t = 0; t < e.cap; ++t)
      if (b->slot[t].state == 0 && std::find(newslots.begin(), newslots.end(), t) == newslots.end()) { s = t; break; }
    if (s < 0) { all = false; continue; }
    const int n2 = bem_num_unknowns(probs[i]);
    if (n2 < 2) return report_error(BEM_ESTATE, "problem has no elements");
    const long long u = take_units(b, n2);
    if (u < 0) { all = false; continue; }
    AsmJob job;
    bem_opts po;
    bem_status st = problem_prepare_batched(probs[i], e.st, &job, &po);
    if (st != BEM_OK) { give_units(b, u, n2); return st; }
    if (po.quad_order != e.o.quad_order || po.form != e.o.form) {
      give_units(b, u, n2);
      return report_error(BEM_EINVAL, "problem quadrature order / form differ from the batch options");
    }
    jobs.push_back(job);
    newslots.push_back(s);
    BatchSlot& sl = b->slot[s];
    sl = BatchSlot();
    sl.p = probs[i];
    sl.n2 = n2;
    sl.u = u;
    b->hA[s] = static_cast<const float2*>(job.A);
    b->hAlo[s] = static_cast<const float2*>(job.Alo);
    b->hn[s] = n2;
    b->hu[s] = u;
    b->htol[s] = e.o.inner_tol;
    slots_out[i] = s;
  }
  if (jobs.empty()) return all ? BEM_OK : report_error(BEM_ENOMEM, "no slot or pool space free");
  // ---- the admitted problems' matrices: the problems whose Bessel arguments stay below Hankel's expansion
  // first, then the others, one launch per group (the first group's kernel leaves out the reduction of the
  // arguments by pi/2); the tile height is tuned on first use ----
  std::vector<AsmJob> ajobs;
  ajobs.reserve(jobs.size());
  for (const AsmJob& jb : jobs)
    if (!jb.asym) ajobs.push_back(jb);
  const int nplain = (int)ajobs.size();
  for (const AsmJob& jb : jobs)
    if (jb.asym) ajobs.push_back(jb);
  const int group_first[2] = {0, nplain}, group_count[2] = {nplain, (int)ajobs.size() - nplain};
  AsmJob* djobs = nullptr;
  long long* dpref = nullptr;
  BCU(cudaMallocAsync(&djobs, ajobs.size() * sizeof(AsmJob), e.st));
  BCU(cudaMallocAsync(&dpref, ajobs.size() * sizeof(long long), e.st));
  BCU(cudaMemcpyAsync(djobs, ajobs.data(), ajobs.size() * sizeof(AsmJob), cudaMemcpyHostToDevice, e.st));
  const Quad q = make_quad_host(e.o.quad_order);
  // tile prefix sums of jobs [first, first + count), from 0; returns the tiles of the range
  auto prefix_for = [&](int ty, int first, int count, std::vector<long long>& pref) {
    pref.resize(count);
    long long acc = 0;
    for (int i = 0; i < count; ++i) { pref[i] = acc; acc += assemble_batched_tiles(ajobs[first + i].n, ty); }
    return acc;
  };
  std::vector<long long> pref;
  int dev = 0;
  cudaGetDevice(&dev);
  if (e.asm_ty == 0 && dev >= 0 && dev < kTunedDevs) e.asm_ty = g_tuned_ty[dev].load(std::memory_order_relaxed);
  if (e.asm_ty == 0) {
    // Tile height (rows of element pairs per 32-column tile): time 4, 8 and 16 once per device on the first
    // problems of the larger group of this batch (about an eighth of its element pairs, at least one problem),
    // keep the fastest.
    const int g = group_count[0] >= group_count[1] ? 0 : 1;
    long long pairs = 0, all_pairs = 0;
    for (int i = 0; i < group_count[g]; ++i) all_pairs += (long long)ajobs[group_first[g] + i].n * ajobs[group_first[g] + i].n;
    int kjobs = 0;
    while (kjobs < group_count[g] && (kjobs == 0 || pairs * 8 < all_pairs)) {
      pairs += (long long)ajobs[group_first[g] + kjobs].n * ajobs[group_first[g] + kjobs].n;
      ++kjobs;
    }
    const int cand[3] = {4, 8, 16};
    float best = 1e30f;
    int best_ty = 8;
    cudaEvent_t t0, t1;
    BCU(cudaEventCreate(&t0));
    BCU(cudaEventCreate(&t1));
    for (int c = 0; c < 3; ++c) {
      const long long tot = prefix_for(cand[c], group_first[g], kjobs, pref);
      BCU(cudaMemcpyAsync(dpref, pref.data(), pref.size() * sizeof(long long), cudaMemcpyHostToDevice, e.st));
      BCU(cudaEventRecord(t0, e.st));
      BCU(launch_assemble_batched(djobs + group_first[g], kjobs, dpref, tot, q, e.o.form, 1, cand[c], e.st, g == 1));
      BCU(cudaEventRecord(t1, e.st));
      BCU(cudaEventSynchronize(t1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (ms < best) { best = ms; best_ty = cand[c]; }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    e.asm_ty = best_ty;
    if (dev >= 0 && dev < kTunedDevs) g_tuned_ty[dev].store(best_ty, std::memory_order_relaxed);
  }
  std::vector<long long> gpref[2];
  for (int g = 0; g < 2; ++g) {
    if (group_count[g] == 0) continue;
    const long long tot = prefix_for(e.asm_ty, group_first[g], group_count[g], gpref[g]);
    BCU(cudaMemcpyAsync(dpref + group_first[g], gpref[g].data(), gpref[g].size() * sizeof(long long),
                        cudaMemcpyHostToDevice, e.st));
    BCU(launch_assemble_batched(djobs + group_first[g], group_count[g], dpref + group_first[g], tot, q, e.o.form, 1,
                                e.asm_ty, e.st, g == 1));
  }
  BCU(cudaStreamSynchronize(e.st));   // pref / jobs are host-local
  cudaFreeAsync(djobs, e.st);
  cudaFreeAsync(dpref, e.st);
  // ---- right-hand sides, x = 0, r = b, ||b||, first inner solve ----
  std::fill(e.h_flag, e.h_flag + e.cap, 0);
  for (size_t i = 0; i < newslots.size(); ++i) {
    const int s = newslots[i];
    BatchSlot& sl = b->slot[s];
    double ang = 0.0;
    for (int t = 0; t < n; ++t)
      if (slots_out[t] == s) ang = angles[t];
    BCU(cudaMemcpyAsync(e.angles + s, &ang, sizeof(double), cudaMemcpyHostToDevice, e.st));
    BCU(launch_rhs_planewave(problem_elem(sl.p), sl.n2 / 2, problem_dom(sl.p), e.o.form, 1, e.angles + s,
                             e.Bv + sl.u, e.st));
    BCU(cudaMemsetAsync(e.X + sl.u, 0, sl.n2 * sizeof(double2), e.st));
    BCU(cudaMemcpyAsync(e.R + sl.u, e.Bv + sl.u, sl.n2 * sizeof(double2), cudaMemcpyDeviceToDevice, e.st));
    BCU(cudaStreamSynchronize(e.st));   // &ang is a local
    sl.state = 1;
    e.h_flag[s] = 1;
  }
  e.dirty = true;
  bem_status st = rebuild_tables(b);
  if (st != BEM_OK) return st;
  BCU(cudaMemcpyAsync(e.flag, e.h_flag, e.cap * sizeof(int), cudaMemcpyHostToDevice, e.st));
  kv_norm<<<e.cap, 256, 0, e.st>>>(view(e), 1);
  BCU(cudaGetLastError());
  BCU(cudaMemcpyAsync(e.h_rnorm, e.rnorm, e.cap * sizeof(double), cudaMemcpyDeviceToHost, e.st));
  BCU(cudaStreamSynchronize(e.st));
  for (int s : newslots) b->slot[s].bnorm = e.h_rnorm[s];
  st = start_flagged(b, newslots);
  if (st != BEM_OK) return st;
  return all ? BEM_OK : report_error(BEM_ENOMEM, "some problems were not admitted (no slot or pool space)");
}

BEM_API bem_status bem_batch_step(bem_batch* b, int* n_running, void* stream) {
  if (!b) return report_error(BEM_EINVAL, "null batch");
  BatchEngine& e = b->e;
  StreamScope scope(e, stream);
  bem_status st = run_iterations(b);
  if (st != BEM_OK) return st;
  st = refine_finished(b);
  if (st != BEM_OK) return st;
  if (n_running) {
    int r = 0;
    for (auto& sl : b->slot) r += (sl.state == 1);
    *n_running = r;
  }
  return BEM_OK;
}

BEM_API bem_status bem_batch_query(bem_batch* b, int slot, int* state, int* iters, double* resid) {
  if (!b || slot < 0 || slot >= b->e.cap) return report_error(BEM_EINVAL, "invalid slot");
  const BatchSlot& sl = b->slot[slot];
  if (state) *state = sl.state;
  if (iters) *iters = sl.iters;
  if (resid) *resid = sl.resid;
  return BEM_OK;
}

BEM_API bem_status bem_batch_take(bem_batch* b, int slot, bem_c64* x_dev, void* stream) {
  if (!b || slot < 0 || slot >= b->e.cap) return report_error(BEM_EINVAL, "invalid slot");
  BatchEngine& e = b->e;
  BatchSlot& sl = b->slot[slot];
  if (sl.state != 2) return report_error(BEM_ESTATE, "slot has no finished result");
  StreamScope scope(e, stream);
  if (x_dev) BCU(cudaMemcpyAsync(x_dev, e.X + sl.u, sl.n2 * sizeof(double2), cudaMemcpyDeviceToDevice, e.st));
  give_units(b, sl.u, sl.n2);
  sl = BatchSlot();
  b->hA[slot] = b->hAlo[slot] = nullptr;
  b->hn[slot] = 0;
  e.dirty = true;
  return BEM_OK;
}

BEM_API long long bem_batch_free_units(const bem_batch* b) {
  if (!b) return 0;
  long long best = 0;
  for (auto& r : b->free_runs) best = std::max(best, r.second);
  return best;
}

BEM_API bem_status bem_batch_solve_planewave(bem_batch* b, int n, bem_problem* const* probs, const double* angles,
                                             bem_c64* const* x_dev, int* iters, double* resid, void* stream) {
  if (!b || n < 1 || !probs || !angles || !x_dev) return report_error(BEM_EINVAL, "invalid argument");
  std::vector<int> slots(n, -1);
  bem_status st = bem_batch_admit(b, n, probs, angles, slots.data(), stream);
  if (st != BEM_OK) {
    for (int s : slots)
      if (s >= 0) { b->slot[s].state = 2; bem_batch_take(b, s, nullptr, stream); }
    return st;
  }
  // the whole solve as one graph launch (device-side loop); host-stepped replays where that is unavailable
  bool looped = false;
  if (!b->e.noloop) {
    StreamScope scope(b->e, stream);
    st = run_device_loop(b);
    if (st == BEM_OK) looped = true;
    else if (!b->e.noloop) return st;
  }
  int running = looped ? 0 : 1;
  for (int guard = 0; running > 0 && guard < 100000; ++guard) {
    st = bem_batch_step(b, &running, stream);
    if (st != BEM_OK) return st;
  }
  bem_status result = BEM_OK;
  for (int i = 0; i < n; ++i) {
    const BatchSlot& sl = b->slot[slots[i]];
    if (iters) iters[i] = sl.iters;
    if (resid) resid[i] = sl.resid;
    if (sl.resid > b->e.o.tol) result = BEM_ENOCONV;
    st = bem_batch_take(b, slots[i], reinterpret_cast<bem_c64*>(x_dev[i]), stream);
    if (st != BEM_OK) return st;
  }
  if (result == BEM_ENOCONV) report_error(BEM_ENOCONV, "some problems did not reach the tolerance");
  return result;
}

}  // extern "C"
