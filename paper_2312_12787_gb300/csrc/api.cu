// C interface of libbem: problem object, validation, assembly and solve drivers.
//
// The drivers sequence the kernels of assemble.cu, matvec.cu, krylov.cu and gemm_tc.cu on the
// caller's stream.  FP64 path: one unrestarted GMRES (paper Sec. 7) in FP64.  Mixed path: iterative
// refinement in FP64 around inner GMRES runs on the complex FP32 matrix.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace bem;

namespace {

thread_local std::string g_err;

bem_status fail(bem_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CU(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(BEM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_Q (three-term recurrence).
void gauss_legendre(int Q, double* t, double* w) {
  for (int i = 0; i < Q; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (Q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= Q; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (Q == 1) { p1 = x; p0 = 1.0; }
      dp = Q * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    // recompute derivative at the converged node
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= Q; ++k) {
      const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = (Q == 1) ? 1.0 : Q * (x * p1 - p0) / (x * x - 1.0);
    t[i] = x;
    w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

bool valid_opts(const bem_opts* o) {
  return o && o->quad_order >= 1 && o->quad_order <= kMaxQuad && o->form >= 0 && o->form <= 3 && o->prec >= 0 &&
         o->prec <= 2 && o->max_iter >= 1 && o->max_iter <= 1000 && o->max_refine >= 1 && o->max_refine <= 100 &&
         o->tol > 0 && std::isfinite(o->tol) && o->inner_tol > 0 && std::isfinite(o->inner_tol) &&
         (o->orth_passes >= 0 && o->orth_passes <= 2) && (o->matrix_free == 0 || o->matrix_free == 1) &&
         !(o->matrix_free && o->prec == BEM_PREC_MIXED_TC) && o->store_bytes >= 0;
}

}  // namespace

struct bem_problem {
  bem_opts o{};
  DomTab dom{};
  std::vector<double> ax, ay, bx, by;
  std::vector<int> P, M;
  int n = 0;
  bool geom_dirty = true;
  double bbox_diag = -1.0;   // diagonal of the elements' bounding box (< 0: not yet computed for this geometry)
  bool mat_dirty = true;
  // device geometry: ax ay bx by mx my tx ty h (9n doubles), their double-float copies (6n floats), P M
  double* d_geom = nullptr;
  int* d_pm = nullptr;
  size_t geom_cap = 0;
  void* d_A = nullptr;
  void* d_Alo = nullptr;
  size_t A_cap = 0;       // bytes of d_A (and d_Alo when mixed)
  // matrix-free mixed problems: the leading element rows that fit in opts.store_bytes, stored as complex FP32
  // (hi) in a compact block (rows i, then rows N + i, of the stored elements i < Es); the rest is recomputed
  float2* d_Hs = nullptr;
  size_t Hs_cap = 0;
  int Es = 0;
  void* d_A16 = nullptr;  // FP16 split copy of the complex FP32 matrix for the tensor-core product
  size_t A16_cap = 0;
  void* d_Alo16 = nullptr;  // the same of the remainder lo (the residual's small terms)
  size_t Alo16_cap = 0;
  bool a16_dirty = true;
  int A_mixed = -1;
  // solve workspace (grow-only)
  char* ws = nullptr;
  size_t ws_cap = 0;
  double* d_small = nullptr;   // angles etc.
  size_t small_cap = 0;
  int* h_pin = nullptr;        // pinned host mirror of counters
  // tensor-core GMRES iterations recorded as a CUDA graph (replayed on an internal stream)
  cudaGraphExec_t ig_exec = nullptr;
  bool ig_loop = false;      // ig_exec is one device-side loop over iterations (conditional WHILE node)
  bool ig_noloop = false;    // building the loop failed once on this device: use replays of 8 iterations
  const void* ig_ws = nullptr;
  const void* ig_a16 = nullptr;
  int ig_n2 = 0, ig_nrhs = 0, ig_m = 0, ig_passes = -1;
  bool ig_fused = false;
  cudaStream_t ig_stream = nullptr;
  cudaEvent_t ig_ev[3] = {nullptr, nullptr, nullptr};
  // measurement: event pairs per phase, kernel launches per phase
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[BEM_PH_COUNT];
  long long launches[BEM_PH_COUNT] = {};
  std::vector<cudaEvent_t> pool;

  ElemDev elem() const {
    ElemDev e;
    e.ax = d_geom; e.ay = d_geom + n; e.bx = d_geom + 2 * n; e.by = d_geom + 3 * n;
    e.mx = d_geom + 4 * n; e.my = d_geom + 5 * n; e.tx = d_geom + 6 * n; e.ty = d_geom + 7 * n;
    e.h = d_geom + 8 * n;
    float* f = reinterpret_cast<float*>(d_geom + 9 * n);
    e.txh = f; e.txl = f + n; e.tyh = f + 2 * n; e.tyl = f + 3 * n; e.hhh = f + 4 * n; e.hhl = f + 5 * n;
    e.P = d_pm; e.M = d_pm + n;
    return e;
  }
  bool mixed() const { return o.prec != BEM_PREC_FP64; }
};

namespace {

cudaEvent_t pool_event(bem_problem* p) {
  if (!p->pool.empty()) {
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Brackets the launches of one phase with events on stream s when profiling is on.
struct Phase {
  bem_problem* p;
  int ph;
  cudaStream_t s;
  cudaEvent_t b = nullptr;
  Phase(bem_problem* p_, int ph_, cudaStream_t s_, int nlaunch) : p(p_), ph(ph_), s(s_) {
    if (!p->prof) return;
    p->launches[ph] += nlaunch;
    b = pool_event(p);
    if (b) cudaEventRecord(b, s);
  }
  void add_launches(int n) {
    if (p->prof) p->launches[ph] += n;
  }
  ~Phase() {
    if (!b) return;
    cudaEvent_t e = pool_event(p);
    if (!e) return;
    cudaEventRecord(e, s);
    p->ev[ph].push_back({b, e});
  }
};

// ---- device memory of problems ---------------------------------------------------------------------
// Problem buffers (matrix copies, Krylov workspace, geometry) come from a per-device memory pool of this
// library that keeps up to kPoolKeepBytes of freed blocks, so a problem created after another one was
// destroyed (a serving loop, the host-buffer entry point) reuses the memory instead of mapping new pages.
// dev_malloc and dev_free are synchronous like cudaMalloc and cudaFree: the allocation is made on an
// internal stream and waited for (usable on every stream on return); the release is cudaFree.  Without pool
// support they are cudaMalloc and cudaFree.
constexpr uint64_t kPoolKeepBytes = 32ull << 30;
constexpr int kPoolDevs = 64;
struct DevPool {
  std::once_flag once;
  cudaMemPool_t pool = nullptr;
  cudaStream_t s = nullptr;
  bool ok = false;
};
DevPool g_pools[kPoolDevs];

DevPool* dev_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kPoolDevs) return nullptr;
  DevPool& d = g_pools[dev];
  std::call_once(d.once, [&d, dev] {
    int supported = 0;
    if (cudaDeviceGetAttribute(&supported, cudaDevAttrMemoryPoolsSupported, dev) != cudaSuccess || !supported) return;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&d.pool, &props) != cudaSuccess) return;
    uint64_t keep = kPoolKeepBytes;
    if (cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) return;
    if (cudaStreamCreateWithFlags(&d.s, cudaStreamNonBlocking) != cudaSuccess) return;
    d.ok = true;
  });
  return d.ok ? &d : nullptr;
}

cudaError_t dev_malloc(void** ptr, size_t bytes) {
  DevPool* d = dev_pool();
  if (!d) return cudaMalloc(ptr, bytes);
  cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes, d->pool, d->s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(d->s);
}
template <typename T> cudaError_t dev_malloc(T** ptr, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(ptr), bytes);
}

// Stream-ordered scratch of one call (freed with cudaFreeAsync on the same stream), from the same pool.
template <typename T> cudaError_t dev_malloc_async(T** ptr, size_t bytes, cudaStream_t s) {
  DevPool* d = dev_pool();
  if (!d) return cudaMallocAsync(reinterpret_cast<void**>(ptr), bytes, s);
  return cudaMallocFromPoolAsync(reinterpret_cast<void**>(ptr), bytes, d->pool, s);
}

// cudaFree also takes stream-ordered allocations back into their pool (after its implicit synchronisation);
// unlike an explicit device synchronisation it leaves stream captures of other threads intact.
void dev_free(void* ptr) {
  if (ptr) cudaFree(ptr);
}

Quad make_quad(int Q) { return bem::make_quad_host(Q); }

bem_status ensure_small(bem_problem* p, size_t doubles) {
  if (doubles <= p->small_cap) return BEM_OK;
  if (p->d_small) dev_free(p->d_small);
  p->d_small = nullptr;
  p->small_cap = 0;
  CU(dev_malloc(&p->d_small, doubles * sizeof(double)));
  p->small_cap = doubles;
  return BEM_OK;
}

bem_status upload_geometry(bem_problem* p, cudaStream_t s) {
  if (!p->geom_dirty) return BEM_OK;
  const int n = p->n;
  if ((size_t)n > p->geom_cap) {
    if (p->d_geom) dev_free(p->d_geom);
    if (p->d_pm) dev_free(p->d_pm);
    p->d_geom = nullptr;
    p->d_pm = nullptr;
    p->geom_cap = 0;
    CU(dev_malloc(&p->d_geom, (size_t)12 * n * sizeof(double)));   // 9n doubles + 6n floats
    CU(dev_malloc(&p->d_pm, (size_t)2 * n * sizeof(int)));
    p->geom_cap = n;
  }
  CU(cudaMemcpyAsync(p->d_geom, p->ax.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(p->d_geom + n, p->ay.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(p->d_geom + 2 * n, p->bx.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(p->d_geom + 3 * n, p->by.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(p->d_pm, p->P.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(p->d_pm + n, p->M.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  {
    Phase ph(p, BEM_PH_GEOMETRY, s, 1);
    CU(launch_elements(p->elem(), n, s));
  }
  // pageable sources: make sure the copies are done before the host vectors can change
  CU(cudaStreamSynchronize(s));
  p->geom_dirty = false;
  return BEM_OK;
}

bem_status check_ready(bem_problem* p) {
  if (!p) return fail(BEM_EINVAL, "null problem");
  if (p->dom.n < 2) return fail(BEM_ESTATE, "domains not set");
  if (p->n < 1) return fail(BEM_ESTATE, "no segments added");
  for (int e = 0; e < p->n; ++e)
    if (p->P[e] >= p->dom.n || p->M[e] >= p->dom.n)
      return fail(BEM_EINVAL, "element %d refers to a domain beyond the %d set", e, p->dom.n);
  // the self-element series is used for k h / 2 < 8 (elements shorter than ~2.5 wavelengths)
  for (int e = 0; e < p->n; ++e) {
    const double h = std::hypot(p->bx[e] - p->ax[e], p->by[e] - p->ay[e]);
    const double kk = std::max(p->dom.k[p->P[e]], p->dom.k[p->M[e]]);
    if (0.5 * kk * h >= 8.0)
      return fail(BEM_EINVAL, "element %d is %.3g wavelengths long; refine the mesh", e, kk * h / (2 * M_PI));
  }
  return BEM_OK;
}

size_t matrix_bytes(int n, bool mixed) {
  const size_t nn = (size_t)2 * n * 2 * n;
  return mixed ? 2 * nn * sizeof(float2) : nn * sizeof(double2);
}

// Element rows of a matrix-free mixed problem that fit in opts.store_bytes (two rows of 2N complex FP32 each).
int stored_element_rows(const bem_problem* p) {
  const size_t per = (size_t)2 * 2 * p->n * sizeof(float2);
  const size_t rows = (size_t)p->o.store_bytes / per;
  return (int)std::min<size_t>(rows, (size_t)p->n);
}

// Whether any Bessel argument k r of an assembly can reach Hankel's expansion (x >= 128, where the kernel needs the
// arguments reduced by pi/2): every collocation point and every quadrature node lie in the bounding box of the
// element end points, so r is at most its diagonal; a margin of 1 below 128 covers the rounding of k r.
bool asym_reachable(bem_problem* p) {
  if (p->ax.empty()) return false;
  if (p->bbox_diag < 0.0) {   // once per geometry
    double x0 = p->ax[0], x1 = x0, y0 = p->ay[0], y1 = y0;
    for (size_t e = 0; e < p->ax.size(); ++e) {
      x0 = std::min({x0, p->ax[e], p->bx[e]});
      x1 = std::max({x1, p->ax[e], p->bx[e]});
      y0 = std::min({y0, p->ay[e], p->by[e]});
      y1 = std::max({y1, p->ay[e], p->by[e]});
    }
    p->bbox_diag = std::hypot(x1 - x0, y1 - y0);
  }
  double kmax = 0.0;
  for (int d = 0; d < p->dom.n; ++d) kmax = std::max(kmax, std::fabs(p->dom.k[d]));
  return kmax * p->bbox_diag >= 127.0;
}

// y = A_hi x (complex FP32, one column) of a matrix-free mixed problem: the stored rows by the FP32 GEMV, the
// others recomputed (FP64 sums, FP32 result).
cudaError_t matvec_partial_f32(bem_problem* p, const float2* x, float2* y, cudaStream_t s, const int* gate) {
  const int n = p->n, n2 = 2 * n, Es = p->Es;
  cudaError_t e = cudaSuccess;
  if (Es > 0) {
    e = launch_matvec_c32_rows(p->d_Hs, n2, n2, Es, 0, 1, x, y, s);
    if (e == cudaSuccess) e = launch_matvec_c32_rows(p->d_Hs + (size_t)Es * n2, n2, n2, Es, n, 1, x, y, s);
  }
  if (e == cudaSuccess)
    e = launch_matvec_free_f32(p->elem(), n, p->dom, make_quad(p->o.quad_order), p->o.form, Es, x, y, s, gate,
                               asym_reachable(p));
  return e;
}

bem_status assemble_impl(bem_problem* p, cudaStream_t s, bool force = false) {
  bem_status st = check_ready(p);
  if (st != BEM_OK) return st;
  st = upload_geometry(p, s);
  if (st != BEM_OK) return st;
  const bool mixed = p->mixed();
  if (p->o.matrix_free) {      // products recompute the entries (mixed problems may keep a stored part)
    if (!force && !p->mat_dirty) return BEM_OK;
    p->Es = mixed ? stored_element_rows(p) : 0;
    if (p->Es > 0) {
      const size_t need = (size_t)2 * p->Es * 2 * p->n * sizeof(float2);
      if (need > p->Hs_cap) {
        if (p->d_Hs) dev_free(p->d_Hs);
        p->d_Hs = nullptr;
        p->Hs_cap = 0;
        if (dev_malloc(&p->d_Hs, need) != cudaSuccess) return fail(BEM_ENOMEM, "stored rows: %zu bytes failed", need);
        p->Hs_cap = need;
      }
      Phase ph(p, BEM_PH_ASSEMBLE, s, 1);
      CU(launch_assemble_rows(p->elem(), p->n, p->dom, make_quad(p->o.quad_order), p->o.form, p->Es, p->d_Hs,
                              (size_t)2 * p->n, s, asym_reachable(p)));
    }
    p->mat_dirty = false;
    return BEM_OK;
  }
  if (!force && !p->mat_dirty && p->A_mixed == (int)mixed) return BEM_OK;
  const size_t nn = (size_t)2 * p->n * 2 * p->n;
  const size_t need = mixed ? nn * sizeof(float2) : nn * sizeof(double2);
  if (need > p->A_cap || p->A_mixed != (int)mixed) {
    if (p->d_A) dev_free(p->d_A);
    if (p->d_Alo) dev_free(p->d_Alo);
    p->d_A = p->d_Alo = nullptr;
    p->A_cap = 0;
    cudaError_t e = dev_malloc(&p->d_A, need);
    if (e != cudaSuccess) return fail(BEM_ENOMEM, "matrix allocation of %zu bytes failed", need);
    if (mixed) {
      e = dev_malloc(&p->d_Alo, need);
      if (e != cudaSuccess) return fail(BEM_ENOMEM, "matrix allocation of %zu bytes failed", need);
    }
    p->A_cap = need;
  }
  const Quad q = make_quad(p->o.quad_order);
  {
    Phase ph(p, BEM_PH_ASSEMBLE, s, 1);
    CU(launch_assemble(p->elem(), p->n, p->dom, q, p->o.form, mixed ? 1 : 0, p->d_A, p->d_Alo, (size_t)2 * p->n, s,
                       asym_reachable(p)));
  }
  p->A_mixed = mixed;
  p->mat_dirty = false;
  p->a16_dirty = true;
  // the no-allocation residual needs an assembled mixed matrix: its one-time set-up on this device (which
  // takes device memory under lazy module loading) belongs here, where the library allocates anyway
  if (mixed) return noalloc_setup();
  return BEM_OK;
}

// The FP16 split copy of the (mixed) matrix that the tensor-core product reads; made once per assembly.
bem_status ensure_a16(bem_problem* p, cudaStream_t s) {
  if (!p->a16_dirty && p->d_A16) return BEM_OK;
  const int n2 = 2 * p->n;
  const size_t need = matvec_tc_a16_bytes(n2);
  if (need > p->A16_cap) {
    if (p->d_A16) dev_free(p->d_A16);
    p->d_A16 = nullptr;
    p->A16_cap = 0;
    if (dev_malloc(&p->d_A16, need) != cudaSuccess) return fail(BEM_ENOMEM, "matrix allocation of %zu bytes failed", need);
    p->A16_cap = need;
  }
  if (need > p->Alo16_cap) {
    if (p->d_Alo16) dev_free(p->d_Alo16);
    p->d_Alo16 = nullptr;
    p->Alo16_cap = 0;
    if (dev_malloc(&p->d_Alo16, need) != cudaSuccess)
      return fail(BEM_ENOMEM, "matrix allocation of %zu bytes failed", need);
    p->Alo16_cap = need;
  }
  {
    Phase ph(p, BEM_PH_OTHER, s, 2);
    CU(launch_tc_prepare_a(static_cast<const float2*>(p->d_A), n2, p->d_A16, s));
    CU(launch_tc_prepare_a(static_cast<const float2*>(p->d_Alo), n2, p->d_Alo16, s));
  }
  p->a16_dirty = false;
  return BEM_OK;
}

// Workspace carve-out for a GMRES block.
struct Carve {
  char* base;
  size_t off = 0;
  template <typename T> T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* r = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return r;
  }
};

size_t krylov_bytes(int n2, int nrhs, int m, bool fp32) {
  const int nc = krylov_nchunk(n2);
  const size_t tb = fp32 ? sizeof(float2) : sizeof(double2);
  size_t b = 0;
  auto add = [&](size_t x) { b = ((b + 255) & ~(size_t)255) + x; };
  add((size_t)(m + 1) * nrhs * n2 * tb);  // V
  add((size_t)nrhs * n2 * tb);            // W
  add((size_t)nrhs * m * (m + 1) * 16);   // H
  add((size_t)nrhs * m * 16);             // cs
  add((size_t)nrhs * m * 16);             // sn
  add((size_t)nrhs * (m + 1) * 16);       // g
  add((size_t)nrhs * m * 16);             // y
  add((size_t)nrhs * 8);                  // beta
  add((size_t)nrhs * 8);                  // hnext
  add((size_t)nrhs * nc * (m + 1) * 16);  // part
  add((size_t)nrhs * nc * 8);             // npart
  add((size_t)nrhs * nc * 8);             // wpart
  add((size_t)nrhs * 4);                  // reo
  add((size_t)nrhs * 4);                  // strict
  add((size_t)nrhs * 4);                  // arrive
  add((size_t)nrhs * 4 * kSyncStride);    // sync
  add(4);                                 // err
  add((size_t)nrhs * (m + 1) * 16);       // hcol
  add((size_t)nrhs * 4);                  // active
  add((size_t)nrhs * 4);                  // iters
  add((size_t)nrhs * 8);                  // resid
  add((size_t)nrhs * 8);                  // tolv
  add(4);                                 // n_active
  add((size_t)nrhs * 4);                  // relaxed
  add(4);                                 // n_unrelaxed
  add(4);                                 // jdev
  add(4);                                 // arrive_all
  // mixed extras: residual r (FP64), rhs copy of the inner solve (FP32 not needed), tc workspace
  add((size_t)nrhs * n2 * 16);
  add(matvec_tc_workspace_bytes(n2, nrhs));
  add((size_t)nrhs * n2 * 16);            // rhs / scratch block (plane waves)
  add(4096);
  return b + 4096;
}

bem_status ensure_ws(bem_problem* p, size_t bytes) {
  if (bytes <= p->ws_cap) return BEM_OK;
  if (p->ws) dev_free(p->ws);
  p->ws = nullptr;
  p->ws_cap = 0;
  cudaError_t e = dev_malloc(&p->ws, bytes);
  if (e != cudaSuccess) return fail(BEM_ENOMEM, "workspace allocation of %zu bytes failed", bytes);
  p->ws_cap = bytes;
  if (!p->h_pin) CU(cudaMallocHost(&p->h_pin, 64 * sizeof(int)));
  return BEM_OK;
}

struct Solver {
  KrylovState st{};
  double2* r = nullptr;      // FP64 residual block (mixed)
  void* tcws = nullptr;
  size_t tcws_bytes = 0;
  double2* rhs = nullptr;    // plane-wave rhs block
};

Solver carve_solver(bem_problem* p, int nrhs, bool fp32) {
  const int n2 = 2 * p->n, m = p->o.max_iter;
  const int nc = krylov_nchunk(n2);
  const size_t tb = fp32 ? sizeof(float2) : sizeof(double2);
  Carve c{p->ws};
  Solver sv;
  KrylovState& st = sv.st;
  st.n = n2; st.nrhs = nrhs; st.m = m; st.basis_fp32 = fp32 ? 1 : 0;
  st.V = c.take<char>((size_t)(m + 1) * nrhs * n2 * tb);
  st.W = c.take<char>((size_t)nrhs * n2 * tb);
  st.H = c.take<double2>((size_t)nrhs * m * (m + 1));
  st.cs = c.take<double2>((size_t)nrhs * m);
  st.sn = c.take<double2>((size_t)nrhs * m);
  st.g = c.take<double2>((size_t)nrhs * (m + 1));
  st.y = c.take<double2>((size_t)nrhs * m);
  st.beta = c.take<double>(nrhs);
  st.hnext = c.take<double>(nrhs);
  st.part = c.take<double2>((size_t)nrhs * nc * (m + 1));
  st.npart = c.take<double>((size_t)nrhs * nc);
  st.wpart = c.take<double>((size_t)nrhs * nc);
  st.reo = c.take<int>(nrhs);
  st.strict = c.take<int>(nrhs);
  st.arrive = c.take<int>(nrhs);
  st.sync = c.take<int>((size_t)nrhs * kSyncStride);
  st.err = c.take<int>(1);
  st.hcol = c.take<double2>((size_t)nrhs * (m + 1));
  st.active = c.take<int>(nrhs);
  st.iters = c.take<int>(nrhs);
  st.resid = c.take<double>(nrhs);
  st.tolv = c.take<double>(nrhs);
  st.n_active = c.take<int>(1);
  st.relaxed = c.take<int>(nrhs);
  st.n_unrelaxed = c.take<int>(1);
  st.jdev = c.take<int>(1);
  st.arrive_all = c.take<int>(1);
  sv.r = c.take<double2>((size_t)nrhs * n2);
  sv.tcws_bytes = matvec_tc_workspace_bytes(n2, nrhs);
  sv.tcws = c.take<char>(sv.tcws_bytes);
  sv.rhs = c.take<double2>((size_t)nrhs * n2);
  return sv;
}

// Bytes of the Krylov basis of a solver (free scratch outside a GMRES run).
size_t basis_bytes(const Solver& sv) {
  return (size_t)(sv.st.m + 1) * sv.st.nrhs * sv.st.n * (sv.st.basis_fp32 ? sizeof(float2) : sizeof(double2));
}

// One unrestarted GMRES run from x0 = 0 on r0 (FP64 block), adding the correction into x.
bem_status gmres_run(bem_problem* p, Solver& sv, const double2* r0, double2* x, const std::vector<double>& tols,
                     std::vector<int>& iters, std::vector<double>& resid, cudaStream_t s, float2* dout = nullptr) {
  KrylovState& st = sv.st;
  const int n2 = st.n, nrhs = st.nrhs;
  const double tol = tols[0];
  CU(cudaMemcpyAsync(const_cast<double*>(st.tolv), tols.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
  const bool fp32 = st.basis_fp32;
  const size_t tb = fp32 ? sizeof(float2) : sizeof(double2);
  const bool use_tc = fp32 && p->o.prec == BEM_PREC_MIXED_TC && nrhs > 1 && matvec_tc_supported(n2, nrhs);
  struct ClearB {   // the operand pointers belong to this run only
    KrylovState& st;
    ~ClearB() { st.b16hi = st.b16lo = nullptr; }
  } clear_b{st};
  if (use_tc) {
    const bem_status a = ensure_a16(p, s);
    if (a != BEM_OK) return a;
    CU(matvec_tc_clear_error(sv.tcws, n2, nrhs, s));
    // the Krylov kernels write each unit-norm basis vector as the product's FP16 operand (scale 1); rows
    // of absent systems stay zero
    matvec_tc_b_operand(sv.tcws, n2, &st.b16hi, &st.b16lo, &st.ldb16);
    CU(cudaMemsetAsync(sv.tcws, 0, matvec_tc_b_bytes(n2), s));
  }
  {
    Phase ph(p, BEM_PH_GIVENS, s, 3);
    CU(krylov_start(st, r0, tol, s));
  }
  // automatic: two passes for the FP64 basis; for the FP32 basis one pass, and a second one only for the
  // systems whose vector the first pass shrank below a tenth of its length (selective reorthogonalisation)
  const int passes = p->o.orth_passes ? p->o.orth_passes : (fp32 ? 0 : 2);
  const int* gate = st.n_active;
  // decided (and the fused kernel's attributes set) before any graph capture below
  const bool fused = krylov_fused(st) != 0;
  // the fused kernel sums the tensor-core product's stream-K partials itself (no reduction launch)
  if (use_tc && fused && !matvec_tc_partials(p->d_A16, n2, nrhs, sv.tcws, &st.tc)) st.tc = TcPartials{};
  // one iteration: product, orthogonalisation, rotations and scaling of the next basis vector (the kernels read
  // the iteration index from the device; only the non-tensor-core products take the basis vector's address)
  int launched = 0;   // iterations queued by the host loop below (the graph path does not count them)
  auto iteration = [&](int j) -> cudaError_t {
    void* Vj = static_cast<char*>(st.V) + (size_t)j * nrhs * n2 * tb;
    cudaError_t e;
    if (use_tc) {   // the GEMM (B = V_j, written by the Krylov kernels), then its stream-K reduction (which the
                    // fused iteration kernel does itself as it stages w)
      {
        Phase ph(p, BEM_PH_MATVEC, s, 1);
        e = launch_matvec_tc(p->d_A16, n2, nrhs, nullptr, static_cast<float2*>(st.W), sv.tcws, sv.tcws_bytes, s,
                             gate, 1, kRelaxFactor > 0.0 ? st.n_unrelaxed : nullptr);
      }
      if (e != cudaSuccess) return e;
      if (!st.tc.part) {
        Phase ph(p, BEM_PH_REDUCE, s, 1);
        e = launch_matvec_tc(p->d_A16, n2, nrhs, nullptr, static_cast<float2*>(st.W), sv.tcws, sv.tcws_bytes, s,
                             gate, 2);
      }
    } else {
      Phase ph(p, BEM_PH_MATVEC, s, 1);
      if (p->o.matrix_free && fp32) {   // stored rows and recomputed rows, column by column
        e = cudaSuccess;
        for (int r = 0; r < nrhs && e == cudaSuccess; ++r)
          e = matvec_partial_f32(p, static_cast<const float2*>(Vj) + (size_t)r * n2,
                                 static_cast<float2*>(st.W) + (size_t)r * n2, s, gate);
      } else if (p->o.matrix_free) {
        e = launch_matvec_free(p->elem(), p->n, p->dom, make_quad(p->o.quad_order), p->o.form, nrhs,
                               static_cast<const double2*>(Vj), static_cast<double2*>(st.W), s, gate,
                               asym_reachable(p));
      } else if (!fp32) {
        e = launch_matvec_c64(static_cast<const double2*>(p->d_A), n2, n2, nrhs, static_cast<const double2*>(Vj),
                              static_cast<double2*>(st.W), s, gate);
      } else {
        e = launch_matvec_c32(static_cast<const float2*>(p->d_A), n2, n2, nrhs, static_cast<const float2*>(Vj),
                              static_cast<float2*>(st.W), st.active, s, gate);
      }
    }
    if (e != cudaSuccess) return e;
    if (fused) {   // one launch: Gram-Schmidt passes and the end of the iteration
      Phase ph(p, BEM_PH_ARNOLDI, s, 1);
      return krylov_fused_step(st, passes, tol, s);
    }
    {
      Phase ph(p, BEM_PH_ARNOLDI, s, krylov_orth_launches(st, passes));
      e = krylov_orthogonalise(st, passes, s);
    }
    if (e != cudaSuccess) return e;
    Phase ph(p, BEM_PH_GIVENS, s, 1);
    return krylov_finish_step(st, tol, s);
  };
  if (use_tc && !p->prof) {
    // The tensor-core path's launches do not depend on the iteration index, so kGraphIters iterations are
    // recorded once per workspace layout as a CUDA graph and replayed on an internal stream ordered after s.
    // The host reads the active count of one replay while the next one runs.
    constexpr int kGraphIters = 8;
    constexpr int kLoopIters = 4;
    if (!p->ig_stream) {
      CU(cudaStreamCreateWithFlags(&p->ig_stream, cudaStreamNonBlocking));
      for (cudaEvent_t& e : p->ig_ev) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (p->ig_exec && (p->ig_ws != p->ws || p->ig_a16 != p->d_A16 || p->ig_n2 != n2 || p->ig_nrhs != nrhs ||
                       p->ig_m != st.m || p->ig_passes != passes || p->ig_fused != fused)) {
      cudaGraphExecDestroy(p->ig_exec);
      p->ig_exec = nullptr;
    }
    cudaStream_t gs = p->ig_stream;
    if (!p->ig_exec) {
      CU(matvec_tc_setup());
      const cudaStream_t user = s;
      s = gs;   // the iteration body launches on the capturing stream
      cudaError_t ce = cudaErrorNotSupported;
      if (!p->ig_noloop) {
        // One graph for the whole inner solve: a WHILE node whose body is kLoopIters iterations; the
        // iteration's last kernel sets the loop condition to (some system still iterating), so the host does
        // not poll and at most kLoopIters - 1 gated iterations run past convergence (one iteration per body
        // made each pass through the loop cost more than the iterations it saved).
        cudaGraph_t graph = nullptr;
        cudaGraphConditionalHandle h = 0;
        ce = cudaGraphCreate(&graph, 0);
        if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        if (ce == cudaSuccess) ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
        if (ce == cudaSuccess) {
          cudaGraph_t body = cp.conditional.phGraph_out[0];
          ce = cudaStreamBeginCaptureToGraph(gs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
          if (ce == cudaSuccess) {
            st.cond_handle = (unsigned long long)h;
            cudaError_t ie = cudaSuccess;
            for (int k = 0; k < kLoopIters && ie == cudaSuccess; ++k) ie = iteration(0);
            st.cond_handle = 0;
            cudaGraph_t out = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(gs, &out);
            ce = ie != cudaSuccess ? ie : ee;
          }
        }
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&p->ig_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
          p->ig_exec = nullptr;
          p->ig_noloop = true;
          (void)cudaGetLastError();   // clear the failure; the replay form below is recorded instead
        }
        p->ig_loop = ce == cudaSuccess;
      }
      if (!p->ig_loop) {
        CU(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
        ce = cudaSuccess;
        for (int k = 0; k < kGraphIters && ce == cudaSuccess; ++k) ce = iteration(0);
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(gs, &graph);
        if (ce == cudaSuccess) ce = ee;
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&p->ig_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
      }
      s = user;
      if (ce != cudaSuccess) {
        p->ig_exec = nullptr;
        return fail(BEM_ECUDA, "recording the GMRES iteration graph failed: %s", cudaGetErrorString(ce));
      }
      p->ig_ws = p->ws; p->ig_a16 = p->d_A16; p->ig_n2 = n2; p->ig_nrhs = nrhs; p->ig_m = st.m;
      p->ig_passes = passes;
      p->ig_fused = fused;
    }
    CU(cudaEventRecord(p->ig_ev[2], s));
    CU(cudaStreamWaitEvent(gs, p->ig_ev[2], 0));
    if (p->ig_loop) {
      CU(cudaGraphLaunch(p->ig_exec, gs));
    } else {
      for (int j = 0, r = 0; j < st.m; j += kGraphIters, ++r) {
        CU(cudaGraphLaunch(p->ig_exec, gs));
        CU(cudaMemcpyAsync(p->h_pin + (r & 1), st.n_active, sizeof(int), cudaMemcpyDeviceToHost, gs));
        CU(cudaEventRecord(p->ig_ev[r & 1], gs));
        if (r > 0) {
          CU(cudaEventSynchronize(p->ig_ev[(r - 1) & 1]));
          if (p->h_pin[(r - 1) & 1] == 0) break;
        }
      }
    }
    CU(cudaEventRecord(p->ig_ev[2], gs));
    CU(cudaStreamWaitEvent(s, p->ig_ev[2], 0));
  } else {
    // Iterations are queued kSyncEvery at a time before the host reads the active count: the GPU never
    // waits for the host between iterations.  Once every system has converged, the queued iterations find
    // their gates closed (n_active = 0, active flags cleared) and return at once.
    constexpr int kSyncEvery = 4;
    for (int j = 0; j < st.m; ++j) {
      CU(iteration(j));
      ++launched;
      if ((j + 1) % kSyncEvery == 0) {
        CU(cudaMemcpyAsync(p->h_pin, st.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (p->h_pin[0] == 0) break;
      }
    }
  }
  {
    Phase ph(p, BEM_PH_UPDATE, s, 2);
    CU(krylov_update_solution(st, x, s, dout));
  }
  std::vector<int> it(nrhs);
  std::vector<double> rs(nrhs);
  CU(cudaMemcpyAsync(it.data(), st.iters, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(rs.data(), st.resid, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  int tc_words[2] = {0, 0}, orth_err = 0;   // error word, relaxed launches
  if (use_tc)
    CU(cudaMemcpyAsync(tc_words, matvec_tc_error_word(sv.tcws, n2, nrhs), 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  const int tc_err = tc_words[0];
  if (fused) CU(cudaMemcpyAsync(&orth_err, st.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (tc_err) return fail(BEM_ETIMEOUT, "tensor-core GEMM wait expired (code %d)", tc_err);
  if (orth_err) return fail(BEM_ETIMEOUT, "a per-system barrier wait of the Gram-Schmidt kernel expired");
  for (int r = 0; r < nrhs; ++r) {
    iters[r] += it[r];
    resid[r] = rs[r];
  }
  if (p->prof && launched > 0) {
    // Iterations queued past the last system's convergence found their gates closed: their product launches
    // did no work, so the per-launch figures of the product phases count only the launches that did.
    const int worked = *std::max_element(it.begin(), it.end());
    const int gated = std::max(0, launched - worked);
    p->launches[BEM_PH_MATVEC] -= gated;
    if (use_tc && !st.tc.part) p->launches[BEM_PH_REDUCE] -= gated;
  }
  if (p->prof && use_tc) {
    // the run's relaxed products (counted on the device; the error word's neighbour is cleared per run)
    p->launches[BEM_PH_RELAXED] += tc_words[1];
  }
  return BEM_OK;
}

// The refinement residual r = b - (hi + lo) x of a mixed problem.  Problems that use the tensor-core product
// form the small terms hi x_lo + lo x_hi on the tensor cores (the FP32 pipes then only sum the exact products
// hi x_hi); that path waits for the stream to read the product's error word.  ws = the solver's basis
// (free outside a GMRES run).
bem_status residual_mixed(bem_problem* p, Solver& sv, int nrhs, const double2* x, const double2* b, double2* r,
                          cudaStream_t s);

// column 2-norms of an FP64 block (host result)
bem_status column_norms(bem_problem* p, Solver& sv, const double2* v, int nrhs, std::vector<double>& out,
                        cudaStream_t s);

// The refinement residual updated by a correction: r -= A d, with the correction d (complex FP32, in the
// solver's work block W) multiplied by the inner solves' own product (tensor-core GEMM or FP32 GEMV/GEMM).
bem_status residual_update(bem_problem* p, Solver& sv, int nrhs, double2* r, cudaStream_t s);

}  // namespace

namespace bem {
cudaError_t launch_column_norms(const double2* v, int n, int nrhs, double* out, cudaStream_t s);
}

namespace {
bem_status column_norms(bem_problem* p, Solver& sv, const double2* v, int nrhs, std::vector<double>& out,
                        cudaStream_t s) {
  {
    Phase ph(p, BEM_PH_OTHER, s, 1);
    CU(launch_column_norms(v, sv.st.n, nrhs, sv.st.beta, s));
  }
  out.resize(nrhs);
  CU(cudaMemcpyAsync(out.data(), sv.st.beta, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return BEM_OK;
}

bem_status residual_mixed(bem_problem* p, Solver& sv, int nrhs, const double2* x, const double2* b, double2* r,
                          cudaStream_t s) {
  const int n2 = 2 * p->n;
  if (p->o.matrix_free) {   // every entry recomputed, FP64 sums: r = b - A x
    Phase ph(p, BEM_PH_RESIDUAL, s, nrhs + 1);
    CU(launch_matvec_free(p->elem(), p->n, p->dom, make_quad(p->o.quad_order), p->o.form, nrhs, x, r, s, nullptr,
                          asym_reachable(p)));
    CU(launch_axpby_neg(b, r, (size_t)nrhs * n2, s));
    return BEM_OK;
  }
  const float2* A = static_cast<const float2*>(p->d_A);
  const float2* Alo = static_cast<const float2*>(p->d_Alo);
  if (p->o.prec == BEM_PREC_MIXED_TC && nrhs > 1 && matvec_tc_supported(n2, nrhs) &&
      basis_bytes(sv) >= residual_tc_ws_bytes(n2, nrhs)) {
    const bem_status a = ensure_a16(p, s);
    if (a != BEM_OK) return a;
    CU(matvec_tc_clear_error(sv.tcws, n2, nrhs, s));
    int nl = 0, tc_err = 0;
    {
      Phase ph(p, BEM_PH_RESIDUAL, s, 0);
      CU(launch_residual_split_tc(A, Alo, n2, p->d_A16, p->d_Alo16, n2, nrhs, x, b, r, sv.st.V, basis_bytes(sv),
                                  sv.tcws, sv.tcws_bytes, s, &nl));
      ph.add_launches(nl);
    }
    CU(cudaMemcpyAsync(&tc_err, matvec_tc_error_word(sv.tcws, n2, nrhs), sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (tc_err) return fail(BEM_ETIMEOUT, "tensor-core GEMM wait expired (code %d)", tc_err);
    return BEM_OK;
  }
  Phase ph(p, BEM_PH_RESIDUAL, s, 0);
  int nl = 0;
  CU(launch_residual_split(A, Alo, n2, n2, nrhs, x, b, r, sv.st.V, s, basis_bytes(sv), &nl));
  ph.add_launches(nl);   // split of x, double-float product [, combination of the K splits]
  return BEM_OK;
}

bem_status residual_update(bem_problem* p, Solver& sv, int nrhs, double2* r, cudaStream_t s) {
  const int n2 = 2 * p->n;
  const float2* d = static_cast<const float2*>(sv.st.W);
  float2* y = static_cast<float2*>(sv.st.V);   // the basis is free between GMRES runs
  const bool tc = p->o.prec == BEM_PREC_MIXED_TC && nrhs > 1 && matvec_tc_supported(n2, nrhs);
  int tc_err = 0;
  {
    Phase ph(p, BEM_PH_RESIDUAL, s, tc ? 5 : 2);   // [column maxima, operand, GEMM, reduction | product], r -= y
    if (tc) {
      const bem_status a = ensure_a16(p, s);
      if (a != BEM_OK) return a;
      CU(matvec_tc_clear_error(sv.tcws, n2, nrhs, s));
      CU(launch_matvec_tc(p->d_A16, n2, nrhs, d, y, sv.tcws, sv.tcws_bytes, s));
      CU(cudaMemcpyAsync(&tc_err, matvec_tc_error_word(sv.tcws, n2, nrhs), sizeof(int), cudaMemcpyDeviceToHost, s));
    } else if (p->o.matrix_free) {
      for (int c = 0; c < nrhs; ++c) CU(matvec_partial_f32(p, d + (size_t)c * n2, y + (size_t)c * n2, s, nullptr));
    } else {
      CU(launch_matvec_c32(static_cast<const float2*>(p->d_A), n2, n2, nrhs, d, y, nullptr, s));
    }
    CU(launch_sub_c32(r, y, (size_t)nrhs * n2, s));
  }
  if (tc) {
    CU(cudaStreamSynchronize(s));
    if (tc_err) return fail(BEM_ETIMEOUT, "tensor-core GEMM wait expired (code %d)", tc_err);
  }
  return BEM_OK;
}

bem_status solve_impl(bem_problem* p, int nrhs, const double2* b, double2* x, int* iters_h, double* resid_h,
                      cudaStream_t s) {
  bem_status st = assemble_impl(p, s);
  if (st != BEM_OK) return st;
  const int n2 = 2 * p->n;
  const bool mixed = p->mixed();
  st = ensure_ws(p, krylov_bytes(n2, nrhs, p->o.max_iter, mixed));
  if (st != BEM_OK) return st;
  Solver sv = carve_solver(p, nrhs, mixed);
  std::vector<int> iters(nrhs, 0);
  std::vector<double> resid(nrhs, 0.0);
  CU(cudaMemsetAsync(x, 0, (size_t)nrhs * n2 * sizeof(double2), s));
  CU(cudaMemsetAsync(sv.st.strict, 0, nrhs * sizeof(int), s));
  bem_status result = BEM_OK;
  if (!mixed) {
    st = gmres_run(p, sv, b, x, std::vector<double>(nrhs, p->o.tol), iters, resid, s);
    if (st != BEM_OK) return st;
    for (int r = 0; r < nrhs; ++r)
      if (resid[r] > p->o.tol) result = BEM_ENOCONV;
  } else {
    std::vector<double> bn, rn;
    st = column_norms(p, sv, b, nrhs, bn, s);
    if (st != BEM_OK) return st;
    CU(cudaMemcpyAsync(sv.r, b, (size_t)nrhs * n2 * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    rn = bn;
    std::vector<int> strict(nrhs, 0);
    std::vector<char> met(nrhs, 0);   // the column met the tolerance; resid[r] keeps its residual from then on
    bool done = false;
    for (int outer = 0; outer < p->o.max_refine && !done; ++outer) {
      // zero the residual of columns that meet the tolerance so the inner solve skips them
      done = true;
      for (int r = 0; r < nrhs; ++r) {
        if (met[r]) continue;
        resid[r] = bn[r] > 0 ? rn[r] / bn[r] : 0.0;
        if (resid[r] <= p->o.tol) {
          met[r] = 1;
          CU(cudaMemsetAsync(sv.r + (size_t)r * n2, 0, n2 * sizeof(double2), s));
        } else {
          done = false;
        }
      }
      if (done) break;
      // each column's inner run only needs to reach what the outer tolerance still asks of it
      std::vector<double> inner_res(nrhs), tols(nrhs);
      for (int r = 0; r < nrhs; ++r)
        tols[r] = rn[r] > 0 ? std::max(p->o.inner_tol, kRefineMargin * p->o.tol * bn[r] / rn[r]) : 1.0;
      const std::vector<int> it_before = iters;
      const std::vector<double> rn_before = rn;
      // Once the residual is below 1e-4 of ||b||, it is updated, r -= A d, with the inner solves' own product of
      // the correction d: d is then a small fraction of x (its relative size follows the residual's), so the
      // product's ~3e-7 relative error enters r at ~3e-7 |A| |d|, far below the tolerance, and the double-float
      // residual b - (hi + lo) x is formed only until then.  Tolerances below 1e-11 keep exact residuals.
      double worst = 0.0;
      for (int r = 0; r < nrhs; ++r)
        if (!met[r]) worst = std::max(worst, bn[r] > 0 ? rn[r] / bn[r] : 0.0);
      const bool update = outer > 0 && p->o.tol >= 1e-11 && worst <= 1e-4;
      st = gmres_run(p, sv, sv.r, x, tols, iters, inner_res, s, update ? static_cast<float2*>(sv.st.W) : nullptr);
      if (st != BEM_OK) return st;
      st = update ? residual_update(p, sv, nrhs, sv.r, s) : residual_mixed(p, sv, nrhs, x, b, sv.r, s);
      if (st != BEM_OK) return st;
      st = column_norms(p, sv, sv.r, nrhs, rn, s);
      if (st != BEM_OK) return st;
      // A column whose step used every iteration or cut its residual by less than 4x lost orthogonality in
      // its FP32 basis under the selective second pass: from now on it runs Gram-Schmidt twice.
      bool changed = false;
      for (int r = 0; r < nrhs; ++r) {
        if (strict[r] || met[r]) continue;
        if (iters[r] - it_before[r] >= p->o.max_iter || rn[r] > 0.25 * rn_before[r]) {
          strict[r] = 1;
          changed = true;
        }
      }
      if (changed) CU(cudaMemcpyAsync(sv.st.strict, strict.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    for (int r = 0; r < nrhs; ++r) {
      if (!met[r]) resid[r] = bn[r] > 0 ? rn[r] / bn[r] : 0.0;
      if (resid[r] > p->o.tol) result = BEM_ENOCONV;
    }
  }
  if (iters_h) std::copy(iters.begin(), iters.end(), iters_h);
  if (resid_h) std::copy(resid.begin(), resid.end(), resid_h);
  if (result == BEM_ENOCONV) fail(BEM_ENOCONV, "tolerance not reached within the iteration limits");
  return result;
}

bem_status rhs_impl(bem_problem* p, int nrhs, const double* angles_h, double2* b, cudaStream_t s) {
  bem_status st = check_ready(p);
  if (st != BEM_OK) return st;
  st = upload_geometry(p, s);
  if (st != BEM_OK) return st;
  for (int r = 0; r < nrhs; ++r)
    if (!std::isfinite(angles_h[r])) return fail(BEM_EINVAL, "angle %d is not finite", r);
  st = ensure_small(p, nrhs);
  if (st != BEM_OK) return st;
  CU(cudaMemcpyAsync(p->d_small, angles_h, nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
  {
    Phase ph(p, BEM_PH_RHS, s, 1);
    CU(launch_rhs_planewave(p->elem(), p->n, p->dom, p->o.form, nrhs, p->d_small, b, s));
  }
  CU(cudaStreamSynchronize(s));   // angles_h may be pageable
  return BEM_OK;
}

}  // namespace

namespace bem {
Quad make_quad_host(int Q) {
  Quad q{};
  q.Q = Q;
  gauss_legendre(Q, q.t, q.w);
  for (int m = 0; m < Q; ++m) {
    q.wh[m] = (float)q.w[m];
    q.wl[m] = (float)(q.w[m] - (double)q.wh[m]);
    q.th[m] = (float)q.t[m];
    q.tl[m] = (float)(q.t[m] - (double)q.th[m]);
  }
  return q;
}

void domtab_finish(DomTab& d) {
  auto split = [](double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
  };
  for (int i = 0; i < d.n; ++i) {
    split(d.k[i], d.kh[i], d.kl[i]);
    split(d.eps[i], d.eh[i], d.el[i]);
    split(-1.0 / (d.k[0] * d.eps[i]), d.gh[i], d.gl[i]);
  }
  split(1.0 / d.k[0], d.ik1h, d.ik1l);
}
bool problem_mixed_matrix(bem_problem* p, const float2** hi, const float2** lo, int* n2) {
  if (!p || !p->mixed() || p->mat_dirty || p->A_mixed != 1 || !p->d_A || !p->d_Alo) return false;
  *hi = static_cast<const float2*>(p->d_A);
  *lo = static_cast<const float2*>(p->d_Alo);
  *n2 = 2 * p->n;
  return true;
}
bem_status report_error(bem_status st, const char* msg) { return fail(st, "%s", msg); }
ElemDev problem_elem(bem_problem* p) { return p->elem(); }
DomTab problem_dom(bem_problem* p) { return p->dom; }
bem_status problem_prepare_batched(bem_problem* p, cudaStream_t s, AsmJob* job, bem_opts* opts) {
  if (!p) return fail(BEM_EINVAL, "null problem");
  if (!p->mixed()) return fail(BEM_EINVAL, "batched solves need a mixed-precision problem");
  if (p->o.matrix_free) return fail(BEM_EINVAL, "batched solves store every matrix (no matrix-free problems)");
  bem_status st = check_ready(p);
  if (st != BEM_OK) return st;
  st = upload_geometry(p, s);
  if (st != BEM_OK) return st;
  const size_t nn = (size_t)2 * p->n * 2 * p->n;
  const size_t need = nn * sizeof(float2);
  if (need > p->A_cap || p->A_mixed != 1) {
    if (p->d_A) dev_free(p->d_A);
    if (p->d_Alo) dev_free(p->d_Alo);
    p->d_A = p->d_Alo = nullptr;
    p->A_cap = 0;
    if (dev_malloc(&p->d_A, need) != cudaSuccess || dev_malloc(&p->d_Alo, need) != cudaSuccess) {
      if (p->d_A) dev_free(p->d_A);
      p->d_A = nullptr;
      return fail(BEM_ENOMEM, "matrix allocation of 2 x %zu bytes failed", need);
    }
    p->A_cap = need;
  }
  job->e = p->elem();
  job->n = p->n;
  job->dom = p->dom;
  job->A = p->d_A;
  job->Alo = p->d_Alo;
  job->asym = asym_reachable(p) ? 1 : 0;
  p->A_mixed = 1;
  p->mat_dirty = false;
  p->a16_dirty = true;
  *opts = p->o;
  return noalloc_setup();   // as in assemble_impl
}
}  // namespace bem

// ================================== C interface ==================================================

extern "C" {

BEM_API void bem_default_opts(bem_opts* o) {
  if (!o) return;
  o->quad_order = 4;
  o->form = BEM_FORM_MOD;
  o->prec = BEM_PREC_FP64;
  o->max_iter = 500;
  o->max_refine = 6;
  o->tol = 1e-10;
  o->inner_tol = 1e-5;
  o->orth_passes = 0;
  o->matrix_free = 0;
  o->store_bytes = 0;
}

BEM_API bem_status bem_problem_create(bem_problem** out, const bem_opts* opts) {
  if (!out) return fail(BEM_EINVAL, "null output pointer");
  *out = nullptr;
  bem_opts o;
  bem_default_opts(&o);
  if (opts) o = *opts;
  if (!valid_opts(&o)) return fail(BEM_EINVAL, "invalid options");
  bem_problem* p = new bem_problem();
  p->o = o;
  *out = p;
  return BEM_OK;
}

BEM_API void bem_problem_destroy(bem_problem* p) {
  if (!p) return;
  if (p->d_geom) dev_free(p->d_geom);
  if (p->d_pm) dev_free(p->d_pm);
  if (p->d_A) dev_free(p->d_A);
  if (p->d_Alo) dev_free(p->d_Alo);
  if (p->d_Hs) dev_free(p->d_Hs);
  if (p->d_A16) dev_free(p->d_A16);
  if (p->d_Alo16) dev_free(p->d_Alo16);
  if (p->ws) dev_free(p->ws);
  if (p->d_small) dev_free(p->d_small);
  if (p->h_pin) cudaFreeHost(p->h_pin);
  if (p->ig_exec) cudaGraphExecDestroy(p->ig_exec);
  for (cudaEvent_t e : p->ig_ev)
    if (e) cudaEventDestroy(e);
  if (p->ig_stream) cudaStreamDestroy(p->ig_stream);
  for (int k = 0; k < BEM_PH_COUNT; ++k)
    for (auto& pr : p->ev[k]) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (auto e : p->pool) cudaEventDestroy(e);
  delete p;
}

BEM_API bem_status bem_set_opts(bem_problem* p, const bem_opts* opts) {
  if (!p || !valid_opts(opts)) return fail(BEM_EINVAL, "invalid options");
  if (opts->quad_order != p->o.quad_order || opts->form != p->o.form || opts->prec != p->o.prec ||
      opts->matrix_free != p->o.matrix_free || opts->store_bytes != p->o.store_bytes)
    p->mat_dirty = true;
  p->o = *opts;
  return BEM_OK;
}

BEM_API bem_status bem_set_domains(bem_problem* p, int n_dom, const double* k, const double* eps) {
  if (!p || !k || !eps) return fail(BEM_EINVAL, "null argument");
  if (n_dom < 2 || n_dom > kMaxDomains) return fail(BEM_EINVAL, "n_dom must be in [2, %d]", kMaxDomains);
  for (int d = 0; d < n_dom; ++d) {
    if (!(k[d] > 0) || !std::isfinite(k[d])) return fail(BEM_EINVAL, "k[%d] must be positive and finite", d);
    if (!(eps[d] > 0) || !std::isfinite(eps[d])) return fail(BEM_EINVAL, "eps[%d] must be positive and finite", d);
  }
  if (eps[0] != 1.0) return fail(BEM_EINVAL, "eps[0] (host medium) must be 1");
  p->dom.n = n_dom;
  for (int d = 0; d < n_dom; ++d) {
    p->dom.k[d] = k[d];
    p->dom.eps[d] = eps[d];
  }
  domtab_finish(p->dom);
  p->mat_dirty = true;
  return BEM_OK;
}

BEM_API bem_status bem_add_segment(bem_problem* p, int n_vert, const double* xy, int dom_P, int dom_M, int closed) {
  if (!p || !xy) return fail(BEM_EINVAL, "null argument");
  if (n_vert < (closed ? 3 : 2)) return fail(BEM_EINVAL, "too few vertices (%d)", n_vert);
  if (dom_P < 0 || dom_M < 0 || dom_P >= kMaxDomains || dom_M >= kMaxDomains || dom_P == dom_M)
    return fail(BEM_EINVAL, "invalid domain pair (%d, %d)", dom_P, dom_M);
  for (int v = 0; v < 2 * n_vert; ++v)
    if (!std::isfinite(xy[v])) return fail(BEM_EINVAL, "vertex coordinate %d is not finite", v);
  const int ne = closed ? n_vert : n_vert - 1;
  for (int e = 0; e < ne; ++e) {
    const int a = e, b = (e + 1) % n_vert;
    if (xy[2 * a] == xy[2 * b] && xy[2 * a + 1] == xy[2 * b + 1])
      return fail(BEM_EINVAL, "zero-length element %d", e);
  }
  for (int e = 0; e < ne; ++e) {
    const int a = e, b = (e + 1) % n_vert;
    p->ax.push_back(xy[2 * a]);
    p->ay.push_back(xy[2 * a + 1]);
    p->bx.push_back(xy[2 * b]);
    p->by.push_back(xy[2 * b + 1]);
    p->P.push_back(dom_P);
    p->M.push_back(dom_M);
  }
  p->n += ne;
  p->geom_dirty = true;
  p->bbox_diag = -1.0;
  p->mat_dirty = true;
  return BEM_OK;
}

BEM_API int bem_num_elements(const bem_problem* p) { return p ? p->n : 0; }
BEM_API int bem_num_unknowns(const bem_problem* p) { return p ? 2 * p->n : 0; }

BEM_API size_t bem_footprint_bytes(const bem_problem* p, int n_rhs) {
  if (!p || n_rhs < 1) return 0;
  const bool mixed = p->o.prec != BEM_PREC_FP64;
  const size_t a16 =
      (!p->o.matrix_free && p->o.prec == BEM_PREC_MIXED_TC && n_rhs > 1) ? 2 * matvec_tc_a16_bytes(2 * p->n) : 0;
  const size_t stored = mixed ? (size_t)2 * stored_element_rows(p) * 2 * p->n * sizeof(float2) : 0;
  return (p->o.matrix_free ? stored : matrix_bytes(p->n, mixed)) + a16 + krylov_bytes(2 * p->n, n_rhs, p->o.max_iter, mixed) +
         (size_t)12 * p->n * 8;
}

BEM_API bem_status bem_assemble(bem_problem* p, void* stream) {
  return assemble_impl(p, static_cast<cudaStream_t>(stream), true);
}

BEM_API bem_status bem_get_matrix(bem_problem* p, int which, bem_c64* A_dev, void* stream) {
  if (!p || !A_dev) return fail(BEM_EINVAL, "null argument");
  if (which != 0 && which != 1) return fail(BEM_EINVAL, "which must be 0 or 1");
  if (p->o.matrix_free) return fail(BEM_ESTATE, "matrix-free problems store no matrix");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bem_status st = assemble_impl(p, s);
  if (st != BEM_OK) return st;
  if (which == 1 && !p->mixed()) return fail(BEM_EINVAL, "which = 1 needs a mixed-precision problem");
  const size_t nn = (size_t)2 * p->n * 2 * p->n;
  CU(launch_matrix_to_c64(p->d_A, p->d_Alo, p->mixed() ? 1 : 0, which, nn, reinterpret_cast<double2*>(A_dev), s));
  return BEM_OK;
}

BEM_API bem_status bem_rhs_planewave(bem_problem* p, int n_rhs, const double* angles, bem_c64* b_dev, void* stream) {
  if (!p || !angles || !b_dev || n_rhs < 1) return fail(BEM_EINVAL, "invalid argument");
  return rhs_impl(p, n_rhs, angles, reinterpret_cast<double2*>(b_dev), static_cast<cudaStream_t>(stream));
}

BEM_API bem_status bem_matvec(bem_problem* p, int n_rhs, const bem_c64* x_dev, bem_c64* y_dev, void* stream) {
  if (!p || !x_dev || !y_dev || n_rhs < 1) return fail(BEM_EINVAL, "invalid argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bem_status st = assemble_impl(p, s);
  if (st != BEM_OK) return st;
  const int n2 = 2 * p->n;
  const double2* x = reinterpret_cast<const double2*>(x_dev);
  double2* y = reinterpret_cast<double2*>(y_dev);
  if (p->o.matrix_free) {
    Phase ph(p, BEM_PH_MATVEC, s, n_rhs);
    CU(launch_matvec_free(p->elem(), p->n, p->dom, make_quad(p->o.quad_order), p->o.form, n_rhs, x, y, s, nullptr,
                          asym_reachable(p)));
    return BEM_OK;
  }
  if (!p->mixed()) {
    Phase ph(p, BEM_PH_MATVEC, s, 1);
    CU(launch_matvec_c64(static_cast<const double2*>(p->d_A), n2, n2, n_rhs, x, y, s));
    return BEM_OK;
  }
  // mixed: convert x to complex FP32, run the solver's kernel, widen the result
  st = ensure_ws(p, krylov_bytes(n2, n_rhs, p->o.max_iter, true));
  if (st != BEM_OK) return st;
  Solver sv = carve_solver(p, n_rhs, true);
  float2* xf = static_cast<float2*>(sv.st.V);
  float2* yf = static_cast<float2*>(sv.st.W);
  {
    Phase ph(p, BEM_PH_OTHER, s, 1);
    CU(launch_convert_c64_c32(x, xf, (size_t)n_rhs * n2, s));
  }
  {
    const bool tc = p->o.prec == BEM_PREC_MIXED_TC && n_rhs > 1 && matvec_tc_supported(n2, n_rhs);
    Phase ph(p, BEM_PH_MATVEC, s, tc ? 4 : 1);   // tensor cores: column maxima, operand, GEMM, reduction
    if (tc) {
      st = ensure_a16(p, s);
      if (st != BEM_OK) return st;
      CU(matvec_tc_clear_error(sv.tcws, n2, n_rhs, s));
      CU(launch_matvec_tc(p->d_A16, n2, n_rhs, xf, yf, sv.tcws, sv.tcws_bytes, s));
      int tc_err = 0;
      CU(cudaMemcpyAsync(&tc_err, matvec_tc_error_word(sv.tcws, n2, n_rhs), sizeof(int), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      if (tc_err) return fail(BEM_ETIMEOUT, "tensor-core GEMM wait expired (code %d)", tc_err);
    } else {
      CU(launch_matvec_c32(static_cast<const float2*>(p->d_A), n2, n2, n_rhs, xf, yf, nullptr, s));
    }
  }
  {
    Phase ph(p, BEM_PH_OTHER, s, 1);
    CU(launch_convert_c32_c64(yf, y, (size_t)n_rhs * n2, s));
  }
  return BEM_OK;
}

BEM_API bem_status bem_residual(bem_problem* p, int n_rhs, const bem_c64* x_dev, const bem_c64* b_dev, bem_c64* r_dev,
                                void* stream) {
  if (!p || !x_dev || !b_dev || !r_dev || n_rhs < 1) return fail(BEM_EINVAL, "invalid argument");
  if ((const void*)r_dev == (const void*)x_dev) return fail(BEM_EINVAL, "r_dev must not alias x_dev");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bem_status st = assemble_impl(p, s);
  if (st != BEM_OK) return st;
  const int n2 = 2 * p->n;
  const double2* x = reinterpret_cast<const double2*>(x_dev);
  const double2* b = reinterpret_cast<const double2*>(b_dev);
  double2* r = reinterpret_cast<double2*>(r_dev);
  if (p->o.matrix_free) {
    Phase ph(p, BEM_PH_RESIDUAL, s, 2);
    // r = b - A x with recomputed entries: product into r, then r = b - r
    CU(launch_matvec_free(p->elem(), p->n, p->dom, make_quad(p->o.quad_order), p->o.form, n_rhs, x, r, s, nullptr,
                          asym_reachable(p)));
    CU(launch_axpby_neg(b, r, (size_t)n_rhs * n2, s));
    return BEM_OK;
  }
  if (!p->mixed()) {
    Phase ph(p, BEM_PH_RESIDUAL, s, 1);
    CU(launch_residual_c64(static_cast<const double2*>(p->d_A), n2, n2, n_rhs, x, b, r, s));
    return BEM_OK;
  }
  st = ensure_ws(p, krylov_bytes(n2, n_rhs, p->o.max_iter, true));
  if (st != BEM_OK) return st;
  Solver sv = carve_solver(p, n_rhs, true);
  return residual_mixed(p, sv, n_rhs, x, b, r, s);
}

BEM_API bem_status bem_solve(bem_problem* p, int n_rhs, const bem_c64* b_dev, bem_c64* x_dev, int* iters,
                             double* resid, void* stream) {
  if (!p || !b_dev || !x_dev || n_rhs < 1) return fail(BEM_EINVAL, "invalid argument");
  return solve_impl(p, n_rhs, reinterpret_cast<const double2*>(b_dev), reinterpret_cast<double2*>(x_dev), iters,
                    resid, static_cast<cudaStream_t>(stream));
}

BEM_API bem_status bem_solve_planewave(bem_problem* p, int n_rhs, const double* angles, bem_c64* x_dev, int* iters,
                                       double* resid, void* stream) {
  if (!p || !angles || !x_dev || n_rhs < 1) return fail(BEM_EINVAL, "invalid argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bem_status st = assemble_impl(p, s);
  if (st != BEM_OK) return st;
  const int n2 = 2 * p->n;
  st = ensure_ws(p, krylov_bytes(n2, n_rhs, p->o.max_iter, p->mixed()));
  if (st != BEM_OK) return st;
  Solver sv = carve_solver(p, n_rhs, p->mixed());
  st = rhs_impl(p, n_rhs, angles, sv.rhs, s);
  if (st != BEM_OK) return st;
  return solve_impl(p, n_rhs, sv.rhs, reinterpret_cast<double2*>(x_dev), iters, resid, s);
}

BEM_API bem_status bem_far_field(bem_problem* p, int n_rhs, const bem_c64* x_dev, int n_ang, const double* ang,
                                 bem_c64* out_dev, void* stream) {
  if (!p || !x_dev || !ang || !out_dev || n_rhs < 1 || n_ang < 1) return fail(BEM_EINVAL, "invalid argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bem_status st = check_ready(p);
  if (st != BEM_OK) return st;
  st = upload_geometry(p, s);
  if (st != BEM_OK) return st;
  // d_small: the angles, then the per-angle element sums (2 x n_ang x N complex)
  const size_t ang_slots = ((size_t)n_ang + 1) & ~(size_t)1;   // keep the complex part 16-byte aligned
  st = ensure_small(p, ang_slots + (size_t)4 * n_ang * p->n);
  if (st != BEM_OK) return st;
  CU(cudaMemcpyAsync(p->d_small, ang, n_ang * sizeof(double), cudaMemcpyHostToDevice, s));
  const Quad q = make_quad(p->o.quad_order);
  {
    Phase ph(p, BEM_PH_FARFIELD, s, 2);
    CU(launch_far_field(p->elem(), p->n, p->dom, q, n_rhs, reinterpret_cast<const double2*>(x_dev), n_ang,
                        p->d_small, reinterpret_cast<double2*>(out_dev),
                        reinterpret_cast<double2*>(p->d_small + ang_slots), s));
  }
  CU(cudaStreamSynchronize(s));
  return BEM_OK;
}

BEM_API bem_status bem_near_field(bem_problem* p, int n_rhs, const bem_c64* x_dev, const double* angles,
                                  int n_pts, const double* pts, const int* dom, bem_c64* out_dev, void* stream) {
  if (!p || !x_dev || !pts || !dom || !out_dev || n_rhs < 1 || n_pts < 1) return fail(BEM_EINVAL, "invalid argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bem_status st = check_ready(p);
  if (st != BEM_OK) return st;
  for (int i = 0; i < n_pts; ++i) {
    if (dom[i] < 0 || dom[i] >= p->dom.n) return fail(BEM_EINVAL, "point %d: domain %d out of range", i, dom[i]);
    if (!std::isfinite(pts[2 * i]) || !std::isfinite(pts[2 * i + 1])) return fail(BEM_EINVAL, "point %d not finite", i);
  }
  st = upload_geometry(p, s);
  if (st != BEM_OK) return st;
  // points, domains and angles travel in one temporary device block
  const size_t bytes = (size_t)2 * n_pts * sizeof(double) + (size_t)n_rhs * sizeof(double) + (size_t)n_pts * sizeof(int);
  char* blk = nullptr;
  CU(dev_malloc_async(&blk, bytes, s));
  double* dp = reinterpret_cast<double*>(blk);
  double* da = dp + 2 * (size_t)n_pts;
  int* dd = reinterpret_cast<int*>(da + n_rhs);
  CU(cudaMemcpyAsync(dp, pts, 2 * (size_t)n_pts * sizeof(double), cudaMemcpyHostToDevice, s));
  if (angles) CU(cudaMemcpyAsync(da, angles, n_rhs * sizeof(double), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(dd, dom, n_pts * sizeof(int), cudaMemcpyHostToDevice, s));
  {
    Phase ph(p, BEM_PH_FARFIELD, s, 1);
    CU(launch_near_field(p->elem(), p->n, p->dom, make_quad(p->o.quad_order), n_rhs,
                         reinterpret_cast<const double2*>(x_dev), n_pts, dp, dd, angles ? da : nullptr,
                         reinterpret_cast<double2*>(out_dev), s));
  }
  CU(cudaFreeAsync(blk, s));
  CU(cudaStreamSynchronize(s));   // host arrays may be pageable
  return BEM_OK;
}

BEM_API bem_status bem_solve_planewave_host(bem_problem* p, int n_rhs, const double* angles, bem_c64* x_host,
                                            int n_ang, const double* ff_ang, bem_c64* ff_host, int* iters,
                                            double* resid, void* stream) {
  if (!p || !angles || n_rhs < 1) return fail(BEM_EINVAL, "invalid argument");
  if (ff_host && (!ff_ang || n_ang < 1)) return fail(BEM_EINVAL, "far-field angles missing");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n2 = (size_t)2 * (p->n);
  double2* xd = nullptr;
  double2* ffd = nullptr;
  CU(dev_malloc_async(&xd, n_rhs * n2 * sizeof(double2), s));
  if (ff_host) CU(dev_malloc_async(&ffd, (size_t)n_rhs * n_ang * sizeof(double2), s));
  bem_status st = bem_solve_planewave(p, n_rhs, angles, reinterpret_cast<bem_c64*>(xd), iters, resid, stream);
  if (st == BEM_OK || st == BEM_ENOCONV) {
    if (ff_host) {
      bem_status st2 = bem_far_field(p, n_rhs, reinterpret_cast<bem_c64*>(xd), n_ang, ff_ang,
                                     reinterpret_cast<bem_c64*>(ffd), stream);
      if (st2 != BEM_OK) st = st2;
      else CU(cudaMemcpyAsync(ff_host, ffd, (size_t)n_rhs * n_ang * sizeof(double2), cudaMemcpyDeviceToHost, s));
    }
    if (x_host) CU(cudaMemcpyAsync(x_host, xd, n_rhs * n2 * sizeof(double2), cudaMemcpyDeviceToHost, s));
  }
  cudaFreeAsync(xd, s);
  if (ffd) cudaFreeAsync(ffd, s);
  CU(cudaStreamSynchronize(s));
  return st;
}

BEM_API bem_status bem_profile_enable(bem_problem* p, int on) {
  if (!p) return fail(BEM_EINVAL, "null problem");
  for (int k = 0; k < BEM_PH_COUNT; ++k) {
    for (auto& pr : p->ev[k]) {
      cudaEventSynchronize(pr.second);
      p->pool.push_back(pr.first);
      p->pool.push_back(pr.second);
    }
    p->ev[k].clear();
    p->launches[k] = 0;
  }
  p->prof = on != 0;
  return BEM_OK;
}

BEM_API bem_status bem_profile_read(bem_problem* p, double* ms, long long* launches) {
  if (!p) return fail(BEM_EINVAL, "null problem");
  for (int k = 0; k < BEM_PH_COUNT; ++k) {
    double t = 0.0;
    for (auto& pr : p->ev[k]) {
      CU(cudaEventSynchronize(pr.second));
      float f = 0.f;
      CU(cudaEventElapsedTime(&f, pr.first, pr.second));
      t += f;
    }
    if (ms) ms[k] = t;
    if (launches) launches[k] = p->launches[k];
  }
  return BEM_OK;
}

BEM_API bem_status bem_test_set_wait_limit(double seconds) {
  if (!(seconds >= 0.0) || seconds > 10.0) return fail(BEM_EINVAL, "wait limit must be in [0, 10] s");
  matvec_tc_set_wait_ns((unsigned long long)(seconds * 1e9));
  krylov_set_wait_ns((unsigned long long)(seconds * 1e9));
  return BEM_OK;
}

BEM_API bem_status bem_test_set_fused_iteration(int on) {
  krylov_set_fused(on);
  return BEM_OK;
}

BEM_API const char* bem_last_error(void) { return g_err.c_str(); }

BEM_API const char* bem_version(void) { return "libbem 0.1 (sm_103a)"; }

}  // extern "C"
