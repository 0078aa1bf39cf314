// Internal declarations shared by the translation units of libbem (not part of the C interface).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>

#include "bem.h"

namespace bem {

// Programmatic dependent launch for the kernels of one GMRES iteration: launch_pdl lets the next kernel of
// the stream be scheduled while its predecessor drains, and the kernel's first statement, pdl_enter(),
// waits until the predecessor has completed and its writes are visible, then lets its own successor be
// scheduled.  So at most two grids are resident at a time, each reads its inputs only after they are
// complete, and the launch latency of each kernel overlaps the tail of the one before (in stream order
// and in the recorded CUDA graph alike).  Without the launch attribute the two instructions do nothing.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

constexpr int kMaxDomains = 64;
constexpr int kMaxQuad = 16;

// Per-element geometry in structure-of-arrays form (device).  Normal = (-ty, tx).
struct ElemDev {
  const double* ax; const double* ay;   // start vertex
  const double* bx; const double* by;   // end vertex
  double* mx; double* my;               // centre (collocation point)
  double* tx; double* ty;               // unit tangent
  double* h;                            // length
  const int* P; const int* M;           // domain the normal points out of / into
  // double-float copies (hi, lo FP32 pairs) of the tangent and of half the length, for the assembly
  float* txh; float* txl; float* tyh; float* tyl; float* hhh; float* hhl;
};

struct DomTab {
  int n;
  double k[kMaxDomains];
  double eps[kMaxDomains];
  // double-float copies (hi, lo) of k_d, eps_d, gim_d = -1/(k_1 eps_d) and 1/k_1 (domtab_finish)
  float kh[kMaxDomains], kl[kMaxDomains];
  float eh[kMaxDomains], el[kMaxDomains];
  float gh[kMaxDomains], gl[kMaxDomains];
  float ik1h, ik1l;
};
// Fill the double-float copies of a DomTab from k and eps (host).
void domtab_finish(DomTab& d);

struct Quad {
  int Q;
  double t[kMaxQuad];
  double w[kMaxQuad];
  float wh[kMaxQuad], wl[kMaxQuad];   // weights in double-float
  float th[kMaxQuad], tl[kMaxQuad];   // nodes in double-float
};

// One problem of a batched assembly launch.
struct AsmJob {
  ElemDev e;
  int n;           // elements
  DomTab dom;
  void* A;         // hi (mixed) or full (FP64) matrix, 2n x 2n row-major
  void* Alo;       // remainder (mixed) or null
  int asym;        // 1 if a Bessel argument of this problem can reach Hankel's expansion (x >= 128)
};

// ---- complex helpers ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// conj(a) * b
__host__ __device__ __forceinline__ double2 cdotc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// the same for complex FP32
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cdotc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// ---- launchers (each returns cudaGetLastError() of its launch) -----------------------------------
cudaError_t launch_elements(const ElemDev& e, int n, cudaStream_t s);
// asym = false: the caller has checked that no Bessel argument reaches Hankel's expansion (asym_reachable in
// api.cu), so the mixed-store kernel leaves out the reduction of the arguments by pi/2.
cudaError_t launch_assemble(const ElemDev& e, int n, const DomTab& dom, const Quad& q, int form, int store_mixed,
                            void* A, void* Alo, size_t lda, cudaStream_t s, bool asym = true);
// y = A x without a stored matrix (entries recomputed in FP64), n elements, nrhs columns of 2n.
// `gate` (optional, device int): when it reads 0 the product is skipped (every system of the block has
// converged; the solver queues several iterations ahead of its convergence check).
// asym as for launch_assemble.
cudaError_t launch_matvec_free(const ElemDev& e, int n, const DomTab& dom, const Quad& q, int form, int nrhs,
                               const double2* x, double2* y, cudaStream_t s, const int* gate = nullptr,
                               bool asym = true);
// The same for complex FP32 x and y (FP64 sums inside) and only the element rows i0 .. n-1 (matrix rows i and
// n + i): the recomputed part of a partly stored matrix in the FP32 inner solves.
cudaError_t launch_matvec_free_f32(const ElemDev& e, int n, const DomTab& dom, const Quad& q, int form, int i0,
                                   const float2* x, float2* y, cudaStream_t s, const int* gate = nullptr,
                                   bool asym = true);
// Element rows i < rows of the matrix as complex FP32 (hi only) into a compact block: row i at H + i * lda,
// row n + i at H + (rows + i) * lda.
cudaError_t launch_assemble_rows(const ElemDev& e, int n, const DomTab& dom, const Quad& q, int form, int rows,
                                 float2* H, size_t lda, cudaStream_t s, bool asym = true);
// Tiles of a problem with n elements for tile height ty (4, 8 or 16 rows of element pairs x 32 columns).
long long assemble_batched_tiles(int n, int ty);
// Mixed store only (store_mixed = 0 returns cudaErrorNotSupported); asym = false when no job's asym is set.
cudaError_t launch_assemble_batched(const AsmJob* jobs_dev, int njobs, const long long* tile_prefix_dev,
                                   long long total_tiles, const Quad& q, int form, int store_mixed, int ty,
                                   cudaStream_t s, bool asym = true);
cudaError_t launch_rhs_planewave(const ElemDev& e, int n, const DomTab& dom, int form, int nrhs,
                                 const double* angles_dev, double2* b, cudaStream_t s);
// scratch: 2 * nang * n complex entries (the per-angle element sums).
cudaError_t launch_far_field(const ElemDev& e, int n, const DomTab& dom, const Quad& q, int nrhs, const double2* x,
                             int nang, const double* ang_dev, double2* out, double2* scratch, cudaStream_t s);
cudaError_t launch_near_field(const ElemDev& e, int n, const DomTab& dom, const Quad& q, int nrhs, const double2* x,
                              int npts, const double* pts_dev, const int* dom_dev, const double* angles_dev,
                              double2* out, cudaStream_t s);
// Matrix to c64 copy for inspection: which 0 -> main (c64 or hi), 1 -> hi + lo.
cudaError_t launch_matrix_to_c64(const void* A, const void* Alo, int mixed, int which, size_t nn, double2* out,
                                 cudaStream_t s);

// y[r] = A x[r] for nrhs columns; A is n x n row-major (lda).  FP64 path.
cudaError_t launch_matvec_c64(const double2* A, size_t lda, int n, int nrhs, const double2* x, double2* y,
                              cudaStream_t s, const int* gate = nullptr);
// y[r] = A x[r] with A complex FP32 (hi only), x and y complex FP32.
cudaError_t launch_matvec_c32(const float2* A, size_t lda, int n, int nrhs, const float2* x, float2* y,
                              const int* active, cudaStream_t s, const int* gate = nullptr);
// The same product for `rows` consecutive stored rows starting at A, written to rows yoff .. yoff + rows - 1 of y
// (columns of n entries; nrhs 1 or 2).
cudaError_t launch_matvec_c32_rows(const float2* A, size_t lda, int n, int rows, int yoff, int nrhs, const float2* x,
                                   float2* y, cudaStream_t s);
// r = b - (hi + lo) x, with FP64 x, b, r (refinement residual) in double-float arithmetic; ws must hold
// 2 * nrhs * n float2 (ws_bytes: its size, 0 = exactly that).  The _f64 variant computes the same in FP64 arithmetic.
// With ws_bytes beyond the x split, the tiled product may split K over CTAs and keep FP64 partials there.
cudaError_t launch_residual_split(const float2* Ahi, const float2* Alo, size_t lda, int n, int nrhs,
                                  const double2* x, const double2* b, double2* r, void* ws, cudaStream_t s,
                                  size_t ws_bytes = 0, int* nlaunch = nullptr);
// The same residual for problems with the tensor-core product: the small terms hi * x_lo + lo * x_hi are two
// tensor-core products (a16 = FP16 split copy of hi, alo16 = the same of lo; tcws = a tensor-core workspace),
// so the FP32-pipe kernel only sums the exact products hi * x_hi.  ws holds residual_tc_ws_bytes(n, nrhs)
// bytes and more for K-split partials.  Needs 2 <= nrhs <= 64.
size_t residual_tc_ws_bytes(int n, int nrhs);
cudaError_t launch_residual_split_tc(const float2* Ahi, const float2* Alo, size_t lda, const void* a16,
                                     const void* alo16, int n, int nrhs, const double2* x, const double2* b,
                                     double2* r, void* ws, size_t ws_bytes, void* tcws, size_t tcws_bytes,
                                     cudaStream_t s, int* nlaunch = nullptr);
cudaError_t launch_residual_c64(const double2* A, size_t lda, int n, int nrhs, const double2* x, const double2* b,
                                double2* r, cudaStream_t s);
// Load the kernels of launch_residual_split (without a tensor-core workspace) on the current device, so that
// a later call does not load them lazily (which takes device memory).
cudaError_t residual_split_preload();
// Set-up of the no-allocation residual on the current device (noalloc.cu): looks up its static scratch
// array and loads its kernels.  Called where the library allocates anyway (assembly of mixed problems).
bem_status noalloc_setup();
// tcgen05 tensor-core GEMM Y = A X (X / Y complex FP32, 2 <= nrhs <= 64) on the FP16 split copy of A that
// launch_tc_prepare_a makes (matvec_tc_a16_bytes(n) bytes, from the complex FP32 matrix A, n x n).  Returns
// cudaErrorNotSupported if the shape is not supported.  The kernel records a bounded-wait expiry in an
// error word inside ws and never clears it: callers clear it (matvec_tc_clear_error) before a run of
// products and read it (matvec_tc_error_word) afterwards.
// x == nullptr: the block's B operand is already in ws in the FP16 x 3 format with scale 1 (the Krylov kernels
// write it for unit-norm basis vectors; matvec_tc_b_operand gives its place).  stage 0: the whole product;
// 1: operand preparation and the GEMM; 2: the stream-K reduction of a stage-1 call with the same arguments.
// relax (optional, device int): when it reads 0 the product multiplies the FP16 hi parts of A and Bt alone (half
// of A's bytes and of Bt's, a relative error of ~2^-11 of the largest entries): the relaxed products of inexact
// GMRES.
cudaError_t launch_matvec_tc(const void* a16, int n, int nrhs, const float2* x, float2* y, void* ws,
                             size_t ws_bytes, cudaStream_t s, const int* gate = nullptr, int stage = 0,
                             const int* relax = nullptr);
void matvec_tc_b_operand(void* ws, int n, void** bhi, void** blo, size_t* ldb);
size_t matvec_tc_b_bytes(int n);
// One-time settings of the tensor-core kernel (shared-memory limit); call before recording it in a graph.
cudaError_t matvec_tc_setup();
// Main-loop wait limit (ns) of the tensor-core kernels launched from now on; 0 restores the default (2 s).
void matvec_tc_set_wait_ns(unsigned long long ns);
cudaError_t matvec_tc_clear_error(void* ws, int n, int nrhs, cudaStream_t s);
size_t matvec_tc_a16_bytes(int n);
cudaError_t launch_tc_prepare_a(const float2* A, int n, void* a16, cudaStream_t s);
size_t matvec_tc_workspace_bytes(int n, int nrhs);
// Device word where the tensor-core kernel records a bounded-wait expiry (0 = none) inside ws; the next word
// counts the relaxed launches (both cleared by matvec_tc_clear_error).
int* matvec_tc_error_word(void* ws, int n, int nrhs);
bool matvec_tc_supported(int n, int nrhs);
struct TcPartials;
// Where a stage-1 product leaves its stream-K partials (layout in tc_operand.cuh), for a consumer that sums them
// itself instead of the stage-2 reduction; false if the shape is not supported.
bool matvec_tc_partials(const void* a16, int n, int nrhs, void* ws, TcPartials* out);

// Element-wise conversions between complex FP64 and FP32 blocks; column 2-norms of an FP64 block.
cudaError_t launch_convert_c64_c32(const double2* in, float2* out, size_t count, cudaStream_t s);
cudaError_t launch_convert_c32_c64(const float2* in, double2* out, size_t count, cudaStream_t s);
// r = b - r (elementwise)
cudaError_t launch_axpby_neg(const double2* b, double2* r, size_t count, cudaStream_t s);
// r -= y (r complex FP64, y complex FP32), elementwise
cudaError_t launch_sub_c32(double2* r, const float2* y, size_t count, cudaStream_t s);
cudaError_t launch_column_norms(const double2* v, int n, int ncol, double* out, cudaStream_t s);

// GMRES building blocks for nrhs systems sharing one matrix; see krylov.cu.
// The stream-K partials of a tensor-core product (tc_operand.cuh): y[s][r] = (sum over the partial tiles that
// cover r's row tile, in CTA order) / rsc[r] for a B operand of scale 1.
struct TcPartials {
  const float* part = nullptr;   // null: none (the product's result is in the output block)
  const float* rsc = nullptr;    // row scales of A's FP16 split (powers of two)
  int kpt = 0;                   // K-steps per row tile
  int G = 0;                     // CTAs of the product
  long long total = 0;           // (row tile, K-step) pairs
};

constexpr int kSyncStride = 32;   // ints between the barrier counters of two systems

// Relaxed products in the tensor-core inner solves (inexact GMRES: once the residual has fallen, the product may
// be less accurate in inverse proportion, Simoncini and Szyld 2003; Bouras and Fraysse 2005): when every active
// system of the block is within kRelaxFactor of its inner tolerance, the product multiplies the FP16 hi parts of A
// and of the basis block alone (half of the bytes, a relative error of ~2^-11 of the largest entries).  The outer
// refinement's residuals use the full product, so a relaxation too early costs iterations, never accuracy.
// 64-system star, per step: factor 0 (off) 26.25 ms; 10: 25.87 ms (116 iterations, final residual 9.0e-9, the
// last ~10 iterations of each inner solve relaxed: 71 against 94 us per product); 30: 26.65 ms (117, 9.2e-9).
constexpr double kRelaxFactor = 10.0;

// Mixed refinement: each inner solve is asked for kRefineMargin x (the residual reduction that the outer
// tolerance still needs).  The inner solves' residual estimates match the updated residuals closely (on the
// 64-system star the final residuals land at margin x tol: 3.0e-9, 5.0e-9, 7.0e-9, 9.0e-9 for 0.3, 0.5, 0.7,
// 0.9), so the margin only guards against an optimistic estimate; a column that still misses the tolerance gets
// another refinement step.  0.9 against 0.3: 116 against 121 iterations, 27.1 against 28.2 ms per step.
constexpr double kRefineMargin = 0.9;
struct KrylovState {
  int n;            // unknowns per system
  int nrhs;         // systems
  int m;            // Krylov dimension limit
  int basis_fp32;   // 1: V, W are float2; 0: double2
  void* V;          // (m+1) x nrhs x n
  void* W;          // nrhs x n
  double2* H;       // nrhs x m x (m+1)   column j of system s at H + (s*m + j)*(m+1)
  double2* cs;      // nrhs x m
  double2* sn;      // nrhs x m
  double2* g;       // nrhs x (m+1)
  double2* y;       // nrhs x m (least-squares solution)
  double* beta;     // nrhs
  double* hnext;    // nrhs: ||w|| after orthogonalisation
  double2* part;    // scratch: nrhs x krylov_nchunk(n) x (m+1) partial dot products
  double* npart;    // scratch: nrhs x krylov_nchunk(n) partial squared norms
  double* wpart;    // scratch: nrhs x krylov_nchunk(n) partial squared norms of w before projection
  int* reo;         // nrhs: 1 if the conditional second Gram-Schmidt pass runs this iteration
  int* strict;      // nrhs: 1 once a refinement step stagnated (the conditional second pass then always runs)
  int* arrive;      // nrhs: CTAs of the first-pass update kernel done (the last one takes the decision)
  int* sync;        // nrhs x kSyncStride: chunk arrivals of the fused iteration kernel (a per-system barrier;
                    // only ever incremented, zeroed at the start of a run), one 128-byte line per system
  int* err;         // 1: nonzero after a bounded wait of the fused iteration kernel ran out (read by the host)
  double2* hcol;    // nrhs x (m+1): projections of the current pass
  int* active;      // nrhs: 1 while iterating
  int* iters;       // nrhs
  double* resid;    // nrhs: estimated relative residual
  const double* tolv;  // nrhs per-system tolerances (overrides the scalar tol when non-null)
  int* n_active;    // device count of active systems (the gate of queued iterations)
  // Relaxed products (inexact GMRES): relaxed[s] is set once system s's residual estimate is within
  // kRelaxFactor of its tolerance (or it stopped); n_unrelaxed counts the systems not yet there.  While it is 0
  // the tensor-core product may drop A's FP16 remainder (see launch_matvec_tc).
  int* relaxed;     // nrhs
  int* n_unrelaxed;
  int* jdev;        // current iteration index (set by the start kernel, advanced after each iteration)
  int* arrive_all;  // systems whose end-of-iteration CTAs are all done (the last one advances jdev)
  // when non-zero: the cudaGraphConditionalHandle of the graph's loop over iterations; the end-of-iteration
  // kernel sets it to (some system still iterating)
  unsigned long long cond_handle;
  // when non-null (FP32 basis feeding the tensor-core product): every new basis vector is also written as
  // the FP16 x 3 operand of the next product (tc_operand.cuh), rows of stride ldb16
  void* b16hi;
  void* b16lo;
  size_t ldb16;
  // when tc.part is set (fused iteration kernel after a tensor-core product): w is the sum of the product's
  // stream-K partials, which the kernel adds up itself (W is not written)
  TcPartials tc;
};
int krylov_nchunk(int n);
cudaError_t krylov_start(const KrylovState& st, const double2* r0, double tol_unused, cudaStream_t s);
// passes: 1, 2, or 0 = one pass plus a second one for the systems whose w the first pass shrank below a tenth
// of its length (selective reorthogonalisation).
cudaError_t krylov_orthogonalise(const KrylovState& st, int passes, cudaStream_t s);
cudaError_t krylov_finish_step(const KrylovState& st, double tol, cudaStream_t s);   // one kernel
int krylov_orth_launches(const KrylovState& st, int passes);   // kernels of krylov_orthogonalise
// Nonzero if the tail of an iteration (both Gram-Schmidt passes, rotations, next basis vector, index advance)
// runs as one cooperative launch for this state (krylov_fused_step, in place of krylov_orthogonalise and
// krylov_finish_step); then st.err reports an expired barrier wait.
int krylov_fused(const KrylovState& st);
void krylov_set_wait_ns(unsigned long long ns);   // barrier wait limit of the fused kernel (0: default 0.5 s)
void krylov_set_fused(int on);                     // 0: separate kernels even where the fused one is usable
cudaError_t krylov_fused_step(const KrylovState& st, int passes, double tol, cudaStream_t s);
// x += V y; with dout, the correction V y is also written there in complex FP32.
cudaError_t krylov_update_solution(const KrylovState& st, double2* x, cudaStream_t s, float2* dout = nullptr);

// For the batch engine: validate, upload geometry and allocate the mixed-precision matrix of p (without
// assembling it), fill its batched-assembly job and mark the matrix as current.  Also reports the
// problem's options.
bem_status problem_prepare_batched(bem_problem* p, cudaStream_t s, AsmJob* job, bem_opts* opts);
// Q-point Gauss-Legendre rule on [-1, 1] (Newton's method on P_Q).
Quad make_quad_host(int Q);
// Element view and domain table of a problem whose geometry is on the device.
ElemDev problem_elem(bem_problem* p);
DomTab problem_dom(bem_problem* p);

// Read-only view of a problem's assembled mixed-precision matrix (for entry points defined outside
// api.cu).  Returns false if the problem has no current mixed-precision matrix.
bool problem_mixed_matrix(bem_problem* p, const float2** hi, const float2** lo, int* n2);
// Record a failure message for bem_last_error() and return st.
bem_status report_error(bem_status st, const char* msg);

}  // namespace bem
