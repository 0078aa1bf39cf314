/*
 * bem.h - C interface of the GB300 Burton-Miller collocation BEM library (libbem).
 *
 * The library assembles and solves the collocation system A y = b of the Calderon-preconditioned
 * Burton-Miller formulation for two-dimensional Helmholtz transmission problems
 * (Matsumoto, Yoshiki, Isakari, arXiv 2312.12787):
 *   - Sec. 2: domains Omega_d with wavenumber k_d and flux coefficient eps_d (w = (1/eps_d) du/dn,
 *     eps_1 = 1), u and w continuous across interfaces, radiation condition in the host Omega_1.
 *   - Sec. 3.3: operators S, D, D*, N with G = (i/4) H0^(1)(k r) (eqs. stmp .. ddtmp, fundamental_sol),
 *     Burton-Miller coefficient alpha = -i/k_1.
 *   - Sec. 5 (eq. calderon_bieb, beta = -alpha) and Sec. 6 (eq. 3dom_calderon_bie, gamma = alpha/eps;
 *     the general recipe at the end of Sec. 6): placement of standard and Burton-Miller rows.
 *   - Sec. 7: constant elements, collocation at element centres, Gauss-Legendre quadrature, GMRES
 *     without restart from x0 = 0.
 *
 * Conventions for every entry point:
 *   - Complex numbers are bem_c64 {re, im} (16 bytes, layout-compatible with double _Complex).
 *   - Pointers named *_dev are CUDA device pointers on the current device; pointers named *_host are
 *     host pointers.  The caller owns every buffer it passes; the library owns the assembled matrix,
 *     the Krylov workspace and any scratch it allocates (freed by bem_problem_destroy).  These come from
 *     a per-device memory pool of the library that keeps up to 32 GiB of freed blocks for the next
 *     problem (so creating problems one after another maps no new pages); allocation and release are
 *     synchronous, and a release waits for the device to be idle, as cudaFree does.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Device work is
 *     stream-ordered on it.  Entry points that return host values (iteration counts, residuals,
 *     host outputs) synchronise the stream before returning.
 *   - Unknown order: y = [u_1 .. u_N, w_1 .. w_N], elements numbered segment by segment in the order
 *     the segments were added, and along each segment in vertex order.  Multiple right-hand sides are
 *     stored one after another: column r of a block X is X + r*2N.
 *   - Every function returns a bem_status; on failure bem_last_error() gives a message (thread-local).
 *     Nothing is written to outputs after an argument error.  BEM_ENOCONV still writes the best iterate.
 *   - Not thread-safe on one bem_problem; distinct problems may be used from distinct threads.
 */
#ifndef BEM_H_
#define BEM_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(_WIN32)
#define BEM_API
#else
#define BEM_API __attribute__((visibility("default")))
#endif

typedef struct { double re, im; } bem_c64;

typedef enum {
  BEM_OK = 0,
  BEM_EINVAL = 1,     /* invalid argument or geometry */
  BEM_ENOMEM = 2,     /* device allocation failed or a footprint limit was exceeded */
  BEM_ENOCONV = 3,    /* GMRES / refinement hit its iteration limit; best iterate written */
  BEM_ETIMEOUT = 4,   /* a bounded device-side wait expired */
  BEM_ECUDA = 5,      /* a CUDA runtime call failed (message gives the call and error) */
  BEM_ESTATE = 6      /* call out of order (e.g. solve before domains were set) */
} bem_status;

/* Row placement of the integral equations (see oracle and Sec. 5-6):
 *  MOD   - the paper's proposal: upper row of each element = standard equation of the domain its normal
 *          points into, times -alpha; lower row = Burton-Miller equation of the domain its normal points
 *          out of, with coefficient alpha/eps (Sec. 6 recipe; eq. calderon_bieb, eq. 3dom_calderon_bie).
 *  ORIG  - eq. 3dom_calderon_bie0: as MOD but interior domains keep standard lower rows (times -alpha).
 *  BETA1 - eq. calderon_bie1: as MOD with the standard rows unscaled.
 *  CONV  - eq. naive_bie / eq. 3dom_conv_bie (up to row order): Burton-Miller (host) or standard
 *          equations of the outward domain first, standard equations of the inward domain second. */
typedef enum { BEM_FORM_MOD = 0, BEM_FORM_ORIG = 1, BEM_FORM_BETA1 = 2, BEM_FORM_CONV = 3 } bem_form;

/* Arithmetic of the solve.  Assembly is the same for every precision: FP64 node geometry and phase k r,
 * then the Hankel values, Gauss sums and entry formulas in double-float arithmetic (pairs of FP32), within
 * about 1e-14 of the largest entry of a block of the FP64 definition.
 *  FP64     - A stored as complex FP64; FP64 matvec, FP64 Arnoldi; one unrestarted GMRES to `tol`.
 *  MIXED    - A stored as complex FP32 (hi) plus its FP32 rounding remainder (lo).  Inner GMRES runs on
 *             hi with FP32 products and an FP32 Krylov basis to `inner_tol`; the outer loop refines
 *             x in FP64 with residuals b - (hi + lo) x accumulated in double-float arithmetic.
 *  MIXED_TC - as MIXED, but the inner matvec of a multi-right-hand-side block runs as one dense complex
 *             GEMM on the tcgen05 tensor cores (hi split into two FP16 parts, hi16 + 2^-11 lo16; three FP16
 *             products per term, FP32 accumulation in tensor memory). */
typedef enum { BEM_PREC_FP64 = 0, BEM_PREC_MIXED = 1, BEM_PREC_MIXED_TC = 2 } bem_prec;

typedef struct {
  int quad_order;     /* Gauss-Legendre nodes per element, 1..16 (paper: 10) */
  int form;           /* bem_form */
  int prec;           /* bem_prec */
  int max_iter;       /* Krylov dimension limit of one GMRES run (no restart), >= 1 */
  int max_refine;     /* outer refinement steps for MIXED / MIXED_TC, >= 1 */
  double tol;         /* target relative residual ||b - A x||_2 / ||b||_2 (paper: 1e-8), > 0 */
  double inner_tol;   /* relative tolerance of each inner GMRES run (MIXED / MIXED_TC), > 0 */
  int orth_passes;    /* classical Gram-Schmidt passes per Arnoldi step: 1, 2 (re-orthogonalised), or 0 =
                         automatic: 2 for the FP64 basis; for the FP32 inner solves of the mixed paths one
                         pass, plus a second one in the iterations where the first shrank the new vector below
                         a tenth of its length (selective reorthogonalisation) */
  int matrix_free;    /* 1: do not store A; products recompute the entries (for matrices that do not fit in the
                         device memory granted to the problem).  FP64: every product recomputes every entry (one
                         assembly each).  MIXED: the leading element rows that fit in store_bytes are stored as
                         complex FP32 (their hi part) and only the other rows are recomputed in the FP32 inner
                         solves; the refinement residual recomputes every entry with FP64 sums (once per solve:
                         later residuals are updated, see bem_solve).  Not for MIXED_TC. */
  long long store_bytes;  /* matrix_free MIXED problems: device bytes for stored rows (each element takes two rows
                         of 2N complex FP32 entries, 32 N bytes); 0 = none.  >= 0. */
} bem_opts;

typedef struct bem_problem bem_problem;

/* Fill *o with the defaults: quad_order 4, MOD, FP64, max_iter 500, max_refine 6, tol 1e-10,
 * inner_tol 1e-5, orth_passes 0 (automatic), matrix_free 0, store_bytes 0. */
BEM_API void bem_default_opts(bem_opts* o);

/* Create an empty problem.  *out receives a library-owned handle (free with bem_problem_destroy).
 * EINVAL if an option is out of range. */
BEM_API bem_status bem_problem_create(bem_problem** out, const bem_opts* opts);
BEM_API void bem_problem_destroy(bem_problem* p);

/* Change the options of an existing problem (quadrature order or form changes invalidate the matrix). */
BEM_API bem_status bem_set_opts(bem_problem* p, const bem_opts* opts);

/* Domain table (Sec. 2): k_host[d] = wavenumber k_d > 0, eps_host[d] = flux coefficient eps_d > 0 with
 * eps_host[0] = 1 (domain 0 is the unbounded host medium).  The paper ties them as k_d = omega sqrt(eps_d);
 * the library takes both as given.  eps_d = -1 would put the eigenvalue cluster of A^2 at the origin
 * (Sec. 5) and is rejected with every other eps_d <= 0.  n_dom in [2, 64]. */
BEM_API bem_status bem_set_domains(bem_problem* p, int n_dom, const double* k_host, const double* eps_host);

/* Append one interface segment: a polyline of n_vert vertices xy_host[2*v], xy_host[2*v+1].  Elements
 * join consecutive vertices; closed != 0 adds the element from the last vertex to the first.  The
 * element normal is the tangent turned by +90 degrees; it must point out of domain dom_P and into
 * domain dom_M (Sec. 2: on the host boundary the normal points away from the host).  EINVAL for
 * fewer than 2 vertices (3 if closed), zero-length elements, or domain ids out of range / equal. */
BEM_API bem_status bem_add_segment(bem_problem* p, int n_vert, const double* xy_host, int dom_P, int dom_M,
                                   int closed);

BEM_API int bem_num_elements(const bem_problem* p);   /* N */
BEM_API int bem_num_unknowns(const bem_problem* p);   /* 2N */

/* Device bytes the assembled matrix and a solve with n_rhs right-hand sides will hold (for admission). */
BEM_API size_t bem_footprint_bytes(const bem_problem* p, int n_rhs);

/* Steps a1 + a3..a5: element geometry on the device, then every entry of A (Gauss-Legendre off the
 * diagonal, exact self terms on it) placed by the selected form.  Always recomputes A (the solve entry
 * points assemble only when the matrix is missing or out of date).  Allocates A on first use. */
BEM_API bem_status bem_assemble(bem_problem* p, void* stream);

/* Copy the assembled matrix into A_dev (2N x 2N complex FP64, row-major, leading dimension 2N).
 * which = 0: the matrix used by the solver (FP64 path: A; mixed: hi), which = 1: hi + lo (mixed only). */
BEM_API bem_status bem_get_matrix(bem_problem* p, int which, bem_c64* A_dev, void* stream);

/* Step a2: b for plane waves u_in = exp(i k_1 (cos t, sin t).x), t = angles_host[r], r < n_rhs.
 * b_dev: n_rhs x 2N.  Host-domain rows get u_in (standard) or u_in + alpha du_in/dn (Burton-Miller),
 * times the row's scale; all other rows are zero (eq. naive_bie, eq. 3dom_calderon_bie). */
BEM_API bem_status bem_rhs_planewave(bem_problem* p, int n_rhs, const double* angles_host, bem_c64* b_dev,
                                     void* stream);

/* Steps a6 / a11 for testing: y = A x for n_rhs columns with the kernel the solver uses
 * (FP64: FP64 GEMV/GEMM; MIXED: FP32 GEMV; MIXED_TC: tensor-core GEMM when n_rhs > 1).  Asynchronous on
 * `stream`, except the tensor-core path, which waits for the stream to read the kernel's error word and
 * returns BEM_ETIMEOUT if one of its bounded waits expired. */
BEM_API bem_status bem_matvec(bem_problem* p, int n_rhs, const bem_c64* x_dev, bem_c64* y_dev, void* stream);

/* Step a9's residual: r = b - A x for n_rhs columns with the solver's FP64-accurate operator (FP64 path:
 * FP64 products of A; mixed paths: (hi + lo) x in double-float arithmetic, the exact products hi x_hi on the
 * FP32 pipes; MIXED_TC with n_rhs >= 2 forms the small terms hi x_lo + lo x_hi as tensor-core products, and
 * then waits for the stream to read the product's error word, returning BEM_ETIMEOUT if one of its bounded
 * waits expired).  x_dev, b_dev, r_dev: n_rhs x 2N complex FP64 (r_dev may alias b_dev, not x_dev). */
BEM_API bem_status bem_residual(bem_problem* p, int n_rhs, const bem_c64* x_dev, const bem_c64* b_dev, bem_c64* r_dev,
                                void* stream);

/* The same residual as bem_residual (mixed-precision problems only; for MIXED_TC with n_rhs >= 2, where
 * bem_residual forms the small terms hi x_lo + lo x_hi on the tensor cores, this one forms them on the FP32
 * pipes, and the two agree to the residual's accuracy) without any device allocation.  The
 * paper has no counterpart: this is a library facility.  bem_residual takes its scratch from the problem's
 * solver workspace and may allocate it; callers that cannot allocate at that point (memory handed to their
 * own arena or caching allocator, latency-bound loops where cudaMalloc would stall, processes near their
 * memory limit) use this entry point instead.  Its scratch is a fixed static device array of 2 x 524288
 * complex FP32 entries (8 MiB) that every GPU loading the library holds until exit; n_rhs * 2N must not
 * exceed 524288 (BEM_EINVAL otherwise).  The problem must already be assembled (BEM_ESTATE otherwise;
 * this call never assembles).  Set-up: the assembly of a mixed-precision problem on a device (bem_assemble,
 * the solve entry points, bem_batch_admit), which allocates anyway, also looks up the array's device address
 * on that device and loads the residual kernels there (under lazy module loading both would otherwise take
 * device memory at their first use); so no call of this entry point allocates, the first one included.  All
 * calls share the one array and each overwrites it: calls whose kernels overlap on the GPU (different
 * streams, or different threads) race on it and must be serialised by the caller.  Nothing in it needs
 * clearing between calls: each call writes every entry it reads. */
BEM_API bem_status bem_residual_noalloc(bem_problem* p, int n_rhs, const bem_c64* x_dev, const bem_c64* b_dev,
                                        bem_c64* r_dev, void* stream);

/* Steps a6..a9: solve A x = b for n_rhs right-hand sides b_dev (n_rhs x 2N) into x_dev.
 * iters_host[r] = total GMRES iterations (matvecs) of column r, resid_host[r] = final relative residual
 * ||b - A x|| / ||b|| (FP64 path: the GMRES estimate; mixed paths: the FP64 refinement residual, formed in
 * double-float arithmetic until it is below 1e-4 of ||b|| and from then on updated as r -= A d with the inner
 * solves' own product of each correction d, whose ~3e-7 relative error enters r at ~3e-7 |A| |d|, far below the
 * tolerance; tolerances below 1e-11 form every refinement residual in double-float).  Either may be NULL. */
BEM_API bem_status bem_solve(bem_problem* p, int n_rhs, const bem_c64* b_dev, bem_c64* x_dev, int* iters_host,
                             double* resid_host, void* stream);

/* a2 + a6..a9 for plane waves (assembles first if needed). */
BEM_API bem_status bem_solve_planewave(bem_problem* p, int n_rhs, const double* angles_host, bem_c64* x_dev,
                                       int* iters_host, double* resid_host, void* stream);

/* Step a10: far-field pattern u_inf(theta_a), a < n_ang, of each of n_rhs solutions x_dev (n_rhs x 2N)
 * into out_dev (n_rhs x n_ang), with u_s(x) = e^{i k_1 |x|} / sqrt|x| (u_inf + O(1/|x|)). */
BEM_API bem_status bem_far_field(bem_problem* p, int n_rhs, const bem_c64* x_dev, int n_ang,
                                 const double* ang_host, bem_c64* out_dev, void* stream);

/* Field at points (the paper's accuracy study evaluates it on a 101 x 101 grid, Sec. 7.1): for each of
 * n_rhs solutions x_dev and each point pts_host[2p], pts_host[2p+1] lying in domain dom_host[p], Green's
 * representation u = [u_in] + sum_j sigma_{d,j} int_j (eps_d G_d w_j - dG_d/dn u_j), element integrals by the
 * problem's Gauss-Legendre rule.  angles_host (n_rhs, or NULL) adds the incident plane wave at host points;
 * NULL gives the scattered field there.  out_dev: n_rhs x n_pts.  Points must not lie on the boundary. */
BEM_API bem_status bem_near_field(bem_problem* p, int n_rhs, const bem_c64* x_dev, const double* angles_host,
                                  int n_pts, const double* pts_host, const int* dom_host, bem_c64* out_dev,
                                  void* stream);

/* End-to-end call with host buffers: assemble (if needed), solve plane waves, far field; copies the
 * traces (n_rhs x 2N) and far fields (n_rhs x n_ang) to the host.  x_host or ff_host may be NULL. */
BEM_API bem_status bem_solve_planewave_host(bem_problem* p, int n_rhs, const double* angles_host,
                                            bem_c64* x_host, int n_ang, const double* ff_ang_host,
                                            bem_c64* ff_host, int* iters_host, double* resid_host, void* stream);

/* ---- Batched solves of many independent problems (mixed precision only) -------------------------------
 * A batch engine owns device pools for up to max_slots resident problems whose unknowns add up to at most
 * pool_unknowns, each with its own matrix (allocated by the problem), Krylov basis (max_iter + 1 vectors),
 * solution, residual and right-hand side.  Admitted problems iterate together: every kernel covers all
 * resident problems (work lists over 64-entry chunks and 8-row blocks), the iteration body is replayed from a
 * CUDA graph, and each problem is refined in FP64 (double-float residuals) when its inner GMRES stops.
 * Problems can be admitted while others iterate (continuous batching); each result is the same as when the
 * problem is solved alone.  Admitted problems must stay alive until their slot is taken.  The engine runs on
 * its own stream, ordered after the caller's stream on entry and before it on exit. */
typedef struct bem_batch bem_batch;
BEM_API bem_status bem_batch_create(bem_batch** out, const bem_opts* opts, int max_slots, long long pool_unknowns);
BEM_API void bem_batch_destroy(bem_batch* b);
/* Admit n problems, each with one plane wave angles_host[i]: assemble all of them in one launch (tile height
 * chosen once per device by timing 4, 8 and 16 on about an eighth of the first admitted batch), form right-hand sides and start their solves.
 * slots_host[i] = slot or -1 when no slot or contiguous pool space was free (BEM_ENOMEM, others admitted).
 * Problems must be MIXED or MIXED_TC with the batch's quad_order and form. */
BEM_API bem_status bem_batch_admit(bem_batch* b, int n, bem_problem* const* probs, const double* angles_host,
                                   int* slots_host, void* stream);
/* Run one graph replay of iterations for every iterating problem and refine the ones whose inner solve
 * stopped; *n_running_host (may be NULL) = problems still iterating. */
BEM_API bem_status bem_batch_step(bem_batch* b, int* n_running_host, void* stream);
/* state: 0 free, 1 iterating, 2 finished (result waiting); iters = GMRES iterations so far; resid = last FP64
 * relative residual. */
BEM_API bem_status bem_batch_query(bem_batch* b, int slot, int* state_host, int* iters_host, double* resid_host);
/* Copy a finished slot's solution (2N complex FP64, may be NULL to discard) and free the slot. */
BEM_API bem_status bem_batch_take(bem_batch* b, int slot, bem_c64* x_dev, void* stream);
/* Largest contiguous run of free unknowns in the pools (admission check). */
BEM_API long long bem_batch_free_units(const bem_batch* b);
/* Admit, iterate to completion and take n problems (they must all fit).  The iterations run as one graph
 * launch: a conditional loop over a body of iterations and a refinement stage whose decisions (tolerance met,
 * refinement limit, next inner tolerance) are taken on the device; where conditional graph nodes are
 * unavailable, replays stepped by the host as in bem_batch_step.  Same results either way. */
BEM_API bem_status bem_batch_solve_planewave(bem_batch* b, int n, bem_problem* const* probs, const double* angles_host,
                                             bem_c64* const* x_dev, int* iters_host, double* resid_host,
                                             void* stream);

/* Per-phase device timing for measurement.  When enabled, every kernel launch of the problem is bracketed
 * by CUDA events recorded on the stream it runs on; bem_profile_read synchronises those events and returns,
 * per phase, the summed device milliseconds and the number of kernel launches since the last enable.
 * Arrays have BEM_PH_COUNT entries.  Enabling resets the counters; it does not change results.  Product
 * launches of GMRES iterations queued after every system of a block had converged (their gate closed, so
 * they did no work) are left out of the MATVEC and REDUCE launch counts; their few microseconds stay in the
 * phase times. */
typedef enum {
  BEM_PH_GEOMETRY = 0,  /* a1: element geometry */
  BEM_PH_ASSEMBLE = 1,  /* a3-a5: matrix entries */
  BEM_PH_RHS = 2,       /* a2 */
  BEM_PH_MATVEC = 3,    /* a6 / a11: GEMV, SIMT GEMM or tensor-core GEMM */
  BEM_PH_ARNOLDI = 4,   /* a7: projections, updates, norms; where the iteration tail is one cooperative launch,
                           also the rotations, the next basis vector and the stream-K sums of the product */
  BEM_PH_GIVENS = 5,    /* a8: Hessenberg column, rotations, residual estimate, basis scaling (start of a run;
                           every iteration only on the separate-kernel path) */
  BEM_PH_UPDATE = 6,    /* a9: least squares and x += V y */
  BEM_PH_RESIDUAL = 7,  /* a9: refinement residual b - (hi + lo) x (its norms count as OTHER) */
  BEM_PH_FARFIELD = 8,  /* a10 */
  BEM_PH_OTHER = 9,     /* conversions, copies, column norms, the FP16 split copy of A */
  BEM_PH_REDUCE = 10,   /* a11: stream-K reduction of the tensor-core GEMM inside GMRES (the GEMM is MATVEC);
                           none where the cooperative iteration kernel sums the partials itself */
  BEM_PH_RELAXED = 11,  /* launch count only (time 0): the MATVEC launches of the tensor-core GEMM that ran relaxed,
                           with A's FP16 remainder dropped (half of A's bytes) */
  BEM_PH_COUNT = 12
} bem_phase;
BEM_API bem_status bem_profile_enable(bem_problem* p, int on);
BEM_API bem_status bem_profile_read(bem_problem* p, double* ms_host, long long* launches_host);

/* Failure-path testing: the limit, in seconds, of the waits in the main loop of the tensor-core product
 * kernels and of the per-system barrier waits of the fused GMRES iteration kernel, for kernels launched from now
 * on (process-wide; 0 restores the defaults of 2 s and 0.5 s; CUDA graphs that a problem recorded earlier keep
 * the limits they were recorded with).  A tensor-core wait that runs out records an error word that the host
 * reads after the product (BEM_ETIMEOUT); the kernel then stops issuing work, waits with the default limit for
 * its own copies and MMAs in flight, frees its tensor memory and returns, so the context stays usable.  A
 * barrier wait that runs out records an error word and the kernel goes on without waiting (its results are then
 * meaningless, every access stays in bounds); the solve ends at its iteration limit and returns BEM_ETIMEOUT.
 * EINVAL outside [0, 10]. */
BEM_API bem_status bem_test_set_wait_limit(double seconds);
/* Testing: on = 0 makes solves started from now on run each GMRES iteration's tail as separate kernels
 * (projections, update, end of iteration: the path of devices without cooperative launches) instead of the
 * single cooperative kernel; on != 0 restores the default.  Process-wide. */
BEM_API bem_status bem_test_set_fused_iteration(int on);

/* Thread-local message of the last failure in this thread ("" if none). */
BEM_API const char* bem_last_error(void);

/* Library version string. */
BEM_API const char* bem_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BEM_H_ */
