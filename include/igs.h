/*
 * igs.h -- C ABI of the GB300 IgA-SGBEM assembly and solve library.
 *
 * The library assembles and solves the symmetric Galerkin system A alpha = beta
 * of the 2D Laplace Dirichlet problem on a spline / NURBS boundary curve by the
 * weighted-quadrature method of Aimi, Calabro, Diligenti, Sampoli, Sangalli,
 * Sestini, "Efficient assembly based on B-spline tailored quadrature rules for
 * the IgA-SGBEM" (arXiv:1703.10016):
 *
 *   A_ij = -(1/2pi) int_I B_i(s) J(s) int_I ln|f(s)-f(t)| B_j(t) J(t) dt ds     (Sect. 3.1, eq. final_1)
 *
 * split as ln|f(s)-f(t)| = K1(s,t) + K2(s,t) (Sect. 3.1), with K1 integrated by
 * the regular weighted rules of Algorithm 1 in both variables (eq. IK1e2) and K2
 * by the regular outer rule and the singular (modified-moment) inner rules of
 * Algorithm 2 (eq. IK1e2_bis).  For closed curves K2 is the periodic three-image
 * logarithm ln|x| + ln|x+L| + ln|x-L| - 2 ln L, x = t - s, L = |I|.
 *
 * Conventions common to every entry point
 *   - Return value: IGS_OK (0) or a negative IGS_E_* code.  No C++ exception
 *     crosses the ABI.  igs_last_error() returns a message for the most recent
 *     failure on the calling thread.
 *   - Input arrays are copied during the call; the caller keeps ownership.
 *     Output arrays are caller-provided.  Handles, rules, factors and device
 *     work buffers are owned by the library and released by igs_destroy_*.
 *   - "HOST" pointers are ordinary host memory (pageable or pinned); "DEVICE"
 *     pointers are device memory on the context's GPU.
 *   - All device work is issued on the context's stream (borrowed if the caller
 *     passed one).  Every entry point returns after its results are complete
 *     in the caller's buffers (the call synchronises the stream when it must
 *     hand data back to the host, and otherwise records completion on the stream:
 *     device outputs are valid for later work on the same stream).
 *   - Calls on one problem handle must be serialised by the caller; distinct
 *     problems may be used from distinct threads only with distinct contexts.
 */
#ifndef IGS_H
#define IGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define IGS_OK                   0
#define IGS_E_INVALID_ARG       -1   /* bad size, pointer, knot vector, degree ... */
#define IGS_E_NO_MEMORY         -2   /* device or host allocation failed          */
#define IGS_E_CUDA              -3   /* a CUDA runtime call failed                */
#define IGS_E_NOT_SPD           -4   /* Cholesky met a non-positive pivot         */
#define IGS_E_NOT_CONVERGED     -5   /* iterative refinement missed its tolerance */
#define IGS_E_TIMEOUT           -6   /* a bounded device wait gave up             */
#define IGS_E_ADMISSION_REFUSED -7   /* request does not fit the memory budget    */
#define IGS_E_STATE             -8   /* call out of order (e.g. solve before assemble) */
#define IGS_E_SINGULAR          -9   /* LU met a zero or non-finite pivot         */

/* precision tiers */
#define IGS_FP64   0   /* every step in FP64                                                    */
#define IGS_MIXED  1   /* kernel evaluation + contraction in FP32 (float-float node differences),
                          rules and moments in FP64; FP32 Cholesky + FP64 iterative refinement   */

/* memory kinds / element types of caller buffers */
#define IGS_MEM_HOST    0
#define IGS_MEM_DEVICE  1
#define IGS_F64         0
#define IGS_F32         1

typedef struct igs_ctx_s*  igs_ctx;
typedef struct igs_geom_s* igs_geom;
typedef struct igs_prob_s* igs_prob;

/* Sizes of a problem (all counts are of the paper's Sect. 3-4 objects). */
typedef struct igs_info {
    int32_t n;          /* N_DoF: number of test/trial functions (closed: N_h)            */
    int32_t degree;     /* d: degree of the discretisation and exactness spaces           */
    int32_t n_elems;    /* N_h: uniform elements of the discretisation                    */
    int32_t n_ref;      /* N_ref: refinement of the exactness space (Sect. 4)             */
    int32_t n_quad;     /* N_quad = 2d + 2 N_ref N_h - 1 nodes eta (Sect. 4)              */
    int32_t n_exact;    /* N_E = N_ref N_h + d exactness functions (Sect. 4)              */
    int32_t n_rhs_pts;  /* N_quad + N_GQ points where u_D is sampled (igs_rhs_points)     */
    int32_t closed;     /* 1 for a closed curve (interior problem), 0 for an open arc     */
    int32_t precision;  /* IGS_FP64 or IGS_MIXED                                          */
    int32_t rules_ready, assembled, factored;
    int32_t rhs_slots;  /* scratch of the double-layer sum per data set, in units of     */
                        /* n_quad doubles (igs_build_rhs_noalloc limit); 0: open arc      */
    int64_t device_bytes; /* device memory currently held by the problem                  */
} igs_info;

/* Per-phase device times of the most recent calls on a problem (milliseconds,
 * CUDA events on the context stream); 0 for phases not run. */
typedef struct igs_timing {
    float rules_ms, geometry_ms, assemble_ms, rhs_ms, factor_ms, solve_ms;
    int32_t ir_iterations;
    int32_t kernel_launches;   /* library kernels launched by the most recent call */
} igs_timing;

/* ----------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to borrow (NULL: the library creates and owns one).  Errors: INVALID_ARG
 * (bad device), CUDA. */
int igs_create(igs_ctx* out, int device, void* cuda_stream);

/* Release the context.  Geometries and problems created from it must have
 * been destroyed first (else IGS_E_STATE). */
int igs_destroy(igs_ctx ctx);

/* Message of the last failing call on this thread ("" if none).  The string
 * is owned by the library and valid until the next call on this thread. */
const char* igs_last_error(void);

/* ---------------------------------------------------------------- geometry */

/* Boundary curve f(s) = sum_i Q_i R_i(s) (Sect. 3): a degree-`degree` B-spline
 * (weights == NULL) or NURBS (weights[n_ctrl] > 0) on the extended knot vector
 * knots[n_knots], n_knots = n_ctrl + degree + 1, non-decreasing; the parameter
 * interval is I = [knots[degree], knots[n_ctrl]].  ctrl_xy is row-major
 * n_ctrl x 2 (x, y).  closed = 1 declares a closed curve (f(a) = f(b); closed
 * curves must be at least C^1 across the seam and oriented counter-clockwise;
 * the periodic convention of Sect. 3 repeats the first `degree` control points
 * at the end, a clamped closed curve repeats the first point).  All arrays are
 * HOST memory and copied.  Errors: INVALID_ARG. */
int igs_create_geometry(igs_ctx ctx, igs_geom* out, int degree, const double* knots, int n_knots,
                        const double* ctrl_xy, const double* weights, int n_ctrl, int closed);
int igs_destroy_geometry(igs_geom geom);

/* ----------------------------------------------------------------- problem */

/* Discretise on `n_elems` uniform elements of I with degree-`degree` B-splines
 * (periodic for a closed curve, clamped for an open arc), exactness space
 * refined `n_ref` times (Sect. 4), precision IGS_FP64 or IGS_MIXED.
 * Limits: 2 <= degree <= 5, 1 <= n_ref <= 4, closed: n_elems >= 2(degree+1),
 * n_ref * n_elems >= 3, n <= 65535.  Errors: INVALID_ARG.
 * Storage of the singular rules: on uniform knots the weight of node m' in
 * the rule at node m depends, away from the ends of I, only on m - m' and on
 * the parity of m' (Algorithm 2 is translation invariant there), so beyond
 * small n_quad the library keeps 24(d+1)+16 explicit columns and d+2 explicit
 * rows at each end plus two sequences of length 2 n_quad - 1: O(n_quad)
 * memory instead of n_quad^2. */
int igs_create_problem(igs_geom geom, igs_prob* out, int degree, int n_elems, int n_ref, int precision);
int igs_destroy_problem(igs_prob prob);

/* Attach another boundary curve to an existing problem, keeping its rules
 * (the rules of Algorithms 1 and 2 depend only on the discretisation, not on
 * the geometry, Sect. 4).  The new curve must be closed iff the old one was
 * and have the same parameter interval I.  Invalidates the assembled matrix,
 * the factor and the right-hand sides.  Errors: INVALID_ARG. */
int igs_set_geometry(igs_prob prob, igs_geom geom);
int igs_problem_info(igs_prob prob, igs_info* out);
int igs_problem_timing(igs_prob prob, igs_timing* out);

/* Build the weighted quadrature rules on the device (FP64):
 *   node vector eta (Sect. 4), regular rules w^(i) by Algorithm 1 (minimum-norm
 *   solution of the local exactness system, eq. reg_exactness), the Gram matrix
 *   G = (B)(B)^T of the collocation matrix and its banded Cholesky factor, the
 *   modified moments mu_j(eta_m) (eq. mod_mom_gen) and the singular rules
 *   w^{eta_m} = (B)^T G^{-1} mu(eta_m) of Algorithm 2.
 * The rules depend only on (n_elems, degree, n_ref, closed) and are reused by
 * every later assemble.  Idempotent.  Errors: NO_MEMORY, CUDA. */
int igs_build_weighted_rules(igs_prob prob);

/* Assemble A (n x n) on the device (eqs. IK1e2 and IK1e2_bis, A = -(I_K1 + I_K2)/(2 pi)).
 * Builds the rules first if needed, then evaluates the geometry at the nodes.
 * The matrix is kept inside the problem for igs_solve.  If A_out != NULL it is
 * also copied out, row-major with leading dimension `ld` >= n (elements), in
 * element type `dtype` (IGS_F64 or IGS_F32) to `mem` (IGS_MEM_HOST/DEVICE).
 * Without A_out the kernels are queued on the context stream and the call
 * returns before they finish, so host work (for instance the Dirichlet data at
 * the igs_rhs_points, downloaded before this call) overlaps them; every later
 * call on the problem is ordered after them, and igs_problem_timing waits for
 * them.  With A_out the call returns after the copy.
 * Errors: INVALID_ARG (ld < n, bad dtype/mem), NO_MEMORY, CUDA (a kernel fault
 * may surface in a later call). */
int igs_assemble(igs_prob prob, void* A_out, int64_t ld, int mem, int dtype);

/* Points where the Dirichlet datum u_D must be sampled for igs_build_rhs:
 * the N_quad nodes f(eta_n), then the N_GQ composite Gauss points of the
 * double-layer inner rule (Sect. 5, b2).  Writes `count` = n_rhs_pts and, if
 * xy_out != NULL and capacity >= count, the points row-major count x 2 (HOST).
 * Requires the rules (built on demand).  Errors: INVALID_ARG, CUDA. */
int igs_rhs_points(igs_prob prob, double* xy_out, int64_t capacity, int64_t* count);

/* Right-hand side of Sect. 5 for `nrhs` (1..8) data sets.  uD (`mem` memory)
 * holds, for each data set k, n_rhs_pts values u_D at the points of
 * igs_rhs_points, data set k at uD[k * n_rhs_pts].  Interior (closed) problem:
 * beta = b1/2 - b2/(2pi) (eq. seconda_BIE); open arc: beta = b1 (eq.
 * prima_BIE).  beta is kept in the problem for igs_solve; if beta_out != NULL
 * it is also written (`mem` memory, n x nrhs, data set k at beta_out[k * n]).
 * Errors: INVALID_ARG, NO_MEMORY, CUDA. */
int igs_build_rhs(igs_prob prob, const double* uD, int nrhs, double* beta_out, int mem);

/* Right-hand side without any device allocation.  The paper has no
 * counterpart: this entry exists for callers that cannot allocate device
 * memory inside a call -- a framework that owns all device memory through its
 * own allocator and forbids others, or a latency-bound serving loop that must
 * stay off the driver's allocator.  It computes the same beta as igs_build_rhs
 * (same kernels), but keeps the double-layer potentials at the nodes in a
 * fixed device array inside the library (16 MiB per GPU, held from library load
 * until process exit) and allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine.
 *   uD:       DEVICE, nrhs x n_rhs_pts (layout of igs_build_rhs)
 *   beta_out: DEVICE, nrhs x n, written (the problem's own beta is not changed)
 * Limits: 1 <= nrhs <= 8 and rhs_slots * n_quad * nrhs <= 2097152 doubles
 * (else INVALID_ARG), with rhs_slots from igs_problem_info: 8 for an FP64
 * closed curve (partial sums of 8 Gauss slices), 1 + ceil(S / n_quad) for a
 * MIXED closed curve (the potentials, then S doubles of treecode moments and
 * FP32 data products; S is about 8 n_quad), 0 for an open arc (no
 * double-layer term, so no scratch and no size limit beyond nrhs).
 * Preconditions: the rules, the node geometry and the rhs points exist (call
 * igs_assemble and igs_rhs_points first), else STATE.  The work is queued on
 * the context stream and not waited for.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) and caches it; make that
 * first call before any stream capture.  All calls share the array: calls
 * that overlap on the GPU race on it.  Errors: INVALID_ARG, STATE, CUDA. */
int igs_build_rhs_noalloc(igs_prob prob, const double* uD, int nrhs, double* beta_out);

/* Solve (A + A^T)/2 alpha = beta (eq. sistlin) by Cholesky.  FP64 tier: FP64
 * factorisation.  MIXED tier: FP32 factorisation and FP64 iterative refinement
 * until ||beta - A_s alpha|| <= 1e-10 ||beta|| (at most 30 steps).
 * beta: NULL to use the problem's last igs_build_rhs result, else `mem`
 * memory, n x nrhs (data set k at beta[k*n]).  alpha_out: `mem` memory, same
 * layout.  resid_out: NULL or HOST array of nrhs final relative residuals.
 * The factor is kept and reused until the next igs_assemble.
 * Errors: STATE (not assembled / no rhs), NOT_SPD, NOT_CONVERGED, CUDA. */
int igs_solve(igs_prob prob, const double* beta, int nrhs, double* alpha_out, double* resid_out, int mem);

/* Representation formula (Sect. 2): the potential u at `count` points x_p
 * off the curve from a solved density.  Closed curve (direct method):
 *   u(x) = -(1/2 pi) int ln|x - y| q(y) dgamma_y + (1/2 pi) int d/dn_y ln|x - y| u_D(y) dgamma_y,
 * q = sum_j alpha_j B_j; open arc (indirect method): only the first term, with
 * the density phi = sum_j alpha_j B_j.  Both integrals use the composite Gauss
 * rule of igs_build_rhs (igs_rhs_points), in FP64 in every tier; the rule is
 * not adapted to a near-singular integrand, so a point closer to the curve
 * than a few refined elements gets a less accurate value, and a point on a
 * Gauss point of the curve a non-finite one.
 *   alpha: `mem` memory, nrhs x n (the layout of igs_solve's alpha_out).
 *   uD:    `mem` memory, nrhs x n_rhs_pts (the layout of igs_build_rhs);
 *          only the values at the Gauss points are read.  Required for a
 *          closed curve, ignored (may be NULL) for an open arc.
 *   xy:    `mem` memory, count x 2 (x_p = (xy[2p], xy[2p+1])).
 *   u_out: `mem` memory, nrhs x count (data set k at u_out[k*count]).
 * Needs no rules, matrix or factor.  Errors: INVALID_ARG (NULL pointer, nrhs
 * outside [1, 8], count < 0, missing uD for a closed curve), NO_MEMORY, CUDA. */
int igs_eval_potential(igs_prob prob, const double* alpha, const double* uD, int nrhs, const double* xy,
                       int64_t count, double* u_out, int mem);

/* Collocation form of the single-layer equation (the remark of Sect. 7: the
 * same quadrature rules serve collocation BEM), closed curves only.  The
 * pointwise form of eq. seconda_BIE is imposed at one node m_i per unknown:
 *   Ac[i][j] = -(1/2 pi) (C0 P + W^s Q)[m_i][j]   (the inner sums of eqs. IK1e2, IK1e2_bis),
 *   beta_c[k][i] = u_D,k(eta_m_i)/2 - v_k(eta_m_i)/(2 pi),
 * v_k the double-layer potential at the nodes (the b2 inner rule of Sect. 5),
 * and Ac alpha = beta_c is solved by LU with partial pivoting.  m_i is the
 * node nearest the centre of the support of B_i (its Greville abscissa),
 * measured periodically, ties to the smaller node index.  Matrix, LU and
 * substitutions in FP64 in every tier; v_k follows the problem's tier.  The
 * LU is unblocked (2n launches): meant for n up to a few thousand.
 *   uD:        `mem` memory, nrhs x n_rhs_pts (the layout of igs_build_rhs).
 *   alpha_out: `mem` memory, nrhs x n.
 *   Ac_out:    NULL or `mem` memory, n x n row-major FP64 (before the LU).
 *   nodes_out: NULL or HOST array of n collocation node indices m_i.
 * Builds the rules and node geometry if missing; leaves the Galerkin matrix,
 * factor and right-hand side alone.  Errors: INVALID_ARG (open arc, n > 16384,
 * nrhs outside [1, 8], NULL uD/alpha_out), SINGULAR, NO_MEMORY, CUDA. */
int igs_collocation(igs_prob prob, const double* uD, int nrhs, double* alpha_out, double* Ac_out, int32_t* nodes_out,
                    int mem);

/* Right-hand side and solve in one call: the same computation as
 * igs_build_rhs followed by igs_solve(prob, NULL, ...), with the same bits
 * (every reduction on the path has a fixed order).  The right-hand side
 * (Sect. 5) is computed on an auxiliary stream of the problem while the
 * factorisation (eq. sistlin) runs on the context stream, so the two
 * overlap when the problem is not yet factored.
 *   uD:        `mem` memory, nrhs x n_rhs_pts (the layout of igs_build_rhs).
 *   alpha_out: `mem` memory, nrhs x n.  resid_out: NULL or HOST, nrhs values.
 * The right-hand side is kept in the problem as after igs_build_rhs.
 * Errors: INVALID_ARG, STATE (not assembled), NOT_SPD, NOT_CONVERGED, TIMEOUT, CUDA. */
int igs_solve_data(igs_prob prob, const double* uD, int nrhs, double* alpha_out, double* resid_out, int mem);

/* Download the assembled A (eq. IK1e2 plus IK1e2_bis, Sect. 5) without
 * assembling again, e.g. after igs_batch_assemble.  Arguments as for
 * igs_assemble's A_out, ld, mem, dtype.  Errors: INVALID_ARG, STATE (not
 * assembled), NO_MEMORY, CUDA. */
int igs_get_matrix(igs_prob prob, void* A_out, int64_t ld, int mem, int dtype);

/* ------------------------------------------------------------ batched form */

/* Many assemblies in one persistent launch.  The paper assembles one matrix at
 * a time (Sect. 5, Algorithm 3); this groups the same computation for a set of
 * MIXED-tier problems: one batched pass evaluates every problem's geometry and
 * node records, then one persistent kernel runs all (problem, tile) units from
 * a shared work list; both are captured in a CUDA graph.  Each problem's A is
 * the one igs_assemble would produce (same per-tile arithmetic).
 *
 * igs_batch_create: `probs` are count MIXED-tier problems of ctx (borrowed;
 *   a problem cannot be destroyed while a batch holds it: STATE).  Problems
 *   may differ in curve, n, degree and N_ref.  Errors: INVALID_ARG.
 * igs_batch_assemble: builds rules where missing (first call), then assembles
 *   every problem; afterwards each problem is in the state igs_assemble leaves
 *   (factor invalidated).  A problem whose geometry was replaced by
 *   igs_set_geometry is picked up (the graph is rebuilt).  ms_out (may be NULL):
 *   device time of the graph.  Errors: INVALID_ARG (a tile's node range above
 *   512 nodes), NO_MEMORY, CUDA.
 * igs_batch_tune: times every configuration (tile 32 or 16 DoFs; unit order
 *   natural, interleaved across problems or largest problem first; the
 *   occupancy limit of CTAs per SM or half of it), `reps` timed runs each
 *   (1..100) after one warm-up, keeps and returns the fastest.
 * igs_batch_set_config / igs_batch_get_config: explicit configuration
 *   (ctas_per_sm 0 = occupancy limit); get returns the last run's time in ms. */
typedef struct igs_batch_s* igs_batch;
#define IGS_ORDER_NATURAL       0   /* problem after problem, tiles row-major */
#define IGS_ORDER_INTERLEAVED   1   /* round-robin over the problems          */
#define IGS_ORDER_LARGEST_FIRST 2   /* problems by tile count, largest first  */
typedef struct igs_batch_config {
    int32_t tile;          /* DoFs per tile side: 16 or 32 */
    int32_t order;         /* IGS_ORDER_* */
    int32_t ctas_per_sm;   /* resident CTAs per SM, 0 = occupancy limit */
    float ms;              /* measured time (outputs only) */
} igs_batch_config;
int igs_batch_create(igs_ctx ctx, igs_batch* out, const igs_prob* probs, int count);
int igs_batch_destroy(igs_batch batch);
int igs_batch_assemble(igs_batch batch, float* ms_out);
int igs_batch_tune(igs_batch batch, igs_batch_config* best_out, int reps);
int igs_batch_set_config(igs_batch batch, const igs_batch_config* cfg);
int igs_batch_get_config(igs_batch batch, igs_batch_config* cfg);

/* ------------------------------------------------------------- served form */

/* A request loop around the method: each request is one Dirichlet problem
 * (a curve, a discretisation and 1..8 data sets) taken through rules,
 * assembly, right-hand sides and solve (Sects. 3-5).  The paper solves one
 * problem at a time; the server runs `slots` requests at once, each on its own
 * CUDA stream and host thread, so their kernels overlap on the device.  A
 * queued request is admitted, in arrival order, as soon as a slot is free and
 * its device-memory estimate fits in what the admitted requests leave of
 * `mem_budget`; a request that could never fit is refused at submission.
 * Each request's result does not depend on what runs beside it.
 *
 * Resident problems: the weighted rules depend only on the discretisation
 * (degree, n_elems, n_ref, precision and the curve's parameter interval), not
 * on the curve (Sect. 4), and a factorisation is valid until the matrix
 * changes.  With cache_budget > 0 each slot keeps the problems of its recent
 * requests (rules, matrix, factor) on the device, up to cache_budget bytes
 * over all slots (least recently used first out).  A request whose
 * discretisation matches a kept problem reuses its rules (the curve is swapped
 * in as by igs_set_geometry); if the curve is also the same, bit for bit, it
 * reuses the assembled matrix and its factor and only builds the right-hand
 * sides and solves.  Kept problems count against mem_budget; an idle slot
 * gives its kept problems up when the oldest queued request does not fit.
 * The reuse changes no arithmetic: results equal those of a fresh request.
 *
 * igs_data_fn: called once per request on a server thread with the request's
 *   right-hand-side points xy[count*2] (HOST, FP64, as igs_rhs_points); fills
 *   uD[k*count + q] for the nrhs data sets and returns 0 (nonzero fails the
 *   request with INVALID_ARG).
 * igs_server_create: device, opts (slots 1..64, mem_budget > 0 bytes,
 *   cache_budget >= 0 bytes of resident problems, 0: none).
 *   Errors: INVALID_ARG, CUDA.
 * igs_server_submit: copies the request (curve arrays included) and returns a
 *   ticket at once.  Errors: INVALID_ARG (malformed), ADMISSION_REFUSED (its
 *   estimate exceeds mem_budget).
 * igs_server_wait: blocks until the request is done or failed, or until
 *   timeout_ms (< 0: no limit) has passed (TIMEOUT); st (may be NULL) gets the
 *   stats.  Errors: INVALID_ARG (unknown ticket), TIMEOUT.
 * igs_server_result: for a finished request, copies alpha[nrhs*n] (HOST, data
 *   set k at alpha[k*n]) and resid[nrhs] (either may be NULL) and forgets the
 *   ticket; a failed request returns its error code (and is forgotten).
 *   Errors: INVALID_ARG, STATE (not finished).
 * igs_server_drain: waits until every submitted request has finished
 *   (TIMEOUT after timeout_ms >= 0).
 * igs_server_destroy: drains, stops the threads, frees everything. */
typedef struct igs_server_s* igs_server;
typedef int (*igs_data_fn)(void* user, const double* xy, int64_t count, int nrhs, double* uD);
typedef struct igs_request {
    int32_t geom_degree;        /* curve, as igs_create_geometry */
    int32_t n_knots;
    const double* knots;
    int32_t n_ctrl;
    const double* ctrl_xy;
    const double* weights;      /* NULL: B-spline */
    int32_t closed;
    int32_t degree;             /* discretisation, as igs_create_problem */
    int32_t n_elems;
    int32_t n_ref;
    int32_t precision;
    int32_t nrhs;               /* 1..8 */
    igs_data_fn data;
    void* user;
} igs_request;
typedef struct igs_server_opts {
    int32_t slots;
    int64_t mem_budget;
    int64_t cache_budget;       /* device bytes of resident problems kept between requests (0: none) */
} igs_server_opts;
#define IGS_REQ_QUEUED  0
#define IGS_REQ_RUNNING 1
#define IGS_REQ_DONE    2
#define IGS_REQ_FAILED  3
typedef struct igs_request_stats {
    int32_t status;             /* IGS_REQ_* */
    int32_t error;              /* IGS_E_* of a failed request */
    int32_t n, nrhs, ir_iterations, slot;
    int64_t device_bytes;       /* admission estimate */
    double queue_ms;            /* submission -> admission */
    double run_ms;              /* admission -> done */
    double latency_ms;          /* submission -> done */
    int32_t reuse;              /* IGS_REUSE_*: what the request took from a resident problem */
    int32_t reserved;
} igs_request_stats;
#define IGS_REUSE_NONE   0      /* rules built for the request */
#define IGS_REUSE_RULES  1      /* rules of a resident problem, curve swapped in */
#define IGS_REUSE_FACTOR 2      /* same curve: rules, matrix and factor reused */
int igs_server_create(int device, const igs_server_opts* opts, igs_server* out);
int igs_server_submit(igs_server server, const igs_request* req, int64_t* ticket);
int igs_server_wait(igs_server server, int64_t ticket, int32_t timeout_ms, igs_request_stats* st);
int igs_server_result(igs_server server, int64_t ticket, double* alpha, double* resid, igs_request_stats* st);
int igs_server_drain(igs_server server, int32_t timeout_ms);
int igs_server_destroy(igs_server server);

/* Diagnostic download of the rules for parity checks (HOST outputs, FP64):
 *   eta[n_quad]; W_band[n_quad * (degree+1)]: W_band[m*(d+1)+r] = w^(i)_m for
 *   the test function i = (first(m) + r) mod n containing eta_m (0 if none),
 *   first[n_quad]: first(m) (may be >= n for the seam node eta = b);
 *   Ws[n_quad * n_quad] (row m = w^{eta_m}, NULL to skip; expanded from the
 *   stored form, n_quad <= 65535).
 * Any output pointer may be NULL.  Errors: STATE, INVALID_ARG, NO_MEMORY, CUDA. */
int igs_get_rules(igs_prob prob, double* eta, double* W_band, int32_t* first, double* Ws);

/* Diagnostic download of the geometry at the nodes (HOST, FP64): xy[n_quad*2]
 * (f(eta_n)), J[n_quad] (|f'(eta_n)|).  Errors: STATE, CUDA. */
int igs_get_node_geometry(igs_prob prob, double* xy, double* J);

/* Self-test of the bounded waits that the triangular solves use between
 * thread blocks: one GPU thread waits for a 64-bit word that nothing writes,
 * with a budget of `budget_s` seconds (clamped to [1e-4, 2]), and must give
 * up.  *gave_up = 1 when the wait ended by its budget (the expected result),
 * 0 otherwise.  The CUDA context stays usable.  Errors: INVALID_ARG, CUDA. */
int igs_selftest_wait(igs_ctx ctx, double budget_s, int* gave_up);

/* Throughput of one arithmetic pipe of the context's GPU, measured by a probe
 * kernel that fills every SM with independent dependency chains of one
 * instruction kind (one warm-up launch, then one launch timed with CUDA
 * events, 10-50 ms).  The paper has no counterpart: these are the measured
 * denominators of the roofline fractions of the assembly and right-hand side
 * kernels, which run on the FP32 FMA and special-function (MUFU) pipes.
 *   kind IGS_PEAK_FP32_FMA: FP32 fused multiply-add, flop/s (2 per FMA)
 *        IGS_PEAK_MUFU_LG2: lg2.approx.f32, instructions/s
 *        IGS_PEAK_MUFU_RCP: rcp.approx.f32, instructions/s
 *        IGS_PEAK_FP64_FMA: FP64 fused multiply-add, flop/s (2 per FMA)
 * *rate (HOST) receives the rate, *ms (HOST, may be NULL) the timed launch's
 * duration.  Allocates 1 KB of device memory for the duration of the call;
 * runs on the legacy default stream and waits for it.
 * Errors: INVALID_ARG (NULL rate, unknown kind), CUDA. */
#define IGS_PEAK_FP32_FMA 0
#define IGS_PEAK_MUFU_LG2 1
#define IGS_PEAK_MUFU_RCP 2
#define IGS_PEAK_FP64_FMA 3
int igs_measure_peak(igs_ctx ctx, int kind, double* rate, double* ms);

#ifdef __cplusplus
}
#endif
#endif /* IGS_H */
