/*
 * gbem.h -- C ABI of the GB300 Galerkin boundary element capacitance library.
 *
 * The library implements the single-dielectric method of Wu & Li, "GBEM:
 * Galerkin Boundary Element Method for 3-D Capacitance Extraction"
 * (arXiv 2203.11733), Sec. 3:
 *
 *   boundary partition    dOmega = U_j I_j into axis-aligned rectangles
 *                         (Sec. 3.1 before Eq. "myequation"; Sec. 3.3: every
 *                         conductor is built from cuboids)        -> gbem_mesh
 *   Galerkin matrix       a_ij = 1/(4 pi |I_i||I_j|) int_Ii int_Ij 1/|x-y|
 *                         (Eq. "matrix", Sec. 3.4)                -> gbem_assemble
 *   Cholesky factor       A is symmetric positive definite (Sec. 3.2,
 *                         Theorem 1), so A = L L^T                -> gbem_factor
 *   solve                 A X = b, b_i = mean of f0 over I_i with f0 = 1 on the
 *                         main net and 0 elsewhere (Eq. "lineareq1")
 *                                                                 -> gbem_solve
 *   charge                Q_n = eps * sum_{I_j on net n} X_j
 *                         (Eq. "electriccharge")                  -> gbem_capacitance
 *
 * and its multi-dielectric case, Sec. 4, for layered stacks (per-layer
 * equations with single- and double-layer integrals, LU)    -> gbem_stack_*
 *
 * Units: lengths in micrometres; A in 1/um; X in um; capacitances in farads,
 * C = eps0 * eps_r * 1e-6 * X (eps0 = 8.8541878128e-12 F/m).  The kernel
 * 1/(4 pi |x-y|) is the paper's u* (Sec. 2.1, Eq. "representation"); the
 * permittivity enters only at the charge step, as in Eq. "electriccharge".
 * Conductors sit in free space (no grounded enclosure unless the caller adds
 * one as an extra conductor held at 0 V).
 *
 * Conventions shared by every call:
 *  - Every call returns a gbem_status; on failure the context keeps a message
 *    readable through gbem_last_error().  No C++ exception crosses the ABI.
 *  - Device memory for handles comes from the allocator passed to
 *    gbem_create() (cudaMalloc/cudaFree when none is given); handles own it
 *    and release it in their *_destroy call.  Host arrays passed in are read
 *    during the call only and stay owned by the caller; so do device arrays
 *    passed to gbem_solve().
 *  - gbem_stream is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  gbem_assemble, gbem_factor and gbem_solve only enqueue work on
 *    it; gbem_capacitance, gbem_matrix_download and gbem_matrix_status wait
 *    for that stream.
 *  - A context and its handles are not thread safe; use one context per
 *    worker thread.
 *  - Matrix layout: N x N column-major, lower triangle significant, padded
 *    internally to a multiple of 128 with the identity.
 */
#ifndef GBEM_H
#define GBEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBEM_OK = 0,
    GBEM_ERR_ARG = -1,      /* invalid argument (null pointer, size, id) */
    GBEM_ERR_OOM = -2,      /* allocator refused, or HBM budget exceeded */
    GBEM_ERR_CUDA = -3,     /* a CUDA runtime call failed */
    GBEM_ERR_NOT_SPD = -4,  /* Cholesky met a non-positive pivot, or LU a
                               zero one (singular stack system) */
    GBEM_ERR_TIMEOUT = -5,  /* a bounded device-side wait gave up */
    GBEM_ERR_NOCONV = -6,   /* iterative refinement missed its tolerance */
    GBEM_ERR_MESH = -7,     /* malformed geometry: empty, degenerate or
                               overlapping boxes, zero-area panel */
    GBEM_ERR_STATE = -8,    /* call out of order (e.g. solve before factor) */
    GBEM_ERR_NODEV = -9     /* context has no device (created with device -1) */
} gbem_status;

typedef enum {
    GBEM_FP64 = 0,  /* every step in FP64 */
    GBEM_MIXED = 1  /* FP32 far-field quadrature and FP32 factor; FP64 near
                       field, FP64 residual and iterative refinement */
} gbem_precision;

typedef void* gbem_stream;

/* A conductor cuboid (Sec. 3.3): lo < hi componentwise, in um. */
typedef struct {
    double lo[3];
    double hi[3];
    int32_t conductor;
} gbem_box;

/* Boundary partition.  Each box edge of length L is divided either uniformly
 * into ceil(L/h) cells (ratio <= 1) or, when ratio > 1 and 0 < h_min < h,
 * with cells h_min, h_min*ratio, ... growing from both ends while below h
 * and the rest split into equal cells no longer than h. */
typedef struct {
    double h;
    double ratio;
    double h_min;
} gbem_mesh_params;

/* Tunables.  Zero fields keep the defaults shown. */
typedef struct {
    double q_near_fp64;   /* gap / largest edge below which a pair uses the
                             closed form in FP64 mode (12) */
    double q_near_mixed;  /* mixed mode: below 0.5 every pair takes the closed
                             form, below q_near_mixed (1.0) the pairs whose
                             largest edges differ by more than 1.5x */
    double ir_tol;        /* relative residual target of refinement (1e-11) */
    int ir_max_iter;      /* refinement iterations at most (10) */
    int nb;               /* Cholesky block size: 64 */
} gbem_tuning;

typedef void* (*gbem_alloc_fn)(size_t bytes, gbem_stream stream, void* user);
typedef void (*gbem_free_fn)(void* ptr, size_t bytes, gbem_stream stream, void* user);

typedef struct gbem_ctx_s gbem_ctx;
typedef struct gbem_mesh_s gbem_mesh_t;
typedef struct gbem_matrix_s gbem_matrix_t;

/* Create a context on CUDA device `device` (or -1 for a host-only context
 * that can mesh but not compute).  hbm_budget caps the bytes the context may
 * hold at once (0 = no cap).  alloc/free may be NULL (cudaMalloc/cudaFree). */
gbem_status gbem_create(gbem_ctx** out, int device, size_t hbm_budget,
                        gbem_alloc_fn alloc, gbem_free_fn free_fn, void* user);
/* Destroy a context.  Its meshes and matrices must be destroyed first. */
void gbem_destroy(gbem_ctx* ctx);
const char* gbem_last_error(const gbem_ctx* ctx);
gbem_status gbem_set_tuning(gbem_ctx* ctx, const gbem_tuning* t);
/* Bytes currently held by the context: its handles' buffers, and the
 * buffers of the last destroyed matrix, which the context keeps (idle) for
 * the next matrix's allocations of the same size and releases at the next
 * matrix destroy, when an allocation would exceed the budget or is refused,
 * and in gbem_destroy. */
size_t gbem_bytes_in_use(const gbem_ctx* ctx);

/* Mesh the surfaces of `nbox` disjoint cuboids (Sec. 3.1, Sec. 3.3).
 * Boxes with the same conductor id form one conductor; boxes may not
 * overlap or touch.  Panels are ordered by conductor (ids ascending), then
 * by the Morton code of the panel centre.  Uploads panel geometry to the
 * device when the context has one. */
gbem_status gbem_mesh(gbem_ctx* ctx, const gbem_box* boxes, int nbox,
                      const gbem_mesh_params* params, gbem_mesh_t** out);

/* The paper's distance-graded partition for one main net (Sec. 3.3): every
 * face is split by bisection of its longer edge until each panel I_j
 * satisfies |I_j| <= p4 if its distance d to the main net is below p5 and
 * |I_j| <= p4 * p3 * (d / p5)^3 otherwise (Sec. 3.3, from the far-field
 * bound |dq/dtau| <= C / |x - x0|^3 of Eq. "electric_derivative"), with
 * p4 = p1 for faces that look toward the main net and p4 = p1 * p2 for faces
 * that look away from it.  A face looks toward the main net when some of the
 * main net lies on the outward side of its plane; the main net's own faces
 * and the inner faces of the enclosure always do.  d is the distance from
 * the panel to the nearest box of the main net.  Areas in um^2, lengths in
 * um.  h_max (0 = none) also caps every panel edge.  With has_enclosure the
 * inner faces of the grounded box [encl_lo, encl_hi] (Sec. 3.1: the
 * boundary of the domain, at potential 0) are meshed as conductor
 * encl_conductor; every box must lie strictly inside it.  The mesh is meant
 * for the column of the capacitance matrix that belongs to the main net. */
typedef struct {
    int32_t main_conductor;
    double p1;
    double p2;
    double p3;
    double p5;
    double h_max;
    int has_enclosure;
    double encl_lo[3];
    double encl_hi[3];
    int32_t encl_conductor;
} gbem_partition_params;
gbem_status gbem_mesh_graded(gbem_ctx* ctx, const gbem_box* boxes, int nbox,
                             const gbem_partition_params* params, gbem_mesh_t** out);

/* Error-driven refinement of a mesh (Sec. 3.2, Proposition "error": the
 * charge error on a net is bounded by C sup_j |I_j| sup_{x in I_j} |dq/dtau|).
 * density[i] is the charge density of panel i of `mesh` (in the order of
 * gbem_mesh_panels) from a solve for the net of interest, e.g. X_i / |I_i|
 * for its column of X; only differences and ratios of it matter.  The
 * tangential derivative on panel j is estimated from the panels of the same
 * conductor that share a segment of its boundary (across face edges too; a
 * common corner alone does not count) as the largest
 * |density_k - density_j| / |c_k - c_j| (c: panel centres), and the
 * indicator is eta_j = |I_j| times that.  Every panel with
 * eta_j >= theta * max_k eta_k (0 <= theta <= 1; nothing when that maximum
 * is 0) is bisected across its longer edge (the first in-plane axis on a
 * tie); the others are kept.  *out receives a new mesh of the same context,
 * conductor ids kept, in the library's panel order; eta (optional, mesh->n
 * entries) the indicators; n_marked (optional) the number of bisected
 * panels.  The input mesh is not changed.  Errors: GBEM_ERR_ARG for a NULL
 * argument, theta outside [0, 1], a non-finite density or more than 2e6
 * panels; GBEM_ERR_OOM. */
gbem_status gbem_mesh_refine(const gbem_mesh_t* mesh, const double* density, double theta, double* eta,
                             gbem_mesh_t** out, int* n_marked);

/* Build a mesh from an explicit panel list, kept in the given order.
 * axis[i] in {0,1,2} is the panel's normal axis; geo[5*i..5*i+4] =
 * {c, lo0, hi0, lo1, hi1}: the plane coordinate and the extents along the two
 * other axes in increasing axis order; cond[i] the conductor id. */
gbem_status gbem_mesh_from_panels(gbem_ctx* ctx, int n, const int8_t* axis,
                                  const double* geo, const int32_t* cond,
                                  gbem_mesh_t** out);

/* A mesh of n flat triangles (general, non-Manhattan conductors; the paper's
 * Galerkin formulation, Sec. 3.1 and Eq. "matrix", with triangles for
 * panels): tri holds 9 doubles per triangle, its three vertices (um);
 * cond[i] the conductor id.  Triangles of one conductor that touch must
 * share whole edges or vertices with identical coordinates.  Entries: the
 * self-integral in closed form, touching pairs by the exact potential of one
 * triangle under a tanh-sinh rule over the other, near pairs by the exact
 * potential under Gauss-Legendre, far pairs by Gauss-Legendre product rules
 * (FP64, about 1e-10 relative; in GBEM_MIXED the far rules run in FP32,
 * about 1e-7, stored as for rectangles and factored in FP32 with
 * refinement).  Such a mesh works with gbem_assemble, gbem_factor,
 * gbem_solve and gbem_capacitance; refinement, batches and
 * gbem_mesh_panels' rectangle arrays return GBEM_ERR_STATE.  GBEM_ERR_MESH
 * for non-finite coordinates or zero area. */
gbem_status gbem_mesh_from_triangles(gbem_ctx* ctx, int n, const double* tri, const int32_t* cond,
                                     gbem_mesh_t** out);
/* The triangles of a triangle mesh (9 doubles each) and their conductor ids;
 * GBEM_ERR_STATE for a rectangle mesh. */
gbem_status gbem_mesh_triangles(const gbem_mesh_t* mesh, double* tri, int32_t* cond);

/* Panel count and conductor count of a mesh. */
gbem_status gbem_mesh_info(const gbem_mesh_t* mesh, int* n_panels, int* n_cond);

/* Host copies of the panels in mesh order (arrays of n_panels, 5*n_panels,
 * n_panels) and the sorted conductor ids (array of n_cond); any pointer may
 * be NULL. */
gbem_status gbem_mesh_panels(const gbem_mesh_t* mesh, int8_t* axis, double* geo,
                             int32_t* cond, int32_t* cond_ids);
void gbem_mesh_destroy(gbem_mesh_t* mesh);

/* Assemble the Galerkin matrix (Eq. "matrix") on `stream`.  Pairs whose gap
 * is below q_near times their largest edge use exact 4-D corner sums of
 * closed-form antiderivatives in FP64; the others use a tensor Gauss-Legendre
 * rule whose order follows the gap (FP64, or FP32 in mixed mode). */
gbem_status gbem_assemble(gbem_mesh_t* mesh, gbem_precision prec, gbem_stream stream,
                          gbem_matrix_t** out);

/* Cholesky factorisation A = L L^T (Sec. 3.2), blocked, on `stream`.  FP64
 * mode factors an FP64 copy in FP64 arithmetic.  Mixed mode factors the FP32
 * copy in place entirely in FP32 arithmetic -- the 64 x 64 diagonal blocks
 * and their inverses included -- with the trailing updates on the tensor
 * cores in 3xTF32; the FP64 refinement of gbem_solve restores the accuracy.
 * A non-positive pivot is recorded and reported by the next waiting call as
 * GBEM_ERR_NOT_SPD. */
gbem_status gbem_factor(gbem_matrix_t* mat, gbem_stream stream);

/* Solve A X = B for nrhs right-hand sides on `stream`.  B_dev and X_dev are
 * device arrays, column-major with leading dimensions ldb, ldx >= N, and may
 * alias.  Mixed mode runs FP64 iterative refinement until the relative
 * residual max_k |B_k - A X_k|_inf / |B_k|_inf is below ir_tol; if ir_iters
 * is not NULL the call waits for the stream and stores the iterations used. */
gbem_status gbem_solve(gbem_matrix_t* mat, const double* B_dev, int nrhs, int ldb,
                       double* X_dev, int ldx, int* ir_iters, gbem_stream stream);

/* Size in bytes of the fixed device scratch used by gbem_solve_noalloc. */
#define GBEM_NOALLOC_SCRATCH_BYTES (16u << 20)

/* gbem_solve without any device allocation.  The paper has no counterpart:
 * this serves callers that cannot allocate device memory at solve time -- a
 * serving worker that reserved its HBM budget up front, an application whose
 * device memory belongs to its own pool and forbids library cudaMalloc calls,
 * or a latency-critical loop that must not risk the device synchronisation
 * cudaMalloc/cudaFree can cause.  Arguments and results are those of
 * gbem_solve (the matrix must be factored).  The work buffers live in one
 * file-scope device array of GBEM_NOALLOC_SCRATCH_BYTES that every GPU using
 * the library holds until the process exits; a call needing more
 * (5 * 8 * padded N * nrhs bytes plus 256 plus 4 bytes per 64 rows, each term
 * rounded up to 256) fails with GBEM_ERR_ARG.  The first call on a device
 * looks up the array's device address; make that first call before any
 * stream capture begins.  Every call copies its status words back and waits
 * for its stream before returning, on success and on every error after the
 * argument checks.  All calls share the array and it keeps the last call's
 * contents: calls that overlap on the GPU race and must be serialised by the
 * caller. */
gbem_status gbem_solve_noalloc(gbem_matrix_t* mat, const double* B_dev, int nrhs, int ldb,
                               double* X_dev, int ldx, int* ir_iters, gbem_stream stream);

/* Self-test of the bounded device waits (no counterpart in the paper: a
 * failure-detection check).  One CTA waits, through the same bounded
 * release-flag wait that every elimination step of the mixed factorisation
 * uses, for a device flag to become 1, with a wall-clock limit of limit_ms
 * (0 < limit_ms <= 10000; the library's own waits use 1 s).  With
 * set_flag != 0 the flag is written before the kernel starts and the call
 * returns GBEM_OK; with set_flag == 0 nothing ever writes it, the wait runs
 * out and the call returns GBEM_ERR_TIMEOUT, after which the context is
 * still usable.  Allocates 256 bytes from the context; waits for the
 * stream. */
gbem_status gbem_selftest_wait(gbem_ctx* ctx, int set_flag, double limit_ms, gbem_stream stream);

/* Arithmetic units whose throughput bounds the assembly: the far field's 1/r
 * evaluations go through the MUFU reciprocal square root, the near field's
 * closed forms (Eqs. "F" and "H", Appendix) through FP64 arithmetic and the
 * FP64 log, atan and sqrt. */
typedef enum {
    GBEM_RATE_DFMA = 0,        /* FP64 fused multiply-add */
    GBEM_RATE_FFMA = 1,        /* FP32 fused multiply-add */
    GBEM_RATE_MUFU_RSQRT = 2,  /* FP32 approximate reciprocal square root */
    GBEM_RATE_DSQRT = 3,       /* FP64 sqrt (with one FP64 add) */
    GBEM_RATE_DLOG = 4,        /* FP64 log (with one FP64 add) */
    GBEM_RATE_DATAN = 5,       /* FP64 atan (with one FP64 add) */
    GBEM_RATE_DRSQRT = 6,      /* FP64 rsqrt (with one FP64 add) */
    GBEM_RATE_COUNT = 7
} gbem_unit_rate;

/* Measurement helper with no counterpart in the paper: the roofline of the
 * assembly needs the rates of the units above on the GPU at hand.  Writes
 * rates[k] = operations per second over the whole device (an FMA counts as
 * one operation) for k = 0 .. n_rates-1 (1 <= n_rates <= GBEM_RATE_COUNT),
 * each the best of three timed launches of independent dependency chains
 * after one warm-up, 8 CTAs of 256 threads per SM.  Takes about 0.3 s;
 * allocates 2.5 MB (152 SMs) from the context for the duration of the call;
 * waits for the stream.  Rates reflect the clocks at the time of the call. */
gbem_status gbem_unit_rates(gbem_ctx* ctx, double* rates, int n_rates, gbem_stream stream);

/* Maxwell capacitance matrix in farads, n_c x n_c row-major into C_host:
 * C[m][k] = charge on conductor m with conductor k at 1 V and the others at
 * 0 V (Eqs. "lineareq1", "electriccharge"), rows and columns in ascending
 * conductor id.  Factors the matrix first if needed.  resid_out (may be
 * NULL) receives the final relative residual.  Waits for the stream. */
gbem_status gbem_capacitance(gbem_mesh_t* mesh, gbem_matrix_t* mat, double eps_r,
                             double* C_host, double* resid_out, gbem_stream stream);

/* Copy the assembled matrix A (both triangles filled) to host memory,
 * N x N column-major.  Waits for the matrix's last stream. */
gbem_status gbem_matrix_download(gbem_matrix_t* mat, double* host);

/* Wait for the matrix's last stream and report a recorded device-side error
 * (GBEM_ERR_NOT_SPD from the factorisation), else GBEM_OK. */
gbem_status gbem_matrix_status(gbem_matrix_t* mat);

/* Tracing.  With timing enabled (level 1 or 2), every call records CUDA
 * events on its stream around each phase; gbem_get_stats waits for those events and adds
 * their elapsed times.  launches counts every kernel launched by the library
 * in this process (all contexts).  reset != 0 clears the counters after
 * reading. */
enum {
    GBEM_PHASE_MESH = 0,      /* panel upload */
    GBEM_PHASE_ASSEMBLE = 1,  /* gbem_assemble kernels */
    GBEM_PHASE_FACTOR = 2,    /* Cholesky */
    GBEM_PHASE_SOLVE = 3,     /* triangular solves, residuals, refinement */
    GBEM_PHASE_REDUCE = 4,    /* right-hand sides and charge reduction */
    GBEM_NPHASE = 5
};
typedef struct {
    double ms[GBEM_NPHASE];
    long long calls[GBEM_NPHASE];
    long long launches;
} gbem_stats;
gbem_status gbem_set_timing(gbem_ctx* ctx, int enable);
gbem_status gbem_get_stats(gbem_ctx* ctx, gbem_stats* out, int reset);

/* Kernel-level tracing.  With gbem_set_timing(ctx, 2) the library also
 * records a CUDA event pair, on the launch stream, around every launch of
 * the kernels below, and adds the algorithmic work that launch was given:
 * bytes that must cross HBM at least once and useful flops (the
 * contraction's 2mnk, not the 3x of the split-precision tensor products).
 * gbem_get_kernel_stats waits for the events and returns per kernel the
 * summed device time, the number of launches, bytes and flops.  reset != 0
 * clears the sums after reading.  The events cost a few microseconds per
 * launch, so time the workload itself with level 1 or 0. */
enum {
    GBEM_KERNEL_ASSEMBLE = 0,  /* one CTA per 32 x 32 tile: Galerkin entries */
    GBEM_KERNEL_FACTOR = 1,    /* FP32 factor, timed as one span per factorisation: its
                                  launches per elimination step (panel, strip update,
                                  next diagonal block, tensor-core tiles) overlap the
                                  rest updates on a second stream */
    GBEM_KERNEL_SWEEP = 2,     /* persistent forward/backward triangular sweeps */
    GBEM_KERNEL_RESIDUAL = 3,  /* residual R = B - A X (FP64, or compensated FP32 in mixed mode) */
    GBEM_NKERNEL = 4
};
typedef struct {
    double ms[GBEM_NKERNEL];
    long long launches[GBEM_NKERNEL];
    double bytes[GBEM_NKERNEL];
    double flops[GBEM_NKERNEL];
} gbem_kernel_stats;
gbem_status gbem_get_kernel_stats(gbem_ctx* ctx, gbem_kernel_stats* out, int reset);

/* Batched extraction: many independent structures (meshes of one context)
 * assembled, factored and solved together in mixed precision.  The whole
 * pipeline -- batched assembly over every tile of every structure, the
 * batched Cholesky (one launch per elimination step for all structures),
 * `iters` FP64 refinement passes, residuals and capacitances -- is captured
 * once into a CUDA graph on the batch's own stream and replayed by each
 * gbem_batch_run (one graph launch).  The meshes' panel data are copied at
 * creation; the meshes may be destroyed afterwards.  iters 0 selects 3.
 * Every structure has at most 16 conductors. */
typedef struct gbem_batch_s gbem_batch_t;
gbem_status gbem_batch_create(gbem_ctx* ctx, int count, gbem_mesh_t* const* meshes, int iters,
                              gbem_batch_t** out);
/* Run the batch after work already enqueued on `stream`, and wait for it.
 * C_host receives the capacitance matrices back to back (structure b's
 * n_c(b) x n_c(b) row-major block at the offset reported by
 * gbem_batch_info); resid_host (may be NULL) the final relative residual of
 * each structure. */
gbem_status gbem_batch_run(gbem_batch_t* batch, double eps_r, double* C_host, double* resid_host,
                           gbem_stream stream);
/* count structures; c_total = total length of C_host; c_offset (array of
 * count, may be NULL) = offset of each structure's block. */
gbem_status gbem_batch_info(const gbem_batch_t* batch, int* count, long long* c_total,
                            long long* c_offset);
void gbem_batch_destroy(gbem_batch_t* batch);

/* Batches in groups.  gbem_batch_create_grouped splits the structures into
 * `groups` parts of similar factorisation work (sum of np^3); each part has
 * its own pooled buffers, stream and graph, and the parts' graphs run
 * concurrently (small structures then need not wait for the elimination
 * steps of the largest).  Results come back in the caller's order; groups 1
 * is gbem_batch_create.  Not in the paper (a batching choice). */
gbem_status gbem_batch_create_grouped(gbem_ctx* ctx, int count, gbem_mesh_t* const* meshes, int groups,
                                      int iters, gbem_batch_t** out);
/* The groups and refinement passes a batch was built with. */
gbem_status gbem_batch_config(const gbem_batch_t* batch, int* groups, int* iters);
/* Autotuner for the batched form.  Tries 1, 2 and 4 groups; for each, the
 * fewest refinement passes (at most max_iters, 0 selects 3) after which
 * every structure's relative residual meets the context's tolerance, then
 * the time of three runs after a warm-up (CUDA events, default stream).  The
 * fastest is returned built in *out, and appended to cache_path (may be NULL)
 * as a line "<key> <groups> <passes> <ms>", keyed by a hash of the count,
 * every structure's order and conductor count, and max_iters; a later call
 * with the same key builds that configuration without timing (from_cache =
 * 1).  The runs execute the batch, so the meshes must be valid; the panels
 * are copied and the meshes may be destroyed afterwards. */
typedef struct {
    int groups;
    int iters;
    double ms;        /* per run when timed, or as cached */
    int from_cache;
} gbem_batch_tuning;
gbem_status gbem_batch_autotune(gbem_ctx* ctx, int count, gbem_mesh_t* const* meshes, int max_iters,
                                const char* cache_path, gbem_batch_t** out, gbem_batch_tuning* report);

/* Extraction server (continuous batching).  Requests are meshed on the host
 * when submitted, so their device footprint is known; they wait in arrival
 * order and are admitted by `slots` worker threads (each with its own
 * context and stream) whenever a worker is free: the first waiting request,
 * in arrival order, that fits in hbm_budget bytes next to the requests
 * already running.  A smaller request may pass the head of the queue while
 * the head waits for memory, at most 8 times; then nothing is admitted
 * before the head, so a large request is not starved.  Admitted
 * requests run concurrently and overlap on the device; geometry, matrix,
 * factor and right-hand sides stay on the device for the request's life.  A
 * request larger than the whole budget completes with GBEM_ERR_OOM.  The
 * paper has no serving layer; every extraction follows Sec. 3 as above. */
typedef struct gbem_server_s gbem_server_t;
typedef struct {
    long long id;       /* the caller's request id */
    int status;         /* gbem_status of the extraction */
    int n_panels;
    int n_cond;
    double residual;    /* final relative residual of the solve */
    double submit_s;    /* seconds since server creation: submitted, */
    double start_s;     /* admitted, */
    double done_s;      /* completed */
    long long c_offset; /* offset of this result's n_cond x n_cond C in the poll buffer */
} gbem_result_info;
gbem_status gbem_server_create(int device, size_t hbm_budget, int slots, gbem_precision prec,
                               gbem_server_t** out);
/* Queue one extraction (boxes and mesh parameters as for gbem_mesh).
 * bytes_needed (may be NULL) receives the device bytes it will hold. */
gbem_status gbem_server_submit(gbem_server_t* srv, long long id, const gbem_box* boxes, int nbox,
                               const gbem_mesh_params* params, double eps_r, size_t* bytes_needed);
/* Move up to max_results completed results into infos (and their capacitance
 * matrices, back to back, into C of c_capacity doubles).  With wait_ms > 0 and
 * nothing completed, wait up to wait_ms for a completion. */
gbem_status gbem_server_poll(gbem_server_t* srv, gbem_result_info* infos, double* C, long long c_capacity,
                             int max_results, int* count, int wait_ms);
gbem_status gbem_server_stats(gbem_server_t* srv, int* queued, int* running, size_t* reserved,
                              size_t* peak_reserved);
/* Stop the workers (each finishes the request it is running; queued requests
 * are dropped) and release everything. */
void gbem_server_destroy(gbem_server_t* srv);

/* Matrix order N and the number of panel pairs by class: pairs evaluated by
 * closed form, and by Gauss-Legendre order 1..6 (counts[0] closed form,
 * counts[n] order n; array of 7).  Waits for the assembly stream. */
gbem_status gbem_matrix_info(gbem_matrix_t* mat, int* n, long long* counts);
/* The pairs of each of the 14 evaluation classes of the assembly (array of
 * 14): counts[0] near parallel and counts[1] near perpendicular pairs
 * (closed-form corner sums in FP64, Sec. 3.4, Eqs. "parallel" and
 * "orthogonal"), counts[2n] and counts[2n + 1] the parallel and
 * perpendicular far pairs of Gauss-Legendre order n = 1..6 (n^4 evaluations
 * of 1/r each).  For a triangle mesh: counts[0] self pairs, [1] pairs
 * sharing a vertex, [2] near pairs, [3..6] far pairs of product-rule order
 * 3..6, the rest 0.  Waits for the assembly stream. */
gbem_status gbem_matrix_class_counts(gbem_matrix_t* mat, long long* counts);
/* Waits for the matrix's last stream, then hands its device buffers to the
 * context, which offers them to the next matrix of the same size (see
 * gbem_bytes_in_use); a context made by the server frees them at once. */
void gbem_matrix_destroy(gbem_matrix_t* mat);

/* ---------------------------------------------------------------------------
 * Several dielectrics (Sec. 4).  A layered stack: the box enclosure
 * [lo, hi] (um) cut by the planes z = z[1] < ... < z[n_layers-1] into
 * n_layers horizontal layers (z[0] = lo[2], z[n_layers] = hi[2]) of relative
 * permittivity eps_r[a], with disjoint cuboid conductors strictly inside the
 * enclosure (no box touches another or the enclosure; a box's bottom and top
 * lie off the layer planes).  A box may cross layer planes, as a via does:
 * its side faces are cut where they cross, and each interface is cut along
 * the footprints of the boxes that cross it and holed there.  face_bc[2k + s] sets the enclosure face normal to axis
 * k at lo[k] (s = 0) or hi[k] (s = 1): GBEM_FACE_GROUND (u = 0),
 * GBEM_FACE_NEUMANN (insulating, du/dn = 0) or a conductor id >= 0 (the
 * face is an electrode held at that conductor's potential).
 *
 * Panels: the conductors' faces cut as gbem_mesh cuts them with cells of at
 * most h; the enclosure faces (side faces cut at every layer plane) and the
 * interfaces z = z[a] with cells of at most h_outer (0: h).
 *
 * The system (Sec. 4, "Linear Equation"): for every layer a and every panel
 * I_i of its boundary one row
 *     (1/2) |I_i| u_i + sum_k Q^a_ik u_k - sum_j U_ij q^a_j = 0,
 * U_ij = int int 1/(4 pi |x-y|), Q^a_ik = int int <x-y, n_a(y)>/(4 pi |x-y|^3)
 * over I_i x I_k, n_a the outward normal of the layer, u and q = du/dn_a
 * constant on every panel.  Across an interface u is continuous and
 * eps_a q^a = -eps_b q^b.  Rows: for a = 0, 1, ... the panels of layer a's
 * boundary in panel order.  Columns: for each panel in order its unknown u
 * (insulating faces and interfaces) and then its unknown q (all panels but
 * insulating faces; on an interface the flux of the layer below).
 * Right-hand side m: conductor cond_ids[m] at 1 V, every other conductor and
 * the grounded faces at 0 V.  The charge of conductor n is
 * eps0 sum over its panels of eps_a q^a_j |I_j| (farads with lengths in um
 * scaled by 1e-6).  Entries by closed-form corner sums for near pairs and
 * Gauss-Legendre for far ones; the matrix is not symmetric and is factored
 * by LU with partial pivoting (see gbem_stack_assemble for the precisions).
 * ------------------------------------------------------------------------- */
#define GBEM_MAX_LAYERS 16
#define GBEM_FACE_GROUND (-1)
#define GBEM_FACE_NEUMANN (-2)
#define GBEM_PANEL_INTERFACE (-3)  /* the cond value of interface panels */

typedef struct {
    double lo[3];
    double hi[3];
    int32_t n_layers;
    double z[GBEM_MAX_LAYERS + 1];
    double eps_r[GBEM_MAX_LAYERS];
    int32_t face_bc[6];
    double h;        /* largest cell edge on conductors */
    double h_outer;  /* largest cell edge on faces and interfaces (0: h) */
    /* graded != 0: the paper's partition for the main net main_conductor
     * instead of uniform cells (h and h_outer then cap the panel edges):
     * conductor faces by the rule of Sec. 3.3 (as gbem_mesh_graded: |I| <= p4
     * within p5 of the main net, p4 p3 (d/p5)^3 beyond, p4 = p1 on faces
     * that look toward the main net and p1 p2 on the others), enclosure faces
     * by the same rule with p4 = p1 (Sec. 4 keeps it for the outer boundary),
     * interfaces by the rule of Sec. 4 (p4 p3 (d/p5)^2 beyond, p4 = p1). */
    int32_t graded;
    int32_t main_conductor;
    double p1, p2, p3, p5;
} gbem_stack;

typedef struct gbem_stack_s gbem_stack_t;

/* Mesh a stack and lay out its system (host); on a device context also
 * upload the geometry.  GBEM_ERR_MESH for boxes outside the enclosure or with
 * a bottom or top on a layer plane, touching boxes, or no conductor; GBEM_ERR_ARG for malformed
 * parameters or more than 32768 equations. */
gbem_status gbem_stack_mesh(gbem_ctx* ctx, const gbem_stack* stack, const gbem_box* boxes, int nbox,
                            gbem_stack_t** out);
gbem_status gbem_stack_info(const gbem_stack_t* s, int* n_panels, int* n_eq, int* n_cond);
/* The panels (each pointer may be NULL): axis, geo (5 per panel: plane,
 * lo0, hi0, lo1, hi1 as gbem_mesh_panels), kind (0 conductor face,
 * 1 enclosure face, 2 interface), cond (conductor id, GBEM_FACE_GROUND,
 * GBEM_FACE_NEUMANN or GBEM_PANEL_INTERFACE), region_a (the layer whose
 * boundary it is; the layer below for an interface), region_b (the layer
 * above an interface, else -1), sign (the outward normal of region_a is
 * sign * e_axis), cond_ids (n_cond, ascending: the right-hand sides). */
gbem_status gbem_stack_panels(const gbem_stack_t* s, int8_t* axis, double* geo, int32_t* kind, int32_t* cond,
                              int32_t* region_a, int32_t* region_b, int8_t* sign, int32_t* cond_ids);
/* Assemble the system and its right-hand sides on the device.  GBEM_FP64:
 * every entry in FP64 (closed forms or Gauss-Legendre, about 1e-11
 * relative), factored by LU in FP64.  GBEM_MIXED: near pairs (gap below 1.5
 * largest edges) in FP64 closed form, far pairs by FP32 Gauss-Legendre
 * (about 1e-7 relative), the system kept in FP64 and factored in FP32, the
 * solve refined against the FP64 system.  Allocates np^2 doubles plus np^2
 * doubles (FP64) or floats (mixed), np = n_eq rounded up to 64, and the
 * solve's buffers; enqueues only. */
gbem_status gbem_stack_assemble(gbem_stack_t* s, gbem_precision prec, gbem_stream stream);
/* The assembled matrix (n_eq x n_eq, row-major) and right-hand sides
 * (n_eq x n_cond, row-major) on the host; either may be NULL.  Waits. */
gbem_status gbem_stack_system(gbem_stack_t* s, double* M_host, double* B_host);
/* Capacitance matrix in farads, n_cond x n_cond row-major into C_host
 * (C[n][m] = charge on conductor cond_ids[n] for right-hand side m).
 * Assembles first (FP64) if needed, factors once (LU, partial pivoting),
 * then corrects X += (LU)^-1 P (B - M X), the residual in FP64 against the
 * assembled system, until max |B - M X| / max |B| over the right-hand sides
 * is at most the context's ir_tol (1e-11), at most ir_max_iter (10) times;
 * resid (may be NULL) receives that ratio.  GBEM_ERR_NOT_SPD if a pivot is
 * exactly zero (singular system), GBEM_ERR_NOCONV if the tolerance is
 * missed (C_host is still written).  Waits for the stream. */
gbem_status gbem_stack_capacitance(gbem_stack_t* s, gbem_stream stream, double* C_host, double* resid);
/* Corrections the last gbem_stack_capacitance made. */
gbem_status gbem_stack_iterations(const gbem_stack_t* s, int* iters);
void gbem_stack_destroy(gbem_stack_t* s);

#ifdef __cplusplus
}
#endif
#endif /* GBEM_H */
