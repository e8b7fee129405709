/*
 * wave.h -- C ABI of the GB300 (sm_103a) damped acoustic wave library.
 *
 * The library implements the hot path of Kukreja et al., "Devito: automated
 * fast finite difference computation" (arXiv 1608.08658):
 *
 *   * the forward leapfrog solve of  m u_tt - lap(u) + eta u_t = q
 *     (Eq. 1 with the damping term of Listing 1), with receiver sampling,
 *   * its exact discrete adjoint (Listing 2, Eq. 4),
 *   * the adjoint-state FWI gradient of the objective of Eq. 2 (Eq. 3).
 *
 * Discretisation (shared with the FP64 oracle by specification only):
 *   a u^{k+1} - b u^k + c u^{k-1} = P_s^T q^k,   k = 0 .. nt-2,
 *   a = m/dt^2 + eta/(2dt),  b = 2m/dt^2 + L,  c = m/dt^2 - eta/(2dt),
 *   u^{-1} = u^0 = 0,   d^n = P_r u^n for n = 0 .. nt-1,
 * where L is the centred Laplacian of even space order 2..16 (Sec. IV-A1)
 * with zero values outside the computational grid, eta is a quadratic sponge
 * in the nbl absorbing points added on every side (Sec. V-D), and P_s / P_r
 * are multilinear (bi/tri-linear) sparse-point interpolation operators (Sec. IV).
 *
 * Conventions common to every entry point
 * ---------------------------------------
 * Axes:   axis 0 is x (fastest in memory); axis 1 is y in 3D or depth z in 2D;
 *         axis 2 is depth z in 3D.  A physical field is a dense C-order array
 *         [N_z][N_y][N_x] (3D) or [N_z][N_x] (2D) of float32.
 * Units:  spacing in m, time in ms, velocity in km/s, squared slowness
 *         m = 1/v^2 in s^2/km^2; frequencies in kHz.
 * Memory: every array argument may be a device pointer (CUDA global memory on
 *         the context's device) or a host pointer (pageable or pinned); the
 *         library detects which and stages host arrays through its own
 *         workspace.  The caller owns all argument buffers; the context owns
 *         its workspace (wavefields, coefficients, snapshots, checkpoints).
 *         Each array must hold the elements documented for its argument: a
 *         raw pointer carries no size, so the library cannot check it (the
 *         Python binding checks every array before the call).
 * Streams: work is enqueued on the CUDA stream passed as `stream`
 *         (cudaStream_t cast to void*, NULL = legacy default stream).  Every
 *         compute entry point returns after that stream has completed the
 *         call's work, so outputs are ready on return.
 * Errors: every call returns an int status, 0 on success (the generated
 *         operator of Listing 3 also returns 0).  Failures never abort the
 *         process and never throw across the ABI; wave_last_error() gives a
 *         one-line description.  A call that fails leaves its outputs
 *         unspecified.
 * Threads: a context may be used by one host thread at a time.
 */
#ifndef WAVE_H_
#define WAVE_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define WAVE_API __attribute__((visibility("default")))
#else
#define WAVE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define WAVE_OK                 0
#define WAVE_ERR_INVALID_ARG    1  /* null pointer, bad size, bad space order, ... */
#define WAVE_ERR_POINT_OUTSIDE  2  /* a source/receiver lies outside the physical domain */
#define WAVE_ERR_UNSTABLE_DT    3  /* dt above the leapfrog stability limit */
#define WAVE_ERR_OUT_OF_MEMORY  4  /* workspace would exceed the budget, or cudaMalloc failed */
#define WAVE_ERR_CUDA           5  /* a CUDA runtime/driver call or kernel launch failed */
#define WAVE_ERR_TIMEOUT        6  /* a bounded device-side wait expired (kernel gave up) */
#define WAVE_ERR_NOT_SUPPORTED  7  /* feature or size not supported by the library or the device */

typedef struct wave_context wave_context;

/* Physical grid plus absorbing layer (Sec. V-D: the layer is added outside the
 * model on every side, so the computational grid has N_d + 2*nbl points per
 * axis and its node 0 sits at origin_d - nbl*spacing_d).
 * sponge_vref (km/s) sets the sponge strength
 *   eta(i) = sum_d eta_max_d (delta_d(i)/nbl)^2,
 *   eta_max_d = 3 * sponge_vref * ln(1000) / (2 * nbl * spacing_d),
 * with delta_d the number of points into the layer (1..nbl); it is a fixed
 * parameter (not derived from m) so that eta does not depend on the model. */
typedef struct {
  int32_t ndim;          /* 2 or 3 */
  int32_t nbl;           /* absorbing points per side, in [0, 2^20] */
  int64_t shape[3];      /* physical points per axis, x-first, each in [2, 2^20]
                            (WAVE_ERR_INVALID_ARG otherwise, and for a computational
                            grid above 2^40 points); shape[2] ignored in 2D.
                            A grid whose axis 1 needs more than 65535 CTA tiles of 14-16
                            rows is WAVE_ERR_NOT_SUPPORTED. */
  double spacing[3];     /* grid spacing per axis, m, > 0 */
  double origin[3];      /* coordinate of physical node 0 per axis, m */
  double sponge_vref;    /* km/s, > 0 when nbl > 0 */
} wave_geometry;

/* A set of off-grid points (sources or receivers): n points, `coords` holds
 * n*ndim float32 values, x-first per point, physical coordinates in m (host
 * or device pointer).  Interpolation (Sec. IV, sparse-point interpolation):
 * per axis t = (p - o)/h on the computational grid, i = floor(t), f = t - i,
 * (i = n-2, f = 1 on the last node); corner weights are products of (1-f, f).
 * Every point must lie inside the physical domain (WAVE_ERR_POINT_OUTSIDE).
 * n is in [0, 2^28) (WAVE_ERR_INVALID_ARG otherwise). */
typedef struct {
  int64_t n;
  const float* coords;
} wave_points;

/* Storage of the forward wavefield for the imaging condition of Eq. 3.
 * FULL_*: every time level u^1..u^{nt-1} is kept (Sec. IV-B4 "save" flag).
 * CHECKPOINT_*: a buffer of F levels (as many as fit the budget / free memory,
 * or the interval set with wave_context_set_checkpoint_interval) first holds
 * the last F levels, stored during the forward sweep; the earlier levels are
 * recomputed segment by segment from exact FP32 checkpoints (u^{k-1}, u^k)
 * into the same buffer once the adjoint sweep has consumed the tail.
 * Recomputation is deterministic: every mode gives the same gradient as the
 * FULL mode of the same format, bit for bit.
 * *_BF16 / *_FP16: snapshots are stored in 16 bits with one power-of-two
 * scale per slab of 64 (x) by 2 (axis 1) points of one plane; all stencil
 * arithmetic and gradient accumulation stay FP32.
 * AUTO: FULL_FP32 if it fits the budget, else CHECKPOINT_FP32. */
typedef enum {
  WAVE_SNAP_FULL_FP32 = 0,
  WAVE_SNAP_FULL_BF16 = 1,
  WAVE_SNAP_FULL_FP16 = 2,
  WAVE_SNAP_CHECKPOINT_FP32 = 3,
  WAVE_SNAP_CHECKPOINT_BF16 = 4,
  WAVE_SNAP_CHECKPOINT_FP16 = 5,
  WAVE_SNAP_AUTO = 6
} wave_snap_mode;

/* ---- context ----------------------------------------------------------- */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * workspace the context may hold (0 = no cap beyond free device memory).
 * Workspace is allocated lazily by the compute calls and reused across calls.
 * Errors: INVALID_ARG (ctx NULL), CUDA (no device / sm_103a kernels cannot run). */
WAVE_API int wave_context_create(wave_context** ctx, int device, size_t hbm_budget_bytes);

/* Release the context and all its workspace.  NULL is accepted. */
WAVE_API int wave_context_destroy(wave_context* ctx);

/* Bytes of device workspace currently held by the context. */
WAVE_API size_t wave_context_workspace_bytes(const wave_context* ctx);

/* Release all workspace (the next call re-allocates what it needs). */
WAVE_API int wave_context_trim(wave_context* ctx);

/* Checkpoint interval S (steps) for CHECKPOINT_* modes; 0 = choose from the
 * budget (default). */
WAVE_API int wave_context_set_checkpoint_interval(wave_context* ctx, int steps);

/* Limit, in nanoseconds, of each bounded wait by which a stencil-step kernel
 * waits for its tile loads or for its own consumer warps (failure detection;
 * the paper has no counterpart).  A wait first suspends in hardware for a
 * short system-dependent window, in which waits for data normally complete;
 * the limit counts from there.  A kernel whose wait runs out records a
 * timeout in the context's device status word, lets every copy it has issued
 * land (those drain waits keep the default limit, so no CTA exits with a copy
 * in flight) and returns; the call then returns WAVE_ERR_TIMEOUT and the
 * context stays usable.  ns = 0 restores the default of 10 s.  Sessions take
 * the limit in force when they are created.  Errors: INVALID_ARG (ctx NULL). */
WAVE_API int wave_context_set_wait_limit_ns(wave_context* ctx, uint64_t ns);

/* Time levels computed per pass over memory by forward modelling without
 * sources (wave_forward / wave_forward_ex with an empty source set: the
 * propagation of a given initial state), at space order 8 in 3D.  levels = 2
 * fuses two leapfrog levels of Listing 1 / Eq. 1 per pass (temporal blocking,
 * listed as future work in Sec. VI): 10 bytes of memory traffic per point
 * update instead of 16, at the price of recomputing the first level on a
 * halo of R points around each tile; the results equal those of single
 * levels up to FP32 rounding.  Calls with sources, other orders, 2D grids,
 * the adjoint, gradient and Born paths always take one level per pass.
 * levels = 1 (the default) always takes one.  Errors: INVALID_ARG (ctx NULL,
 * levels not 1 or 2). */
WAVE_API int wave_context_set_time_blocking(wave_context* ctx, int levels);

/* Work decomposition of the plain 3D forward steps (the leapfrog update of
 * Eq. 1 with the source injection and receiver interpolation of Sec. III-C;
 * a scheduling choice with no counterpart in the paper).  The default
 * decomposition cuts each column of 64 x BY points into z chunks of equal
 * length, one CTA each; on grids that fill the GPU only a few times over, the
 * last wave of CTAs leaves most of it idle.  Column segments instead lay the
 * columns end to end and give every resident CTA an equal run of planes
 * (crossing from one column into the next where it must); such a step also
 * injects its source row and samples its receiver row itself, so that a time
 * step is one launch.  mode 1 (the default) takes segments where a cost model
 * of the two decompositions favours them (grids of fewer than 4 waves), 0
 * never, 2 always.  Results are identical bit for bit in every mode.  Steps
 * that store snapshots and the adjoint, gradient and Born sweeps keep the z
 * chunks.  Errors: INVALID_ARG (ctx NULL, mode not 0, 1 or 2). */
WAVE_API int wave_context_set_column_segments(wave_context* ctx, int mode);

/* Host-only: the column segments the plain 3D step takes for a grid of
 * `columns` columns (x tiles of 64 times axis-1 tiles of BY points) of nz
 * planes, whose z-chunk grid has `chunks` chunks per column, with `slots`
 * resident CTAs.  A CTA's cost is its planes plus 4 + R plane times for every
 * column segment it starts (the fill of its register queue); the runs are cut
 * along the tile-major plane sequence so that the largest cost is as small as
 * the run count allows, at most one run per max(16, 2R) planes and per slot.
 * Segments are taken for grids of fewer than 4 waves where that cost is at
 * least 3 % below the z-chunk grid's, or always with force != 0.
 *   run_start: out, n_runs + 1 entries: run b covers planes
 *              [run_start[b], run_start[b+1]) of the sequence (column c holds
 *              planes c*nz .. c*nz + nz - 1); may be NULL when cap = 0;
 *   n_runs:    out, the number of runs, 0 where the z chunks are kept.
 * Errors: INVALID_ARG (columns, nz, chunks or slots < 1, space_order not even
 * in [2, 16], n_runs NULL, more than cap - 1 runs). */
WAVE_API int wave_column_runs_for(long long columns, int nz, int chunks, int space_order, long long slots, int force,
                                  long long* run_start, int cap, int* n_runs);

/* Host-only: the number of chunks the streamed axis of the plain 3D step is cut
 * into for a grid of `columns` column tiles of nz planes with `slots` resident
 * CTAs (the z-chunk grid has columns * chunks CTAs).  Chunks keep at least
 * max(32, 4R) planes; where that still allows 8 waves of CTAs, the count is
 * the one, among those giving 8 to 16 waves, whose last wave is fullest (the
 * smallest within 1 % of the best), else the most chunks allowed.
 *   chunks: out, the number of chunks (>= 1).
 * Errors: INVALID_ARG (columns, nz or slots < 1, space_order not even in
 * [2, 16], chunks NULL). */
WAVE_API int wave_z_chunks_for(long long columns, int nz, int space_order, long long slots, int* chunks);

/* Test hook of the same failure-detection path (no counterpart in the paper):
 * the context's next stencil-step launch issues none of its tile loads, so
 * every wait of its consumer warps runs out after the wait limit, the kernel
 * records the timeout and returns, and the call returns WAVE_ERR_TIMEOUT.
 * Nothing faults and no wait is unbounded; later launches run normally.  Set a
 * short limit first: with the default, each wave of resident CTAs of that one
 * launch waits 10 s.  A session captured after this call takes the withheld
 * launch into its graph.  Errors: INVALID_ARG (ctx NULL). */
WAVE_API int wave_context_withhold_next_loads(wave_context* ctx);

/* Storage plan of the context's last wave_gradient / wave_jacobian_adjoint
 * call: snapshot buffer levels F, parts per checkpointed segment k, and the
 * number of checkpointed segments (0 = full storage). */
WAVE_API int wave_context_storage_plan(const wave_context* ctx, int* levels, int* parts, int* segments);

/* The storage plan wave_gradient chooses for the forward wavefield of Eq. 3
 * (the snapshots the imaging condition reads), for given sizes; host-only, no
 * device work, usable without a GPU.  A buffer of `levels` snapshot levels
 * holds the last levels of the forward sweep; the earlier levels are covered by
 * `segments` checkpointed segments of parts * levels levels, each starting at
 * an exact FP32 checkpoint of two wavefields and rebuilt part by part in the
 * reverse sweep (segments = 0: every level stored).
 *   nt:          time levels (>= 2);
 *   level_bytes: bytes of one stored snapshot level (> 0);
 *   field_bytes: bytes of one FP32 wavefield (a checkpoint holds two);
 *   avail_bytes: memory for the buffer and the checkpoints;
 *   checkpoint:  0 = store every level (full storage), else plan checkpoints;
 *   checkpoint_interval: > 0 fixes the buffer at that many levels (one part
 *                per segment), 0 = the smallest parts per segment (1, 2, 4
 *                .. 64) for which a buffer fits, with the largest such buffer.
 * levels, parts, segments may be NULL.
 * Errors: INVALID_ARG (nt < 2, level_bytes = 0, checkpoint_interval < 0);
 * OUT_OF_MEMORY (with checkpoint and no fixed interval, when not even a
 * one-level buffer with its checkpoints fits). */
WAVE_API int wave_storage_plan_for(int nt, size_t level_bytes, size_t field_bytes, size_t avail_bytes, int checkpoint,
                                   int checkpoint_interval, int* levels, int* parts, int* segments);

/* Text of a status code, and the last error message of a context. */
WAVE_API const char* wave_error_string(int status);
WAVE_API const char* wave_last_error(const wave_context* ctx);

/* ---- method -------------------------------------------------------------- */

/* Forward modelling (Listing 1; Eq. 1 with damping).
 * m:     physical squared slowness, dense [N_z][N_y][N_x] (2D: [N_z][N_x]).
 * src:   n_s source points; q: source traces [nt][n_s] (row k enters the
 *        update of time row k, producing u^{k+1}; row nt-1 is unused).
 * rec:   n_r receiver points; d_out: receiver data [nt][n_r], d^n = P_r u^n.
 * dt:    time step (ms), must not exceed wave_dt_max() for v_max = 1/sqrt(min m).
 * nt:    number of time levels (>= 2); space_order: even, 2..16.
 * Errors: INVALID_ARG, POINT_OUTSIDE, UNSTABLE_DT, OUT_OF_MEMORY, CUDA, TIMEOUT. */
WAVE_API int wave_forward(wave_context* ctx, const wave_geometry* geom, const float* m,
                 const wave_points* src, const float* q, const wave_points* rec,
                 float* d_out, float dt, int nt, int space_order, void* stream);

/* Same as wave_forward with optional initial and final states on the
 * computational grid (dense [n_z][n_y][n_x] float32, n_d = N_d + 2 nbl):
 * u_init_prev = u^{-1}, u_init = u^0 (NULL = zero, the initial condition of
 * Eq. 1); u_final_prev = u^{nt-2}, u_final = u^{nt-1} are written when not
 * NULL.  Used to check single steps of the stencil against the oracle. */
WAVE_API int wave_forward_ex(wave_context* ctx, const wave_geometry* geom, const float* m,
                    const wave_points* src, const float* q, const wave_points* rec,
                    float* d_out, float dt, int nt, int space_order,
                    const float* u_init_prev, const float* u_init,
                    float* u_final_prev, float* u_final, void* stream);

/* Adjoint modelling (Listing 2 read as the exact transpose of wave_forward;
 * Eq. 4 with P_r^* applied to receiver-side traces).
 * y:     receiver-side traces [nt][n_r] (row 0 has no effect: u^0 is fixed);
 * q_out: source-side traces [nt][n_s] = F^T y; row nt-1 is zero.
 * Recursion: lam_{j-1} = (b lam_j - c lam_{j+1} + P_r^T y^j)/a, j = nt-1..1,
 * lam_{nt-1} = lam_nt = 0, q_out^k = P_s lam_k.
 * Errors: as wave_forward. */
WAVE_API int wave_adjoint(wave_context* ctx, const wave_geometry* geom, const float* m,
                 const wave_points* src, const wave_points* rec, const float* y,
                 float* q_out, float dt, int nt, int space_order, void* stream);

/* FWI gradient by the adjoint-state method (Eq. 2-4).
 * Runs the forward model, forms the residual r = P_r u - d_obs [nt][n_r], the
 * objective phi = 0.5 sum r^2 (accumulated in FP64) and the gradient
 *   g = -(1/dt^2) sum_{j=1}^{nt-1} u^j (lam_{j-1} - 2 lam_j + lam_{j+1})
 * with lam the adjoint field for y = r, folded onto the physical grid by the
 * transpose of the edge-replicating padding.
 * grad_out: physical grid, same layout as m.  phi_out: host double (may be NULL).
 * resid_out: optional [nt][n_r] residual (NULL = not returned).
 * snap_mode: a wave_snap_mode value.
 * Errors: as wave_forward; OUT_OF_MEMORY when the chosen storage cannot fit. */
WAVE_API int wave_gradient(wave_context* ctx, const wave_geometry* geom, const float* m,
                  const wave_points* src, const float* q, const wave_points* rec,
                  const float* d_obs, float* grad_out, double* phi_out, float* resid_out,
                  int snap_mode, float dt, int nt, int space_order, void* stream);

/* Multi-shot FWI gradient: the objective of Eq. 2 summed over shots s,
 * phi = sum_s phi_s, and its gradient sum_s grad_s, for nshots independent
 * sources on the same model and geometry.  srcs[i] / recs[i] are the points of
 * shot i, q[i] its traces [nt][n_s,i], d_obs[i] its observed data [nt][n_r,i]
 * (host or device pointers).  Shots run one after another on the GPU, each
 * shot's imaging term accumulating into one computational-grid gradient that
 * is folded once.  Other arguments and errors as wave_gradient. */
WAVE_API int wave_gradient_shots(wave_context* ctx, const wave_geometry* geom, const float* m, int nshots,
                                 const wave_points* srcs, const float* const* q, const wave_points* recs,
                                 const float* const* d_obs, float* grad_out, double* phi_out, int snap_mode,
                                 float dt, int nt, int space_order, void* stream);

/* Gradient back-propagation for a given receiver-side adjoint source: same as
 * wave_gradient but with the residual replaced by `y` [nt][n_r] (so that
 * grad_out = J^T y, the vector-Jacobian product of the map m -> d used by an
 * autograd backward pass).  d_out, if not NULL, receives the forward data. */
WAVE_API int wave_jacobian_adjoint(wave_context* ctx, const wave_geometry* geom, const float* m,
                          const wave_points* src, const float* q, const wave_points* rec,
                          const float* y, float* grad_out, float* d_out,
                          int snap_mode, float dt, int nt, int space_order, void* stream);

/* ---- resident requests (serving) ------------------------------------------ */

/* A session is one forward-modelling request (Listing 1) kept resident on the
 * device so that many requests of different grids and space orders can be in
 * flight at once, each on its own CUDA stream, and advanced a few steps at a
 * time by a host scheduler (continuous batching).  Its device memory (two
 * wavefield slots, coefficients, staged model and source traces, receiver
 * data, point structures) is allocated at creation, counted against the
 * context's budget and released by wave_session_destroy.  Steps are issued as
 * replays of a CUDA graph of `graph_chunk` steps captured at creation (the
 * sparse kernels read the time row from a device counter), plus ordinary
 * launches for the steps that do not fill a whole chunk.  Results are the same
 * as wave_forward's for the same inputs. */
typedef struct wave_session wave_session;

/* Device bytes a session for these arguments would hold (admission by HBM
 * footprint).  Validates the geometry and points like wave_forward. */
WAVE_API int wave_session_footprint(wave_context* ctx, const wave_geometry* geom, const wave_points* src,
                                    const wave_points* rec, int nt, int space_order, size_t* bytes_out);

/* Create a session: copies m [N_z][N_y][N_x] and q [nt][n_s] (host or device)
 * into its own memory, checks dt, builds the point structures, captures the
 * step graph (graph_chunk even, 0 = no graph) on `stream`; returns after the
 * stream has completed the set-up.  Errors: as wave_forward. */
WAVE_API int wave_session_create(wave_context* ctx, wave_session** session, const wave_geometry* geom,
                                 const float* m, const wave_points* src, const float* q, const wave_points* rec,
                                 float dt, int nt, int space_order, int graph_chunk, void* stream);

/* Enqueue about `steps` more time steps (whole graph chunks when possible) on
 * the session's stream without waiting; *steps_left receives the number of
 * steps not yet enqueued. */
WAVE_API int wave_session_advance(wave_session* session, int steps, int* steps_left);

/* Batched advance of several resident sessions (continuous batching of the
 * serving loop; Listing 1 steps of Eq. 1 for every request): enqueue up to
 * `steps` more time steps of each of the n sessions on `stream` without
 * waiting, with one stencil launch per step for all sessions of the same space
 * order, dimension and spacing variant, and one source-injection and one
 * receiver-sampling launch per step for all of them.  A session whose steps
 * run out during the call takes no part in the later launches.  Each session
 * keeps its own fields, tensor maps and step count, and its results equal
 * those of wave_session_advance and of wave_forward bit for bit.  All sessions
 * must share one context; a session must not be advanced on another stream
 * while this call's work is in flight.  Sessions created with graph_chunk = 0
 * suit this call (their captured graphs are not used).  The request tables
 * are staged through a page-locked buffer of the context, which the next call
 * rewrites only after this call's upload has completed.
 * Errors: INVALID_ARG (NULL or foreign sessions, n or steps negative); CUDA;
 * OUT_OF_MEMORY (table workspace beyond the budget). */
WAVE_API int wave_sessions_advance(wave_session* const* sessions, int n, int steps, void* stream);

/* *done = 1 when every step has been enqueued and has completed. */
WAVE_API int wave_session_query(wave_session* session, int* done);

/* Copy the receiver data [nt][n_r] to d_out (host or device) once all steps
 * are enqueued; waits for the session's stream. */
WAVE_API int wave_session_read(wave_session* session, float* d_out);

/* Release the session's device memory (waits for its stream). NULL accepted. */
WAVE_API int wave_session_destroy(wave_session* session);

/* Budget left for new sessions and workspace (0 when the context has no cap). */
WAVE_API size_t wave_context_budget_free(const wave_context* ctx);

/* Linearised (Born) modelling: dd = J dm, the derivative of wave_forward's
 * receiver data with respect to m in the direction dm (J is the Jacobian whose
 * transpose Eq. 3 applies; wave_jacobian_adjoint computes J^T y).  The
 * scattered field solves the rows of Eq. 1 differentiated in m:
 *   a du^{k+1} - b du^k + c du^{k-1} = -dm (u^{k+1} - 2u^k + u^{k-1}) / dt^2,
 * du^{-1} = du^0 = 0, dd^n = P_r du^n; dm is padded like m.
 * dm: physical grid like m; d_out: [nt][n_r].  Errors: as wave_forward. */
WAVE_API int wave_born(wave_context* ctx, const wave_geometry* geom, const float* m, const float* dm,
                       const wave_points* src, const float* q, const wave_points* rec, float* d_out, float dt,
                       int nt, int space_order, void* stream);

/* ---- helpers (host-side, no device work) ---------------------------------- */

/* Centred second-derivative weights [w_0, w_1, .., w_R], R = space_order/2
 * (Sec. IV-A1; closed form w_0 = -2 sum 1/j^2,
 * w_j = 2 (-1)^{j+1} (R!)^2 / (j^2 (R-j)! (R+j)!)).  w_out holds R+1 doubles. */
WAVE_API int wave_fd_weights(int space_order, double* w_out);

/* Sparse-point interpolation operator P of a point set (Sec. IV; P_s and P_r
 * of the discretisation above), read back from the structure the library
 * builds to inject at and sample these points; host-only, no device work,
 * usable without a GPU.
 *   geom: as for wave_forward; pts: coordinates in HOST memory;
 *   index_out: pts->n * 2^ndim int64, the computational-grid points of each
 *     point's cell as linear indices of the dense computational grid, x
 *     fastest: (iz * n_y + iy) * n_x + ix in 3D, iz * n_x + ix in 2D
 *     (n_d = N_d + 2 nbl);
 *   weight_out: pts->n * 2^ndim float32 weights; entry c of a point is the
 *     cell corner whose axis-a index is the upper one when bit a of c is set.
 * Errors: INVALID_ARG (NULL pointer, bad geometry, n < 0 or n >= 2^28);
 * POINT_OUTSIDE (a point outside the physical domain). */
WAVE_API int wave_interpolation_operator(const wave_geometry* geom, const wave_points* pts, int64_t* index_out,
                                         float* weight_out);

/* Leapfrog stability limit dt_max = 2 / (v_max sqrt(sum_d (sum_j |w_j|)/h_d^2))
 * for the undamped scheme; returns a negative value on invalid input. */
WAVE_API double wave_dt_max(int ndim, const double* spacing, int space_order, double v_max);

/* Ricker wavelet r(t_n) = (1 - 2 (pi f0 (t_n - t0))^2) exp(-(pi f0 (t_n - t0))^2),
 * t_n = n dt, n = 0..nt-1 (Sec. V-D source); q_out: nt float32 (host or device). */
WAVE_API int wave_ricker(float* q_out, int nt, float dt, float f0, float t0);

/* ---- allocation-free entry point ------------------------------------------ */

/* The paper has no counterpart to this entry point.  It exists for callers
 * that cannot allocate device memory at the time they need the objective:
 * plug-ins whose host application owns every device allocation through its own
 * pool, and services that must not touch the allocator once a run has started
 * (an allocation there can stall on a device-wide synchronisation or fail under
 * memory pressure at the worst moment).
 *
 * wave_objective_noalloc computes the residual r = d - d_obs and the objective
 * phi = 0.5 * sum r^2 (FP64 accumulation) of Eq. 2 for n receiver samples, the
 * same values wave_gradient returns in resid_out / phi_out, without creating a
 * context and without calling cudaMalloc, cudaFree or any allocating routine.
 * Its scratch is a file-scope device array of WAVE_OBJECTIVE_NOALLOC_MAX_N /
 * WAVE_OBJECTIVE_NOALLOC_CHUNK + 1 doubles (256 KiB plus 8 bytes) that every
 * GPU which loads the library holds until the process exits.
 *   d, d_obs: device arrays of n float32 on the current CUDA device;
 *   r_out:    device array of n float32 receiving r, or NULL;
 *   phi_out:  host double receiving phi;
 *   stream:   CUDA stream (NULL = legacy default); the call copies phi to the
 *             host and returns after the stream has completed its work.
 * The first call on a device looks up the scratch array's device address (with
 * that device current).  The address is kept per device together with the id
 * of the CUDA context it was found in: after a device reset (cudaDeviceReset)
 * the next call sees a new context and looks the address up again.
 * Every call on a device shares the same scratch and overwrites it; calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  Nothing in the scratch needs to start at zero.
 * Errors: INVALID_ARG (NULL pointer, n < 0, n > WAVE_OBJECTIVE_NOALLOC_MAX_N,
 * or an array that is not device memory of the current device); CUDA. */
#define WAVE_OBJECTIVE_NOALLOC_CHUNK 8192LL
#define WAVE_OBJECTIVE_NOALLOC_MAX_N 268435456LL /* 2^28 samples */
WAVE_API int wave_objective_noalloc(const float* d, const float* d_obs, float* r_out, int64_t n,
                                    double* phi_out, void* stream);

/* ---- instrumentation --------------------------------------------------- */

/* Kernel kinds for wave_context_kernel_stats. */
#define WAVE_KERNEL_STEP        0  /* stencil step (forward/adjoint, any epilogue) */
#define WAVE_KERNEL_STEP_SNAP   1  /* stencil step storing a snapshot */
#define WAVE_KERNEL_STEP_GRAD   2  /* adjoint step with the imaging condition */
#define WAVE_KERNEL_SPARSE      3  /* source injection / receiver sampling */
#define WAVE_KERNEL_OTHER       4  /* set-up, residual, fold, snapshot store, copies */
#define WAVE_KERNEL_KINDS       5

/* Enable (1) or disable (0) CUDA-event timing of the context's kernels on the
 * stream they are launched on: every 4th launch of each kind (the first, the
 * fifth, ...) is bracketed by a pair of timing events.  Disabled by default. */
WAVE_API int wave_context_set_profiling(wave_context* ctx, int enable);

/* Launch count (always counted) and total time in ms of one kernel kind since
 * the last reset: the mean event time of its timed launches times its launch
 * count (0 when none was timed); totals over all kinds when kind < 0. */
WAVE_API int wave_context_kernel_stats(wave_context* ctx, int kind, int64_t* launches, double* total_ms);
WAVE_API int wave_context_reset_stats(wave_context* ctx);

/* Compile-time configuration of the stencil-step kernel that the library
 * launches for one (space_order, ndim, kernel, equal_spacing), for profiling
 * records: a measurement taken on a kernel stays valid while this list and the
 * kernel's source are unchanged.  The paper has no counterpart (its code
 * generator fixes such choices per problem, Sec. IV-B).  Host-only: no device
 * work, usable without a GPU.
 *   kernel: 0 plain step, 1/2/3 step storing an FP32/BF16/FP16 snapshot,
 *           4/5/6 adjoint step with the imaging condition reading an
 *           FP32/BF16/FP16 snapshot, 7 Born background step, 8 scattered step;
 *   equal_spacing: nonzero when every axis has the same spacing (selects the
 *           equal-spacing variant where one exists);
 *   out:    receives up to n_out ints, in this order: radius, ndim, kernel,
 *           equal-spacing variant used (0/1), x outputs per CTA, axis-1 outputs
 *           per CTA, x halo, threads per CTA, CTAs per SM asked of the register
 *           allocator, lead-plane design (0/1), planes prefetched, queue-feed
 *           ring stages, per-point ring stages, output planes per queue move,
 *           output planes per renamed queue group, dynamic shared memory bytes.
 *   n_values: receives the number of values of the configuration (16); at
 *           most n_out of them are written.
 * Errors: INVALID_ARG (invalid order, ndim or kernel, NULL out or n_values,
 * n_out < 1). */
WAVE_API int wave_step_kernel_layout(int space_order, int ndim, int kernel, int equal_spacing, int* out, int n_out,
                                     int* n_values);

#ifdef __cplusplus
}
#endif
#endif /* WAVE_H_ */
