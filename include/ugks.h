/*
 * ugks.h -- C ABI of the GB300 UGKS velocity-block sweep.
 *
 * The library advances the reduced distributions h, b and the conservative
 * variables W of the unified gas-kinetic scheme (UGKS) on an unstructured
 * face-list mesh with a discrete velocity grid, one GPU, one CUDA stream.
 * Method: arXiv 2606.15720, Sec. 2.1 (discretisation) and Algorithm 5 (one
 * time step); the velocity-block sweep of Sec. 2.2.2 and Algorithms 1 and 4
 * is the device execution unit.
 *
 * Conventions for every entry point:
 *   * Pointers passed in are HOST pointers unless stated otherwise; the
 *     library copies what it needs at create time and never keeps a caller
 *     pointer.  Output buffers are caller-allocated host memory.
 *   * Every call returns a ugks_status.  On failure the message of the last
 *     error is available from ugks_last_error(ctx) (or ugks_last_error(NULL)
 *     for failures before a context exists).  After UGKS_ERR_CUDA a context
 *     is unusable except for ugks_destroy.
 *   * ugks_step is asynchronous on the context's stream; calls that return
 *     data (moments, residual, get_f, state) synchronise that stream.
 *     Non-finite or non-physical states detected on the device latch into a
 *     status word that the next ugks_moments or ugks_residual reports as
 *     UGKS_ERR_NONFINITE; a bounded device wait that gave up (shared-memory
 *     staging whose copies did not complete) latches UGKS_ERR_TIMEOUT the
 *     same way.  ugks_get_f and ugks_get_state return the raw state
 *     regardless, so that it can be inspected.
 *   * A context is not thread-safe; distinct contexts are independent.
 *   * Units: R = 1/2 (so lambda = 1/T, p = rho T / 2), velocities in
 *     sqrt(2 R T_ref), lengths in the mesh's unit.
 */
#ifndef UGKS_H
#define UGKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ugks_ctx ugks_ctx; /* opaque; owned by the library */

typedef enum {
  UGKS_OK = 0,
  UGKS_ERR_INVALID_ARGUMENT = 1, /* NULL pointer, bad size or parameter */
  UGKS_ERR_MESH = 2,             /* inconsistent mesh (indices, areas, volumes, normals) */
  UGKS_ERR_VGRID = 3,            /* empty grid, negative or non-finite weights */
  UGKS_ERR_OUT_OF_MEMORY = 4,    /* device or host allocation failed */
  UGKS_ERR_CUDA = 5,             /* a CUDA runtime call failed */
  UGKS_ERR_NONFINITE = 6,        /* NaN/Inf or non-positive density / temperature */
  UGKS_ERR_TIMEOUT = 7,          /* a bounded device wait (shared-memory staging) gave up */
  UGKS_ERR_UNSUPPORTED = 8       /* valid request this build does not implement */
} ugks_status;

enum { UGKS_BC_WALL = 1, UGKS_BC_FARFIELD = 2, UGKS_BC_OUTFLOW = 3 };
enum { UGKS_MODEL_BGK = 0, UGKS_MODEL_SHAKHOV = 1 };
enum { UGKS_LIMITER_NONE = 0, UGKS_LIMITER_VENKATAKRISHNAN = 1, UGKS_LIMITER_BARTH_JESPERSEN = 2 };
enum { UGKS_STORAGE_F64 = 0, UGKS_STORAGE_F32 = 1, UGKS_STORAGE_F16 = 2, UGKS_STORAGE_BF16 = 3 };
enum { UGKS_SWEEP_AUTO = 0, UGKS_SWEEP_TILED = 1, UGKS_SWEEP_BLOCKED = 2, UGKS_SWEEP_BLOCKED_FUSED = 3 };

/* Boundary condition of the faces whose neighbour is -(index+1).
 * WALL: diffuse isothermal wall (Sec. 2.1, Eq. 36-38) with wall velocity u
 *       (tangential) and temperature T; rho is ignored (the wall density
 *       follows from the non-penetration condition, Eq. 38).
 * FARFIELD: ghost cell holds the Maxwellian of (rho, u, T).
 * OUTFLOW: ghost cell holds the Maxwellian of the interior cell's W. */
typedef struct {
  int32_t type;
  double rho;
  double u[3];
  double T;
} ugks_bc;

/* Face-list mesh (Sec. 2.1, Eq. 20, 24).  Cells are 0..n_cells-1.
 *   cell_volume[n_cells] > 0, cell_centroid[n_cells][dim]
 *   face_owner[n_faces] in [0, n_cells)
 *   face_neighbor[n_faces]: >= 0 interior cell (different from the owner), or
 *       -(b+1) for boundary condition bc[b]
 *   face_area[n_faces] > 0; face_normal[n_faces][dim] unit, owner -> neighbour
 *   face_centroid[n_faces][dim] in the owner's frame
 *   face_shift[n_faces][dim] or NULL: translation added to the neighbour
 *       centroid across this face (periodic faces); NULL means zero.
 * At most 32 faces per cell. */
typedef struct {
  int32_t dim; /* 1, 2 or 3 */
  int64_t n_cells, n_faces;
  const double *cell_volume;
  const double *cell_centroid;
  const int64_t *face_owner;
  const int64_t *face_neighbor;
  const double *face_area;
  const double *face_normal;
  const double *face_centroid;
  const double *face_shift;
  int32_t n_bc;
  const ugks_bc *bc;
} ugks_mesh;

/* Discrete velocity grid (Sec. 2.1, Eq. 21-22): u[n_v][dim], weight[n_v] >= 0
 * (the velocity-cell volumes omega_k).  The library pads it to a multiple of
 * the velocity block (Sec. 2.2.2, Eq. 47) with zero-weight points.
 * Optional tensor-product declaration: tensor_n[d] > 0 for d < dim declares
 * u[k] = (axis[0][i0], ..., axis[dim-1][i_{dim-1}]) with
 * k = i0 + tensor_n[0] (i1 + tensor_n[1] i2) (first axis fastest) and
 * n_v = the product of the tensor_n; the library checks it against u
 * (UGKS_ERR_VGRID if it does not hold).  All zero: not declared, the library
 * detects the structure from u.  When the fastest axis has 32 points (one
 * velocity block per line) the kernels evaluate Maxwellians as a product of
 * a per-line and a per-point factor (the separable exponentials of a tensor
 * grid). */
typedef struct {
  int64_t n_v;
  const double *u;
  const double *weight;
  int32_t tensor_n[3];
  const double *axis[3];
} ugks_vgrid;

/* Gas and scheme parameters.
 *   model: BGK (Pr must be 1) or Shakhov (Sec. 2.1, Eq. 3; K must be 0)
 *   K: internal degrees of freedom (K_xi = K + 3 - dim, Eq. 2)
 *   mu = mu_ref T^omega, tau = mu / p
 *   dt: dt_override if > 0, else cfl * min_i |Omega_i| / max_k sum_f S_f max(u_k . n_f, 0)
 *   limiter: slope limiter of the least-squares reconstruction, venkat_K its constant
 *   shock_tau_fix: add dt |p_l - p_r| / (p_l + p_r) to the interface relaxation time
 *   storage: precision of the stored distribution: F64 (FP64 arithmetic),
 *     F32 (FP32 arithmetic), or F16 / BF16: FP32 arithmetic with f stored as
 *     deviations from a per-cell reference Maxwellian (the Maxwellian of the
 *     cell's W when the row was written), scaled per row of 32 velocities by
 *     the row's largest deviation, in FP16 / BF16; blocked sweep only, at most
 *     8 faces per cell.  Moments, W and the interface coefficients stay FP64.
 *   tile_cells: cells per tile of the tiled sweep, 0 = automatic
 *   sweep: device organisation of the velocity-block sweep (Sec. 2.2.2,
 *     Table B.1), UGKS_SWEEP_*: BLOCKED runs, per velocity block, the
 *     reconstruction (K2), the micro fluxes of every face (K1, written to a
 *     per-face buffer) and the first stage (K3) as three grid-wide kernels;
 *     BLOCKED_FUSED runs K1 and K3 as one kernel in which each cell evaluates
 *     the fluxes of its own faces (an interior face is evaluated by both of
 *     its cells, its moments added by the owner; the same arithmetic, one
 *     DRAM pass over the per-face buffer instead of three); TILED runs one
 *     persistent kernel over spatial tiles held in shared memory; AUTO picks
 *     BLOCKED.  All give the same result up to rounding order.
 *   block_velocities: velocities per block of the blocked sweep (32, 64,
 *     128, or 256 for dim 3 with one reduced distribution (K_xi = 0);
 *     0 = automatic: 256 where allowed, else 128) */
typedef struct {
  int32_t model;
  int32_t K;
  double Pr, omega, mu_ref;
  double cfl, dt_override;
  int32_t limiter;
  double venkat_K;
  int32_t shock_tau_fix;
  int32_t storage;
  int32_t tile_cells;
  int32_t sweep;
  int32_t block_velocities;
} ugks_params;

/* Creates a solver context.  Copies mesh, grid and W_init (host,
 * [n_cells][dim+2] conservative (rho, rho U, rho E); NULL = the state of
 * bc[0]) to the device, renumbers cells for locality, precomputes geometry
 * and the time step, and sets h, b to the discrete Maxwellians of W_init.
 * cuda_stream: a cudaStream_t to run on, or NULL for a library-owned stream.
 * Errors: INVALID_ARGUMENT, MESH, VGRID, UNSUPPORTED, OUT_OF_MEMORY, CUDA. */
ugks_status ugks_create(const ugks_mesh *mesh, const ugks_vgrid *vgrid, const ugks_params *params,
                        const double *W_init, void *cuda_stream, ugks_ctx **out);

/* Advances n_steps >= 0 UGKS time steps (Algorithm 5), asynchronously. */
ugks_status ugks_step(ugks_ctx *ctx, int32_t n_steps);

/* Allocation-free variant of ugks_step, for callers that must not allocate
 * device memory once the solver is set up: for example a host application
 * whose device memory pool is owned by another allocator (a framework's
 * caching allocator holds it), or a latency-critical loop in which the
 * device-wide synchronisation that cudaMalloc / cudaFree can imply is not
 * acceptable.  The paper has no counterpart; this is an interface addition.
 * It advances n_steps >= 0 steps exactly like ugks_step, with the context's
 * own inputs and outputs, but the velocity-block sweep's scratch (blocked
 * sweep: the gradients and micro fluxes of one block and the face
 * accumulators; tiled sweep: the face accumulators) lives in one file-scope
 * device array of 16 MiB that every GPU loading this library holds until exit.  It
 * calls no cudaMalloc, cudaFree or other allocating routine.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress,
 * once per device); make that first call before any stream capture.  All
 * calls share the array and each call overwrites it (the accumulators are
 * cleared by the kernel), so calls whose work overlaps on the GPU (other
 * streams, other contexts) race on it.  At the end of each step the face
 * accumulators are copied (device to device, on the context's stream) into
 * the context's own buffer, so ugks_surface after a static step reports that
 * context's wall fluxes even when another context has used the array since.
 * Contexts whose scratch needs more
 * than 16 MiB are rejected with UGKS_ERR_INVALID_ARGUMENT and a message
 * naming the size; use ugks_step for them. */
ugks_status ugks_step_static_scratch(ugks_ctx *ctx, int32_t n_steps);

/* Copies W (host, [n_cells][dim+2], original cell order) and, if q_out is not
 * NULL, the heat flux of the current distribution ([n_cells][dim], Eq. 13). */
ugks_status ugks_moments(ugks_ctx *ctx, double *W_out, double *q_out);

/* Copies the residual of the last step, res_out[dim+2]:
 * R_m = sqrt(sum_i (W_im^{n+1} - W_im^n)^2 / n_cells).  Zero before any step. */
ugks_status ugks_residual(ugks_ctx *ctx, double *res_out);

/* Surface quantities of the last step on every diffuse-wall face, from the
 * moments of the wall flux (Sec. 2.1; the paper evaluates the macroscopic
 * surface quantities from the moments of the wall flux without printing
 * formulas, read here as): with n the face normal pointing out of the gas,
 * F the time-integrated face flux of Eq. 28 and P = F_momentum / dt,
 *   p_w = P . n,  tau_w = P - p_w n,  q_w = (F_energy - U_w . F_momentum) / dt.
 * faces[n] receives the wall faces (original indices, ascending) and
 * vals[n][dim+2] the values (p_w, tau_w[0..dim-1], q_w).  If freestream =
 * (rho, U[0..dim-1], T) is not NULL, coef[n][3] receives
 *   C_p = (p_w - rho T/2) / (rho |U|^2 / 2),  C_t = |tau_w| / (rho |U|^2 / 2),
 *   C_h = q_w / (rho |U|^3 / 2).
 * *n_wall always receives the number of wall faces; the arrays must hold at
 * least that many (cap), else UGKS_ERR_INVALID_ARGUMENT.  Zero before the
 * first step.  Synchronises the context stream.  Blocked sweep only
 * (UGKS_ERR_UNSUPPORTED for the tiled sweep). */
ugks_status ugks_surface(ugks_ctx *ctx, const double *freestream, int64_t cap, int64_t *n_wall, int64_t *faces,
                         double *vals, double *coef);

/* Thirteen-moment fields of the current state, per cell (original order),
 * out[n_cells][n13] with n13 = 2 dim + 2 + dim (dim + 1) / 2:
 *   rho, U[dim], T (of W), the deviatoric stress sigma_ij = sum_k w c_i c_j h
 *   - p delta_ij (p = rho T / 2) in the order xx, xy, (xz), yy, (yz), zz, and
 *   the heat flux q[dim] (Eq. 13), all about U of W.  The paper has no such
 * call: these are the fields of the learned warm start.  FP64 or FP32
 * storage (else UGKS_ERR_UNSUPPORTED); synchronises the context stream. */
ugks_status ugks_moments13(ugks_ctx *ctx, double *out);

/* Resets the state to the Chapman-Enskog (Grad 13-moment) distribution of
 * the given fields (layout of ugks_moments13; rho, T > 0), reduced over xi:
 *   h = H [1 + 2 lam^2/rho sigma_ij c_i c_j - lam tr(sigma)/rho
 *          + 4 lam^2/((K+5) rho) (q.c)(2 lam |c|^2 - (dim+2))]
 *   b = kappa H [1 + 2 lam^2/rho sigma_ij c_i c_j - lam (K_xi+2) tr(sigma)/(K_xi rho)
 *          + 4 lam^2/((K+5) rho) (q.c)(2 lam |c|^2 - dim)]
 * (H the Maxwellian of rho, U, lam = 1/T; kappa = K_xi/(2 lam); the trace
 * terms give the K_xi components of xi the stress -tr(sigma)/K_xi each, so
 * that the full stress is trace-free and the moments of f return rho, E and
 * sigma; with K_xi = 0, sigma must be trace-free), W from
 * rho, U, T; the step counter restarts at 0.  A warm start for steady
 * solves; the paper has no such call.  FP64 or FP32 storage. */
ugks_status ugks_init_moments13(ugks_ctx *ctx, const double *fields);

/* Time step in use. */
ugks_status ugks_dt(const ugks_ctx *ctx, double *dt_out);

/* Number of reduced distributions (2 when K_xi > 0, else 1) and padded grid size. */
ugks_status ugks_sizes(const ugks_ctx *ctx, int32_t *n_reduced, int64_t *n_v_padded);

/* Spatial dimension, number of cells and of faces of the context's mesh. */
ugks_status ugks_mesh_sizes(const ugks_ctx *ctx, int32_t *dim, int64_t *n_cells, int64_t *n_faces);

/* Copies the distribution of selected cells (original indices) as FP64:
 * out[n][n_reduced][n_v] (h then b). */
ugks_status ugks_get_f(ugks_ctx *ctx, const int64_t *cells, int64_t n, double *out);

/* Checkpoint / restart: full state as FP64, W[n_cells][dim+2] and
 * f[n_reduced][n_cells][n_v], original cell order; the step counter. */
ugks_status ugks_get_state(ugks_ctx *ctx, double *W, double *f, int64_t *step);
ugks_status ugks_set_state(ugks_ctx *ctx, const double *W, const double *f, int64_t step);

/* Per-kernel device time accumulated since the last reset (CUDA events on the
 * context stream, recorded only while enabled).  names/ms/count arrays of
 * length cap; returns the number of kernels in *n. */
ugks_status ugks_stats_enable(ugks_ctx *ctx, int32_t on);
ugks_status ugks_stats(ugks_ctx *ctx, int32_t cap, const char **names, double *ms, int64_t *count, int32_t *n);

/* One-shot solve with host buffers: create, n_steps steps, copy W_out
 * ([n_cells][dim+2]) and res_out ([dim+2]), destroy. */
ugks_status ugks_solve(const ugks_mesh *mesh, const ugks_vgrid *vgrid, const ugks_params *params,
                       const double *W_init, int32_t n_steps, double *W_out, double *res_out);

ugks_status ugks_destroy(ugks_ctx *ctx);

/* ---- Batches of cases (uneven meshes and velocity grids) ----
 * The paper steps one case over many ranks; a batch steps many independent
 * cases on one GPU.  Each case is an ordinary context (its own mesh, grid,
 * parameters, time step and coefficients; blocked sweep only).
 * ugks_batch_step advances every case by n_steps: two steps of every case are
 * captured once into one CUDA graph, each case on its own forked stream so
 * that small cases run concurrently, and each graph launch advances all cases
 * by two steps (an odd remainder runs as ordinary steps).  Work is queued on
 * cuda_stream (NULL: a library-owned stream); the cases' own calls
 * (ugks_moments, ...) are ordered after it. */
typedef struct ugks_batch ugks_batch;

/* Creates n contexts from meshes[i], vgrids[i], params[i] and W_init[i]
 * (W_init or W_init[i] may be NULL as in ugks_create).  A case whose
 * (cells, velocities, dim, reduced distributions, storage) was tuned earlier
 * in this process reuses that shape (ugks_batch_autotune). */
ugks_status ugks_batch_create(int32_t n, const ugks_mesh *const *meshes, const ugks_vgrid *const *vgrids,
                              const ugks_params *params, const double *const *W_init, void *cuda_stream,
                              ugks_batch **out);

/* Autotuner of the sweep's shape (Sec. 2.2.2: the velocity block is the
 * tiling unit): for every case not tuned yet, a coordinate search over the
 * block size (32, 64, 128 and, where compiled, 256 velocities that its
 * buffers allow), then the organisation of the fluxes and the first stage
 * (split kernels or one fused kernel, UGKS_SWEEP_BLOCKED / _FUSED), then the
 * number of velocity chunks of the second stage (the allocated count and its
 * halves down to an eighth).  Each shape is timed on the device over the
 * second of two steps; the fastest is kept.  These steps advance the cases
 * (shapes differ only in the summation order of the moments).  The choice is
 * cached for the process per (cells, velocities, dim, reduced distributions,
 * storage). */
ugks_status ugks_batch_autotune(ugks_batch *batch);

ugks_status ugks_batch_step(ugks_batch *batch, int32_t n_steps);

/* The context of case i (owned by the batch; do not destroy it). */
ugks_status ugks_batch_context(ugks_batch *batch, int32_t i, ugks_ctx **ctx);

/* Block size in use for case i (velocities per block) and the autotuner's
 * timings, ms_per_step[4]: ms per step at 32, 64, 128, 256 velocities per
 * block (0 = not run). */
ugks_status ugks_batch_tuning(ugks_batch *batch, int32_t i, int32_t *block_velocities, double *ms_per_step);

/* The shape case i runs with (after ugks_batch_autotune: the tuned one):
 * velocities per block, fused (1) or split (0) fluxes and first stage,
 * second-stage velocity chunks, the tuned ms per step (0 if taken from the
 * process cache or not tuned) and the number of shapes timed.  Any output
 * pointer may be NULL. */
ugks_status ugks_batch_shape(ugks_batch *batch, int32_t i, int32_t *block_velocities, int32_t *fused,
                             int32_t *stage2_chunks, double *ms_per_step, int32_t *trials);

ugks_status ugks_batch_destroy(ugks_batch *batch);

/* The same two calls under the names of the boundary's first proposal:
 * ugks_create_batch = ugks_batch_create, ugks_step_batch = ugks_batch_step. */
ugks_status ugks_create_batch(int32_t n, const ugks_mesh *const *meshes, const ugks_vgrid *const *vgrids,
                              const ugks_params *params, const double *const *W_init, void *cuda_stream,
                              ugks_batch **out);
ugks_status ugks_step_batch(ugks_batch *batch, int32_t n_steps);

/* ---- Learned warm start ----
 * The paper has no learned component; its conclusion lists steady-state
 * acceleration as future work.  This interface addition starts steady solves
 * from a learned prediction of the converged fields instead of the
 * freestream.  The predictor is a multilayer perceptron
 *   y = W_L tanh(... tanh(W_1 x + b_1) ...) + b_L
 * (hidden_layers tanh layers of `width` units, linear output) whose input is
 * the per-cell feature vector of ugks_mlp_features and whose output is the
 * thirteen-moment fields of ugks_moments13 (n_out = 2 dim + 2 + dim (dim+1)/2).
 * Inputs and outputs are normalised x' = (x - shift) / scale with the
 * network's scaling (ugks_mlp_set_scaling / ugks_mlp_fit_scaling).  Weights
 * and activations are BF16 with FP32 accumulation on the tensor cores;
 * master weights, biases, gradients and Adam moments are FP32.  Training
 * minimises the mean-squared error over samples and outputs (normalised) by
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).  All calls are
 * synchronous on the network's stream and take host arrays, row-major. */
typedef struct ugks_mlp ugks_mlp;

/* Glorot-uniform weights drawn from splitmix64(seed), zero biases, unit
 * scaling.  1 <= n_in, n_out, width <= 4096, hidden_layers >= 1. */
ugks_status ugks_mlp_create(int32_t n_in, int32_t n_out, int32_t width, int32_t hidden_layers, uint64_t seed,
                            void *cuda_stream, ugks_mlp **out);

/* Scaling of inputs ([n_in] shift and scale) and outputs ([n_out]); scales > 0. */
ugks_status ugks_mlp_set_scaling(ugks_mlp *net, const float *in_shift, const float *in_scale,
                                 const float *out_shift, const float *out_scale);
ugks_status ugks_mlp_get_scaling(const ugks_mlp *net, float *in_shift, float *in_scale, float *out_shift,
                                 float *out_scale);

/* Sets the scaling to the mean and standard deviation (floored at 1e-6 times
 * the largest magnitude, else 1) of each column of X[n][n_in] and Y[n][n_out]. */
ugks_status ugks_mlp_fit_scaling(ugks_mlp *net, const float *X, const float *Y, int64_t n);

/* Number of parameters; get / set them as FP32, layer by layer W_l
 * ([out][in], row-major) then b_l.  Setting resets the Adam state. */
ugks_status ugks_mlp_param_count(const ugks_mlp *net, int64_t *count);
ugks_status ugks_mlp_get_params(ugks_mlp *net, float *params);
ugks_status ugks_mlp_set_params(ugks_mlp *net, const float *params);

/* Gradient of the loss on n <= 4096 samples (X[n][n_in], Y[n][n_out],
 * unnormalised) with respect to the parameters (layout of get_params), and
 * the loss itself (normalised units) if loss is not NULL. */
ugks_status ugks_mlp_gradients(ugks_mlp *net, const float *X, const float *Y, int64_t n, float *grads,
                               double *loss);

/* `epochs` passes of Adam with learning rate lr over X, Y in mini-batches of
 * `batch` <= 4096 samples, shuffled each epoch by splitmix64(seed); *loss_out
 * receives the mean batch loss of the last epoch.  UGKS_ERR_NONFINITE if the
 * loss stops being finite. */
ugks_status ugks_mlp_train(ugks_mlp *net, const float *X, const float *Y, int64_t n, int32_t epochs,
                           int32_t batch, float lr, uint64_t seed, double *loss_out);

/* Y[n][n_out] (unnormalised) of X[n][n_in]. */
ugks_status ugks_mlp_predict(ugks_mlp *net, const float *X, int64_t n, float *Y);

/* Feature vectors of a mesh's cells, out[n_cells][6] =
 *   (mach, log10 kn, centroid x, y, z (0 beyond dim), wall distance),
 * the wall distance being the distance from the cell centroid to the nearest
 * centroid of a face with a WALL boundary condition (0 without walls),
 * computed on the device. */
ugks_status ugks_mlp_features(ugks_mlp *net, const ugks_mesh *mesh, double mach, double kn, float *out);

/* Warm start of a context: predicts the thirteen-moment fields of
 * every cell from its features and resets the context to their
 * Chapman-Enskog distribution (ugks_init_moments13).  The predicted stress
 * and heat flux of a cell are scaled by one factor in (0, 1] where needed so
 * that |sigma_ij| <= p/2 and |q| <= p sqrt(T)/2 (p = rho T / 2): bounded
 * Grad corrections keep f positive at thermal speeds.  Freestream fallback:
 * a cell whose prediction is not finite or has rho <= 0 or T <= 0 gets the
 * fields of freestream = (rho, U[dim], T) with zero stress and heat flux;
 * *n_fallback (if not NULL) receives their number.  mesh must be the mesh the
 * context was created from; net must have n_in = 6 and the n_out of its dim. */
ugks_status ugks_mlp_warm_start(ugks_mlp *net, ugks_ctx *ctx, const ugks_mesh *mesh, double mach, double kn,
                                const double *freestream, int64_t *n_fallback);

ugks_status ugks_mlp_destroy(ugks_mlp *net);

/* Message of the last error of net, or of the calling thread when net is NULL. */
const char *ugks_mlp_last_error(const ugks_mlp *net);

/* Message of the last error of ctx, or of the calling thread when ctx is NULL. */
const char *ugks_last_error(const ugks_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* UGKS_H */
