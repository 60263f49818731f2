/*
 * gsis.h -- C ABI of the GB300 library for the general synthetic iterative scheme
 * (GSIS) of "Accelerated simulation of multiscale gas-radiation coupling flows via a
 * general synthetic iterative scheme".
 *
 * The library solves the steady kinetic model of Section 2.1 (Eq. kinetic_equation:
 * three reduced gas distributions f0, f1, f2 and the gray radiative intensity I_R)
 * with the unstructured finite-volume discrete velocity method of Section 5
 * (Eq. dis_micro).  A problem is stated the way the paper states it: a mesh, a
 * discrete velocity grid, a photon direction grid and the model parameters go in;
 * macroscopic fields (Eq. getmoment) come out.
 *
 * Conventions
 *  - Every entry point returns int: GSIS_OK (0) or a negative GSIS_ERR_* code.  No
 *    C++ exception, abort or exit crosses this boundary.  gsis_strerror() names a
 *    code; gsis_last_error() gives the context's last detailed message.
 *  - All pointers passed in are HOST pointers owned by the caller.  gsis_create()
 *    copies everything it needs; the caller may free its arrays afterwards.  The
 *    library owns every byte of device memory it uses.
 *  - Output buffers are caller-owned host memory; their length (in elements) is
 *    passed and checked, GSIS_ERR_INVALID_ARG if too short.
 *  - One context belongs to one host thread at a time.  All device work of a
 *    context is ordered on the CUDA stream given at creation (NULL: the legacy
 *    default stream): work the library runs on streams of its own (the photon sweep,
 *    staged copies) starts after, and is waited for by, that stream through events.
 *    Calls that return host data synchronise that stream.
 *  - Doubles at the boundary whatever the internal precision.
 *
 * Reduced velocity spaces: with dim in-plane velocity components (dim = spatial
 * dimension) and m = 3 - dim hidden ones, the gas state is four planes per cell and
 * discrete velocity, in the order
 *      [F0, H0, f1, f2],  F0 = int f0 dxi_hidden,  H0 = int |xi_hidden|^2 f0 dxi_hidden,
 * f1, f2 integrated over xi_hidden.  In 3-D the H0 plane is unused (zero).
 */
#ifndef GSIS_H
#define GSIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define GSIS_OK                 0
#define GSIS_ERR_INVALID_ARG   -1   /* bad pointer, size, parameter or buffer length   */
#define GSIS_ERR_OUT_OF_MEMORY -2   /* device or host allocation failed                 */
#define GSIS_ERR_CUDA          -3   /* a CUDA runtime call failed (see gsis_last_error) */
#define GSIS_ERR_DIVERGED      -4   /* NaN/Inf or a negative density/temperature        */
#define GSIS_ERR_NOT_CONVERGED -5   /* gsis_solve hit max_outer before tol_outer        */
#define GSIS_ERR_TIMEOUT       -6   /* a bounded device wait ran out                    */
#define GSIS_ERR_BAD_MESH      -7   /* inconsistent connectivity or geometry            */
#define GSIS_ERR_UNSUPPORTED   -8   /* valid request that this build does not implement */

/* ---- per-cell field record (doubles), used by gsis_init_fields / get_fields --
 *  0 rho | 1..3 u | 4 T_t | 5 T_r | 6 T_v | 7 T_R | 8..10 q_t | 11..13 q_r |
 *  14..16 q_v | 17..19 q_R | 20..25 sigma (xx, yy, zz, xy, xz, yz)            */
#define GSIS_NF 26

/* ---- boundary patches ------------------------------------------------------ */
#define GSIS_PATCH_WALL     0  /* gas: diffuse, fully accommodating at (T_t, u);
                                  photons: black at T_t                           */
#define GSIS_PATCH_FARFIELD 1  /* incoming: equilibrium of (rho, u, T_t, T_r, T_v, T_R) */
#define GSIS_PATCH_SYMMETRY 2  /* mirror plane: molecules and photons reflect specularly
                                  (what enters at xi is what leaves at xi - 2 (xi.n) n);
                                  the synthetic equations take the Rusanov flux against the
                                  cell state with its normal velocity reversed, no viscous,
                                  conductive or radiative flux.  The velocity and photon
                                  sets must be symmetric under the reflection (gsis_create
                                  returns INVALID_ARG otherwise); the patch's state fields
                                  are ignored.  Not combinable with velocity sharding.      */

typedef struct {
    int32_t kind;               /* GSIS_PATCH_*                                    */
    double rho;                 /* far field only                                  */
    double u[3];                /* wall velocity or far-field velocity             */
    double T_t, T_r, T_v, T_R;  /* wall temperature is T_t                         */
} gsis_patch;

/* Unstructured finite-volume mesh (Section 5): faces with owner and neighbour.
 * face_nbr[f] >= 0 is the neighbour cell; face_nbr[f] = -1 - p marks a boundary face
 * of patch p.  face_normal is the unit normal from owner to neighbour (outward on the
 * boundary), [n_faces][dim] row-major.  Areas are lengths in 2-D and 1 in 1-D.
 * Cells are relaxed in blocks of consecutive indices: number them with locality.
 * Cells have at most 4 faces (segments, triangles, quadrilaterals, tetrahedra); the
 * least-squares stencil (face neighbours and their face neighbours) holds at most 12
 * cells in 1-D and 2-D and 16 in 3-D (UNSUPPORTED beyond).
 * 3-D meshes run CIS and GSIS (the synthetic equations with five conservative gas
 * variables, rho u in three components) in FP32 or FP64 with tc_moments = 0; the learned
 * closure's samples (gsis_mlp_samples, gsis_warm_start with use_mlp) and velocity shards
 * are built for 1-D and 2-D and return UNSUPPORTED on a 3-D context.
 * Periodic domains: period[a] > 0 makes axis a periodic with that period (0: not
 * periodic; period NULL: no axis is).  The mesh itself joins the cells across each seam
 * by ordinary interior faces (face_nbr >= 0, one face centroid); every difference of
 * centroids the library forms (least-squares stencils, face offsets, face distances) is
 * then the minimal image along the periodic axes.  A periodic pair of patches is thus a
 * seam of interior faces, and the Fourier analysis of Section 4 is posed on such a domain.
 * Errors: INVALID_ARG (a negative or non-finite period). */
typedef struct {
    int32_t dim;                      /* 1, 2 or 3                                      */
    int64_t n_cells, n_faces;
    const int32_t *face_owner;        /* [n_faces]            */
    const int32_t *face_nbr;          /* [n_faces]            */
    const double *face_normal;        /* [n_faces][dim]       */
    const double *face_area;          /* [n_faces]            */
    const double *face_centroid;      /* [n_faces][dim]       */
    const double *cell_volume;        /* [n_cells]            */
    const double *cell_centroid;      /* [n_cells][dim]       */
    int32_t n_patches;
    const gsis_patch *patches;        /* [n_patches]          */
    const double *period;             /* [dim] or NULL (see below) */
} gsis_mesh;

/* Discrete velocities xi [n][dim] and weights w [n]: sum_i w_i phi(xi_i) approximates
 * the integral over the reduced velocity space (Section 6 uses uniform grids). */
typedef struct { int32_t n; const double *xi; const double *w; } gsis_velocity_quad;

/* Photon directions omega [n][3] (unit vectors) and weights w [n], sum w = 4 pi.
 * Transport uses the first dim components of omega. */
typedef struct { int32_t n; const double *omega; const double *w; } gsis_photon_quad;

/* Model parameters of Section 2.1. */
typedef struct {
    double d_r, d_v;            /* rotational / vibrational degrees of freedom; d_v is used
                                   when dv_temperature_dependent is 0                         */
    double Z_r, Z_v;            /* collision numbers                                          */
    double omega;               /* viscosity index: tau = sqrt(2/pi) T_t^(omega-1) Kn / rho   */
    double Sc;                  /* Schmidt number in the Mason-Monchick matrix A              */
    double Kn, Kn_p;            /* gas and photon Knudsen numbers                             */
    double sigma_R;             /* dimensionless Stefan-Boltzmann constant                    */
    int32_t k_eff_density_scaled; /* 0: k_eff = 1/Kn_p; 1: k_eff = rho/Kn_p                  */
    const double *A;            /* 3x3 row-major relaxation-rate matrix, or NULL for the
                                   Mason-Monchick form of Section 2.1                         */
    double Tv_ref;              /* characteristic vibrational temperature (units of T_0)      */
    int32_t dv_temperature_dependent; /* 1: d_v(T_v) = 2 x / (e^x - 1), x = Tv_ref / T_v
                                   (Section 2.1): e_v = d_v(T_v) rho T_v / 2, T_tv and the
                                   total T solved by Newton, A and the NSF conductivities at
                                   the local d_v(T_v) (unless A is given), source Jacobian of
                                   the synthetic equations re-derived; 0: d_v constant       */
} gsis_model_params;

#define GSIS_FP32 0             /* f and I stored and updated in FP32 */
#define GSIS_FP64 1             /* plain FP64 everywhere              */

/* Solver parameters (Section 5 and Section 6). */
typedef struct {
    int32_t precision;          /* GSIS_FP32 or GSIS_FP64                                   */
    int32_t order;              /* 1: first-order upwind residual; 2: Venkatakrishnan-limited
                                   linear reconstruction (Eq. deltaflux_micro)               */
    int32_t relax_block;        /* point relaxation: forward + backward Gauss-Seidel inside
                                   blocks of this many consecutive cells (1..64)            */
    double cfl_meso, cfl_macro; /* pseudo time step dt = CFL dx / (|u| + c_s)              */
    double venkat_K;            /* limiter constant, eps^2 = (K dx)^3                       */
    int32_t n_cis_precond;      /* CIS iterations before GSIS starts                        */
    int32_t max_outer, max_inner, macro_sweeps;
    double tol_outer, tol_inner;
    double sync_relax;          /* w in f^{k+1} = f^{k+1/2} + w [f_eq(M^{k+1}) - f_eq(M^{k+1/2})],
                                   0 < w <= 1 (Section 3 has w = 1)                          */
    int32_t macro_fp32;         /* GSIS_FP32 contexts only: precision of the synthetic
                                   equations' residual side (gradients, fluxes, high-order
                                   terms, D) and of the neighbours' flux increments in the
                                   relaxation sweeps; the sweeps' diagonal solves, the
                                   updates of W and the norms stay FP64.
                                   0 (default): FP64.  1: FP32.  2: FP32 except the last 16
                                   inner iterations of every solve and the high-order terms,
                                   which are FP64.                                           */
    int32_t tc_moments;         /* GSIS_FP32 contexts only: where the gas velocity moments
                                   (Eq. getmoment) are contracted.  0: CUDA cores;
                                   1: tensor cores (split-TF32 tcgen05) in the standalone and
                                   synchronisation passes, CUDA cores in the sweep epilogue;
                                   2: tensor cores in the sweep epilogue too (relaxation
                                   blocks that divide 16 cells; other blocks keep the
                                   CUDA-core epilogue).  FP64 contexts ignore it.            */
    double positivity;          /* 0 <= theta < 1: after each kinetic sweep every value of f and
                                   I is at least theta times its value before the sweep (a bound
                                   on the implicit update, an extension of Section 5 that
                                   leaves every steady state unchanged; it lets the order-2
                                   defect correction start from impulsive hypersonic states).
                                   0: off, the paper's scheme.                               */
    int32_t defect_correction;  /* 1: every GSIS synthetic solve (Section 3, step 2) solves
                                   R(W) - R(W_h) + r_h = 0 instead of R(W) = 0, with W_h the
                                   conservative variables of M^{k+1/2} and r_h the velocity
                                   moments, in the rows of the synthetic equations, of the
                                   kinetic residual (Eq. dis_micro's right-hand side) at
                                   f^{k+1/2} with the coefficients of M^{k+1/2}.  At a kinetic
                                   steady state r_h = 0 and W_h solves it, so GSIS keeps the
                                   kinetic discretisation's steady state as its fixed point
                                   (the paper's synthetic equations match it only to the
                                   discretisation error, which leaves an eps floor).  Costs one
                                   slope pass and one residual-only sweep per GSIS iteration.
                                   With GSIS_FP32 storage the residual moments are FP32 sums
                                   whose rounding the offset carries into every solve (eps then
                                   stops near 1e-6 to 1e-5): meant for GSIS_FP64.
                                   An extension; 0 (default) is the paper's step.  Not with
                                   velocity shards (UNSUPPORTED).                            */
} gsis_solver_params;

typedef struct gsis_ctx gsis_ctx;

/* Create a solver context: validates and copies the problem, builds the device
 * geometry, allocates the distribution planes (two copies of [n_cells][V][4] and of
 * [n_cells][n_omega] in the chosen precision) and sets f to the equilibrium of a
 * uniform unit state.  cuda_stream is a cudaStream_t (may be NULL).
 * Errors: INVALID_ARG, BAD_MESH, UNSUPPORTED, OUT_OF_MEMORY, CUDA. */
int gsis_create(const gsis_mesh *mesh, const gsis_velocity_quad *vq, const gsis_photon_quad *pq,
                const gsis_model_params *model, const gsis_solver_params *solver,
                void *cuda_stream, gsis_ctx **out);

/* Release every resource of the context (NULL is a no-op). */
void gsis_destroy(gsis_ctx *ctx);

/* Static description of a status code; never NULL. */
const char *gsis_strerror(int code);

/* Last detailed error message of the context ("" if none); valid until the next call. */
const char *gsis_last_error(const gsis_ctx *ctx);

/* Set f to the multi-temperature local equilibrium of per-cell states
 * M [n_cells][GSIS_NF] (rho, u, T_t, T_r, T_v, T_R used; the moments of Eq. getmoment):
 * F0 = rho f_eq(T_t), H0 = m T_t F0, f1 = (d_r/2) T_r F0, f2 = (d_v/2) T_v F0,
 * I = sigma_R T_R^4 / pi.  Then the macroscopic fields are taken from the new f. */
int gsis_init_fields(gsis_ctx *ctx, const double *M, int64_t len);

/* Set the distributions from host FP64 arrays f [n_cells][n_xi][4] and I [n_cells][n_omega]
 * (rounded to the storage precision), then take the macroscopic fields from them. */
int gsis_set_distributions(gsis_ctx *ctx, const double *f, int64_t f_len, const double *I, int64_t I_len);

/* Copy the current distributions to host FP64 arrays of the same layout. */
int gsis_get_distributions(gsis_ctx *ctx, double *f, int64_t f_len, double *I, int64_t I_len);

/* Same as gsis_set_distributions but from host buffers already in the storage
 * precision (float for GSIS_FP32, double for GSIS_FP64), layout [n_cells][n_xi][4] and
 * [n_cells][n_omega].  Pinned buffers make the copies asynchronous on the context
 * stream; the call returns without synchronising. */
int gsis_upload_distributions(gsis_ctx *ctx, const void *f, const void *I);

/* Double-buffered uploads: copy the next state while the current one is being computed.
 * gsis_stage_distributions starts an asynchronous copy of host buffers in the storage
 * precision (layout as gsis_upload_distributions; pinned for true asynchrony) into a
 * staging pair of device buffers, on a copy stream of the context's own.  It waits on the
 * device only for the previous commit, never for the compute stream's current work, and
 * returns at once; the host buffers must stay valid until the copy completes (it has when
 * the commit's work has run).  The first call allocates the staging pair (the size of the
 * distributions) and the copy stream.  gsis_commit_staged makes the staged state current
 * on the context stream (waiting for the copy there, not on the host) and takes its fields
 * as gsis_refresh_fields does.  One upload can be staged at a time.  The paper has no
 * counterpart: this is how the step overlaps its host-to-device input with compute.
 * Errors: INVALID_ARG (null buffer, a second stage before a commit, a commit with nothing
 * staged), OUT_OF_MEMORY, CUDA. */
int gsis_stage_distributions(gsis_ctx *ctx, const void *f, const void *I);
int gsis_commit_staged(gsis_ctx *ctx);

/* Recompute the macroscopic fields from the distributions now on the device (the velocity
 * moments of Eq. getmoment and the fields of Section 2, the same pass that follows an
 * upload), asynchronously on the context stream.  In FP32 contexts with tc_moments >= 1
 * the gas moments are one split-TF32 tensor-core contraction per (16-cell tile, 64
 * velocities).  Synchronises the context stream to read the device error word.
 * Errors: INVALID_ARG, TIMEOUT (see gsis_set_wait_limit), CUDA. */
int gsis_refresh_fields(gsis_ctx *ctx);

/* Macroscopic fields of the current distributions, [n_cells][GSIS_NF] doubles. */
int gsis_get_fields(gsis_ctx *ctx, double *out, int64_t len);

/* Same, asynchronously into a caller buffer (pinned for true asynchrony) on the
 * context stream; the caller synchronises the stream before reading it. */
int gsis_download_fields_async(gsis_ctx *ctx, double *out, int64_t len);

#define GSIS_MODE_CIS  0        /* conventional iteration: one kinetic step                */
#define GSIS_MODE_GSIS 1        /* kinetic step + synthetic equations + synchronisation    */

/* One outer iteration from the current distributions f^k (Section 3):
 * CIS:  moments M^k -> reference distributions -> one implicit sweep (Eq. dis_micro)
 *       for gas and photons -> f^{k+1} and M^{k+1}.
 * GSIS: the same kinetic step gives f^{k+1/2} and M^{k+1/2}; the high-order terms of
 *       Eq. (getHoTs) from f^{k+1/2} are frozen and the synthetic equations (Eq.
 *       macroscopic_equation, implicit form Eq. delta_macro) are relaxed in FP64 for up
 *       to max_inner pseudo-time steps of macro_sweeps point-relaxation sweeps, until
 *       ||R|| <= tol_inner ||R_0||, giving M^{k+1} (in a domain bounded by walls only,
 *       rescaled to the total mass of M^k); then f^{k+1} = f^{k+1/2} + sync_relax
 *       [f_eq(M^{k+1}) - f_eq(M^{k+1/2})] and likewise for I.
 * *eps_out (may be NULL) receives the convergence measure of Section 6 between M^k
 * and M^{k+1}.  This call synchronises the stream to read eps.
 * Errors: DIVERGED (non-finite or non-positive density/temperature), TIMEOUT (a
 * tensor-core completion wait ran out, see gsis_set_wait_limit), CUDA, INVALID_ARG. */
int gsis_step(gsis_ctx *ctx, int32_t mode, double *eps_out);

/* Iterate to a steady state (Section 6): CIS for the first n_cis_precond iterations
 * (mode GSIS_MODE_GSIS; counted from the last time the distributions were set, so a
 * resumed run continues the count of the run it was exported from) or throughout
 * (GSIS_MODE_CIS), then GSIS, until eps < tol or max_outer iterations.  max_outer <= 0 and tol <= 0 take the solver parameters'
 * values.  *iters_out (may be NULL) receives the number of iterations; eps_history (may
 * be NULL, else at least max_outer doubles, caller-owned) receives eps of each.
 * Errors: NOT_CONVERGED (max_outer reached; the state is kept), DIVERGED, CUDA. */
int gsis_solve(gsis_ctx *ctx, int32_t mode, int32_t max_outer, double tol, int32_t *iters_out,
               double *eps_history);

/* Same iteration without reading eps back: the device work is queued on the context
 * stream and the call returns at once.  gsis_last_eps() synchronises and returns the
 * measure of the most recent iteration. */
int gsis_step_async(gsis_ctx *ctx, int32_t mode);
int gsis_last_eps(gsis_ctx *ctx, double *eps_out);

/* The synthetic solve of the most recent GSIS iteration: inner iterations taken and the
 * first and last residual norms ||R||_2.  Synchronises the context stream. */
int gsis_macro_stats(gsis_ctx *ctx, int32_t *inner_iters, double *r0, double *rn);

/* ---- checkpoint / resume -----------------------------------------------------------
 * The iteration state of Section 3's outer loop is the distributions f^k and I^k and the
 * macroscopic fields M^k they define (the next iteration's reference distributions,
 * shift velocities and convergence measure all follow from these), plus the outer
 * iteration count since the distributions were set and the eps of each iteration that
 * was read.  gsis_export_state writes that state into a caller-owned HOST buffer of at
 * least gsis_state_size() bytes: a header (magic, version, dim, precision, n_xi,
 * n_omega, n_cells, iteration count, history length, last eps), then the eps history
 * (doubles), M^k ([n_cells][GSIS_NF] doubles), f ([n_cells][n_xi][4]) and I
 * ([n_cells][n_omega]) in the context's storage type, unpadded.  gsis_import_state
 * loads such an image into a context created with the same mesh, quadratures, model and
 * solver parameters; the iterations that follow reproduce the exporting run's bit for
 * bit.  Both synchronise the context stream.
 * Errors: INVALID_ARG (null or short buffer; an image of another version, dimension,
 * precision or size), CUDA. */
int gsis_state_size(const gsis_ctx *ctx, int64_t *bytes);
int gsis_export_state(gsis_ctx *ctx, void *buf, int64_t len);
int gsis_import_state(gsis_ctx *ctx, const void *buf, int64_t len);

/* Outer iterations since the distributions were last set (*iter) and the eps history
 * kept by the context (up to len values into eps, caller-owned; *n_out its length). */
int gsis_get_history(const gsis_ctx *ctx, int64_t *iter, double *eps, int64_t len, int64_t *n_out);

/* ---- velocity-space sharding (several GPUs, one process each) ----------------------
 * With the fields M^k fixed, every discrete velocity's (and photon direction's) sweep is
 * independent: the kinetic step of Section 3 partitions by velocity, as the paper's own
 * parallel runs do.  Each rank creates a context whose velocity and photon sets are one
 * contiguous range of the full sets (in the same order on every rank), then calls
 * gsis_shard_setup with the FULL sets: the wall re-emission normalisation and the
 * replicated synthetic equations use them.  The exchange buffer (gsis_shard_buffer:
 * `count` doubles in device memory owned by the context, valid until gsis_destroy) holds
 * this rank's per-cell moment sums, wall outflow and kinetic boundary-flux sums; the
 * caller sums it over the ranks IN PLACE (an all-reduce on the context stream) after
 * every gsis_shard_refresh, gsis_shard_begin and gsis_shard_mid, and before the next
 * phase call:
 *   refresh (after the distributions are set): refresh(0), sum, end(NULL), refresh(1),
 *     sum, end(NULL) - moments about zero, then about the velocity found;
 *   CIS iteration:  begin(CIS), sum, end(&eps);
 *   GSIS iteration: begin(GSIS), sum, mid, sum, end(&eps) - the synthetic solve runs on
 *     every rank with identical inputs and gives identical results.
 * Every rank then holds the same fields and eps as an unsharded context.  A shard
 * refuses gsis_step, gsis_step_async, gsis_solve and gsis_warm_start (UNSUPPORTED).
 * The paper has no counterpart beyond the partitioning itself.
 * Errors: INVALID_ARG (null pointers, full sets smaller than the shard, phase calls out
 * of order, a context that is already a shard), OUT_OF_MEMORY, CUDA; end also DIVERGED
 * and TIMEOUT like gsis_step. */
int gsis_shard_setup(gsis_ctx *ctx, int32_t n_xi_all, const double *xi_all, const double *w_all,
                     int32_t n_omega_all, const double *omega_all, const double *wo_all);
int gsis_shard_buffer(gsis_ctx *ctx, void **dev_ptr, int64_t *count);
int gsis_shard_refresh(gsis_ctx *ctx, int32_t pass);
int gsis_shard_begin(gsis_ctx *ctx, int32_t mode);
int gsis_shard_mid(gsis_ctx *ctx);
int gsis_shard_end(gsis_ctx *ctx, double *eps_out);

/* ---- failure detection -------------------------------------------------------------
 * Every device-side wait in the library is bounded.  The tensor-core moment contraction
 * waits for its MMA chain on an mbarrier; this sets the number of polls of that first
 * wait (default 2^22, about a second).  When it runs out the CTA skips the accumulator,
 * issues no further chain, waits for the outstanding one with the full default bound
 * before it frees its tensor memory, and sets an error bit: the step (or
 * gsis_refresh_fields) then returns GSIS_ERR_TIMEOUT and the context stays usable.
 * A budget of 0 makes every such wait run out at once (a test of the error path).
 * The paper has no counterpart.  Errors: INVALID_ARG (negative budget). */
int gsis_set_wait_limit(gsis_ctx *ctx, int32_t polls);

/* ---- learned closure (warm start) -----------------------------------------------
 * A perceptron 16 -> 128 -> 128 -> 128 -> 12 (GELU hidden layers) maps the state of a
 * cell to its high-order terms (Eq. getHoTs):
 *   inputs  rho, u_x, u_y, T_t, T_r, T_v, T_R, the magnitudes of their least-squares
 *           gradients (T_R through e_R), Kn, 1/Kn_p;
 *   outputs HoT_sigma (xx, xy, yy, zz) / (rho T_t), HoT_q (t, r, v, R) x (x, y) /
 *           (rho T_t^1.5).
 * Weights are used in BF16 with FP32 accumulation; FP32 master weights are trained by
 * Adam on the mean squared error of standardised outputs.  The parameter blob
 * (GSIS_MLP_NPARAM floats) is W0 b0 W1 b1 W2 b2 W3 b3 (W row-major [out][in]) followed
 * by the input and output standardisation (x_mean[16] x_std[16] y_mean[12] y_std[12]).
 * All buffers are host memory owned by the caller; sample arrays are row-major. */
#define GSIS_MLP_NPARAM 36804
#define GSIS_MLP_NW 36748

/* He-normal weights from a seeded generator, zero biases, identity standardisation. */
int gsis_mlp_init(gsis_ctx *ctx, uint64_t seed);
int gsis_mlp_set_params(gsis_ctx *ctx, const float *params, int64_t len);
int gsis_mlp_get_params(gsis_ctx *ctx, float *params, int64_t len);
/* Features X [n_cells][16] and targets Y [n_cells][12] (Y may be NULL) of the current
 * fields: training samples taken from the solver's own iterations. */
int gsis_mlp_samples(gsis_ctx *ctx, float *X, float *Y, int64_t n_cells);
/* Standardisation from the samples, then epochs of shuffled mini-batches of `batch`
 * rows (seeded); *loss_out (may be NULL) receives the last batch's loss. */
int gsis_mlp_train(gsis_ctx *ctx, const float *X, const float *Y, int64_t n, int32_t epochs, int32_t batch,
                   double lr, uint64_t seed, double *loss_out);
/* Outputs (in target units) for raw inputs. */
int gsis_mlp_predict(gsis_ctx *ctx, const float *X, int64_t n, float *Y);
/* Loss on standardised targets and its gradient with respect to W0..b3 (grad: NULL or
 * GSIS_MLP_NW floats), without updating the parameters. */
int gsis_mlp_loss_grad(gsis_ctx *ctx, const float *X, const float *Y, int64_t n, double *loss, float *grad);
/* Warm start: n_presolve synthetic solves from the current fields with high-order terms
 * predicted by the network (use_mlp = 1) or zero (use_mlp = 0, the NSF limit), then
 * f = f_eq(M) and I = sigma_R T_R^4 / pi.  GSIS from there converges to the kinetic
 * solution whatever the prediction: the network only moves the starting point.
 * Errors: INVALID_ARG (use_mlp without a trained or set network), CUDA. */
int gsis_warm_start(gsis_ctx *ctx, int32_t n_presolve, int32_t use_mlp);

/* Kernel timing.  While enabled, the library brackets each of its kernel launches with
 * CUDA events on the stream it runs on and accumulates device time per kernel id.
 * gsis_profile_read fills up to n entries of names/ms/launches (arrays of length n)
 * and sets *n_out to the number of kernel ids. */
int gsis_profile_enable(gsis_ctx *ctx, int32_t on);
int gsis_profile_reset(gsis_ctx *ctx);
int gsis_profile_read(gsis_ctx *ctx, int32_t n, const char **names, double *ms, int64_t *launches,
                      int32_t *n_out);

/* Total number of kernels the context has launched since creation. */
int64_t gsis_launch_count(const gsis_ctx *ctx);

/* Sizes chosen by the library: padded velocity count, padded photon count, number of
 * velocity chunks per cell and the relaxation block size actually used. */
int gsis_get_layout(const gsis_ctx *ctx, int32_t *v_pad, int32_t *o_pad, int32_t *n_chunks,
                    int32_t *block);

/* Allocation-free velocity moments.  The paper has no counterpart: this entry point
 * serves callers that cannot allocate device memory, e.g. a host framework that owns the
 * whole device heap through its own pool allocator, or a plugin that may only use the
 * buffers it is handed.  Such callers cannot create a context, because gsis_create
 * allocates.
 *
 * Computes the per-cell field record (GSIS_NF doubles: rho, u, T_t, T_r, T_v, T_R, the
 * four heat fluxes, the six stress components, as gsis_get_fields) of DEVICE-resident
 * distributions:
 *   xi [n_xi][dim], w [n_xi], omega [n_omega][3], wo [n_omega]   doubles, device
 *   f  [n_cells][n_xi][4] planes [F0, H0, f1, f2], I [n_cells][n_omega]  in the
 *      storage type of `precision` (float for GSIS_FP32, double for GSIS_FP64), device
 *   fields [n_cells][GSIS_NF] doubles, device (output)
 * on cuda_stream (NULL: the legacy default stream); the call returns after queueing.
 * The gas moments are summed about each cell's own mean velocity (found in a first pass),
 * so FP32 storage keeps the heat fluxes to 1e-5 of rho T^1.5 at hypersonic speeds.
 *
 * It calls no cudaMalloc/cudaFree and no allocating library routine.  Its shift
 * velocities and partial sums live in one 32 MiB file-scope device array that every GPU
 * loading the library holds until the process exits; sizes that do not fit,
 *   n_cells * 24 + (n_cells * ceil(n_xi/128) * 20 + n_cells * ceil(n_omega/128) * 4)
 *   * sizeof(storage) > 32 MiB,
 * are rejected with GSIS_ERR_INVALID_ARG before anything is launched.  The first call on
 * a device looks up the array's device address (with that device current) and caches it
 * for the life of the process; make that first call before any stream capture, and make
 * no call after cudaDeviceReset on that device.  All calls share the array: calls whose
 * kernels overlap on one GPU race on it.
 * Errors: INVALID_ARG (null pointer, non-positive size, too large), UNSUPPORTED (dim 3),
 * CUDA (address lookup or launch failure). */
int gsis_moments_static(int32_t dim, int32_t precision, int64_t n_cells, int32_t n_xi, const double *xi,
                        const double *w, int32_t n_omega, const double *omega, const double *wo,
                        const void *f, const void *I, double d_r, double d_v, double sigma_R, double *fields,
                        void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GSIS_H */
