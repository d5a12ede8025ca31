/*
 * igamg.h -- C ABI of the GB300 (sm_103a) extrapolated geometric-multigrid
 * solver for isogeometric (tensor-product B-spline) Poisson problems.
 *
 * Method: Mouhssine, Ratnani, Sadok, "Vector extrapolation methods applied to
 * geometric multigrid solvers for isogeometric analysis" (2024).
 *   - model problem and discrete system A^h u^h = b^h ............ Sec. 2, Eq. (1)-(3)
 *   - open knot vectors, Cox-de Boor B-splines ...................... Sec. 2.3, Eq. (moneq)
 *   - coarse grid 2h, prolongation P, restriction R = P^T ........... Sec. 2, Eq. (4)
 *   - mu-cycle (V-cycle for mu = 1) ................................. Sec. 2.1, Algorithm 2
 *   - multigrid as the fixed-point map s_{k+1} = G(s_k) ............. Sec. 2.5, Eq. (fixedpoint)
 *   - RRE / MPE extrapolation ........................................ Sec. 3, Algorithms 3-4
 *   - restarted extrapolation ........................................ Sec. 3.2, Algorithm 5
 *
 * Conventions for every entry point
 *   - Every call returns an igamg_status; nothing throws or aborts.  After a
 *     failure igamg_last_error() gives a one-line message (per thread).
 *   - "d_" pointers are CUDA device pointers on the current device; "h_"
 *     pointers are host pointers.  The caller owns every pointer it passes; the
 *     library never frees them and keeps none of them after the call returns.
 *   - Grid vectors hold the interior unknowns only (homogeneous Dirichlet data
 *     removes the first and last B-spline per direction): m_d = n_d + p - 2
 *     per direction, C order with x fastest, index = i + m_x (j + m_y k).
 *   - "stream" is a cudaStream_t (NULL = legacy default stream).  Calls only
 *     enqueue work on it unless stated otherwise; igamg_solve synchronises it.
 *   - Scratch memory: calls that need it take (d_ws, ws_bytes); query the size
 *     with igamg_workspace_bytes().  The hot path allocates no device memory.
 *   - The context owns the device copies of its 1D factors, transfer
 *     operators and coarse-solve data (allocated by igamg_assemble, freed by
 *     igamg_destroy).  One context must not be used by two threads at once.
 */
#ifndef IGAMG_H
#define IGAMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IGAMG_OK = 0,
    IGAMG_EINVAL = 1,      /* bad argument (size, degree, dimension, pointer, alignment) */
    IGAMG_ENOMEM = 2,      /* host or device allocation failed, or workspace too small */
    IGAMG_ECUDA = 3,       /* a CUDA runtime call failed */
    IGAMG_ENOTCONV = 4,    /* max_cycles reached; d_x still holds the last iterate */
    IGAMG_EBREAKDOWN = 5,  /* non-finite residual (NaN/Inf in the data or the iteration) */
    IGAMG_ETIMEOUT = 6     /* a bounded device-side wait gave up */
} igamg_status;

typedef enum { IGAMG_EXTRAP_NONE = 0, IGAMG_RRE = 1, IGAMG_MPE = 2 } igamg_extrap;

/* Arithmetic of the multigrid cycle.  IGAMG_FP64: everything in FP64.
 * IGAMG_FP32_IR: V-cycles in FP32 inside FP64 iterative refinement; residuals,
 * the extrapolation Gram/least-squares solve and iterate updates in FP64.
 * IGAMG_FP32_IR_LEARNED: as FP32_IR, with the finest-level post-smoothing
 * replaced by the learned network (igamg_set_smoother). */
typedef enum { IGAMG_FP64 = 0, IGAMG_FP32_IR = 1, IGAMG_FP32_IR_LEARNED = 2 } igamg_prec;

/* Smoother of the multigrid cycle (igamg_set_cycle). */
typedef enum { IGAMG_SMOOTH_GS = 0, IGAMG_SMOOTH_JACOBI = 1 } igamg_smoother;

/* igamg_solve flags */
#define IGAMG_FLAG_X0_GIVEN 1u   /* start from d_x instead of s_0 = 0 */
#define IGAMG_FLAG_ABS_TOL  2u   /* test ||b - A t|| <= tol instead of ||b - A t|| / ||b|| <= tol */
#define IGAMG_FLAG_NO_GRAPH 4u   /* enqueue kernels directly instead of replaying a CUDA graph */
#define IGAMG_FLAG_HOST_LOOP 8u  /* test the residual on the host after every restart cycle (one graph
                                    launch and one synchronisation per cycle) instead of running the
                                    restart loop on the GPU */

typedef struct igamg_ctx igamg_ctx;

/* ---------------------------------------------------------------- set-up */

/* Create a problem context: dimension dim in {2, 3}, spline degree p in
 * [1, 7], n_elems[d] >= 2 elements in direction d (x first) on a uniform open
 * knot vector of [0, 1] (Sec. 2.3), and n_levels grids (0 = coarsen until every
 * direction has <= 8 elements).  Coarse grids keep every other breakpoint
 * (mesh 2h, Sec. 2), plus the last one when the count is odd.
 * Errors: EINVAL for dim/p/n out of range or too many levels; ENOMEM. */
igamg_status igamg_setup(int dim, int p, const int* n_elems, int n_levels, igamg_ctx** out);

/* Host assembly + one upload: per level and direction the banded 1D Galerkin
 * mass M_d and stiffness K_d ((p+1)-point Gauss quadrature per element), the
 * 1D prolongation P_d by knot insertion, the inverse diagonal of A on every
 * level, and the generalised eigenpairs K V = M V Lambda used for the exact
 * coarsest-grid solve.  Errors: ECUDA, ENOMEM. */
igamg_status igamg_assemble(igamg_ctx* ctx);

/* Sizes: number of levels, and per level (0 = coarsest) the interior unknowns
 * per direction.  h_m must hold 3*n_levels ints (unused directions get 1). */
igamg_status igamg_info(const igamg_ctx* ctx, int* n_levels, int* h_m);

/* Copy a 1D factor of `level` and direction d to the host, in banded form:
 * which = 0 mass M, 1 stiffness K (rows x (2p+1), entry [i][k] = F[i][i+k-p]),
 * 2 prolongation P from level-1 (dense rows_fine x cols_coarse).
 * h_out must hold rows*cols doubles; rows/cols are returned. */
igamg_status igamg_get_factor(const igamg_ctx* ctx, int level, int d, int which,
                              double* h_out, int* rows, int* cols);

/* Scratch bytes needed by igamg_solve for restart number k and precision. */
size_t igamg_workspace_bytes(const igamg_ctx* ctx, int k, int prec);

/* Load vector b_I = int f phi_I on the finest grid with (p+1)^dim Gauss points
 * per element (Sec. 2, Eq. (2)) for the sine series
 *   f = sum_k c[k_{dim-1}..k_0] prod_d sin((k_d+1) pi x_d),
 * h_coeffs holding modes^dim doubles (x mode fastest).  Writes d_b (finest N). */
igamg_status igamg_rhs_sine(igamg_ctx* ctx, int modes, const double* h_coeffs, double* d_b,
                            void* stream);

/* --------------------------------------- general operator (Sec. 4.3) */

/* The full elliptic problem of Sec. 4.3, Eq. (fullelliptic):
 *   -div(A grad u) + B . grad u + c u = f,  u = 0 on the boundary,
 * A SPD, on the image of the unit square under a map F (the unit square
 * itself, or e.g. the quarter annulus of Table 15), 2D.  Galerkin
 * discretisation on the tensor B-spline space of igamg_setup (degree p,
 * n_elems[2] uniform elements, at most 1024 per direction), (p+1)-point Gauss
 * quadrature per element and direction; the map enters as the transformed
 * coefficients |J| J^{-1} A J^{-T}, |J| J^{-1} B, |J| c and |J| f on the unit
 * square (J = DF).  Coarse operators: the Galerkin product P^T A P of Eq. (4)
 * with the knot-insertion P; the coarsest level is solved with its dense
 * inverse.  igamg_solve then runs Algorithm 5 (RRE or MPE; A is not
 * symmetric, so RRE is GMRES-like and MPE FOM-like) around Algorithm 2 with
 * the context's cycle (igamg_set_cycle: multicolour Gauss-Seidel, (p+1)^2
 * colours, or weighted Jacobi; V or W), FP64 only (IGAMG_FP64); igamg_apply,
 * igamg_smooth and igamg_vcycle act on the stencil levels.  The calls that
 * only exist for the Poisson problem (igamg_rhs_sine, igamg_smooth_f32,
 * igamg_autotune, the learned smoother, the probe) return IGAMG_EINVAL.
 * Order: igamg_setup_general -> igamg_quadrature_points -> evaluate the
 * problem's functions there -> igamg_assemble_general -> igamg_rhs_points ->
 * igamg_solve.
 * Errors: EINVAL (sizes, a Jacobian with det <= 0, a singular coarsest
 * operator), ECUDA, ENOMEM. */
igamg_status igamg_setup_general(int p, const int* n_elems, int n_levels, igamg_ctx** out);
/* Number of quadrature points nq = (n_x (p+1)) (n_y (p+1)) and their
 * parameter coordinates (xi, eta) in [0,1]^2, x fastest: h_xi, h_eta hold nq
 * doubles each.  The caller maps them by F and evaluates A, B, c, f there. */
long igamg_quadrature_count(const igamg_ctx* ctx);
igamg_status igamg_quadrature_points(const igamg_ctx* ctx, double* h_xi, double* h_eta);
/* Assembles every level on the host and uploads it (may be called again with
 * new coefficients).  h_coef: 6 nq doubles, A11, A12, A22, B1, B2, c at the
 * mapped points (coefficient-major: h_coef[k nq + q]); h_jac: 4 nq doubles,
 * dF1/dxi, dF1/deta, dF2/dxi, dF2/deta at the points, or NULL for the unit
 * square (F = identity). */
igamg_status igamg_assemble_general(igamg_ctx* ctx, const double* h_coef, const double* h_jac);
/* Load vector b_I = int f phi_I (with |J|) from h_f: nq values of f at the
 * mapped points; writes d_b (finest N) and synchronises `stream`. */
igamg_status igamg_rhs_points(igamg_ctx* ctx, const double* h_f, double* d_b, void* stream);

/* ---------------------------------------------------------------- solve */

/* Restarted extrapolation (Algorithm 5) around the V-cycle (Algorithm 2, mu=1,
 * one multicolour Gauss-Seidel sweep before and after the coarse correction,
 * (p+1)^dim colours, ascending before and descending after).
 * Each restart cycle runs k+1 V-cycles from s_0, extrapolates t by RRE
 * (Algorithm 3) or MPE (Algorithm 4) through the Gram matrix of the
 * differences, and stops when ||b - A t|| / ||b|| <= tol (or the absolute test
 * with IGAMG_FLAG_ABS_TOL); else s_0 := t.  With IGAMG_EXTRAP_NONE each cycle
 * is a single V-cycle and k is ignored.  k in [1, 12].
 * d_b: finest right-hand side (read only).  d_x: solution (written; read as
 * s_0 with IGAMG_FLAG_X0_GIVEN).  h_hist (may be NULL) receives max_cycles+1
 * relative residuals: entry 0 for s_0, entry c after cycle c.  h_cycles and
 * h_vcycles receive the restart cycles and V-cycles run.
 * The restart loop runs on the GPU: one CUDA graph holds a conditional WHILE
 * node around the restart cycle, whose last kernel applies the accuracy test
 * to the residual and sets the loop condition, so a solve is one graph launch
 * and one host synchronisation (not with IGAMG_FLAG_HOST_LOOP or
 * IGAMG_FLAG_NO_GRAPH, for IGAMG_FP32_IR_LEARNED, whose stall fallback
 * switches smoothers between cycles, or for max_cycles >= 2047: then the
 * host tests the residual after every cycle).  Same arithmetic either way.
 * Returns OK on convergence, ENOTCONV after max_cycles (d_x = last iterate),
 * EBREAKDOWN on a non-finite residual, ETIMEOUT when a bounded device wait of
 * a single-launch sweep gave up.  Synchronises `stream`. */
igamg_status igamg_solve(igamg_ctx* ctx, const double* d_b, double* d_x, double tol,
                         int extrap, int k, int max_cycles, int prec, unsigned flags,
                         void* d_ws, size_t ws_bytes, void* stream,
                         double* h_hist, int* h_cycles, int* h_vcycles);

/* --------------------------------------------- components (FP64, for checks) */

/* y = A_level x, A = sum_d K_d (x) prod_{e!=d} M_e (matrix free, sum-factorised). */
igamg_status igamg_apply(igamg_ctx* ctx, int level, const double* d_x, double* d_y,
                         void* d_ws, size_t ws_bytes, void* stream);

/* One multicolour Gauss-Seidel sweep on `level`, in place on d_x
 * (descending = 0: colours ascending; 1: descending). */
igamg_status igamg_smooth(igamg_ctx* ctx, int level, double* d_x, const double* d_b,
                          int descending, void* d_ws, size_t ws_bytes, void* stream);

/* The same sweep in FP32 (the smoother of FP32 V-cycles).  The row partial
 * sums T_M, T_K of d_x live in the workspace (sized for IGAMG_FP32_IR);
 * sums_current = 1 reuses them as the previous igamg_smooth_f32 call on this
 * level and workspace left them (valid only if d_x has not changed since),
 * 0 recomputes them first. */
igamg_status igamg_smooth_f32(igamg_ctx* ctx, int level, float* d_x, const float* d_b, int descending,
                              int sums_current, void* d_ws, size_t ws_bytes, void* stream);

/* d_coarse = P_level^T d_fine (restriction from `level` to level-1). */
igamg_status igamg_restrict(igamg_ctx* ctx, int level, const double* d_fine, double* d_coarse,
                            void* d_ws, size_t ws_bytes, void* stream);

/* d_fine += P_level d_coarse (prolongation from level-1 to `level`). */
igamg_status igamg_prolong(igamg_ctx* ctx, int level, const double* d_coarse, double* d_fine,
                           void* d_ws, size_t ws_bytes, void* stream);

/* d_e = A_0^{-1} d_r on the coarsest level (fast diagonalisation). */
igamg_status igamg_coarse_solve(igamg_ctx* ctx, const double* d_r, double* d_e, void* stream);

/* One V-cycle (Algorithm 2, mu = 1) in place on the finest d_x with right side
 * d_b, in the given precision (FP32_IR: one refinement step
 * x += sigma V32(0; (b - A x) / sigma)). */
igamg_status igamg_vcycle(igamg_ctx* ctx, double* d_x, const double* d_b, int prec,
                          void* d_ws, size_t ws_bytes, void* stream);

/* One RRE / MPE extrapolation (Algorithms 3-4, via the Gram matrix of the
 * differences) on q+2 iterates of length n stored at d_S + j*ld (j = 0..q+1):
 * writes t to d_t, the q+2 combination weights to h_gamma (gamma_{q+1} is
 * non-zero only on the breakdown fallback) and the q actually used to h_qused
 * (-1 = fallback t = s_{q+1}).  Needs igamg_extrap_workspace_bytes(n, q). */
size_t igamg_extrap_workspace_bytes(long n, int q);
igamg_status igamg_extrapolate(long n, int q, int method, const double* d_S, long ld,
                               double* d_t, double* h_gamma, int* h_qused,
                               void* d_ws, size_t ws_bytes, void* stream);

/* Allocation-free igamg_extrapolate, for callers that cannot allocate device
 * memory where they extrapolate (a host framework that owns all device
 * allocations and forbids cudaMalloc on its hot path, since cudaMalloc can
 * block the device and fail on fragmented memory; code under a fixed memory
 * budget with no allocator to hand scratch through).  The paper has no
 * counterpart: this is an interface variant only; the arithmetic is that of
 * igamg_extrapolate.
 * Scratch is a 240 KiB array built into the library, resident on every GPU
 * that loads it until the process exits; every restart number q in [1, 12]
 * fits (larger requests return EINVAL).  The first call on a device looks up
 * the array's device address, so make it before any stream capture.  All
 * calls share the array: calls whose GPU work overlaps (e.g. on two streams)
 * race and must be serialised.  Arguments and results are those of
 * igamg_extrapolate without (d_ws, ws_bytes); synchronises `stream`. */
igamg_status igamg_extrapolate_noalloc(long n, int q, int method, const double* d_S, long ld,
                                       double* d_t, double* h_gamma, int* h_qused, void* stream);

/* ------------------------------------------- Gauss-Seidel sweep schedule */

/* Form of the multicolour Gauss-Seidel sweep (Sec. 2.4; the same colours,
 * order and arithmetic either way, so the results are identical).  The
 * single-launch form runs a whole sweep in one kernel launch, each row
 * starting as soon as the rows within reach of earlier colours are done
 * (persistent CTAs claim rows in colour order and wait on per-row flags in
 * the workspace); the other form runs one launch per row phase ((p+1)^(dim-1)
 * per sweep).  Per precision of the cycle (FP32 V-cycles of the mixed forms,
 * FP64 cycles): 0 = row phases on every level, 1 = one launch on every level,
 * N >= 2 = one launch on levels with at least N rows (m_y m_z), -1 =
 * unchanged.  Defaults: 2D row phases; 3D one launch from 8192 rows.
 * igamg_autotune picks the threshold by timing.  Errors: EINVAL. */
igamg_status igamg_set_sweep_form(igamg_ctx* ctx, int single_launch_fp32, int single_launch_fp64);
void igamg_get_sweep_form(const igamg_ctx* ctx, int* single_launch_fp32, int* single_launch_fp64);

/* Bound of every device-side wait of the single-launch sweeps, in seconds
 * (process-wide, default 1; read when work is enqueued or a restart graph is
 * captured).  A wait that runs out sets an error word in the workspace and
 * the kernel finishes normally; igamg_solve and igamg_batch_solve then return
 * IGAMG_ETIMEOUT (the iterate is not meaningful), and igamg_device_status
 * reports it after component calls.  test_unset_flag = 1 makes every sweep
 * CTA first wait on a word that nothing sets, so that the wait runs out: it
 * exists to test this path and slows every sweep by the limit. */
void igamg_set_wait_limit(double seconds, int test_unset_flag);

/* Synchronises `stream` and returns IGAMG_ETIMEOUT (clearing the word) when
 * a bounded device-side wait of a call that used workspace d_ws gave up
 * since the word was last cleared, else IGAMG_OK. */
igamg_status igamg_device_status(const igamg_ctx* ctx, void* d_ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------- learned smoother */

/* A small convolutional network used as the finest-level post-smoother of
 * IGAMG_FP32_IR_LEARNED solves (the paper has no learned component; this is
 * the build's extension of the smoothing step of Algorithm 2).  Three 3x3
 * zero-padded convolutions without biases, 1 -> 16 -> 16 -> 1 channels, ReLU
 * after the first two; BF16 activations, FP32 accumulation, the 16 -> 16
 * layer on the tensor cores.  Weights: igamg_cnn_num_weights() FP32 values,
 * W1[co][tap] (144), W2[co][ci][tap] (2304), W3[ci][tap] (144), tap =
 * 3 (dy+1) + (dx+1) reading pixel (y+dy, x+dx).  Images: batch x H x W FP32,
 * x fastest. */
int igamg_cnn_num_weights(void);
size_t igamg_cnn_workspace_bytes(int batch, int H, int W);
/* d_y = network(d_r). */
igamg_status igamg_cnn_forward(int batch, int H, int W, const float* d_r, const float* d_w, float* d_y,
                               void* d_ws, size_t ws_bytes, void* stream);
/* d_loss[0] = 0.5 mean((network(d_r) - d_e)^2) and d_grad = its gradient with
 * respect to the weights (deterministic reductions). */
igamg_status igamg_cnn_grad(int batch, int H, int W, const float* d_r, const float* d_e, const float* d_w,
                            float* d_grad, float* d_loss, void* d_ws, size_t ws_bytes, void* stream);
/* One Adam step (bias-corrected) on n parameters; step counts from 1. */
igamg_status igamg_adam_step(int n, float* d_w, const float* d_g, float* d_m, float* d_v, int step, float lr,
                             float b1, float b2, float eps, void* stream);

/* Use the network with weights d_w (device, caller-owned, must outlive the
 * solves) as the finest-level post-smoother of IGAMG_FP32_IR_LEARNED solves:
 * after the coarse correction x += network(b - A x) replaces the Gauss-Seidel
 * sweep.  When a restart cycle reduces the relative residual by less than
 * the factor stall_ratio (e.g. 0.9), the solve falls back to plain
 * Gauss-Seidel post-smoothing for its remaining cycles;
 * igamg_smoother_fell_back() reports whether the last solve did.  2D
 * problems only (IGAMG_EINVAL otherwise); d_w = NULL unsets the network. */
igamg_status igamg_set_smoother(igamg_ctx* ctx, const float* d_w, double stall_ratio);
int igamg_smoother_fell_back(const igamg_ctx* ctx);

/* Coarse tail of FP32 V-cycles (the paper's V-cycle, Algorithm 2, with a
 * different schedule): levels 0..lc run in one kernel launch instead of one
 * launch per smoothing phase and transfer pass.  2D: on one CTA (levels of at
 * most 6000 unknowns that together fit its shared memory; the default) or on
 * a thread-block cluster (igamg_set_tail_ctas).  3D: on a 16-CTA cluster (the
 * default) or 8.  Same arithmetic up to FP32 rounding order.
 * igamg_coarse_tail_level() returns lc (0: none or disabled);
 * igamg_set_coarse_tail(ctx, 0) switches it off (on by default), e.g. to
 * compare schedules.  FP64 cycles never use it (on GB300 the per-level FP64
 * kernels spread over all SMs are faster). */
int igamg_coarse_tail_level(const igamg_ctx* ctx);
igamg_status igamg_set_coarse_tail(igamg_ctx* ctx, int enable);

/* Launch schedule of the FP32 V-cycles: gs_threads caps the threads of the
 * GS row CTAs (0 = default 512, else 128, 256 or 512); tail_levels sets the
 * coarse tail to levels 0..tail_levels (clipped to the feasible maximum; 0 =
 * off, -1 = unchanged).  Arithmetic is unchanged up to FP32 rounding order. */
igamg_status igamg_set_schedule(igamg_ctx* ctx, int gs_threads, int tail_levels);
void igamg_get_schedule(const igamg_ctx* ctx, int* gs_threads, int* tail_levels);

/* Where the coarse tail runs: ctas = 1 on one CTA (2D only), 8 or 16 on one
 * thread-block cluster of that many CTAs (2D and 3D).  The cluster form splits
 * every tail level's grid rows into contiguous bands, one per CTA, kept in
 * that CTA's shared memory; the rows a step needs from a neighbouring band
 * are read from the neighbour's shared memory (distributed shared memory),
 * and cluster barriers order the steps (3D: each CTA also keeps copies of
 * the rows within reach of its band, written by their owners).  Its levels
 * are limited by the shared memory of one CTA per band (2D: about 257^2
 * unknowns on 16 CTAs; 3D: about 33^3), not by 6000 unknowns.  Same colours, order and operators (FP32 rounding order
 * aside).  Switching keeps the tail depth where the other form has it, else
 * takes its deepest; igamg_tail_levels_available() gives the deepest tail
 * level of each form (0: none), igamg_get_tail_ctas() the form in use.
 * igamg_autotune times every form and depth.  The first use of a cluster-tail
 * depth (3D: the default one at set-up) builds, once, each CTA's unchanging
 * shared memory (operator data, transfer tables, neighbour-row addresses)
 * into device memory the context owns and frees in igamg_destroy; every cycle
 * then copies it in.  Where that memory cannot be had, 2D falls back to the
 * one-CTA tail and 3D to per-level launches.  Errors: EINVAL (ctas not 1, 8
 * or 16). */
igamg_status igamg_set_tail_ctas(igamg_ctx* ctx, int ctas);
int igamg_get_tail_ctas(const igamg_ctx* ctx);
int igamg_tail_levels_available(const igamg_ctx* ctx, int ctas);

/* Cycle of Algorithm 2 (Sec. 2.4) used by every solve, cycle and autotune
 * call of this context.  smoother: IGAMG_SMOOTH_GS (default; multicolour
 * Gauss-Seidel, (p+1)^dim colours, ascending before and descending after the
 * coarse correction) or IGAMG_SMOOTH_JACOBI (weighted Jacobi
 * x += omega D^{-1} (b - A x), the smoother of the paper's experiments in
 * Sec. 4 with omega = 2/3; omega in (0, 2), ignored for GS).  mu = 1 is the
 * V-cycle (default), mu = 2 the W-cycle (the coarse problem of every level
 * above the coarsest is approximated by two cycles from a zero start).
 * nu1 = nu2 = 1; the coarsest level is solved directly.  FP32 2D V-cycles
 * (either smoother) run their coarse levels in the one-CTA tail
 * (igamg_set_coarse_tail); W-cycles run per-level kernels throughout.  With
 * anything but the default Gauss-Seidel V-cycle, IGAMG_FP32_IR_LEARNED solves
 * and igamg_vcycle_probe return IGAMG_EINVAL.  Errors: IGAMG_EINVAL for other
 * values. */
igamg_status igamg_set_cycle(igamg_ctx* ctx, int smoother, int mu, double omega);
void igamg_get_cycle(const igamg_ctx* ctx, int* smoother, int* mu, double* omega);

/* Launch overlap (process-wide, on by default): the kernels of the V-cycle,
 * refinement and extrapolation chain are launched with programmatic stream
 * serialisation, so that each kernel's CTAs are scheduled while its
 * predecessor drains and start work the moment the predecessor's writes are
 * visible.  Same kernels, same order, same results; only the gaps between
 * launches shrink.  Takes effect for launches enqueued, and restart-cycle
 * graphs captured, after the call (a context recaptures its graph on its next
 * solve when the setting differs from the one it was captured with). */
void igamg_set_launch_overlap(int enable);
int igamg_get_launch_overlap(void);

/* Autotuner: times `reps` FP32 V-cycles (zero start, constant right side) for
 * every GS row-CTA cap in {128, 256, 512} (2D) and every coarse-tail depth,
 * on the given stream, and keeps the fastest schedule.  The workspace must be
 * sized for IGAMG_FP32_IR; its contents are overwritten.  Synchronises the
 * stream; typically a few tens of milliseconds. */
igamg_status igamg_autotune(igamg_ctx* ctx, void* d_ws, size_t ws_bytes, void* stream, int reps);

/* One FP64 V-cycle in place on the finest d_x (as igamg_vcycle) that also
 * copies the iterate at the point just before the finest-level post-smoothing
 * (after the coarse correction) to d_x_mid: the network's training input. */
igamg_status igamg_vcycle_probe(igamg_ctx* ctx, double* d_x, const double* d_b, double* d_x_mid,
                                void* d_ws, size_t ws_bytes, void* stream);

/* Training pairs of the learned post-smoother, generated by the solver
 * itself: restarted RRE(k) (Algorithm 5 with Algorithm 3) in FP64 from s_0 =
 * 0 on right side d_b, every V-cycle probed as in igamg_vcycle_probe.  For
 * each V-cycle (in order, up to max_pairs) with probed iterate x_mid it
 * writes the pair r = b - A x_mid, e = u_h - x_mid (d_uh: the discrete
 * solution, e.g. an igamg_solve to 1e-13), both scaled by the same c > 0 so
 * that e has unit root-mean-square, as FP32 rows of length N into d_R and d_E
 * (pair i at offset i N).  Stops after the restart whose extrapolant passes
 * ||b - A t|| / ||b|| <= tol, or after max_restarts.  h_pairs receives the
 * number of pairs written.  Workspace: igamg_training_workspace_bytes(ctx,
 * k).  Synchronises `stream` once per restart.  Errors: EINVAL (also for a
 * context whose cycle is not the Gauss-Seidel V-cycle), ENOMEM, EBREAKDOWN. */
size_t igamg_training_workspace_bytes(const igamg_ctx* ctx, int k);
igamg_status igamg_training_pairs(igamg_ctx* ctx, const double* d_b, const double* d_uh, int k, double tol,
                                  int max_restarts, float* d_R, float* d_E, int max_pairs, void* d_ws,
                                  size_t ws_bytes, void* stream, int* h_pairs);

/* ---------------------------------------------------------------- batches */

/* Many independent problems of uneven size and degree, solved together.
 * Problem i: dimension dim, degree p[i], n[i] elements per direction.  The
 * right-hand sides and solutions are packed back to back in one vector; use
 * igamg_batch_layout for the offsets (count+1 entries, last = total length).
 * Each problem runs the restarted extrapolation of igamg_solve with its own
 * convergence test; problems that converge stop while the others continue.
 * (The paper treats one problem at a time; batching is an interface
 * extension of Algorithm 5.) */
typedef struct igamg_batch igamg_batch;
igamg_status igamg_batch_create(int count, int dim, const int* p, const int* n, igamg_batch** out);
igamg_status igamg_batch_layout(const igamg_batch* batch, long* h_offsets);
size_t igamg_batch_workspace_bytes(const igamg_batch* batch, int k, int prec);
/* h_coeffs: count blocks of modes^dim sine coefficients (see igamg_rhs_sine). */
igamg_status igamg_batch_rhs_sine(igamg_batch* batch, int modes, const double* h_coeffs, double* d_b,
                                  void* stream);
/* extrap: IGAMG_RRE or IGAMG_MPE.  h_cycles, h_status, h_res (may be NULL):
 * per problem the restart cycles run, its igamg_status and its final relative
 * residual.  Returns OK when every problem converged, else the first
 * non-OK status.  Synchronises `stream`. */
igamg_status igamg_batch_solve(igamg_batch* batch, const double* d_b, double* d_x, double tol, int extrap,
                               int k, int max_cycles, int prec, void* d_ws, size_t ws_bytes, void* stream,
                               int* h_cycles, int* h_status, double* h_res);
/* Where the batch's restart loops run.  enable = 1 (default): on the GPU, in
 * one CUDA graph whose independent branches hold, per problem, a kernel that
 * starts its loop (unless it converged at s_0 = 0) and a conditional WHILE
 * node around its restart cycle, ended on the device by its own accuracy
 * test; a batched solve is then one graph launch and one host
 * synchronisation.  enable = 0: rounds of per-problem restart-cycle graphs on
 * 128 streams, the host testing every residual after each round.  Same
 * arithmetic either way.  Errors: EINVAL for a null batch. */
igamg_status igamg_batch_set_device_loop(igamg_batch* batch, int enable);
/* Every problem's coarse tail on one CTA (ctas = 1) or on a cluster of 8 or
 * 16 CTAs (igamg_set_tail_ctas), each at that form's deepest level.  The
 * members' clusters run concurrently like their other kernels.  Errors:
 * EINVAL. */
igamg_status igamg_batch_set_tail_ctas(igamg_batch* batch, int ctas);
/* Autotunes the batch: for every degree, igamg_autotune on the problem of
 * median size, with the one-CTA coarse tail only (the members run
 * concurrently, and a cluster tail ties up 8 or 16 SMs for a latency-bound
 * stretch the others could use); the problems of that degree take its GS
 * row-CTA cap and a coarse tail down to the same level size.  The workspace
 * is the batch workspace (sized for IGAMG_FP32_IR); its contents are
 * overwritten. */
igamg_status igamg_batch_autotune(igamg_batch* batch, void* d_ws, size_t ws_bytes, void* stream, int reps);
void igamg_batch_destroy(igamg_batch* batch);

/* ---------------------------------------------------------------- misc */

void igamg_destroy(igamg_ctx* ctx);
const char* igamg_status_str(int status);
const char* igamg_last_error(void);
/* Number of kernel launches this thread has enqueued (including graph nodes
 * replayed), for launch accounting in benchmarks. */
long long igamg_launch_count(void);

/* Per-kernel timing for measurement.  After igamg_profile_start(), every
 * kernel of the solver that this thread enqueues directly (not while a stream
 * is captured into a graph: use IGAMG_FLAG_NO_GRAPH | IGAMG_FLAG_HOST_LOOP)
 * is bracketed by CUDA events on its own stream.  igamg_profile_stop()
 * synchronises on them, ends the profile and returns the number of launches
 * recorded; the first cap of them are written in launch order: the kernel's
 * name (NUL-terminated, at most name_len bytes each, in h_names, may be NULL),
 * its duration in microseconds (h_us) and its grid size in CTAs (h_grid).
 * The events serialise the stream, so launches lose their overlap. */
void igamg_profile_start(void);
long igamg_profile_stop(int cap, char* h_names, int name_len, double* h_us, int* h_grid);

#ifdef __cplusplus
}
#endif
#endif /* IGAMG_H */
