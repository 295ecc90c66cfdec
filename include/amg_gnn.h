/*
 * amg_gnn.h -- C ABI of the GB300 (sm_103a) GNN-smoothed algebraic multigrid
 * pressure solver ("Acceleration of an algebraic multigrid pressure solver
 * using graph neural networks").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices follow the symmetric positive definite sign convention: positive
 *   diagonal, non-positive off-diagonal couplings (the negative of the
 *   negative semi-definite operator of Sec. 2.1).  A must be symmetric with
 *   every diagonal entry present in its pattern.
 * - CSR arrays are 0-based, int32 row pointers and column indices with
 *   ascending columns inside each row, float64 values.
 * - Host pointers are read during the call only; the library copies what it
 *   keeps.  Device pointers ("d_" prefix) are caller-owned device memory on
 *   the context's device and must stay valid until the work enqueued on the
 *   given stream has finished.  A NULL stream means the legacy default stream.
 * - Every int-returning call returns AMG_OK (0) or a negative AMG_ERR_* code;
 *   amg_last_error() then describes the failure.  Errors from argument checks
 *   leave the context unchanged.  A context is not thread-safe.
 */
#ifndef AMG_GNN_H
#define AMG_GNN_H

#ifdef __cplusplus
extern "C" {
#endif

#define AMG_OK               0
#define AMG_ERR_ARG         -1  /* invalid argument or size                         */
#define AMG_ERR_CUDA        -2  /* a CUDA runtime call failed                       */
#define AMG_ERR_NOT_SPD     -3  /* coarsest matrix not positive definite            */
#define AMG_ERR_DIVERGED    -4  /* residual not finite or > 1e3 x initial residual  */
#define AMG_ERR_STAGNATED   -5  /* best residual of the last 10 V-cycles not 1% below
                                   the best of the 10 before them               */
#define AMG_ERR_MAXITER     -6  /* max_iter V-cycles without reaching the tolerance */
#define AMG_ERR_DEVICE_FLAG -7  /* a kernel reported an invalid index or value      */
#define AMG_ERR_STATE       -8  /* call made in the wrong order (e.g. no hierarchy) */

/* precision of the V-cycle (the outer residual/update are always FP64) */
#define AMG_FP64         0
#define AMG_FP32_IN_FP64 1

/* smoother of the V-cycle */
#define AMG_SMOOTHER_JACOBI 0   /* relaxed Jacobi, Q^-1 = omega D^-1 (Sec. 2.3)          */
#define AMG_SMOOTHER_GNN    1   /* sparse pseudo-inverse from coefficients (Sec. 3.1)    */
#define AMG_SMOOTHER_CHEB   2   /* Chebyshev polynomial in D^-1 A (fixed-coefficient baseline) */

/* outer iteration around the V-cycle */
#define AMG_OUTER_REFINE 0      /* stationary correction x += V(b - A x) (Sec. 2.1)       */
#define AMG_OUTER_PCG    1      /* conjugate gradients preconditioned by one V-cycle      */

/* arithmetic of the GCIN node linears (layers 2..4) */
#define AMG_GNN_FP32 0   /* FP32 CUDA-core FMAs                                  */
#define AMG_GNN_BF16 1   /* tcgen05 tensor cores: BF16 operands, FP32 accumulation */

#define AMG_GCIN_NUM_PARAMS 55045       /* App. A.1: GCIN width 64 */
#define AMG_GCIN_NUM_PARAMS_H32 37189   /* App. B.3: the halved GCIN width 32 */

typedef struct amg_ctx amg_ctx;

typedef struct {
    int n_rows;
    int n_cols;
    long long nnz;
    const int *row_ptr;   /* n_rows + 1 */
    const int *col;       /* nnz        */
    const double *val;    /* nnz        */
} amg_csr;

typedef struct {
    int nu1;          /* pre-smoothing sweeps per level  (Sec. 4: 2)                 */
    int nu2;          /* post-smoothing sweeps per level (Sec. 4: 2)                 */
    int max_levels;   /* hierarchy depth cap (Table train_hyper: 10)                 */
    int max_coarse;   /* stop coarsening at n <= max_coarse (64)                     */
    int max_iter;     /* V-cycle cap of a solve (Sec. 4: 500)                        */
    int precision;    /* AMG_FP64 or AMG_FP32_IN_FP64                                */
    int smoother;     /* AMG_SMOOTHER_JACOBI or AMG_SMOOTHER_GNN                     */
    double omega;     /* Jacobi relaxation (Sec. 4: 2/3)                             */
    double theta;     /* Ruge-Stueben strength threshold (Sec. 4: 0.25)              */
    int device;       /* CUDA device ordinal                                         */
    int gnn_precision;/* AMG_GNN_BF16 (default) or AMG_GNN_FP32                      */
    int outer;        /* AMG_OUTER_REFINE (default) or AMG_OUTER_PCG: FP64 conjugate
                         gradients with the V-cycle (zero initial guess) as the
                         preconditioner and the flexible coefficient
                         beta = z_k.(r_k - r_{k-1}) / (z_{k-1}.r_{k-1}); the history
                         then holds the recurrence residual, and a breakdown
                         (z.r <= 0 or p.Ap <= 0) ends the solve with
                         AMG_ERR_DIVERGED leaving x at the last iterate           */
    int fused_sweeps; /* 0 (default): one kernel per pass.  1: on levels too
                         large for the L2 cache, each smoothing phase of the
                         V-cycle (with the residual for restriction, or with the
                         prolongation-correction) runs as one wavefront kernel
                         that re-reads A from L2 instead of HBM, with the
                         pseudo-inverse values evaluated on the fly in FP32
                         (same operators; slower on GB300 so far: the passes are
                         bound by load latency, not by HBM bandwidth)            */
} amg_options;

/* Fill *opt with the paper's settings: nu1 = nu2 = 2, max_levels = 10,
 * max_coarse = 64, max_iter = 500, FP32 V-cycle in FP64 refinement, Jacobi,
 * omega = 2/3, theta = 0.25, device 0, BF16 tensor-core GCIN linears
 * (Sec. 4, Table train_hyper). */
void amg_default_options(amg_options *opt);

/* Create a context bound to opt->device.  *ctx receives the handle (NULL on
 * error).  Errors: AMG_ERR_ARG for out-of-range options, AMG_ERR_CUDA. */
int amg_create(amg_ctx **ctx, const amg_options *opt);

/* Release every host and device resource of ctx (NULL is allowed). */
void amg_destroy(amg_ctx *ctx);

/* Message of the last failing call on ctx (never NULL; "" after success).
 * With ctx == NULL: the message of the last failing amg_create. */
const char *amg_last_error(const amg_ctx *ctx);

/* ------------------------------------------------------------------------
 * Setup phase (Sec. 2.2; Algorithm 1 step 2), host C++ -- off the hot path.
 * ------------------------------------------------------------------------ */

/* Setup-AMG-Hierarchy: build {A_l, P_l, R_l} from A by classical
 * Ruge-Stueben coarsening (strength theta), direct interpolation, R = P^T and
 * the Galerkin product A_c = R A P (Sec. 2.2), until n <= max_coarse, the
 * level cap, or a coarse level keeping > 90% of the points; then upload it to
 * the device and factor the coarsest level (as amg_load_hierarchy).
 * Replaces any previous hierarchy and resets the smoother to Jacobi.
 * Errors: AMG_ERR_ARG (non-square, bad CSR), AMG_ERR_NOT_SPD, AMG_ERR_CUDA. */
int amg_setup(amg_ctx *ctx, const amg_csr *A);

/* C/F split of amg_setup_device (flags; 0 = PMIS alone) */
#define AMG_SPLIT_SECOND_PASS 1 /* then the round-parallel second pass         */
#define AMG_SPLIT_RS_BLOCKS   2 /* block-local RS first pass instead of PMIS   */

/* amg_setup with every level built on the device and the Ruge-Stueben first
 * pass (Sec. 2.2, Sec. 4: classical RS, theta = 0.25) in a parallel form:
 *  - AMG_SPLIT_RS_BLOCKS: the rows are cut into consecutive blocks of B rows
 *    and the classical first pass (largest measure first, ties to the lowest
 *    index) runs on each block's induced strength subgraph, one CTA per block
 *    (B = the largest of 4096, 2048, ..., 128 with at most 32768 strong
 *    pairs inside every block; with one block this is amg_setup's split); then
 *    every F point with strong dependencies but none on a C point (its
 *    couplings all leave its block) becomes C.  Numberings with locality (a
 *    mesh order, RCM) keep the coarse grids within a few percent of RS;
 *  - otherwise PMIS (De Sterck, Yang & Heys 2006) on the same strength
 *    graph: measure lambda_i = |S_i^T| + r_i (FP64), points with
 *    |S_i^T| = 0 start as F, then rounds in which every undecided point that
 *    beats all undecided points of S_i u S_i^T (larger lambda, ties to the
 *    lower index) becomes C and every undecided point with a strong
 *    dependency on a new C point becomes F.
 * Level l draws r_i (i = 0 .. n_l - 1) as the top 53 bits of output i + 1 of
 * splitmix64 started at seed + l, times 2^-53.  AMG_SPLIT_SECOND_PASS then
 * runs rounds in which every F point j with a strong F partner i (j in S_i)
 * sharing no strong C point with it counts those pairs v_j, and each such j
 * that beats every such candidate in S_j u S_j^T (v + r, ties to the lower
 * index) becomes C, until every strong F-F pair has a common strong C point
 * (denser coarse levels, fewer V-cycles).  split = 0 / 1 keep the PMIS
 * meanings of the former second_pass flag.  Direct interpolation, R = P^T and
 * A_c = R (A P) as amg_setup, on the device; the levels are copied device to
 * device into the solve's memory and reach the host only when asked for
 * (amg_get_level copies a level's entries once).  A (host CSR) is
 * copied.  Same stopping rules and errors as amg_setup, AMG_ERR_ARG for an
 * unknown split; AMG_ERR_CUDA also covers device allocation failures.  PMIS
 * with the second pass keeps about half the points per level, so meshes of
 * millions of rows need max_levels of about 16 to keep the coarsest level
 * within the dense solve's 4096 rows. */
int amg_setup_device(amg_ctx *ctx, const amg_csr *A, unsigned long long seed, int split);

/* Load a caller-built hierarchy: A[0..n_levels-1] (finest first),
 * P[0..n_levels-2] (n_l x n_{l+1}) and R[0..n_levels-2] (n_{l+1} x n_l);
 * R may be NULL, then R = P^T is formed.  Copies everything to the device,
 * computes s_l = max|A_l - D_l| for every level (Sec. 3.1) and factors the
 * coarsest A by dense Cholesky on the device (FP64).
 * Errors: AMG_ERR_ARG (sizes disagree), AMG_ERR_NOT_SPD, AMG_ERR_CUDA. */
int amg_load_hierarchy(amg_ctx *ctx, int n_levels, const amg_csr *A, const amg_csr *P, const amg_csr *R);

/* Number of levels of the loaded hierarchy (0 if none). */
int amg_num_levels(const amg_ctx *ctx);

/* Sizes of level `level`: rows, nnz of A_l and nnz of P_l (0 on the
 * coarsest level).  Any output pointer may be NULL. */
int amg_level_info(const amg_ctx *ctx, int level, int *n, long long *nnz_A, long long *nnz_P);

/* Copy level `level`'s A_l and P_l (host hierarchy) into caller buffers
 * sized by amg_level_info; the P buffers are ignored (may be NULL) on the
 * coarsest level.  Errors: AMG_ERR_ARG, AMG_ERR_STATE. */
int amg_get_level(const amg_ctx *ctx, int level, int *A_row_ptr, int *A_col, double *A_val,
                  int *P_row_ptr, int *P_col, double *P_val);

/* Smoother scale s_l = max |A_l - D_l| of every level as computed on the
 * device (Sec. 3.1); s_out has amg_num_levels() entries. */
int amg_get_scales(const amg_ctx *ctx, double *s_out);

/* ------------------------------------------------------------------------
 * Smoother selection (Sec. 2.3, Sec. 3.1)
 * ------------------------------------------------------------------------ */

/* Relaxed Jacobi on every level: Q^-1 = omega D^-1 (Sec. 2.3). */
int amg_set_jacobi(amg_ctx *ctx, double omega);

/* Sparse pseudo-inverse smoother (Sec. 3.1) on every smoothed level l from
 * c[5 l .. 5 l + 4] = (d0, d1, d2, o1, o2):
 *   q_ii^-1 = (d0 + d1 x + d2 x^2) / a_ii,        x = a_ii / s_l
 *   q_ij^-1 = (o1 x + o2 x^2) / (a_ii + a_jj),    x = a_ij / s_l.
 * c holds n_rows >= amg_num_levels() - 1 rows (extra rows ignored).
 * The Q^-1 values are assembled on the device once, in FP64 and in the
 * V-cycle precision.  c = (omega, 0, 0, 0, 0) reproduces weighted Jacobi. */
int amg_set_coeffs(amg_ctx *ctx, const double *c, int n_rows);

/* The same smoother with one coefficient row per node instead of per level
 * (a generalisation; the paper's coefficients are per level): c holds, level
 * by level for l = 0 .. amg_num_levels() - 2, n_l rows of
 * (d0, d1, d2, o1, o2) (host, n_values = 5 sum_l n_l doubles, copied).
 * q_ii^-1 uses node i's (d0, d1, d2); q_ij^-1 uses the mean of nodes i's and
 * j's (o1, o2), so Q^-1 stays symmetric.  Rows all equal to c_l give exactly
 * amg_set_coeffs' values.  Errors: AMG_ERR_ARG (wrong n_values, NULL or
 * non-finite values), AMG_ERR_STATE (no hierarchy), AMG_ERR_CUDA. */
int amg_set_node_coeffs(amg_ctx *ctx, const double *c, long long n_values);

/* Read back the smoother values of level `level` on A_l's pattern (nnz_A
 * entries, FP64 copy).  Jacobi leaves zeros off the diagonal. */
int amg_get_smoother(const amg_ctx *ctx, int level, double *q_out);

/* ------------------------------------------------------------------------
 * Coefficient network (Sec. 3.2, App. A.1; Algorithm 1 steps 3-6)
 * ------------------------------------------------------------------------ */

/* Load the GCIN parameters (copied to the device): n floats in the flat
 * order conv1 W(2xH) b(H); conv2..4 W(HxH) b(H); IN1..4 gamma(H) beta(H);
 * readout1..4 W(2Hx32) b(32); LN gamma(128) beta(128); head W(128x128)
 * b(128), W(128x64) b(64), W(64x5) b(5); weights [in][out] row-major.  The
 * GCIN width H follows from n: AMG_GCIN_NUM_PARAMS -> H = 64 (App. A.1),
 * AMG_GCIN_NUM_PARAMS_H32 -> H = 32 (App. B.3).  Errors: AMG_ERR_ARG (any
 * other n, or theta NULL), AMG_ERR_CUDA. */
int gnn_load_params(amg_ctx *ctx, const float *theta, long long n);

/* Batched GCIN inference over every level graph of the loaded hierarchy
 * (node features [a_ii, deg_i], edge weights a_ij, self-loop weight a_ii),
 * then amg_set_coeffs with the result.  c_out (host, may be NULL) receives
 * amg_num_levels() rows of 5.  Errors: AMG_ERR_STATE (no hierarchy or no
 * parameters), AMG_ERR_CUDA. */
int gnn_predict_coeffs(amg_ctx *ctx, double *c_out);

/* ------------------------------------------------------------------------
 * Solve phase (Sec. 2.1, 2.2; Algorithm 1 step 9) -- the hot path
 * ------------------------------------------------------------------------ */

/* Solve A x = b.  x holds the initial guess on entry and the last iterate on
 * return.  Each V-cycle runs in the context's precision as a preconditioner
 * of an FP64 iterative refinement x <- x + V(b - A x) (identical to the
 * stationary V-cycle iteration of Sec. 2.1 in exact arithmetic).  Stops when
 * ||b - A x||_2 / ||b||_2 <= rtol or after max_iter cycles.
 * n_vcycles (may be NULL) receives the number of V-cycles; res_hist (may be
 * NULL, max_iter + 1 entries) the relative residual before cycle 0 and after
 * every cycle.  Returns AMG_OK, AMG_ERR_DIVERGED, AMG_ERR_STAGNATED or
 * AMG_ERR_MAXITER (x and res_hist are filled in every case), AMG_ERR_STATE,
 * AMG_ERR_CUDA.  Host vectors of n_0 doubles. */
int amg_solve(amg_ctx *ctx, const double *b, double *x, double rtol, int *n_vcycles, double *res_hist);

/* amg_solve with device vectors d_b, d_x (n_0 doubles each) enqueued on
 * `stream` (a cudaStream_t); n_vcycles/res_hist are host outputs and the
 * call returns after the solve has finished on the stream. */
int amg_solve_device(amg_ctx *ctx, const double *d_b, double *d_x, double rtol, void *stream,
                     int *n_vcycles, double *res_hist);

/* One V-cycle from a zero initial guess: d_e = B d_r (Sec. 2.2), in the
 * context's precision (inputs/outputs FP64, n_0 each).  Asynchronous. */
int amg_vcycle_device(amg_ctx *ctx, const double *d_r, double *d_e, void *stream);

/* n_sweeps smoothing steps u <- u + Q_l^-1 (b - A_l u) on level `level`
 * (d_b, d_u: n_l doubles; d_u is updated in place).  Asynchronous. */
int amg_smooth_device(amg_ctx *ctx, int level, const double *d_b, double *d_u, int n_sweeps, void *stream);

/* d_y = A_l d_x on level `level` in the context's precision.  Asynchronous. */
int amg_spmv_device(amg_ctx *ctx, int level, const double *d_x, double *d_y, void *stream);

/* Relative validation metric of Sec. 3.3 on right-hand side b (host, n_0):
 * log10(||r_n^GNN|| / ||r_n^omega-J||) after n = n_cycles V-cycles from x = 0
 * with the current pseudo-inverse smoother and with omega-Jacobi (the paper
 * compares residuals after cycle n+1; more than one cycle exposes smoothers
 * that reduce the first residual well but converge slowly).  *metric is
 * +inf when the learned smoother diverges, -inf when only Jacobi does.
 * A value >= 0 means the learned smoother does not beat Jacobi.
 * Errors: AMG_ERR_ARG (n_cycles outside 1..10000), AMG_ERR_STATE, AMG_ERR_CUDA. */
int amg_judge(amg_ctx *ctx, const double *b, int n_cycles, double *metric);

/* Judge and reroute (the fallback of the learned smoother).  Runs n_cycles
 * (>= 4) V-cycles from x = 0 on b with each smoother and compares
 *   m1 = log10(||r_n^GNN|| / ||r_n^J||)                       (Sec. 3.3) and
 *   m2 = the same log-ratio for the reduction over the last n/4 cycles,
 * which exposes smoothers that start well but converge slowly; n is the
 * last cycle, or the first at which either relative residual is <= 1e-12 if
 * earlier (past it both runs sit at rounding level).  *metric = max(m1, m2)
 * (+inf when the learned smoother diverges, or alone stagnates above 1e-12).
 * If it is not negative the context falls back to omega-Jacobi and
 * amg_last_error reports the rerouting; *smoother receives the smoother in
 * use afterwards.  metric/smoother may be NULL. */
int amg_reroute(amg_ctx *ctx, const double *b, int n_cycles, double *metric, int *smoother);

/* When amg_reroute keeps the learned smoother it also arms an in-solve check
 * for the mesh (kept across coefficient updates, cleared by a new
 * hierarchy): if some 10 consecutive V-cycles of a later solve with the
 * learned smoother reduce the residual by less than half the decades Jacobi
 * gained over 10 cycles in the probe, the solve switches to Jacobi and
 * continues from the current iterate (history and V-cycle count continue).
 * Returns 1 if the last solve on ctx did so. */
int amg_last_solve_rerouted(const amg_ctx *ctx);

/* Chebyshev baseline smoother (not in the paper: the fixed-coefficient
 * polynomial the learned smoother is compared with).  Each pre- and
 * post-smoothing phase of the V-cycle applies the degree-`degree`
 * Chebyshev polynomial in D^-1 A once (degree residual evaluations),
 * on the interval [rho/30, 1.1 rho] with rho the largest eigenvalue of
 * D^-1 A estimated by 20 power iterations from v_i = frac(i 2654435761 / 2^32)
 * + 0.5 (FP64, on the host, once per hierarchy), by the three-term recurrence
 *   d = D^-1 r / theta;  d <- rho_k rho_{k-1} d + (2 rho_k / delta) D^-1 r,
 *   rho_0 = delta / theta, rho_k = 1 / (2 theta / delta - rho_{k-1}), u <- u + d,
 * theta = (hi + lo)/2, delta = (hi - lo)/2.  amg_smooth_device applies the
 * polynomial n_sweeps times.  degree: 1..16.  Errors: AMG_ERR_ARG, AMG_ERR_STATE. */
int amg_set_chebyshev(amg_ctx *ctx, int degree);

/* The Chebyshev interval of level `level`: rho (power estimate), theta, delta. */
int amg_get_chebyshev(const amg_ctx *ctx, int level, double *rho, double *theta, double *delta);

/* ------------------------------------------------------------------------
 * Measurement aids (no counterpart in the paper; used for roofline timing)
 * ------------------------------------------------------------------------ */

/* Kernels selectable in amg_kernel_launch. */
#define AMG_K_RESIDUAL  0   /* r = b - A_l u                          (V-cycle precision) */
#define AMG_K_PINV      1   /* u += Q_l^-1 r   (needs coefficients)    (V-cycle precision) */
#define AMG_K_JACOBI    2   /* u' = u + omega D^-1 (b - A_l u)         (V-cycle precision) */
#define AMG_K_RESTRICT  3   /* b_{l+1} = R_l r                         (V-cycle precision) */
#define AMG_K_PROLONG   4   /* u += P_l e_{l+1}                        (V-cycle precision) */
#define AMG_K_OUTER     5   /* FP64 r = b - A_0 x with norm partials   (level 0 only)      */
#define AMG_K_VCYCLE    6   /* one whole V-cycle from level 0          (level ignored)     */
#define AMG_K_MASWEEP   7   /* u' = u + w - (Q^-1 A) u single pass   (latency-optimised levels) */
#define AMG_K_WF_PRE    8   /* wavefront chain: pre-smoothing from zero + residual (HBM-sized levels) */
#define AMG_K_WF_POST   9   /* wavefront chain: prolongation-correction + post-smoothing            */
#define AMG_K_EMPTY    10   /* an empty one-CTA kernel with the solve's dependent-launch attribute
                               (the floor of a chain of launches; level ignored)                 */

/* Launch `reps` back-to-back instances of one solve-path kernel on level
 * `level`, using the context's own work vectors, asynchronously on
 * `stream`; the caller brackets the call with events to time it.  *bytes
 * (may be NULL) receives the algorithmic bytes one launch moves, every
 * array element counted once (values, indices and vectors at their storage
 * width).  Errors: AMG_ERR_ARG (unknown kernel or level), AMG_ERR_STATE. */
int amg_kernel_launch(amg_ctx *ctx, int kernel, int level, int reps, void *stream, double *bytes);

/* Algorithmic bytes of one V-cycle with the current smoother/precision. */
int amg_vcycle_bytes(const amg_ctx *ctx, double *bytes);

/* Number of kernels this library has launched in this process so far. */
long long amg_launch_count(void);

/* Allocation-free residual norm.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- applications that
 * reserve all device memory up front in their own pool, or that run it in a
 * time-critical loop where a driver allocation (which may synchronise the
 * device or fail under memory pressure) is not acceptable.
 *
 * Computes r = b - A x in FP64 for a caller-owned CSR matrix already on the
 * device (n rows, nnz entries; same layout rules as amg_csr), stores r in d_r
 * when d_r is not NULL, and writes d_out[0] = ||b - A x||_2 and
 * d_out[1] = ||b||_2.  Every input and output is caller-owned device memory;
 * the call allocates nothing.  Its only scratch is a fixed array of
 * 2 x 1216 doubles (19,456 bytes) compiled into the library, which every GPU
 * that loads the library holds until the process exits.
 *
 * Limits: 0 <= n <= 67,108,863 rows (the row-group thread index must fit a
 * 32-bit int) and 0 <= nnz <= 2^31 - 1; anything larger is rejected with
 * AMG_ERR_ARG.  The first call on a device looks up the scratch array's
 * device address (once per device, with that device current); make that
 * first call before any stream capture.  The address is cached for the life
 * of the process: do not call this entry point on a device after
 * cudaDeviceReset of that device.  All calls on a device share the
 * scratch array, so calls whose work overlaps on the GPU (e.g. on two
 * concurrent streams) race and give wrong norms; serialise them.  The array
 * keeps the last call's contents, and every call overwrites the slots it
 * reads.  Asynchronous on `stream` (a cudaStream_t) of the current device.
 * Errors: AMG_ERR_ARG, AMG_ERR_CUDA; amg_last_error(NULL) describes them. */
int amg_residual_norm_noalloc(int n, long long nnz, const int *d_row_ptr, const int *d_col,
                              const double *d_val, const double *d_b, const double *d_x, double *d_r,
                              double *d_out, void *stream);

/* Self-test of the tensor-core node linear (no counterpart in the paper):
 * runs the GCIN layer kernel once on 128 nodes of an identity graph, so that
 * y = round_bf16(x) round_bf16(W) + bias with FP32 accumulation (x: 128 x 64,
 * W: 64 x 64 [in][out], bias: 64, y and h: 128 x 64, host, row-major; h
 * receives the BF16-rounded x).  no_commit != 0 issues no MMA, so the
 * kernel's bounded mbarrier wait runs out: *flag becomes 1, the kernel frees
 * its tensor memory and returns, and the context stays usable (about 0.2 s).
 * Allocates and frees its own device buffers; synchronises the device.
 * Errors: AMG_ERR_ARG, AMG_ERR_CUDA. */
int gcin_tc_selftest(int device, int no_commit, const float *x, const float *W, const float *bias, float *y,
                     float *h, int *flag);

/* ------------------------------------------------------------------------
 * Training (Sec. 3.3, Algorithm 1, Table train_hyper)
 * ------------------------------------------------------------------------ */

typedef struct gcin_trainer gcin_trainer;

/* Trainer owning the parameters, their gradient and Adam moments on
 * `device`; precision AMG_GNN_FP32 or AMG_GNN_BF16 selects the arithmetic of
 * the forward node linears (the backward runs in FP32 on the same rounded
 * operands).  theta0: n_params floats (copied); n_params is
 * AMG_GCIN_NUM_PARAMS (width 64) or AMG_GCIN_NUM_PARAMS_H32 (width 32), and
 * gcin_trainer_get_params / gcin_trainer_backward return that many values.
 * Errors: AMG_ERR_ARG (NULL pointer, precision or n_params), AMG_ERR_CUDA. */
int gcin_trainer_create(gcin_trainer **tr, int device, int precision, const float *theta0, long long n_params);
void gcin_trainer_destroy(gcin_trainer *tr);
const char *gcin_trainer_last_error(const gcin_trainer *tr);
int gcin_trainer_get_params(const gcin_trainer *tr, float *theta_out);

/* Replace the trainer's parameters with theta (host, n floats, n = the
 * count it was created with; copied); Adam moments are kept.  The next
 * backward needs a new forward.  Errors: AMG_ERR_ARG, AMG_ERR_CUDA. */
int gcin_trainer_set_params(gcin_trainer *tr, const float *theta, long long n);

/* Batched inference over every level of every problem (Algorithm 1 step 6),
 * keeping the activations for gcin_trainer_backward.  c_out (host) receives
 * sum_m amg_num_levels(problems[m]) rows of 5, problem by problem. */
int gcin_trainer_forward(gcin_trainer *tr, int n_problems, amg_ctx *const *problems, double *c_out);

/* Backward of the last forward: dc (host, same layout as c_out) -> the
 * parameter gradient (kept on the device; dtheta_out, host, may be NULL). */
int gcin_trainer_backward(gcin_trainer *tr, const double *dc, double *dtheta_out);

/* Clip the kept gradient to global norm max_norm, then one Adam step
 * (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr. */
int gcin_trainer_adam_step(gcin_trainer *tr, double lr, double max_norm);

/* Loss of one problem (Sec. 3.3, u_0 = 0) and its gradient:
 *   L = sum_{n=1}^{n_vc} log10(||r_n|| / ||r_{n-1}||) = log10(||f - A u_nvc|| / ||f||),
 * u_n = one V-cycle of the pseudo-inverse smoother with coefficients c
 * (n_levels rows of 5) applied to u_{n-1}, f host (n_0); dL/dc (host,
 * n_levels rows of 5, zero on the coarsest level) from the hand-written
 * adjoint of the n_vc chained V-cycles.  n_vc = 1 is the paper's primary
 * loss, n_vc > 1 its multi-V-cycle loss.  Runs in the context's precision.
 * Errors: AMG_ERR_ARG (n_vc outside 1..64), AMG_ERR_STATE, AMG_ERR_DIVERGED
 * (zero or non-finite residual), AMG_ERR_CUDA. */
int amg_loss_grad(amg_ctx *ctx, const double *c, const double *f, int n_vc, double *loss, double *dc);

#ifdef __cplusplus
}
#endif
#endif /* AMG_GNN_H */
