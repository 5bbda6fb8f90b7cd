/*
 * pint.h -- C ABI of the GB300 library for the parareal all-at-once partially
 * explicit splitting scheme (Wang, Yang, Leung, "Parallel in time partially
 * explicit splitting scheme for high contrast linear multiscale diffusion
 * problems", arXiv:2411.09244).
 *
 * Problem (Section 2, eq. (2.1)): u_t - div(kappa grad u) = f on the unit
 * square, u = 0 on the boundary, u(0) = u0; find the multiscale solution
 * u_H^n at the coarse times t_n = n T / N (Algorithm 1).
 *
 * Conventions shared by every call
 *   - Every call returns a pint_status: PINT_OK (0) or a negative code.
 *     No call aborts, prints or exits; pint_last_error() gives a one-line
 *     message for the last failure on the calling thread.
 *   - Arrays are FP64 unless stated, row-major, fine-grid nodal arrays use
 *     node (i, j) -> j*(n_f+1) + i (x fastest), cell arrays (ci, cj) ->
 *     cj*n_f + ci.
 *   - "ptr" arguments may be host or device memory: the library inspects
 *     each pointer and stages host buffers through its own device buffers
 *     with cudaMemcpyAsync on the context's stream.  The caller keeps
 *     ownership of everything it passes; the library owns every buffer it
 *     allocates and frees them in pint_destroy().
 *   - All GPU work runs on the stream given to pint_setup_fine_grid (a
 *     cudaStream_t passed as void*; NULL = legacy default stream).  Calls
 *     that return host-visible results synchronise that stream before
 *     returning.  The solves read convergence norms on the host between
 *     launches, so they cannot themselves be captured into a caller's CUDA
 *     graph; internally the PINT_MIXED solve captures each WR iteration once
 *     (on a private stream of the context) and launches the graph on the
 *     context's stream.
 *   - One context is not thread-safe; distinct contexts are independent and
 *     may be driven from different host threads at once (pint_batch_solve
 *     does so).
 */
#ifndef PINT_H
#define PINT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pint_ctx pint_ctx;
typedef int pint_status;

enum {
  PINT_OK = 0,
  PINT_ERR_BAD_ARG = -1,       /* invalid size, pointer or call order      */
  PINT_ERR_OOM = -2,           /* device allocation failed                 */
  PINT_ERR_CUDA = -3,          /* a CUDA runtime call failed               */
  PINT_ERR_UNSTABLE_DT = -4,   /* Delta t violates the Section 3.2 bound   */
  PINT_ERR_NOT_CONVERGED = -5, /* parareal stopped at k_max above eps      */
  PINT_ERR_NONFINITE = -6,     /* NaN/Inf in a jump or WR update norm      */
  PINT_ERR_SINGULAR = -7,      /* a Cholesky pivot was not positive        */
  PINT_ERR_STATE = -8,         /* stage called before its prerequisites    */
  PINT_ERR_TIMEOUT = -9        /* a bounded device wait ran out            */
};

/* precision of the fine propagator:
 *   PINT_FP64      every step in FP64
 *   PINT_MIXED     WR contractions on the tensor cores (TF32 hi/lo split,
 *                  FP32 accumulation), time solve and recurrence in FP32,
 *                  FP64 coarse states; then one refinement pass: the residual
 *                  of the fine scheme over the trajectory (double-float
 *                  contractions) drives a correction solve whose coarse
 *                  step (the diagonal (M11 + Delta t A11) solve and the
 *                  couplings) runs in FP64.  The parareal jump and
 *                  convergence norm of eq. (2.8) is FP64 throughout.
 *   PINT_MIXED_F32 the same with FP32 CUDA-core contractions (comparison) */
enum { PINT_FP64 = 0, PINT_MIXED = 1, PINT_MIXED_F32 = 2 };

/* flags for pint_assemble_reduced */
enum {
  PINT_ALLOW_UNSTABLE = 1,
  PINT_FINE_SEQUENTIAL = 2,
  PINT_AUTOTUNE = 4,
  PINT_COARSE_FP64 = 8,
  PINT_REFINE_FP64 = 16,
  PINT_CARRY_LAGS = 32,
  PINT_ADJOINT_RESPONSE = 64,
  PINT_COARSE_GRID = 128
};

typedef struct {
  int n_f, nc, J, ell;
  int n_blocks;       /* nc*nc                                             */
  int n_raw;          /* all CEM/NLMC bases (matrix + fracture + enrichment) */
  int L;              /* fracture bases (eq. (3.7))                         */
  int d1, d2;         /* dim V_H1, dim V_H2                                 */
  double gamma;       /* eq. (4.15), largest L2 cosine between the spaces  */
  double lambda_max22;/* sup_{V_H2} ||v||_a^2 / ||v||^2                     */
  double dt_max;      /* (1 - gamma^2) / lambda_max22 (Section 3.2)         */
  double setup_ms;    /* device time of the last setup stage                */
  double T;           /* final time of the assembled time grid (0 before)   */
  double Dt, dt;      /* coarse step T / N and fine step Delta t / P        */
} pint_space_info;

#define PINT_MAX_ITERS 512

typedef struct {
  int K1;                     /* parareal F sweeps done                   */
  int converged;              /* 1 if the jump fell below eps              */
  int wr_total;               /* WR iterations summed over all F sweeps    */
  int wr_iters[PINT_MAX_ITERS];   /* WR iterations of F sweep k          */
  double jumps[PINT_MAX_ITERS];   /* eq. (2.8) jump after sweep k        */
  double solve_ms;            /* device time of the solve (CUDA events)    */
  double f_ms, g_ms, prolong_ms; /* split of solve_ms                       */
  int launches;               /* kernels launched inside the solve         */
  int hot_launches;           /* launches of the WR contraction kernels     */
  double hot_ms;              /* their summed device time (CUDA events)     */
  double hot_flops;           /* their algorithmic flops: 4 d1 d2 per column
                                 of each contraction (two per WR iteration) */
} pint_stats;

/*
 * pint_setup_fine_grid -- Section 2 (fine FEM, eq. (2.2)); the fine mass and
 * stiffness matrices M_f, A_f of Section 3.2.  Q1 elements on n_f x n_f
 * square cells of side 1/n_f, kappa constant per cell.
 *   out          receives a new context (free with pint_destroy)
 *   n_f          fine cells per side, 4 <= n_f <= 4096
 *   kappa_cells  ptr, n_f*n_f cell coefficients, all > 0
 *   stream       cudaStream_t for all work of this context (void*)
 * Errors: BAD_ARG (sizes, non-positive kappa), OOM, CUDA.
 */
pint_status pint_setup_fine_grid(pint_ctx** out, int n_f, const double* kappa_cells,
                                 void* stream);

/*
 * pint_build_multiscale_spaces -- Section 3: per coarse block the NLMC
 * indicator functions of the matrix and of each high-conductivity component
 * (eqs. (3.4)-(3.5)) plus J CEM eigen-enrichment functions from eq. (3.1);
 * the oversampled constraint energy minimising bases of eq. (3.2) on
 * K_i^+ = K_i enlarged by ell coarse layers; psi_bar and the split
 * V_H1 / V_H2 of eq. (3.7).
 *   nc    coarse blocks per side (n_f % nc == 0, n_f/nc <= 32)
 *   J     eigen-enrichment functions per block (0 = NLMC only)
 *   ell   oversampling layers (>= 1)
 *   info  optional, receives the dimensions (gamma/lambda are filled by
 *         pint_assemble_reduced)
 * Errors: BAD_ARG, STATE (no fine grid), SINGULAR (a window system not
 * positive definite), OOM, CUDA.
 */
pint_status pint_build_multiscale_spaces(pint_ctx* ctx, int nc, int J, int ell,
                                         pint_space_info* info);

/*
 * pint_assemble_reduced -- eq. (3.8): M_ij = Psi_i^T M_f Psi_j,
 * A_ij = Psi_i^T A_f Psi_j; gamma of eq. (4.15); the time grid of Section
 * 4.3 (N coarse intervals of Delta t = T/N, each split into P steps of
 * dt = Delta t / P) and the WR parameter alpha of eq. (4.1).  Also the
 * eigenbases Q (A11 Q = M11 Q Lambda1, Q^T M11 Q = I) and Q2 (same for
 * (A22, M22)) in which the fine and coarse steps are solved.
 *   T, N, P, alpha   time grid and WR parameter (0 < alpha < 1, P <= 64);
 *                    T <= 0 asks the library for the final time: 90% of
 *                    the Section 3.2 bound on the coarse step,
 *                    T = 0.9 N (1 - gamma^2) / lambda_max(A22, M22),
 *                    rounded down to two significant digits (info->T)
 *   precision        PINT_FP64 or PINT_MIXED
 *   flags            PINT_ALLOW_UNSTABLE: do not reject a Delta t above
 *                    dt_max (Section 3.2 condition);
 *                    PINT_FINE_SEQUENTIAL (PINT_FP64 only; BAD_ARG with
 *                    the mixed paths): the fine propagator of Algorithm 1
 *                    is the fine scheme stepped P times on all active
 *                    intervals at once instead of the WR all-at-once solve
 *                    (same fixed point; a comparison mode without the
 *                    paper's counterpart);
 *                    PINT_COARSE_FP64: on the mixed paths, the first
 *                    (low-precision) solve's coarse sweeps run in FP64 too
 *                    (by default they run with FP32 couplings on one
 *                    thread-block cluster, or grid-wide where no cluster
 *                    holds the coupling; the correction solve's are always
 *                    FP64);
 *                    PINT_COARSE_GRID: on the mixed paths, the first
 *                    solve's coarse sweeps run grid-wide with FP32
 *                    couplings even where a cluster holds the coupling (the
 *                    form otherwise used only for large couplings);
 *                    PINT_REFINE_FP64: on the mixed paths, the refinement
 *                    residual's two contractions run in FP64 (by default
 *                    in double-float arithmetic, about 48 bits, on the FP32
 *                    pipe);
 *                    PINT_CARRY_LAGS (PINT_FP64 only; a comparison mode
 *                    without the paper's counterpart): the lagged increments
 *                    of eqs. (2.4)-(2.5) are carried across the coarse
 *                    boundaries instead of restarted, so the limit is the
 *                    scheme run uninterrupted over [0, T]; the parareal state
 *                    is (u, w) at t_n and one fine step earlier, F steps the
 *                    fine scheme P times with the carried lags (all active
 *                    intervals at once), G takes one coarse step with the
 *                    fine increment extrapolated to the coarse spacing as its
 *                    lag and returns the linearly interpolated lag; eq. (2.7)
 *                    acts on the whole state, eq. (2.8) on (u, w);
 *                    pint_sequential_solve then gives the uninterrupted scheme;
 *                    PINT_ADJOINT_RESPONSE: pint_adjoint takes the
 *                    amplitude gradient from the interval's unit-source
 *                    response, <lambda_{n+1}, s>, instead of recomputing the
 *                    fine adjoint inside each interval (see pint_adjoint);
 *                    PINT_AUTOTUNE: on the PINT_MIXED path, the tile width,
 *                    K split and row pairing of each tensor-core contraction
 *                    shape are measured (CUDA events, best of the cost
 *                    model's top candidates) the first time the shape is met, and kept
 *                    in the process-wide table of pint_tuning_*; without
 *                    the flag the cost model's choice (or a loaded entry of
 *                    the table) is used
 *   info             optional, receives gamma, lambda_max22, dt_max and
 *                    the time grid T, Dt, dt
 * Errors: BAD_ARG (also a non-finite T, or T <= 0 when no stable T exists),
 * STATE, UNSTABLE_DT (Delta t > dt_max without the flag; info is still
 * filled), SINGULAR, OOM, CUDA.  Every call replaces the time grid; work
 * cached for the previous one (captured WR iterations, the low-precision
 * operator copies) is discarded.  A call that fails with BAD_ARG, SINGULAR,
 * OOM or CUDA after its argument checks leaves no time grid: solves return
 * STATE until an assembly succeeds (UNSTABLE_DT keeps the new grid).
 */
pint_status pint_assemble_reduced(pint_ctx* ctx, double T, int N, int P, double alpha,
                                  int precision, int flags, pint_space_info* info);

/*
 * pint_parareal_solve -- Algorithm 1 (update eq. (2.7), stopping rule eq.
 * (2.8)): initial G sweep, then F sweeps by the all-at-once WR propagator
 * of Section 4.2 on every coarse interval at once, each followed by the
 * sequential coarse correction, until max_n ||u_H^{n,k} - u_H^{n,k-1}||_L2
 * <= eps, k = N or k = k_max; then prolongation to the fine grid.
 *   u0_nodes    ptr, (n_f+1)^2 initial values (boundary values ignored)
 *   f_shape     ptr, (n_f+1)^2 source shape g; the source on interval n is
 *               amp[n] * g
 *   amp         ptr or NULL (all ones), N amplitudes
 *   eps         jump tolerance: >= 0 absolute; < 0 relative, |eps| times
 *               the largest M_H norm of the states of the initial G sweep
 *               (max over n = 1..N)
 *   k_max       maximum F sweeps (1..N)
 *   wr_tol      WR stop: max over intervals and steps of the L2 norm of the
 *               update of u or w; >= 0 absolute, < 0 relative to the same
 *               state scale as eps
 *   wr_max      maximum WR iterations per F sweep (>= 1)
 *   u_out       ptr or NULL, N x (n_f+1)^2: u_H at t_1..t_N on the fine grid
 *   coarse_out  ptr or NULL, (N+1) x (d1+d2): (u_n, w_n) coefficients in the
 *               V_H1 / V_H2 bases at t_0..t_N
 *   stats       optional
 * Errors: BAD_ARG, STATE, NOT_CONVERGED (outputs and stats still written; on
 * PINT_MIXED it means the correction solve stopped at k_max above eps),
 * NONFINITE (a non-finite WR update or jump; the context stays usable),
 * TIMEOUT (a bounded device wait ran out), OOM, CUDA.
 */
pint_status pint_parareal_solve(pint_ctx* ctx, const double* u0_nodes, const double* f_shape,
                                const double* amp, double eps, int k_max, double wr_tol,
                                int wr_max, double* u_out, double* coarse_out,
                                pint_stats* stats);

/*
 * pint_sequential_solve -- the limit of Algorithm 1: the fine splitting
 * scheme eqs. (2.4)-(2.5) stepped sequentially over all N*P fine steps,
 * restarting the lag terms at every coarse boundary.  Same arguments and
 * outputs as pint_parareal_solve (no stats).
 */
pint_status pint_sequential_solve(pint_ctx* ctx, const double* u0_nodes, const double* f_shape,
                                  const double* amp, double* u_out, double* coarse_out);

/*
 * pint_adjoint -- gradient of the observation misfit
 * J = 1/2 sum_{n=1..N} sum_o (u_H^n(x_o) - d_{o,n})^2 with respect to u0
 * and the amplitudes, through the transposed parareal sweeps (the forward
 * map of Algorithm 1 at its limit is affine in (u0, amp); the paper does
 * not treat differentiation).  Runs the forward solve (the context's
 * precision), keeps the coarse states as checkpoints, then parareal
 * backwards in time with the transposed fine scheme on all intervals at once
 * and the transposed coarse step (FP64 on the FP64 path, FP32 transposed
 * sweeps on the low-precision paths).  The amplitude gradient recomputes
 * the fine adjoint inside each interval from the boundary adjoint (the
 * coarse states are the only checkpoints; the map is linear, so no state
 * inside an interval is stored): dJ/da_n = sum_p <mu_p, c>, the transposed
 * fine scheme stepped P times from lambda_{n+1} on all intervals at once, c
 * the step's unit source term (PINT_ADJOINT_RESPONSE: <lambda_{n+1}, s>).
 *   obs_nodes   ptr (int32, host or device), n_obs node ids in [0, (n_f+1)^2)
 *   data        ptr, N x n_obs observations d_{o,n}
 *   u0_nodes, f_shape, amp   as in pint_parareal_solve
 *   eps, k_max, wr_tol, wr_max  controls of the forward solve; the backward
 *               sweep stops when the summed change of the adjoint states is
 *               below 1e-14 (FP64) or 1e-7 (FP32) of their largest norm, or
 *               at k = N, where it is exact
 *   misfit      host double*, receives J (may be NULL)
 *   grad_u0     ptr or NULL, (n_f+1)^2
 *   grad_amp    ptr or NULL, N
 * Errors: as pint_parareal_solve; BAD_ARG for an observation id out of range.
 */
pint_status pint_adjoint(pint_ctx* ctx, const int* obs_nodes, int n_obs, const double* data,
                         const double* u0_nodes, const double* f_shape, const double* amp,
                         double eps, int k_max, double wr_tol, int wr_max, double* misfit,
                         double* grad_u0, double* grad_amp);

/*
 * pint_get_reduced -- copy a reduced quantity (for inspection and tests).
 *   which  0 M11, 1 A11, 2 M22, 3 A22, 4 M12, 5 A12 (row-major d_i x d_j),
 *          6 load F1 and F2 of f_shape (d1 then d2; pass f_shape in aux),
 *          7 the raw-basis Gram matrices G_M (n_raw^2),
 *          8 per raw basis: kind (0 matrix, 1 fracture, 2 enrichment) and
 *            owner block, as doubles (2*n_raw),
 *          9 wall time of the setup stages in ms (6 doubles: block
 *            eigenproblems, oversampled basis solves, Galerkin products,
 *            reduced matrices, spectral bases, time-grid operators)
 *   out    ptr, large enough for the quantity
 *   aux    ptr or NULL, extra input for which = 6
 */
pint_status pint_get_reduced(pint_ctx* ctx, int which, double* out, const double* aux);

/*
 * pint_prolong -- u_h = Psi1 u + Psi2 w on the fine grid (Algorithm 1's
 * output u_H = u + w), for `count` coefficient vectors.
 *   coarse  ptr, count x (d1+d2)
 *   u_out   ptr, count x (n_f+1)^2
 */
pint_status pint_prolong(pint_ctx* ctx, const double* coarse, int count, double* u_out);

/*
 * pint_prolong_noalloc -- the same result as pint_prolong, for callers that
 * cannot call cudaMalloc or any other allocating routine: host runtimes that
 * own the device allocator and forbid allocations outside it, real-time
 * loops that must not touch the allocator, callers with no allocator.  The
 * paper has no counterpart: this is a service entry point of the library.
 * The call allocates and frees nothing: its scratch
 * (count * (d1 + d2 + n_raw) doubles) lives in a file-scope device array of
 * 2^20 doubles (8 MB, held by every GPU that loads the library until exit).
 *   coarse  DEVICE pointer, count x (d1+d2)
 *   u_out   DEVICE pointer, count x (n_f+1)^2
 * The context's device (the one current at pint_setup_fine_grid) must be
 * current.  The work is queued on the context's stream and the call returns
 * without waiting for it: u_out is ready once that stream reaches it.
 * Errors: BAD_ARG (host pointers, another device current, or
 * count * (d1 + d2 + n_raw) > 2^20), STATE, CUDA.  The first call on a
 * device looks the array's device address up (cudaGetSymbolAddress) and
 * caches it.  All calls share the array, which keeps the last call's
 * contents, so calls whose work overlaps on the GPU (other streams, threads
 * or contexts on the same device) race; each call writes every scratch
 * element before reading it.
 */
pint_status pint_prolong_noalloc(pint_ctx* ctx, const double* coarse, int count, double* u_out);

/* pint_apply_G / pint_apply_F -- one application of the coarse propagator
 * (one step of eqs. (2.4)-(2.5) with step Delta t) or of the WR fine
 * propagator (Section 4.2) to `count` states (count <= N), with source
 * amplitudes amp (ptr, count values, or NULL = ones) of f_shape.
 *   in, out  ptr, count x (d1+d2) coefficient vectors
 *   wr_iters host int*, receives the WR iterations (F only, may be NULL) */
pint_status pint_apply_G(pint_ctx* ctx, const double* in, int count, const double* f_shape,
                         const double* amp, double* out);
pint_status pint_apply_F(pint_ctx* ctx, const double* in, int count, const double* f_shape,
                         const double* amp, double wr_tol, int wr_max, double* out,
                         int* wr_iters);

/* pint_get_info -- current dimensions and diagnostics. */
pint_status pint_get_info(pint_ctx* ctx, pint_space_info* info);

/* pint_destroy -- free every device buffer of the context (NULL is a no-op). */
pint_status pint_destroy(pint_ctx* ctx);

/*
 * pint_batch_solve -- many independent instances (uneven grids, spaces and
 * time grids): pint_parareal_solve of every item, each on its own context
 * and that context's stream, from `workers` host threads inside the
 * library.  Items are taken longest first (estimated work: fine unknowns x
 * N x P), so that the uneven instances finish together; the kernels of
 * different instances overlap on the GPU.
 *   items    host array of count items; each names a distinct context
 *            (a context is driven by one thread at a time) and the
 *            arguments of pint_parareal_solve; status receives the item's
 *            own result
 *   count    >= 0
 *   workers  host threads (<= 0: min(count, 16))
 * Returns OK when every item is OK, else the first failing item's status
 * (NOT_CONVERGED only when no item failed otherwise), with "item i: ..." in
 * pint_last_error.  Errors of the call itself: BAD_ARG (NULL items with
 * count > 0, NULL or repeated context).
 */
typedef struct {
  pint_ctx* ctx;
  const double* u0_nodes;
  const double* f_shape;
  const double* amp;
  double eps;
  int k_max;
  double wr_tol;
  int wr_max;
  double* u_out;
  double* coarse_out;
  pint_stats* stats;
  pint_status status;   /* out */
} pint_batch_item;

pint_status pint_batch_solve(pint_batch_item* items, int count, int workers);

/*
 * Autotuner table (process-wide, shared by all contexts and host threads).
 * One row per contraction shape of the WR fine propagator's two tensor-core
 * contractions, as 7 ints: M (rows: d1 or d2), Kp (padded K), ncols (active
 * intervals x P), maxs (largest K split the consumer sums), tn (tile width,
 * 128..256, a multiple of 32), s (K split, 1..maxs, Kp a multiple of 16 s),
 * pair (0 or 1: clusters of two CTAs take adjacent row tiles and share each
 * B tile by multicast; a pair entry is ignored where such clusters cannot be
 * resident); and the measured time of one launch in microseconds (0 when set
 * by hand).
 * These calls touch no device state and need no GPU.
 *   pint_tuning_count  number of rows
 *   pint_tuning_get    copies up to cap rows (host int[cap][7], host
 *                      float[cap] or NULL) in key order; *count receives the
 *                      number copied.  Errors: BAD_ARG (NULL rows/count,
 *                      cap < 0)
 *   pint_tuning_set    merges count rows (host, same layout; us may be NULL);
 *                      nothing is merged if any row is invalid.  Errors:
 *                      BAD_ARG (invalid row, named in pint_last_error)
 *   pint_tuning_clear  empties the table
 * The table is read by PINT_MIXED solves whether or not PINT_AUTOTUNE is set.
 */
int pint_tuning_count(void);
pint_status pint_tuning_get(int* rows, float* us, int cap, int* count);
pint_status pint_tuning_set(const int* rows, const float* us, int count);
pint_status pint_tuning_clear(void);

/*
 * pint_set_wait_limit -- diagnostic control of failure detection: the polls
 * a grid-barrier wait of the FP64 coarse sweep makes before it gives up
 * (process-wide; spins < 0 restores the default of 4194304, about 0.1 s).
 * A wait that gives up records an error flag; the kernel returns, the solve
 * returns PINT_ERR_TIMEOUT and the context stays usable.  0 makes every
 * such wait give up at once, to exercise that path.  Returns the previous
 * limit.  Touches no device state.
 */
int pint_set_wait_limit(int spins);

/*
 * pint_set_sweep_smem -- tuning control of the FP64 coarse sweep (the G step
 * and update of Algorithm 1, eq. (2.7)): the most dynamic shared memory, in
 * bytes, one block of the sweep may use to keep its rows of the coupling
 * operators resident for the whole sweep (process-wide; bytes < 0 restores
 * the default of 204800).  Couplings whose per-block share does not fit are
 * read from global memory at every coarse step instead; both variants form
 * the same products (summed in another order), so results agree to rounding
 * whatever this value.  0
 * selects the streaming variant for every shape.  Returns the previous value.
 * Touches no device state.
 */
int pint_set_sweep_smem(int bytes);

/* pint_last_error -- message of the last failing call on this thread. */
const char* pint_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PINT_H */
