/*
 * ipm_mf.h -- C ABI of a GB300 (sm_103a) multifrontal LDL^T factorise/solve
 * library for the regularised linear systems of an interior point method
 * (Zanetti & Gondzio, "A factorisation-based regularised interior point
 * method using the augmented system", arXiv 2508.04370).
 *
 * The library factorises, at every IPM iteration and on a fixed pattern,
 * either the regularised augmented system (Sec. 3.2, Eq. regul_matrix)
 *
 *        K = [ -(Theta^-1 + rho I)   A^T     ]          (n + m unknowns)
 *            [        A             delta I  ]
 *
 * or the regularised normal equations (Eq. normeq with Eq. regul_matrix)
 *
 *        M = A (Theta^-1 + rho I)^-1 A^T + delta I       (m unknowns),
 *
 * and solves K [dx; dy] = [r7; r1] (Eq. augsys; for the normal equations dy
 * solves M dy = r1 + A Theta~ r7 and dx = Theta~ (A^T dy - r7), Eq. normeq).
 *
 * Conventions shared by every call:
 *   - A is m x n in compressed sparse columns: colptr[n+1] (int64),
 *     rowidx[nnz] (int32), 0-based, rows sorted inside each column, no
 *     duplicates.  The pattern is copied at ipm_analyse; the caller keeps
 *     ownership of its arrays.
 *   - Pointers documented as "device" are CUDA device pointers owned by the
 *     caller and accessed in stream order on the given stream.  Pointers
 *     documented as "host" are ordinary host memory.
 *   - Streams are passed as `void *` holding a cudaStream_t (NULL = legacy
 *     default stream), so this header needs no CUDA header.
 *   - Return value: 0 = success, negative = error (nothing was changed
 *     unless stated), positive = success with a warning.
 *   - A context is not thread-safe: one host thread at a time.
 *   - Nothing in this library traps or aborts the GPU: device-side problems
 *     (non-finite pivots, expired bounded waits) are recorded in a device
 *     status word and returned by the next call that synchronises
 *     (ipm_get_info, ipm_sync_status, the *_host calls).
 */
#ifndef IPM_MF_H
#define IPM_MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define IPM_OK 0
#define IPM_ERR_INVALID_ARG (-1)
#define IPM_ERR_NOT_ANALYSED (-2)
#define IPM_ERR_OOM (-3)
#define IPM_ERR_CUDA (-4)
#define IPM_ERR_NONFINITE (-5)     /* NaN/Inf in Theta, a pivot or a residual */
#define IPM_ERR_DEVICE_TIMEOUT (-6) /* a bounded device-side wait expired */
#define IPM_ERR_NOT_FACTORISED (-7)
#define IPM_ERR_NO_DEVICE (-8)
#define IPM_ERR_SCRATCH_TOO_SMALL (-9) /* ipm_solve_noalloc: problem exceeds its fixed work space */
#define IPM_WARN_DYNREG_APPLIED 1   /* at least one pivot was lifted (Sec. 4.5) */
#define IPM_WARN_LARGE_REG 2        /* a lift exceeded opt.large_reg (Sec. 4.6 end) */
#define IPM_WARN_REFINE_NOT_CONVERGED 3

/* forms (Sec. 4.2) */
#define IPM_FORM_AUTO 0
#define IPM_FORM_AUGMENTED 1
#define IPM_FORM_NORMAL 2

/* fill-reducing orderings (Sec. 4.2) */
#define IPM_ORD_AMD 0      /* approximate minimum degree (Amestoy, Davis, Duff) */
#define IPM_ORD_ND 1       /* nested dissection, minimum degree on the leaves */
#define IPM_ORD_USER 2     /* caller-supplied permutation */
#define IPM_ORD_NATURAL 3  /* identity (tests) */

/* precision of the Schur-complement updates (Sec. 4.4 dgemm updates) */
#define IPM_PREC_FP64 0    /* everything in FP64 */
#define IPM_PREC_MIXED 1   /* FP32-accurate tensor-core updates (3xTF32, FP32 accumulation) on large
                              fronts; FP64 pivots, regularisation, residual, refinement */
#define IPM_PREC_SLICED 2  /* FP64-accurate tensor-core updates on large fronts: each row of the panel
                              operands is scaled by a power of two and split into eight 7-bit digits,
                              the digit products run as exact bf16 MMAs with FP32 accumulation and are
                              recombined in integers (about 2^-54 of the largest operand entry of a
                              row, where FP64 GEMM gives 2^-53 of each product); FP64 elsewhere.
                              For both tensor-core modes: if refinement cannot reach omega_target
                              from such a factorisation, ipm_solve factorises again in FP64, solves
                              again, and later factorisations stay in FP64 (an IPM's Theta spread only
                              widens); ipm_info counts these fallbacks. */

/* order of the large fronts' 32-column steps (Sec. 4.3 tree-level parallelism) */
#define IPM_SCHED_AUTO 0        /* the dependency order where it takes at most 4/5 of the level order's
                                   steps and levels for the level kernel hold under 1/10 of them; else
                                   the level order */
#define IPM_SCHED_LEVELS 1      /* level by level: the large fronts of a tree level step through their
                                   panels together, the next level starts when the level is done */
#define IPM_SCHED_DEPENDENCY 2  /* each large front starts two steps after its last large child's last
                                   panel (and after the small-front levels of its small children), so
                                   the steps follow the longest chain of panels in the tree instead of
                                   the sum over levels of each level's widest front; no level kernel */

typedef struct ipm_ctx ipm_ctx;

typedef struct ipm_options {
    int32_t nb;               /* pivot-block width (Sec. 4.4 "32, 64 or 128"); default 32 */
    int32_t amalg_width;      /* merge a child into its parent when the width stays <= this; 16 */
    double amalg_zero_frac;   /* ... or when explicit zeros stay <= this fraction; < 0 (the default, -1):
                                 0.1 or 0.2, whichever gives the smaller modelled factorisation time
                                 (front flops at 1 TFLOP/s + 60 us per tree level); the value used is
                                 reported in ipm_info.amalg_zero_frac */
    double eps_piv;           /* dynamic-regularisation floor eps_piv * ||K||_1 (Sec. 4.5: "of the order of
                                 magnitude of machine precision"); 2.220446049250313e-16 */
    double large_reg;         /* a lift larger than this raises IPM_WARN_LARGE_REG; 1e-4 */
    int32_t precision;        /* IPM_PREC_FP64, IPM_PREC_MIXED or IPM_PREC_SLICED; FP64 */
    int32_t mixed_min_front;  /* tensor-core modes: fronts with f >= this use tensor-core updates; 256 */
    double omega_target;      /* refinement stops at this backward error; 1e-12 */
    int32_t refine_max;       /* at most this many refinement steps per solve; 10 */
    int32_t gmres_restarts;   /* when classical refinement of an FP64 factor stalls above omega_target, up to
                                 this many restarts of GMRES(8) on K c = r preconditioned by the factor follow
                                 (an extension of Sec. 4.5; 0 = the paper's classical refinement only; a
                                 stalled tensor-core factor falls back to FP64 instead); 6 */
    int32_t nd_leaf;          /* nested dissection stops at subgraphs of this size; 128 */
    double dense_row_factor;  /* AMD treats degree > max(16, f*sqrt(N)) as dense; 10 */
    int32_t device;           /* CUDA device ordinal; 0 */
    int32_t spin_limit_log2;  /* dependency waits of the persistent solve and of the level kernel give up
                                 after 2^this polls (each >= 64 ns) and report IPM_ERR_DEVICE_TIMEOUT;
                                 -1 = give up at once (tests of the failure path); 24 */
    int32_t verbose;          /* print analysis statistics to stderr; 0 */
    int32_t level_kernel;     /* FP64 large fronts: 1 = one persistent, dependency-driven launch per tree
                                 level (diagonal blocks, triangular solves and trailing updates of all the
                                 level's large fronts); 0 = one launch per kernel and pivot block; 1 */
    int32_t pivoting;         /* 0 = 1x1 pivots with static and dynamic regularisation (Sec. 4.4-4.5, Prop. 3),
                                 for the quasi-definite regularised K; 1 = the Bunch-Kaufman variation of
                                 Sec. 4.5 for matrices that are not quasi-definite (e.g. rho = delta = 0): 1x1
                                 and 2x2 pivots chosen inside each 32-column pivot block of a front (pre-swap of
                                 the largest remaining diagonal, the alpha = (1 + sqrt 17)/8 tests, a pivot below
                                 eps_piv ||K||_1 lifted to that size with its sign), interchanges only among the
                                 front's fully-summed columns, no delayed pivots.  One CTA per front (a
                                 correctness path, not tuned for speed); augmented system and IPM_PREC_FP64
                                 only; fronts up to 12,800 rows; no ipm_graph_capture or ipm_solve_noalloc
                                 (IPM_ERR_INVALID_ARG); the factor's blocks come from ipm_get_pivots; 0 */
    int32_t schedule;         /* IPM_SCHED_AUTO, IPM_SCHED_LEVELS or IPM_SCHED_DEPENDENCY; AUTO.  Both
                                 orders give the same factor bit for bit (every entry receives the
                                 same updates in the same order) */
} ipm_options;

typedef struct ipm_info {
    int32_t m, n, N, form, ordering;
    int32_t nsuper, nlevels, nfronts_small, nfronts_large;
    int32_t max_front, max_k;
    int64_t nnz_A, nnz_K_lower, nnz_L;      /* nnz_L: entries of L in the supernodal structure,
                                               sum of k f - k (k - 1) / 2, unit diagonal included */
    double flops_factor;                    /* sum over fronts of sum_{i=1..k} (f-i)(f-i+3) */
    double flops_tensor;                    /* part of flops_factor in tensor-core updates */
    int64_t device_bytes;                   /* device memory held by the context */
    int32_t npos, nneg, ndynreg;            /* inertia and number of lifted pivots */
    double max_dynreg;                      /* largest |lift| */
    double norm_K1;                         /* ||K||_1 (or ||M||_1) of the last factorisation */
    int32_t refine_steps;                   /* refinement steps of the last solve (GMRES iterations included) */
    int32_t gmres_iters;                    /* GMRES iterations of the last solve (0: classical refinement sufficed) */
    double omega;                           /* backward error of the last solve, on K */
    double omega_hist[16];                  /* omega after 0, 1, ... refinement steps */
    int32_t status;                         /* device status word of the last factorise/solve */
    double ms_analyse;                      /* host wall time of ipm_analyse */
    double est_cost_ne, est_cost_as;        /* AS/NE chooser: modelled seconds per IPM iteration
                                               (Sec. 4.2; -1 when the normal equations were abandoned) */
    int64_t nnz_ne_seen;                    /* entries of A A^T counted before the chooser stopped */
    int32_t precision_fallbacks;            /* mixed path: refactorisations in FP64 so far */
    int32_t mixed_active;                   /* 1 while tensor-core updates are in use */
    int32_t tune_small_threads[3];          /* threads per small-front CTA, size classes f <= 32, 64, 128 */
    double tune_level_ratio;                /* level-kernel threshold (see ipm_autotune) */
    double tune_ms;                         /* best factorisation time the autotuner measured; 0 before */
    double amalg_zero_frac;                 /* amalgamation threshold the analysis used */
    int32_t tune_level_ctas_per_sm;         /* CTAs per SM of the level kernel (0 before the first factorisation) */
    int32_t graph_kernels;                  /* kernel nodes of the graph ipm_graph_capture built (0: none) */
    int32_t schedule;                       /* order of the large fronts' steps in use: IPM_SCHED_LEVELS or
                                               IPM_SCHED_DEPENDENCY */
    int32_t steps_levels;                   /* 32-column steps of the large fronts in the level order */
    int32_t steps_dependency;               /* ... in the dependency order */
    int32_t nfronts_thin;                   /* large fronts of one pivot block (k <= 32, f <= 512, FP64 updates)
                                               that a level outside the level kernel runs whole, one CTA each */
} ipm_info;

/* Fill *opt with the defaults listed above. */
void ipm_default_options(ipm_options *opt);

/* Create a context.  opt may be NULL (defaults).  Allocates no device memory. */
int ipm_create(ipm_ctx **out, const ipm_options *opt);

/* Release the context, its device arena and any captured graph. */
int ipm_destroy(ipm_ctx *ctx);

/* Symbolic analysis, done once per pattern (Sec. 4.2-4.3): choose the form
 * (AUTO runs the augmented-system symbolic first and abandons forming the
 * normal equations once they hold more entries than L of the augmented
 * system, Sec. 4.2; otherwise it compares modelled per-iteration costs:
 * factorisation flops at 1 TFLOP/s FP64, three solves' worth of L traffic at
 * 6.7 TB/s and the formation of A Theta~ A^T; ties and AUTO + USER order are
 * resolved to / rejected in favour of the augmented system), order
 * (AMD / ND / USER / NATURAL), build the elimination
 * tree, postorder, column counts, fundamental supernodes and amalgamation,
 * the front row lists, the extend-add maps, the tree levels and the device
 * plan.  Host only: the device arena is allocated by the first
 * ipm_set_values.
 *   m, n      sizes of A (m >= 0, n >= 0)
 *   colptr    host, n+1 entries
 *   rowidx    host, colptr[n] entries
 *   user_perm host, N entries (N = n+m for the augmented system, m for the
 *             normal equations), perm[new] = old; read only for IPM_ORD_USER
 * The normal equations need, for every entry of A A^T, the list of columns
 * contributing to it; a pattern needing more than 2^28 such pairs (dense
 * rows) is rejected for IPM_FORM_NORMAL and never chosen by AUTO.
 * Errors: IPM_ERR_INVALID_ARG for a malformed pattern or permutation, the
 * AUTO + USER combination, or normal equations beyond the pair limit. */
int ipm_analyse(ipm_ctx *ctx, int32_t m, int32_t n, const int64_t *colptr, const int32_t *rowidx,
                int32_t form, int32_t ordering, const int32_t *user_perm);

/* Batched analysis of `count` independent LPs, factorised together as one
 * block-diagonal system (a forest); per-instance arrays are concatenated:
 *   ms[count], ns[count], colptrs (sum(n_i+1) entries, each instance
 *   starting at 0), rowidxs (sum nnz_i entries).  The combined unknowns are
 *   [x_0; ...; x_{c-1}; y_0; ...; y_{c-1}] (all primal blocks, then all dual
 *   blocks), so the batch behaves exactly like one LP with a block-diagonal
 *   A.  Form is the augmented system. */
int ipm_analyse_batch(ipm_ctx *ctx, int32_t count, const int32_t *ms, const int32_t *ns,
                      const int64_t *colptrs, const int32_t *rowidxs, int32_t ordering);

/* Checkpoint of the symbolic analysis (Sec. 4.2: the symbolic phase runs once
 * per sparsity pattern).  ipm_save_analysis writes everything ipm_analyse (or
 * ipm_analyse_batch) computed to the file at `path` (host string);
 * ipm_load_analysis reads such a file into a context instead of calling
 * ipm_analyse, releasing any device state the context held.  The file is
 * self-contained (the pattern of A included) and checked on reading: a
 * missing, truncated or foreign file gives IPM_ERR_INVALID_ARG and leaves the
 * context unchanged.  Saving before any analysis gives IPM_ERR_NOT_ANALYSED. */
int ipm_save_analysis(const ipm_ctx *ctx, const char *path);
int ipm_load_analysis(ipm_ctx *ctx, const char *path);

/* Values of A (device, colptr[n] doubles in the CSC order given at analyse).
 * They are copied into the context, so the pointer need not stay valid.
 * The first call allocates the device arena (call it before any stream
 * capture).  Errors: IPM_ERR_NOT_ANALYSED, IPM_ERR_OOM, IPM_ERR_CUDA. */
int ipm_set_values(ipm_ctx *ctx, const double *Ax_dev, void *stream);

/* Numeric factorisation of K (or M) for the given Theta (device, n doubles,
 * every entry > 0 and finite) and static regularisation rho, delta >= 0
 * (Sec. 4.5: added to each pivot after it has been computed, with sign -1
 * for the primal block and +1 for the dual block).  Pivots whose magnitude
 * falls below max(eps_piv ||K||_1, Prop. 3 bound) are lifted (dynamic
 * regularisation).  Enqueued on `stream`; returns without synchronising.
 * Non-finite input or pivots set IPM_ERR_NONFINITE in the device status. */
int ipm_factorise(ipm_ctx *ctx, const double *theta_dev, double rho, double delta, void *stream);

/* Solve K [dx; dy] = [r7; r1] with the last factorisation, followed by
 * iterative refinement on the regularised K (Sec. 4.5) until the
 * component-wise backward error is <= omega_target, refine_max steps were
 * taken, or a step fails to halve it; then, for an FP64 factor still above
 * the target, up to gmres_restarts cycles of GMRES(8) preconditioned by the
 * factor, and for a tensor-core factor an FP64 refactorisation and a second
 * solve (the mixed path's fallback).  All pointers device: r7, dx have n
 * entries, r1, dy have m.  Inputs and outputs may not alias.  The decisions
 * are taken on the host: the call synchronises `stream` once per refinement
 * step (ipm_graph_capture gives the device-driven version without host
 * synchronisation). */
int ipm_solve(ipm_ctx *ctx, const double *r7_dev, const double *r1_dev, double *dx_dev, double *dy_dev,
              void *stream);

/* One IPM iteration's linear algebra from host memory: copy Theta (n) and
 * `nrhs` right-hand sides (r7 blocks of n then r1 blocks of m, rhs k at
 * r7_host + k*n and r1_host + k*m) to the device, factorise, solve each rhs
 * with refinement, and copy the solutions back (dx_host, dy_host, same
 * layout).  Synchronises `stream` and returns the device status. */
int ipm_iterate_host(ipm_ctx *ctx, const double *theta_host, double rho, double delta, int32_t nrhs,
                     const double *r7_host, const double *r1_host, double *dx_host, double *dy_host,
                     void *stream);

/* Synchronise `stream` and return (and clear) the device status word. */
int ipm_sync_status(ipm_ctx *ctx, void *stream);

/* Statistics of the analysis and of the last factorise/solve; synchronises
 * the device.  Returns the device status of the last operations. */
int ipm_get_info(ipm_ctx *ctx, ipm_info *out);

/* Symbolic results in the factorisation order (for bit-exact tests); any
 * pointer may be NULL.  Sizes: perm, etree, colcount N; snode_ptr nsuper+1;
 * sn_parent nsuper; sn_rptr nsuper+1; sn_rows sn_rptr[nsuper].
 * perm[new] = old is the fill-reducing order composed with the postorder of
 * its elimination tree. */
int ipm_get_symbolic(const ipm_ctx *ctx, int32_t *perm, int32_t *etree, int64_t *colcount,
                     int32_t *snode_ptr, int32_t *sn_parent, int64_t *sn_rptr, int32_t *sn_rows);

/* Sizes needed by ipm_get_symbolic / ipm_get_factor. */
int ipm_get_sizes(const ipm_ctx *ctx, int32_t *N, int32_t *nsuper, int64_t *nrows_total, int64_t *nnz_L_stored);

/* Copy the factor to host memory (tests): L_host holds, supernode after
 * supernode, the f x k column-major block of each front (rows in sn_rows
 * order, unit diagonal stored as 1, entries above it 0); D_host and
 * dynreg_host have N entries in the factorisation order.  Synchronises. */
int ipm_get_factor(ipm_ctx *ctx, double *L_host, double *D_host, double *dynreg_host);

/* The pivoting mode's factor (opt.pivoting = 1, after a factorisation; host
 * arrays of N entries in the factorisation order, any may be NULL): lperm[p]
 * is the local index, within its supernode's fully-summed columns, of the
 * unknown the front's interchanges moved to position p (the supernode's
 * columns c0 .. c0+k-1 hold c0 + lperm[c0 .. c0+k-1]; ipm_get_factor's L and D
 * are in this interchanged order); Doff[p] = D(p+1, p) of a 2x2 block
 * starting at p, else 0; bsize[p] = 1 or 2 at a block's first position, 0 at
 * a 2x2 block's second.  Synchronises.  Errors: IPM_ERR_INVALID_ARG without
 * the pivoting mode, IPM_ERR_NOT_FACTORISED. */
int ipm_get_pivots(ipm_ctx *ctx, int32_t *lperm_host, double *Doff_host, int32_t *bsize_host);

/* Capture one IPM iteration's linear algebra into one CUDA graph owned by the
 * context (Sec. 4.2: the pattern and the symbolic analysis are reused by
 * every iteration): a copy of Theta (device, n) into the context, the
 * factorisation, then `nsolves` refined solves with right-hand side k at
 * r7_dev + k*n, r1_dev + k*m and solution k at dx_dev + k*n, dy_dev + k*m
 * (all device).  The pointers must stay valid; every replay reads Theta and
 * the right-hand sides afresh, so an IPM loop writes new values there and
 * calls ipm_graph_launch.  Inside the graph the refinement decisions are
 * taken on the device: refine_max steps are captured and the kernels of a
 * step exit at entry once omega <= omega_target, omega failed to halve or
 * the step limit is reached.  When classical refinement ends above the
 * target, GMRES refinement (gmres_restarts cycles of GMRES(8), as in
 * ipm_solve) follows inside the graph as a conditional node that the device
 * enables only then; its kernels return at entry once it is done.  A 3xTF32
 * factorisation that cannot be refined to the target sets
 * IPM_WARN_REFINE_NOT_CONVERGED (no FP64 fallback inside a graph).  Call after ipm_set_values.  The capture runs on a
 * stream private to the context (`stream` is unused and may be NULL); the
 * graph can then be launched on any stream. */
int ipm_graph_capture(ipm_ctx *ctx, const double *theta_dev, double rho, double delta, const double *r7_dev,
                      const double *r1_dev, double *dx_dev, double *dy_dev, int32_t nsolves, void *stream);
int ipm_graph_launch(ipm_ctx *ctx, void *stream);

/* Number of kernel launches enqueued by the last ipm_factorise and the last
 * ipm_solve (for launch accounting). */
int ipm_launch_counts(const ipm_ctx *ctx, int32_t *factorise_launches, int32_t *solve_launches);

/* Allocation-free solve of the augmented system (the paper has no
 * counterpart).  It exists for callers that cannot allocate device memory
 * when they need a solve: a host library or an optimisation callback that
 * runs under a fixed device-memory budget, or that must not change the
 * device's allocation state (an allocation there can fail, or make a caching
 * allocator release and re-reserve memory).  Its work vectors live in one
 * file-scope device array of 2^21 doubles (16 MiB) that every GPU loading
 * this library holds until the process exits; the call makes no cudaMalloc,
 * cudaFree or other allocating call.  Arguments as ipm_solve.
 * It is a simpler variant, not a copy, of ipm_solve:
 *   - it runs the per-level triangular sweeps (one launch per tree level)
 *     instead of the persistent sweeps, so its solution agrees with
 *     ipm_solve's to the refinement accuracy, not bit for bit;
 *   - classical refinement only: no GMRES, and a tensor-core factor whose
 *     refinement stalls is not refactorised in FP64; the call then returns
 *     IPM_WARN_REFINE_NOT_CONVERGED with the best iterate it reached;
 *   - its decisions are taken on the host: it synchronises `stream` after
 *     the first solve and after every refinement step;
 *   - ipm_get_info reports its backward error and step count afterwards.
 * Limits, checked before anything is enqueued (IPM_ERR_SCRATCH_TOO_SMALL):
 * the work needs 7 N + sum over supernodes of (f_s - k_s) doubles (N
 * unknowns, f_s - k_s the contribution rows of supernode s), and the largest
 * front must fit the sweeps' shared memory (at most 25,600 rows).
 * The first call on a device looks up the array's device address with that
 * device current.  All calls share the array: calls that overlap on the GPU
 * (other streams, other threads, other contexts) race and must be
 * serialised by the caller.  Every work vector is written before it is read
 * within a call, so the previous call's contents need no clearing. */
int ipm_solve_noalloc(ipm_ctx *ctx, const double *r7_dev, const double *r1_dev, double *dx_dev, double *dy_dev,
                      void *stream);

/* Autotuner for the launch shapes of the factorisation (the batching and
 * tiling the paper's CPU scheme leaves to the implementation, Sec. 4.3):
 * factorises `reps` + 1 times per candidate on `stream` with the given Theta
 * (device, n doubles), rho and delta, and keeps, by coordinate descent (a
 * candidate must be at least 2% faster than the incumbent, by the median),
 *   - the level-kernel threshold: a tree level runs its large fronts in one
 *     persistent launch when their FP64 work at 1 TFLOP/s is below ratio x
 *     (35 us per 32-column panel of its widest front); candidates 0 (never),
 *     0.25, 0.5 (default), 1, 2, 1e30 (always);
 *   - the threads per small-front CTA of each size class present (f <= 32:
 *     32 or 64; f <= 64: 64 or 128; f <= 128: 128 or 256);
 *   - the level kernel's CTAs per SM: as many as fit (default) or one (see
 *     ipm_set_level_ctas).
 * The choices never change the arithmetic of any entry: the factors are the
 * same bit for bit.  They are reported by ipm_get_info and kept by the
 * context; tune before ipm_graph_capture (a captured graph keeps the launch
 * shapes it was captured with).  Synchronises `stream`.  Leaves the context
 * factorised with the last candidate's (identical) factors.
 * Errors: IPM_ERR_NOT_ANALYSED before ipm_set_values, IPM_ERR_INVALID_ARG for
 * reps outside [1, 20], and those of ipm_factorise. */
int ipm_autotune(ipm_ctx *ctx, const double *theta_dev, double rho, double delta, int32_t reps, void *stream);

/* Set the launch shapes ipm_autotune would choose, e.g. to reproduce a
 * configuration: small_threads (host, 3 entries, may be NULL to keep) gives
 * the threads per small-front CTA of the size classes f <= 32, 64, 128, each
 * 32, 64, 128, 256 or 0 (the default 32 / 64 / 128); level_ratio >= 0 sets
 * the level-kernel threshold (a negative value keeps it).  Results are the
 * same bit for bit whatever the shapes.  Takes effect at the next
 * factorisation (not in an already captured graph).
 * Errors: IPM_ERR_INVALID_ARG for another width or a NaN ratio. */
int ipm_set_launch_shapes(ipm_ctx *ctx, const int32_t *small_threads, double level_ratio);

/* CTAs per SM of the persistent level kernel: 0 (the default) as many as
 * fit, else per_sm (at most as many as fit).  One CTA per SM gives each SM
 * sub-partition's FP64 pipe to one CTA's pivot chain, which shortens the
 * chains of latency-bound levels; more keep more trailing tiles in flight.
 * ipm_autotune tries one against the default.  Items are taken in ticket
 * order whatever the grid, so waits still end and the factors are the same
 * bit for bit.  Takes effect at the next factorisation (not in an already
 * captured graph).
 * Errors: IPM_ERR_INVALID_ARG for a negative per_sm or one above 64. */
int ipm_set_level_ctas(ipm_ctx *ctx, int32_t per_sm);

/* Test hook for the pivot reciprocal (Sec. 4.4-4.5: every column of L is the
 * pivot column scaled by 1/d).  For n doubles x (device) writes the
 * reciprocal the factorisation uses (hardware estimate plus one third-order
 * Newton-Raphson step, division outside [2^-1000, 2^1000] in magnitude) to
 * rcp and CUDA's correctly rounded 1.0 / x to quo (both device, n doubles),
 * on `stream` without synchronising.  Errors: IPM_ERR_INVALID_ARG for n < 0
 * or a null pointer with n > 0. */
int ipm_test_recip_pivot(const double *x_dev, double *rcp_dev, double *quo_dev, int64_t n, void *stream);

/* ------------------------------------------------------------ measurement */
/* FP64 peaks of `device`, the denominators of the FP64 rooflines (the pivot
 * blocks, triangular solves and FP64 updates of Sec. 4.4 run on these
 * units): DFMA chains and mma.sync.m8n8k4.f64 chains over every SM, best of
 * three timed runs after one untimed (CUDA events), 2 flops per FMA.
 * Allocates and frees a small device buffer and synchronises the device's
 * work it starts; takes about a second.  Outputs (host) in TFLOP/s.
 * Errors: IPM_ERR_INVALID_ARG for a null output, IPM_ERR_CUDA. */
int ipm_measure_fp64_peak(int32_t device, double *dfma_tflops, double *dmma_tflops);

/* Kernel classes reported by ipm_kernel_stats. */
#define IPM_K_SMALL_FRONTS 0   /* fused assemble+factorise of fronts f <= 128 (shared memory) */
#define IPM_K_LARGE_ASSEMBLE 1 /* extend-add into large fronts */
#define IPM_K_LARGE_PANEL 2    /* triangular solve of a 32-column panel; the persistent level kernel
                                  (all large-front work of a level) is counted here */
#define IPM_K_LARGE_UPDATE 3   /* trailing (Schur-complement) update, FP64 */
#define IPM_K_LARGE_UPDATE_TC 4 /* trailing update on tensor cores (IPM_PREC_MIXED or IPM_PREC_SLICED) */
#define IPM_K_FORWARD 5        /* forward + diagonal solve (one persistent sweep) */
#define IPM_K_BACKWARD 6       /* backward solve (one persistent sweep) */
#define IPM_K_RESIDUAL 7       /* residual, |K||x|, |K|e and backward error */
#define IPM_K_OTHER 8          /* norms, statistics, permutations, vector updates, diagonal-block
                                  inverses for the solves */
#define IPM_K_SLICE 9          /* reserved (0 launches): the sliced path's digit slices are written by the
                                  panel's triangular solve, counted in IPM_K_LARGE_PANEL */
#define IPM_K_PIVOT_BLOCK 10   /* pivot blocks of a 32-column step, launched per step (the level kernel's
                                  are counted in IPM_K_LARGE_PANEL) */
#define IPM_K_COUNT 11

typedef struct ipm_kernel_stat {
    int64_t launches;  /* launches recorded since the last reset */
    double ms;         /* summed device time between CUDA events around each launch */
    double flops;      /* algorithmic floating-point operations of those launches */
    double bytes;      /* algorithmic HBM bytes of those launches */
} ipm_kernel_stat;

/* Enable (1) or disable (0) per-launch CUDA events for ipm_kernel_stats.
 * Events are recorded on the stream each kernel is launched on. */
int ipm_set_profiling(ipm_ctx *ctx, int32_t enable);

/* Synchronise, fold the recorded events into per-class totals and copy
 * IPM_K_COUNT entries to out (host array); reset != 0 clears the totals. */
int ipm_kernel_stats(ipm_ctx *ctx, ipm_kernel_stat *out, int32_t reset);

/* Launch trace of the profiled launches folded since the last call (the
 * folding happens here and in ipm_kernel_stats): synchronises, then writes
 * up to cap records in issue order (host arrays of cap entries): kernel
 * class, stream index (streams numbered in order of first appearance),
 * start and end in ms measured from the first launch folded in the same
 * batch (the events of one batch are those recorded between two folds).
 * *count receives the number of records (which may exceed cap); the trace
 * is then cleared.  For timelines: which launches overlap, where the
 * critical stream waits. */
int ipm_kernel_trace(ipm_ctx *ctx, int32_t *cls, int32_t *stream, double *start_ms, double *end_ms, int32_t cap,
                     int32_t *count);

#ifdef __cplusplus
}
#endif
#endif /* IPM_MF_H */
