/*
 * slu.h -- C ABI of the irregular-block sparse LU library for B300 (sm_103a).
 *
 * The library factors a square sparse matrix A = L U (L unit lower, U upper,
 * no row exchanges) over the structure-aware irregular 2-D block grid of
 * "A Structure-Aware Irregular Blocking Method for Sparse LU Factorization"
 * (Hu et al.), and solves with the factors.
 *
 *   slu_analyze  host: symmetric pattern, symbolic factorization,
 *                diagonal block pointer (Section 4.2, Algorithm 2),
 *                percentage sampling and irregular blocking (Section 4.3,
 *                Algorithm 3) or regular blocking, and the block task plan
 *                of the right-looking blocked LU (Section 2.2, Algorithm 1).
 *                slu_analyze_device runs the symbolic factorization and
 *                Algorithms 2 and 3 on the GPU, with the same plan.
 *   slu_factor   GPU: value scatter, then per level of the block dependency
 *                structure GETRF / GESSM / TSTRF / SSSSM (Algorithm 1's four
 *                block operations), each block sparse or dense by density.
 *   slu_solve    GPU: block forward / backward substitution, optionally
 *                wrapped in FP64 iterative refinement.
 *
 * Conventions shared by every entry point:
 *   - Matrices are CSC, 0-based: colptr int64[n+1], rowidx int32[nnz].
 *     Row indices inside a column may come in any order; duplicates are an
 *     error (SLU_ERR_INVALID_ARG).
 *   - "host" pointers are read during the call only; the library copies what
 *     it keeps.  "device" pointers are CUDA device memory owned by the caller
 *     and must stay valid until the work enqueued on `stream` has finished.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  All device work of a call is enqueued on it.  Calls return
 *     after enqueueing unless stated otherwise.
 *   - Dense right-hand sides are column-major with a leading dimension.
 *   - No call throws.  On failure a call returns a status other than SLU_OK
 *     and slu_last_error() describes the failure (thread-local string).
 *   - Plans and handles are opaque and freed only by their destroy call.
 *     A handle refers to its plan, which must outlive it.
 *   - Sharing.  The first slu_factor of a plan copies the plan's arrays to
 *     the current device, and every handle of that plan reads them there:
 *     all handles of one plan must live on one device (analyse the pattern
 *     again for another device), and the first slu_factor of a plan must
 *     not run concurrently with another call on the same plan.  A handle
 *     owns scratch buffers and recorded graphs: calls on one handle must
 *     come from one host thread at a time, and their GPU work must not
 *     overlap (one stream per handle, or streams ordered by events).
 *     Different handles are independent.
 */
#ifndef SLU_H
#define SLU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SLU_OK = 0,
    SLU_ERR_INVALID_ARG = 1,     /* bad size, pointer, pattern or option   */
    SLU_ERR_OUT_OF_MEMORY = 2,   /* host or device allocation failed       */
    SLU_ERR_CUDA = 3,            /* a CUDA runtime call or launch failed   */
    SLU_ERR_SINGULAR = 4,        /* zero pivot with perturbation disabled  */
    SLU_ERR_NOT_CONVERGED = 5,   /* refinement missed its tolerance        */
    SLU_ERR_TIMEOUT = 6,         /* a bounded device-side wait expired     */
    SLU_ERR_NOT_SUPPORTED = 7    /* option combination not implemented     */
} slu_status;

typedef enum {
    SLU_BLOCKING_IRREGULAR = 0,  /* Algorithm 3 on the sampled curve        */
    SLU_BLOCKING_REGULAR = 1,    /* fixed-size blocks of regular_block rows */
    SLU_BLOCKING_REGULAR_SELECT = 2
                                 /* fixed-size blocks whose size a selection
                                    tree picks from the order and the filled
                                    nonzeros (slu_select_regular_block)     */
} slu_blocking;

typedef enum {
    SLU_PREC_FP64 = 0,           /* factors stored and computed in FP64     */
    SLU_PREC_FP32 = 1            /* factors in FP32 (diagonal-block pivots
                                    tested in FP64; dense Schur tiles on the
                                    tensor cores as split-precision 3xTF32
                                    with FP32 accumulation), solves refined
                                    in FP64                                 */
} slu_precision;

typedef struct {
    int32_t blocking;            /* slu_blocking                            */
    int32_t regular_block;       /* block size for SLU_BLOCKING_REGULAR     */
    int32_t sample_points;       /* Algorithm 3: samples S (paper: 1000)    */
    int32_t step;                /* Algorithm 3: window width (paper: 2)    */
    int32_t max_num;             /* Algorithm 3: forced boundary after this
                                    many skips (paper: 3)                   */
    int32_t stride;              /* window advance (1 = the listed loop)    */
    int32_t b_min;               /* S = min(sample_points, n / b_min)       */
    int32_t precision;           /* slu_precision                           */
    double dense_threshold;      /* block stored dense if nnz >= thr*bI*bJ  */
    int32_t pivot_perturb;       /* 1: |pivot| < tau -> +-tau and counted   */
    double pivot_tau_rel;        /* tau = pivot_tau_rel * max|A|; 0 = the
                                    default 2^-26 (pivots are FP64 in both
                                    precisions)                             */
    double refine_tol;           /* stop when backward error <= this        */
    int32_t refine_max_iter;     /* < 0 never refine; 0 = default (none for
                                    FP64, 30 for FP32); > 0 that many       */
    int64_t wait_budget_ms;      /* bound of every dependency wait of the
                                    persistent launch (slu_set_persistent),
                                    ms; <= 0 means 2000                     */
    int32_t tc_passes;           /* FP32 dense Schur tiles: 3 = tensor cores,
                                    split precision 3xTF32 (the products
                                    keep FP32 accuracy), 1 = tensor cores,
                                    one TF32 pass with FP32 accumulation
                                    (refinement recovers the accuracy), 0 =
                                    FP32 pipe, executing only the 8 x 4
                                    sub-tiles whose operands hold nonzeros
                                    (for structurally sparse dense-stored
                                    blocks, where a dense tile multiplies
                                    mostly zeros)                           */
} slu_opts;

/* Phases of slu_analyze, the index of slu_plan_info.phase_ms:
 *   INPUT     checks of the pattern, A's CSR view and its sorted columns;
 *   SYMBOLIC  pattern(A + A^T), elimination tree, struct L, filled L+U
 *             pattern (Section 1, the symbolic factorization);
 *   BLOCKING  Algorithm 2's diagonal block pointer, the sampling of Section
 *             4.3 with Algorithm 3, or the regular sizes;
 *   BLOCKS    non-empty blocks, storage layout, local patterns;
 *   TASKS     levels of the block DAG and the per-level task lists;
 *   MAPS      flop counts per kernel class and the A -> storage map. */
enum {
    SLU_PHASE_INPUT = 0,
    SLU_PHASE_SYMBOLIC = 1,
    SLU_PHASE_BLOCKING = 2,
    SLU_PHASE_BLOCKS = 3,
    SLU_PHASE_TASKS = 4,
    SLU_PHASE_MAPS = 5,
    SLU_PHASE_COUNT = 6
};

typedef struct {
    int64_t n;
    int64_t nnz_a;               /* entries of the input pattern            */
    int64_t nnz_sym;             /* entries of pattern(A + A^T) + diagonal  */
    int64_t nnz_lu;              /* entries of the filled L+U pattern       */
    int64_t flops;               /* sum_k (l_k + 2 l_k u_k)                 */
    int32_t nblocks_1d;          /* p: blocks per dimension                 */
    int32_t nlevels;             /* levels of the block dependency DAG      */
    int64_t nblocks;             /* non-empty 2-D blocks                    */
    int64_t ndense;              /* blocks stored dense                     */
    int64_t storage_elems;       /* value slots incl. explicit zeros        */
    int64_t n_getrf, n_gessm, n_tstrf;
    int64_t n_ssssm_targets, n_ssssm_pairs;
    int32_t max_block;           /* largest block dimension                 */
    int32_t samples;             /* S actually used                         */
    double analyze_ms;           /* host time of slu_analyze                */
    int32_t regular_block;       /* regular blocking: the block size used
                                    (the largest over batch members for
                                    SLU_BLOCKING_REGULAR_SELECT); else 0    */
    double phase_ms[SLU_PHASE_COUNT]; /* analyze_ms by phase (SLU_PHASE_*)  */
} slu_plan_info;

typedef struct {
    int64_t nperturb;            /* pivots replaced by +-tau                */
    double tau;                  /* perturbation threshold used             */
} slu_factor_info;

typedef struct {
    int32_t iterations;          /* refinement steps taken                  */
    double backward_error;       /* max over RHS of ||b-Ax||_inf /
                                    (||A||_inf ||x||_inf + ||b||_inf); -1
                                    when not computed                       */
} slu_solve_info;

/* Kernel classes for slu_stats. */
enum {
    SLU_KC_PREP = 0,             /* max|A|, ||A||_inf, value scatter        */
    SLU_KC_GETRF = 1,
    SLU_KC_PANEL = 2,            /* GESSM + TSTRF                           */
    SLU_KC_SSSSM = 3,
    SLU_KC_SOLVE = 4,            /* solve: pull of solved blocks            */
    SLU_KC_RESID = 5,            /* residual, norms, update                 */
    SLU_KC_INV = 6,              /* inverses of dense diagonal factors      */
    SLU_KC_DIAG = 7,             /* solve: diagonal-block step              */
    SLU_KC_PERSIST = 8,          /* the persistent level walk (all classes) */
    SLU_KC_COUNT = 9
};

typedef struct {
    int64_t launches;            /* kernels launched through this handle    */
    int64_t calls[SLU_KC_COUNT]; /* launches per class while profiling      */
    double ms[SLU_KC_COUNT];     /* summed CUDA-event durations per class   */
} slu_stats;

typedef struct slu_plan slu_plan;
typedef struct slu_handle slu_handle;

/* Fill *opts with the defaults: irregular blocking, S = 1000, step 2,
 * max_num 3, stride 1, b_min 32, regular_block 128, FP64, dense threshold
 * 0.6, perturbation on, refine_tol 1e-14, refine_max_iter 0 (the
 * precision's default), wait budget 2000 ms. */
void slu_opts_default(slu_opts *opts);

/* Host-only analysis (Sections 4.2-4.3, Algorithms 2 and 3; Algorithm 1's
 * block task lists).  colptr/rowidx: host, CSC of A's pattern (n x n).
 * The analysis runs on up to 16 host threads (the hardware concurrency, or
 * the environment variable SLU_HOST_THREADS when it is a positive number);
 * the plan is the same for every thread count.
 * opts: host, NULL for defaults.  *out receives a new plan on success;
 * the caller keeps ownership of the arrays, which the plan copies.
 * Errors: SLU_ERR_INVALID_ARG for n outside [0, 2^31 - 2], a NULL array,
 * colptr[0] != 0, a decreasing colptr, a row index outside [0, n), a
 * repeated (row, column) entry or a bad option; SLU_ERR_NOT_SUPPORTED for
 * a blocking the kernels cannot take (a block over 65535 rows, or sparse
 * blocks whose column or row index lists pass 2^31 entries);
 * SLU_ERR_OUT_OF_MEMORY when a host allocation fails.  *out is NULL on any
 * error and slu_last_error() says which check failed. */
slu_status slu_analyze(int64_t n, const int64_t *colptr, const int32_t *rowidx,
                       const slu_opts *opts, slu_plan **out);

/* Batch analysis: `count` independent square matrices (member q: order
 * n[q], CSC colptr[q] / rowidx[q], host) analysed as one block-diagonal
 * system of order sum n[q].  Each member is blocked on its own (its own
 * diagonal block pointer, samples and Algorithm 3), and the level lists of
 * all members are merged, so one launch per level and kernel class walks
 * every member's tasks of that level.  Values, right-hand sides and
 * solutions of the batch plan are the members' concatenated in order
 * (values: member 0's CSC values, then member 1's, ...; rows likewise).
 * Refinement measures the backward error of every member separately and
 * stops when the largest is <= refine_tol.  Every member is checked as
 * slu_analyze checks its pattern, and its colptr before any of its row
 * indices is read; count < 1, a NULL n, colptr or rowidx array, or a total
 * order above 2^31 - 2 is SLU_ERR_INVALID_ARG. */
slu_status slu_analyze_batch(int32_t count, const int64_t *n,
                             const int64_t *const *colptr,
                             const int32_t *const *rowidx,
                             const slu_opts *opts, slu_plan **out);

/* slu_analyze / slu_analyze_batch with the steps that walk the pattern
 * entry by entry on the current GPU, enqueued on `stream`: the symmetric
 * pattern, the elimination tree, struct L and the filled L+U pattern (the
 * symbolic factorization of Section 1), Algorithm 2's per-row counts and
 * prefix sum (Section 4.2), and the sampling of the percentage curve with
 * Algorithm 3 (Section 4.3, one CTA per batch member).  The pattern checks,
 * the block plan and the task lists stay on the host.  The plan equals
 * slu_analyze's (slu_plan_digest is the same); slu_plan_info.phase_ms
 * reports the device phases' time including their copies.  The pattern
 * stays host memory; the call returns when the device work has finished
 * and uses temporary device memory (about 16 bytes per entry of pattern(A
 * + A^T) and per filled entry) allocated stream-ordered from the device's
 * default pool.  Errors: those of slu_analyze, SLU_ERR_OUT_OF_MEMORY when a
 * device allocation fails, SLU_ERR_CUDA when a CUDA call fails. */
slu_status slu_analyze_device(int64_t n, const int64_t *colptr,
                              const int32_t *rowidx, const slu_opts *opts,
                              void *stream, slu_plan **out);
slu_status slu_analyze_batch_device(int32_t count, const int64_t *n,
                                    const int64_t *const *colptr,
                                    const int32_t *const *rowidx,
                                    const slu_opts *opts, void *stream,
                                    slu_plan **out);

slu_status slu_plan_query(const slu_plan *plan, slu_plan_info *info);

/* General-matrix front end (host; the paper's inputs arrive reordered and
 * its solvers pivot statically, Sections 1 and 2.1).  slu_reorder computes
 * for an n x n matrix (CSC, host; rows within a column in any order):
 *   SLU_REORDER_SCALE: a maximum-product transversal -- the row matched to
 *     each column so that the product of the matched |a_ij| is largest, by
 *     shortest augmenting paths on the costs log(max_i |a_ij|) - log |a_ij|
 *     -- and, from its optimal duals, row and column scales under which
 *     every matched entry has magnitude 1 and no entry exceeds 1 (MC64's
 *     option 5 objective and scaling); needs values;
 *   SLU_REORDER_ORDER: a fill-reducing symmetric ordering, nested dissection
 *     of the graph of B + B^T (B: A with the matched entries, or A's own
 *     diagonal without SCALE, on the diagonal) by recursive bisection at the
 *     middle level of a breadth-first level structure from a pseudo-
 *     peripheral node; separators after the parts they split; parts of at
 *     most `leaf` nodes keep their order.
 * Outputs (host, n each): rowperm, colperm with the reordered matrix
 *   R(k, l) = rowscale[rowperm[k]] * A(rowperm[k], colperm[l]) * colscale[colperm[l]],
 * whose diagonal holds the matched entries; rowscale, colscale may be NULL
 * (all ones without SCALE).  A x = b is then R y = b' with
 * b'[k] = rowscale[rowperm[k]] b[rowperm[k]] and x[colperm[l]] =
 * colscale[colperm[l]] y[l] (slu_permute_scale).  Errors: SLU_ERR_SINGULAR
 * when A is structurally singular (no perfect matching, or an empty
 * column), SLU_ERR_INVALID_ARG for a bad pattern or flags, NaN or infinite
 * values. */
#define SLU_REORDER_SCALE 1
#define SLU_REORDER_ORDER 2
slu_status slu_reorder(int64_t n, const int64_t *colptr, const int32_t *rowidx,
                       const double *values, int32_t flags, int32_t leaf,
                       int32_t *rowperm, int32_t *colperm, double *rowscale,
                       double *colscale);

/* R in CSC (rows sorted) from A and slu_reorder's outputs (host): out_colptr
 * int64[n+1], out_rowidx int32[nnz], out_values double[nnz] (may be NULL;
 * values may then be NULL).  rowscale / colscale NULL mean ones.
 * SLU_ERR_INVALID_ARG when rowperm or colperm is not a permutation. */
slu_status slu_reorder_apply(int64_t n, const int64_t *colptr, const int32_t *rowidx,
                             const double *values, const int32_t *rowperm,
                             const int32_t *colperm, const double *rowscale,
                             const double *colscale, int64_t *out_colptr,
                             int32_t *out_rowidx, double *out_values);

/* Device gather / scatter with scaling for the reordered system (all
 * device memory, column-major n x nrhs): inverse = 0:
 *   Y(k, c) = scale[perm[k]] X(perm[k], c)     (b' from b, with rowperm, rowscale)
 * inverse = 1:
 *   Y(perm[k], c) = scale[perm[k]] X(k, c)     (x from y, with colperm, colscale)
 * scale may be NULL (ones); X and Y must not overlap. */
slu_status slu_permute_scale(int64_t n, int32_t nrhs, const int32_t *perm,
                             const double *scale, const double *X, int64_t ldx,
                             double *Y, int64_t ldy, int32_t inverse, void *stream);

/* Regular-size selection policy (SLU_BLOCKING_REGULAR_SELECT).  PanguLU,
 * the regular-blocking solver the paper compares against, picks its block
 * size with a selection tree over the matrix order and the number of
 * nonzeros after symbolic factorization (Section 1; Section 5.2 compares
 * irregular blocking with it and with the best size of a sweep).  The
 * paper does not print the tree.  This one was fitted to B300 timings of
 * the FP64 factor + solve over the regular sizes {32, 64, 128, 256} on the
 * seeded grid, convection-diffusion and circuit families; it splits on n
 * and on the filled density nnz_lu / n (entries per column).  Returns the
 * block size for an n x n matrix with nnz_lu filled entries (1 <= result
 * <= max(n, 1)); pure host function. */
int32_t slu_select_regular_block(int64_t n, int64_t nnz_lu);

/* Copies of the plan's host arrays, for bit-exact checks.  Every output is
 * host memory sized from slu_plan_query:
 *   blockptr int64[n+1]  diagonal block pointer of the filled pattern
 *   ptr      int64[p+1]  block boundaries
 *   colptr   int64[n+1], rowidx int32[nnz_lu]: filled L+U pattern, rows
 *            sorted; this is also the order of slu_export_factors' values
 * Any output pointer may be NULL to skip it. */
slu_status slu_plan_export(const slu_plan *plan, int64_t *blockptr,
                           int64_t *ptr, int64_t *colptr, int32_t *rowidx);

/* Block list (sorted by block column, then block row) and levels:
 *   bi, bj int32[nblocks], bnnz int64[nblocks], dense uint8[nblocks],
 *   level int32[p]. */
slu_status slu_plan_export_blocks(const slu_plan *plan, int32_t *bi,
                                  int32_t *bj, int64_t *bnnz, uint8_t *dense,
                                  int32_t *level);

/* Task lists, per level concatenated; level l owns entries
 * [off[l], off[l+1]) of each list (off arrays int64[nlevels+1]).
 *   getrf  int32[n_getrf]              diagonal block I
 *   gessm  int32[2*n_gessm]            (I, J)
 *   tstrf  int32[2*n_tstrf]            (J, I)
 *   tgt    int32[2*n_ssssm_targets]    (K, J), sorted per level
 *   srcoff int64[n_ssssm_targets+1], src int32[n_ssssm_pairs]: sources I of
 *          each target, ascending. */
slu_status slu_plan_export_tasks(const slu_plan *plan, int64_t *getrf_off,
                                 int32_t *getrf, int64_t *gessm_off,
                                 int32_t *gessm, int64_t *tstrf_off,
                                 int32_t *tstrf, int64_t *tgt_off,
                                 int32_t *tgt, int64_t *srcoff, int32_t *src);

/* GPU numerical factorization.  values: device, float64[nnz_a] in the CSC
 * order of the pattern given to slu_analyze.  Allocates the factor storage
 * (device memory on the current device) and enqueues the factorization on
 * `stream`.  The call synchronizes the stream before returning (it reads
 * the perturbation count), so *info is final.  *out receives a new handle;
 * with SLU_ERR_SINGULAR a handle is still returned (factors not usable).
 * SLU_ERR_TIMEOUT reports that a tensor-core tile's bounded wait for its own
 * MMAs ran out (that tile's update was skipped; factors not usable).
 * SLU_ERR_INVALID_ARG reports a NaN or infinite entry in values (found by
 * the max|a| reduction on the device; slu_refactor reports it when info is
 * requested).
 * The handle owns a second, non-blocking stream: each level's Schur updates
 * whose target lies outside the next level's block rows and columns run
 * there, forked from `stream` after the level's panels and joined back
 * before the next level's updates, so every launch stays ordered after
 * earlier work on `stream` and completes before later work on it. */
slu_status slu_factor(const slu_plan *plan, const double *values,
                      void *stream, slu_handle **out, slu_factor_info *info);

/* Batch factorization of independent matrices (Section 2.2's level walk
 * over many matrices at once; the batching form).  plans: count host
 * pointers to single-matrix plans from slu_analyze, all with equal options
 * (else SLU_ERR_NOT_SUPPORTED); values: count device pointers, values[q]
 * float64[nnz_a of plans[q]] in the CSC order of that plan's pattern.  The
 * call builds the batch plan of the members' patterns (the analysis of
 * slu_analyze_batch, on the host, each member blocked on its own), gathers
 * the values into one device array, and factors every member in the same
 * per-level launches on `stream` (the deferred Schur updates on a second
 * stream, as slu_factor).  out: host array of count handle pointers; out[q]
 * behaves as slu_factor's handle for plans[q] (slu_solve,
 * slu_solve_transpose, slu_export_factors, slu_refactor of that member
 * alone, slu_handle_destroy), its factors equal to slu_factor's for that
 * plan bit for bit.  The members' factors live in one shared device
 * allocation, freed with the last of the count handles; each handle owns
 * its own solve state.  The perturbation threshold tau uses max|a| over
 * all members (as a slu_analyze_batch plan does); info (may be NULL)
 * receives the batch's perturbation count and tau.  Synchronizes the
 * stream.  Returns SLU_OK or SLU_ERR_SINGULAR (handles returned, as
 * slu_factor); on any other status every out[q] is NULL and nothing is
 * kept.  A member plan must not be destroyed while its handle lives. */
slu_status slu_factor_batch(int32_t count, const slu_plan *const *plans,
                            const double *const *values, void *stream,
                            slu_handle **out, slu_factor_info *info);

/* Re-run the factorization into an existing handle with new values of the
 * same pattern; no allocation.  Enqueues only (info may be NULL; if not
 * NULL the call synchronizes and fills it). */
slu_status slu_refactor(slu_handle *h, const double *values, void *stream,
                        slu_factor_info *info);

/* Graph mode: when enabled, slu_refactor records its launch sequence into
 * a CUDA graph on its first call (and again whenever `values` differs from
 * the recorded pointer) and replays the graph afterwards.  The stream given
 * to slu_refactor must then be a created stream, not the legacy NULL
 * stream, and profiling is ignored while recording. */
slu_status slu_set_graph(slu_handle *h, int32_t enable);

/* X = A^{-1} B.  B, X: device, float64, column-major n x nrhs with leading
 * dimensions ldb, ldx >= n, 1 <= nrhs <= 64; X may alias B.  With
 * refinement (FP32 factors by default, or refine_max_iter > 0) the call
 * iterates r = b - A x in FP64 until the backward error is <= refine_tol,
 * synchronizing once per iteration, and returns SLU_ERR_NOT_CONVERGED (X
 * holding the last iterate) if it stops at the iteration limit.  A non-NULL
 * info also makes an unrefined solve compute the backward error (one
 * residual, synchronizing).  Refinement and info use a workspace that the
 * handle allocates on first use.  The level sweeps run as a CUDA graph that
 * the handle records (on a private stream, over a vector buffer it
 * allocates) the first time a right-hand-side count is solved and replays
 * on `stream` afterwards; with profiling enabled they are launched
 * directly. */
slu_status slu_solve(const slu_handle *h, const double *B, int64_t ldb,
                     int32_t nrhs, double *X, int64_t ldx, void *stream,
                     slu_solve_info *info);

/* Lam = A^{-T} G through the stored factors (U^T then L^T); no refinement.
 * Same layout rules as slu_solve. */
slu_status slu_solve_transpose(const slu_handle *h, const double *G,
                               int64_t ldg, int32_t nrhs, double *Lam,
                               int64_t ldl, void *stream);

/* Gradient of a loss l(x), x = A^{-1} B, with respect to the stored values
 * of A, given Lam = A^{-T} (dl/dx) (slu_solve_transpose) and X:
 *   grad[p] = - sum_c Lam(row_p, c) X(col_p, c)
 * over the entries p of A's pattern in the CSC order given to slu_analyze
 * (dA = -Lam X^T restricted to the pattern).  Lam, X: device, column-major
 * n x nrhs; grad: device float64[nnz_a]. */
slu_status slu_grad_values(const slu_handle *h, const double *Lam, int64_t ldl,
                           const double *X, int64_t ldx, int32_t nrhs,
                           double *grad, void *stream);

/* Factor values in the order of the plan's filled pattern (slu_plan_export
 * colptr/rowidx): rows < col hold U, the diagonal holds U's, rows > col hold
 * L.  out: device float64[nnz_lu]. */
slu_status slu_export_factors(const slu_handle *h, double *out, void *stream);

/* Persistent launch (the batching form's "one launch" for the level walk;
 * no counterpart in the paper's A100 design, which launches per task).
 * When enabled, slu_refactor runs every level of every matrix of the plan
 * (many members for a slu_analyze_batch plan) in ONE kernel launch after
 * the value scatter: persistent CTAs (one per SM for FP64, two for FP32)
 * take tasks in the order of a work list built on the host -- per level the
 * GETRF, inverse, panel and Schur-tile tasks of all members, in that phase
 * order, the Schur tiles split into those the next level reads and the
 * deferred rest -- and before each task wait until the member's tasks it
 * depends on are done (device-side counters, acquire/release at GPU scope:
 * the previous phase of the member's chain, and the deferred tiles that may
 * touch the task's blocks).  Tickets are taken
 * in list order, so a CTA only waits for tasks that running CTAs hold.
 * Each wait is bounded by opts.wait_budget_ms; one that runs out stops the
 * launch and the next synchronizing call reports SLU_ERR_TIMEOUT (the
 * factors are then not usable; the context stays usable).  The factors
 * are bit for bit those of the per-level launches.  Graph mode records the
 * persistent launch like any other.  Supported when every block is stored
 * dense and every diagonal block has explicit inverses (dense_threshold 0
 * and blocks of at most 384 rows), else SLU_ERR_NOT_SUPPORTED. */
slu_status slu_set_persistent(slu_handle *h, int32_t enable);

/* The persistent launch's work list, 7 int32 per task in ticket order:
 * kind (0 GETRF, 1 inverse, 2 panel, 3 Schur tile read by the next level,
 * 4 deferred Schur tile), index into that kind's task list of the plan, two
 * (counter, count) waits (counter -1: none), and the counter the task
 * increments when done; counter ((member * nlevels) + level) * 5 + kind
 * counts the finished tasks of that member, level and kind.
 * slu_persistent_tasks copies min(cap, count) tasks
 * into tasks (host) and the count into *count (the list is built by
 * slu_set_persistent).  slu_set_persistent_tasks replaces the list with
 * `count` tasks (at most the built list's length) from host memory after
 * checking that every kind, index and counter is in range
 * (SLU_ERR_INVALID_ARG otherwise); it does not check
 * that the waits can be met -- a wait that cannot is stopped by the bound
 * above. */
slu_status slu_persistent_tasks(const slu_handle *h, int32_t *tasks, int64_t cap,
                                int64_t *count);
slu_status slu_set_persistent_tasks(slu_handle *h, const int32_t *tasks,
                                    int64_t count);

/* Persistent solve: every sweep of slu_solve, slu_solve_transpose and the
 * refinement runs as ONE launch per four right-hand sides instead of two
 * per level.  Persistent CTAs take tasks in the order of a work list built
 * on the host at the first solve -- per level, in the sweep's order, the
 * pulls of already solved blocks into the level's blocks (one per source
 * block and row chunk), then the level's diagonal blocks -- and before each
 * task wait until what it reads is done (device-side counters, acquire and
 * release at GPU scope: a pull waits for the block row whose solution it
 * reads, a diagonal block for every pull into it).  A block therefore
 * starts as soon as its own sources are solved, with no barrier per level.
 * Each wait is bounded by opts.wait_budget_ms; one that runs out stops the
 * launch, and the next solve that synchronizes (refinement, or info
 * requested) reports SLU_ERR_TIMEOUT.  The solutions are bit for bit those
 * of the per-level launches (same operations in the same order).  Supported
 * when every diagonal block has explicit inverses (dense and at most 384
 * rows, e.g. dense_threshold 0), else SLU_ERR_NOT_SUPPORTED; enable = 0
 * returns to the per-level launches. */
slu_status slu_set_persistent_solve(slu_handle *h, int32_t enable);

/* Profiling: while enabled, every kernel launch of the handle is bracketed
 * by a pair of CUDA events on its stream, and slu_handle_stats sums their
 * durations per kernel class (it synchronizes on every recorded event).  Enabling
 * clears the accumulated figures; the launch counter runs always. */
slu_status slu_set_profiling(slu_handle *h, int32_t enable);
slu_status slu_handle_stats(slu_handle *h, slu_stats *out);

/* Per-launch record of the launches profiled since the last
 * slu_set_profiling / slu_handle_stats call, in launch order: kernel class,
 * CUDA-event duration (ms), factorization level (-1 outside the level loop)
 * and grid size in CTAs (negative for the generic sparse GESSM/TSTRF and
 * SSSSM kernels, 0 where not recorded).  Copies min(cap, count) records
 * into whichever of the host arrays cls, ms, level, ctas are non-NULL and
 * the count into *count; synchronizes on every recorded event; does not consume
 * the records. */
slu_status slu_handle_trace(slu_handle *h, int64_t cap, int32_t *cls,
                            float *ms, int32_t *level, int32_t *ctas,
                            int64_t *count);

/* Algorithmic flops of the factorization by kernel class, from the filled
 * pattern: with l_k the entries of L(:,k) inside k's diagonal block and
 * l'_k those below it, GETRF does l_k + 2 l_k^2, GESSM + TSTRF
 * l'_k + 4 l_k l'_k and SSSSM 2 l'_k^2 (they sum to l + 2 l^2 per column).
 * out: host double[3] = {getrf, panel, ssssm}. */
slu_status slu_plan_flops(const slu_plan *plan, double *out);

/* Allocation-free refined solve (no counterpart in the paper).
 *
 * The same computation as slu_solve with refinement (and with the backward
 * error always computed, per member for a slu_analyze_batch handle), for
 * callers that may not allocate device memory when they solve: a process
 * whose device memory is budgeted and handed out entirely at start-up, an
 * application whose framework owns all device memory through its own pool,
 * or a latency-critical loop that cannot afford cudaMalloc's implicit
 * synchronization.  slu_solve allocates its refinement workspace on first
 * use; this call allocates nothing (no cudaMalloc, cudaFree or allocating
 * library routine, and no host buffer either).  Its residual and reduction
 * scratch is a fixed array in the library's device image,
 * SLU_NOALLOC_MAX_ELEMS + 256 doubles (about 8 MiB), which every GPU that
 * loads the library holds until the process exits.
 *
 * Arguments as slu_solve, except that X must not alias B, the current
 * device must be the handle's (else SLU_ERR_INVALID_ARG), and the residual
 * plus the reduction words must fit the array: n * nrhs <=
 * SLU_NOALLOC_MAX_ELEMS and, rounded up to 32, plus 3 * nrhs words per
 * matrix (one, or each member of a batch) plus one, <= SLU_NOALLOC_MAX_ELEMS
 * + 256 (else SLU_ERR_INVALID_ARG with a message naming the limit).  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps
 * the previous call's contents (the call clears what it needs zeroed);
 * calls whose GPU work overlaps race on it and must be ordered by the
 * caller.  Synchronizes the stream once per refinement iteration. */
#define SLU_NOALLOC_MAX_ELEMS (1 << 20)
slu_status slu_solve_refine_noalloc(const slu_handle *h, const double *B,
                                    int64_t ldb, int32_t nrhs, double *X,
                                    int64_t ldx, void *stream,
                                    slu_solve_info *info);

/* Plan cache.  The host analysis of a large pattern can take seconds (the
 * irregular blocking costs more preprocessing than regular blocking, which
 * Section 5.4 accepts for the faster factorization), and its result is
 * plain host data: a plan can be written out and loaded again instead of
 * analysing the pattern anew.  The paper has no counterpart.
 *
 * slu_plan_serialize: with buf == NULL stores the number of bytes the plan
 * needs in *size.  Otherwise buf (host, *size bytes) receives the plan: a
 * 48-byte header (magic, format version, byte-order mark, layout
 * fingerprint, checksum of the payload, payload size, analysis time) and
 * every host array and setting the factorization and the solves use; *size
 * is set to the bytes written.  A buffer smaller than needed is
 * SLU_ERR_INVALID_ARG with *size set to the size needed.
 *
 * slu_plan_deserialize: a new plan from such a buffer (host, read during the
 * call only), equal field for field to the one written (the same digest).
 * A buffer that is not a plan, is truncated, fails its checksum or
 * describes a plan that fails slu_plan_check is SLU_ERR_INVALID_ARG; one
 * written by a build of the library whose plan layout or format version
 * differs, or with another byte order, is SLU_ERR_NOT_SUPPORTED (analyse
 * the pattern again).
 *
 * slu_plan_digest: a 64-bit checksum of the plan's contents (the analysis
 * time excluded), equal for equal plans; the checksum a serialized plan
 * carries. */
slu_status slu_plan_serialize(const slu_plan *plan, void *buf, int64_t *size);
slu_status slu_plan_deserialize(const void *buf, int64_t size, slu_plan **out);
slu_status slu_plan_digest(const slu_plan *plan, uint64_t *digest);

/* Plan invariants (no counterpart in the paper): every index the
 * factorization and the solves take from the plan lies inside the array or
 * block it addresses, every offset array is nondecreasing and ends at its
 * array's length, and every task relates the blocks its kernel expects
 * (GESSM/TSTRF panels of their diagonal block, Schur sources L_KI and U_IJ
 * of their target K,J with I < K,J, tiles inside their target), and that
 * the kernels' task lists carry every task of Algorithm 1 exactly once
 * (chunks and tiles covering each task once, sources in ascending order
 * per target).  Host only, N log N in the plan's size (3 s for a plan of
 * 354 M filled entries); slu_plan_deserialize runs it on every loaded plan.
 * SLU_OK, or SLU_ERR_INVALID_ARG naming the first violated invariant in
 * slu_last_error(). */
slu_status slu_plan_check(const slu_plan *plan);

void slu_plan_destroy(slu_plan *plan);
void slu_handle_destroy(slu_handle *h);
const char *slu_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SLU_H */
