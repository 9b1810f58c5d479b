/*
 * jv.h -- C ABI of libjavelin_gb, a GB300 (sm_103a) implementation of the
 * hot path of Javelin (Booth & Bolet, arXiv 1812.06160): level-scheduled
 * numeric ILU(0) on a CSR matrix's own pattern, the L and U sparse
 * triangular solves ("stri"), CSR spmv, the dependency analysis that feeds
 * them, and two extensions (transposed solves for a differentiable
 * preconditioner apply, and single-precision factors inside double-precision
 * Krylov iterations).
 *
 * General conventions
 *   - Matrices are square CSR, 0-based, int32 indices, n >= 1, nnz < 2^31,
 *     columns strictly ascending inside every row and the diagonal stored
 *     (Sec. III, Fig. 1 visits the columns of a row in ascending order and
 *     divides by a_{col,col}).
 *   - Every array argument is a DEVICE pointer of the current CUDA device
 *     unless its comment says "host".  Dense vectors with several right-hand
 *     sides are row-major n x nrhs (element (i, c) at i * nrhs + c).
 *   - The caller owns every value and vector buffer.  The handle copies the
 *     pattern inside jv_analyze (the caller may free rowptr/colidx after it
 *     returns) and owns all analysis arrays; pointers returned by jv_get_*
 *     stay valid until jv_destroy.
 *   - All work is enqueued on the handle's stream.  With options.check != 0
 *     (the default) every compute call then synchronises that stream and
 *     returns the device status of the work it enqueued; with check == 0 the
 *     call returns after enqueueing and device-side errors (zero pivot, spin
 *     timeout) accumulate in the handle until jv_status_sync.
 *   - A handle may be used by one stream at a time: calls that overlap on the
 *     device share the handle's scratch words and would race.
 *   - Return value: JV_OK (0) or one of the negative JV_ERR_* codes below.
 *     Host-side argument errors are detected before anything is enqueued.
 */
#ifndef JV_H
#define JV_H

#ifdef __cplusplus
extern "C" {
#endif

#define JV_OK 0
#define JV_ERR_ARG (-1)           /* bad argument (null pointer, size, aliasing, dtype) */
#define JV_ERR_PATTERN (-2)       /* column out of range, unsorted or duplicate; bad rowptr */
#define JV_ERR_NO_DIAG (-3)       /* a row without its diagonal entry */
#define JV_ERR_ZERO_PIVOT (-4)    /* u_ii == 0 or not finite (no pivoting, Sec. III) */
#define JV_ERR_TIMEOUT (-5)       /* a sync-free wait exceeded spin_timeout_cycles */
#define JV_ERR_CUDA (-6)          /* a CUDA runtime call failed */
#define JV_ERR_NOMEM (-7)         /* device allocation failed */
#define JV_ERR_INTERNAL (-8)      /* analysis invariant violated */
#define JV_ERR_NOT_CONVERGED (-9) /* Krylov driver hit its iteration limit */

typedef struct jv_handle_s *jv_handle;

typedef enum { JV_F64 = 0, JV_F32 = 1 } jv_dtype;

/* Scheduling of the factor and the solves.
 * LEVEL:    one launch per level (the barrier-per-level "CSR-LS" schedule of
 *           Sec. VI; rows of a level run concurrently).
 * SYNCFREE: one launch; rows are claimed in level order and each waits only
 *           on its own dependencies (the point-to-point synchronisation of
 *           Sec. III-A, Fig. 4, with per-row flags in global memory).
 * HYBRID:   the two-stage split of Sec. III-A (Fig. 2): levels that pass the
 *           stage test (stage_min_rows, stage_max_density, stage_position
 *           below) run one launch per level, and every maximal run of the
 *           other levels -- thin or dense levels between wide ones (Fig. 3)
 *           and the tail -- runs as one sync-free launch. */
typedef enum { JV_MODE_LEVEL = 0, JV_MODE_SYNCFREE = 1, JV_MODE_HYBRID = 2 } jv_mode;

/* The four dependency structures built by jv_analyze.
 * LOWER:   lower(A), forward solve and factor (Sec. III: levels of lower(A)).
 * UPPER:   upper(A), backward solve (levels counted from row n-1).
 * UPPER_T: U^T, forward solve over the columns of U (adjoint).
 * LOWER_T: L^T, backward solve over the columns of L (adjoint). */
typedef enum { JV_LOWER = 0, JV_UPPER = 1, JV_UPPER_T = 2, JV_LOWER_T = 3 } jv_structure;

typedef struct {
    int mode;                       /* jv_mode; default JV_MODE_SYNCFREE */
    int reorder;                    /* 1: work on B = P A P^T with P the level order of
                                       lower(A) (Sec. III: nonzeros permuted into the level
                                       ordering); every vector and value array passed to
                                       the handle is then in B's order.  Default 0. */
    int check;                      /* 1 (default): synchronise and return device status */
    int long_row;                   /* solve rows with more dependencies than this run one
                                       row per warp (lanes cooperate); shorter rows run one
                                       row per lane, 32 to a warp.  0 = default (24) */
    long long spin_timeout_cycles;  /* bound on every sync-free wait; 0 = default (2^32) */
    int fault_row;                  /* TEST ONLY: this row never publishes its result, so
                                       its dependants time out.  -1 (default) = off. */
    int sf_ctas_per_sm;             /* sync-free launches run a persistent grid of this many
                                       CTAs per SM (bounds how many rows poll at once);
                                       0 = default (1; 2 for solves with several
                                       right-hand sides, whose tasks are single rows) */
    int sf_backoff_ns;              /* longest pause between two polls of a value that is not
                                       ready; 0 = default, negative = never pause */
    int band_rows;                  /* sync-free band schedule: rows per band (> 0), one CTA
                                       per band, local levels inside it.  0 or -1 = the
                                       level-ordered schedule (the default: on GB300 it is
                                       the faster one for every workload measured) */
    int sf_gate_levels;             /* sync-free factor's level gate: a task polls its operands
                                       only once the tasks of all levels below (its level -
                                       this) have finished, sleeping until then; 0 = poll from
                                       the start; -1 (default) = automatic: enough levels to
                                       hold about 64 tasks, at least 1 (narrow levels want a
                                       wider gate).  (The solves do not gate: on GB300 it
                                       slowed them.) */
    int milu;                       /* 1: the handle's factor is modified ILU(0) -- an update
                                       a_ij -= l_ik u_kj whose column j is outside row i's
                                       pattern is applied to a_ii instead of being dropped
                                       (row sums of L U equal A's); 0 (default): ILU(0).
                                       Not offered with band_rows > 0 (JV_ERR_ARG). */
    int sym_levels;                 /* 1: schedule on the levels of lower(A + A^T) and
                                       upper(A + A^T) (Sec. III's option) instead of lower(A)
                                       and upper(A): the factor, the L and U^T solves share
                                       the first, the U and L^T solves the second.  Results
                                       are unchanged; with reorder = 1 the level-order
                                       permutation then keeps A's lower/upper split for any
                                       pattern.  0 (default).  Not offered with
                                       band_rows > 0 (JV_ERR_ARG). */
    /* Stage test of the two-stage schedules (Sec. III-A: minimal rows per
       level, row density, relative position).  A level belongs to the upper
       stage when it has at least stage_min_rows rows, its mean row length is
       at most stage_max_density times the matrix's mean, and it starts before
       row stage_position * n of the level order; every other level is
       second-stage material.  Used by JV_MODE_HYBRID and er_corner. */
    int stage_min_rows;             /* 0 = default (1024) */
    double stage_max_density;       /* 0 = no density limit (default) */
    double stage_position;          /* 0 = no position limit (default); in (0, 1] */
    int er_corner;                  /* 1: Even-Rows second stage for the factor (Sec. III-B,
                                       Fig. 8).  The corner is the tail of levels of lower(A)
                                       that starts where every later level is second-stage
                                       material, shortened from its top until it fits one
                                       CTA's shared memory.  The upper stage (mode LEVEL,
                                       SYNCFREE or HYBRID) factors the rows above it; then
                                       one CTA runs FACTOR_L -- every corner row's updates
                                       from the rows above the corner, all rows at once --
                                       and factors the corner level by level in shared
                                       memory.  Each row still takes its updates in
                                       ascending column order, so the factor is ILU(0)'s
                                       exactly.  The corner's rows must be the last rows of
                                       the handle's order (reorder = 1 guarantees it; else
                                       JV_ERR_ARG); a tail too large for shared memory leaves
                                       the corner empty (jv_info.corner_rows = 0).  The
                                       one-column solves get corners of their own the same
                                       way: the tail levels of each structure, when they are
                                       the last rows (L, U^T) or the first rows (U, L^T),
                                       solved by one CTA in shared memory after the upper
                                       stage, with every row's sum in the serial order
                                       (jv_info.solve_corner_rows).  Not offered with
                                       band_rows > 0 (JV_ERR_ARG).  0 = off (default). */
    int no_graphs;                  /* 1: issue the launch sequences of LEVEL and HYBRID (one
                                       launch per upper-stage level) one by one.  0 (default):
                                       the first call of a sequence captures it into a CUDA
                                       graph, later calls with the same operation, dtypes,
                                       buffers and mode replay it (up to 16 graphs per
                                       handle; inside a stream capture of the caller's own
                                       the launches go into that capture). */
    int exact;                      /* 1: every FP64 result equals the serial algorithm's
                                       bit for bit: the factor divides by each pivot as
                                       Fig. 1 does, and every sum runs in the serial order.
                                       0 (default), these departures, each deterministic
                                       run to run and within a few units in the last
                                       place per operation (sums: relative to the sum of
                                       the terms' magnitudes):
                                       - the FP64 factor's row k computes 1/u_kk once, by
                                         Newton's iteration, when u_kk is final, and every
                                         multiplier is l_ik = a_ik * (1/u_kk) (the
                                         division sequence it replaces is the longest run
                                         of FP64 work on the critical path);
                                       - an FP64 factor entry of a one-warp row that
                                         receives more than 32 updates (a hub row's
                                         diagonal) sums them over the warp's lanes, each
                                         lane's share in ascending step order, then a
                                         fixed tree, and adds the total to a_ij;
                                       - a solve row with more dependencies than long_row
                                         splits its sum over the warp's lanes the same
                                         way, so its chain is about 1/32 as long;
                                       - spmv rows longer than spmv_long_row likewise.
                                       Either way the U / U^T solves form s / u_ii from
                                       1/u_ii, computed before a row's operands arrive,
                                       and one correction step (Markstein's), which gives
                                       the division's own result, the one-lane solve rows
                                       and the factor's other arithmetic keep the serial
                                       order, and FP32 divides (its pipe is full width). */
    int spmv_long_row;              /* with exact = 0, spmv rows longer than this split their
                                       sum over the 32 lanes of a warp (each lane's share in
                                       ascending column order, then a fixed tree; the
                                       result is deterministic run to run); shorter rows,
                                       and every row with exact = 1, sum in the serial
                                       order, one row per lane.  0 = default (128). */
} jv_options;

typedef struct {
    int n, nnz;
    int nnz_lower, nnz_upper;   /* strictly lower / strictly upper entries */
    int nlev[4];                /* levels per jv_structure */
    int nlong[4];               /* rows run one per warp, per jv_structure */
    int nlong_factor;           /* rows the factor runs one per warp */
    int band_rows[4];           /* band size per jv_structure, 0 when the band schedule
                                   is not used for it */
    int nband_levels[4];        /* local levels over all bands */
    long long npairs;           /* update pairs of the symbolic factorisation (flops of the
                                   factor = 2 npairs + nnz_lower) */
    int mode, reorder;
    int hybrid_launches[4];     /* launches of a JV_MODE_HYBRID solve per jv_structure
                                   (one per upper-stage level + one per sync-free run) */
    int hybrid_launches_factor; /* the same for an FP64 factor (levels above its corner) */
    int corner_rows[2];         /* rows of the Even-Rows corner per factor jv_dtype (the
                                   FP32 corner holds about twice the rows); 0: none */
    int corner_levels[2];       /* levels of lower(A) each corner spans */
    int solve_corner_rows[4][2];/* rows of the one-column solve corner per jv_structure;
                                   [1]: factor and x both FP32, [0]: otherwise */
    int spmv_wide_rows;         /* rows the spmv sums over a warp (spmv_long_row) */
} jv_info;

/* Fill *opt with the defaults above. */
void jv_default_options(jv_options *opt);

/* The stage test of the two-stage schedules (Sec. III-A), on the host: what
 * jv_analyze applies to each level structure, exported so that a caller can
 * preview the split.  Nothing here touches a GPU.
 * nlev: levels.  level_ptr[nlev+1] (host): the first position of every level
 * in level order (level_ptr[0] = 0, strictly increasing, level_ptr[nlev] =
 * n).  dep_sum[nlev] (host): the sum of the dependency counts of each
 * level's rows, or NULL (then opt->stage_max_density must be 0).  opt: the
 * stage_min_rows / stage_max_density / stage_position options, NULL for the
 * defaults.  Writes upper[nlev] (host): 1 for an upper-stage level, 0 for
 * second-stage material, and *tail (may be NULL): the first level of the run
 * of second-stage levels that ends the structure (nlev if there is none).
 * The hybrid schedule launches each upper-stage level on its own and each
 * maximal run of other levels as one sync-free launch; the Even-Rows corner
 * lies within [tail, nlev).  Returns JV_OK or JV_ERR_ARG. */
int jv_stage_plan(int nlev, const int *level_ptr, const long long *dep_sum, int n,
                  const jv_options *opt, unsigned char *upper, int *tail);

/* Dependency analysis (Sec. II level scheduling; Sec. III-A upper stage).
 * n, nnz: matrix order and stored entries.  rowptr[n+1], colidx[nnz]: device
 * CSR pattern (values are not needed).  opt: host pointer or NULL for the
 * defaults.  stream: a cudaStream_t (NULL = legacy default stream) that
 * becomes the handle's stream.  *out (host) receives the new handle.
 * Validates the pattern (JV_ERR_PATTERN / JV_ERR_NO_DIAG with the offending
 * row readable through jv_status_sync's bad_row), finds diag_ptr, builds the
 * CSC of the pattern, the level of every row for all four jv_structure DAGs
 * (longest dependency path, computed by peeling dependency-free rows on the
 * GPU), the level sets (rows grouped by level, ascending row index inside a
 * level, by a stable GPU radix sort), and the per-level work lists.  With
 * opt->reorder it also builds B = P A P^T and analyses B.  Synchronous. */
int jv_analyze(int n, int nnz, const int *rowptr, const int *colidx,
               const jv_options *opt, void *stream, jv_handle *out);

/* Row of the last jv_analyze failure on this host thread (pattern or
 * missing-diagonal errors), -1 if none or not row-specific. */
int jv_last_bad_row(void);

/* Release every device array the handle owns.  NULL is ignored. */
void jv_destroy(jv_handle h);

/* Change the handle's stream (cudaStream_t) / scheduling mode (any jv_mode:
 * the stage test and the corner are planned by jv_analyze whatever the mode)
 * / check flag. */
int jv_set_stream(jv_handle h, void *stream);
int jv_set_mode(jv_handle h, int mode);
int jv_set_check(jv_handle h, int check);

/* Numeric ILU(0) -- Sec. III, Fig. 1 (up-looking, row by row; no pivoting).
 * vals[nnz] (dtype vals_t) are A's values in the handle's order; lu[nnz]
 * (dtype lu_t) receives L (strictly lower part, unit diagonal implied) and U
 * (diagonal and strictly upper part) in the same pattern.  lu == vals is
 * allowed when the dtypes match (in place); vals_t = F64 with lu_t = F32
 * fuses the down-cast.  Arithmetic is done in lu_t, in the order of Fig. 1:
 * every update a_ij -= l_ik u_kj is one fused multiply-add; the multiplier
 * l_ik is the division a_ik / u_kk (FP32, or FP64 with options.exact = 1) or,
 * by default in FP64, a_ik times the pivot's reciprocal (see
 * jv_options.exact).  The pivot test (u_ii == 0 or not finite ->
 * JV_ERR_ZERO_PIVOT) is done in double.  Device scratch (the pivot array,
 * the work area of rows too long for shared memory) is allocated on the
 * first call that needs it and kept by the handle.
 * bad_row (host, may be NULL): the smallest failing row, or -1. */
int jv_ilu0_factor(jv_handle h, jv_dtype vals_t, const void *vals,
                   jv_dtype lu_t, void *lu, int *bad_row);

/* Forward substitution with the unit lower factor (Sec. VI, stri):
 * x = L^-1 b.  lu: factor from jv_ilu0_factor (dtype lu_t, which is also the
 * arithmetic type).  b (dtype b_t) and x (dtype x_t) are n x nrhs row-major,
 * nrhs >= 1; x must not overlap b.  Every row sums its terms in the serial
 * order (ascending columns), one fused multiply-add each -- except, by
 * default, a one-column row with more dependencies than options.long_row,
 * which sums by lanes and a fixed tree (jv_options.exact).  A one-column
 * solve keeps a handle-owned copy of x (allocated on first use) that its
 * rows poll. */
int jv_lsolve(jv_handle h, jv_dtype lu_t, const void *lu, jv_dtype b_t,
              const void *b, jv_dtype x_t, void *x, int nrhs);

/* Backward substitution with U (Sec. VI): x = U^-1 b.  Same arguments. */
int jv_usolve(jv_handle h, jv_dtype lu_t, const void *lu, jv_dtype b_t,
              const void *b, jv_dtype x_t, void *x, int nrhs);

/* Transposed solves for the adjoint of z = U^-1 L^-1 r (not in the paper):
 * x = L^-T b (backward over the columns of L) and x = U^-T b (forward over
 * the columns of U), through the CSC built by jv_analyze.  Same arguments. */
int jv_lsolve_t(jv_handle h, jv_dtype lu_t, const void *lu, jv_dtype b_t,
                const void *b, jv_dtype x_t, void *x, int nrhs);
int jv_usolve_t(jv_handle h, jv_dtype lu_t, const void *lu, jv_dtype b_t,
                const void *b, jv_dtype x_t, void *x, int nrhs);

/* spmv (Sec. I; Sec. VI leaves it to future work): y = alpha A x + beta y.
 * vals[nnz], x[n], y[n] all of dtype t; beta == 0 never reads y.
 * x must not overlap y.  Each row's products are added with one fused
 * multiply-add each in ascending column order (the serial spmv's result),
 * except, by default, rows longer than options.spmv_long_row, summed by the
 * lanes of a warp and a fixed tree (jv_options.exact).  16-byte aligned
 * vals take wider loads on matrices with rows over 32 entries (same
 * result). */
int jv_spmv(jv_handle h, jv_dtype t, const void *vals, const void *x, void *y,
            double alpha, double beta);

/* Pattern-restricted outer product for the factor gradient (not in the
 * paper): for every entry p = (i, j) of the chosen part,
 *   g[p] = alpha * sum_c a[i, c] * b[j, c]       (c < nrhs),
 * which = 0: strictly lower part (gradient of L), which = 1: diagonal and
 * strictly upper part (gradient of U).  Other entries of g are untouched.
 * a, b: n x nrhs row-major; g[nnz]; all of dtype t. */
int jv_masked_outer(jv_handle h, jv_dtype t, int which, const void *a,
                    const void *b, int nrhs, double alpha, void *g);

/* With opt.reorder: out[t] = in[vmap[t]] maps A-ordered values to B order
 * (Sec. III: values copied into the level-ordered CSR). */
int jv_permute_values(jv_handle h, jv_dtype t, const void *in, void *out);

/* With opt.reorder: inverse == 0: out[r, :] = in[perm[r], :] (A order -> B
 * order); inverse == 1: out[perm[r], :] = in[r, :].  in/out n x nrhs. */
int jv_permute_vector(jv_handle h, jv_dtype t, int inverse, const void *in,
                      void *out, int nrhs);

/* Read-only views of the analysis (device pointers owned by the handle).
 * Any output pointer may be NULL. */
int jv_get_info(jv_handle h, jv_info *info);
int jv_get_levels(jv_handle h, int which, int *nlev, const int **level_ptr,
                  const int **level_rows, const int **lev);
int jv_get_pattern(jv_handle h, const int **rowptr, const int **colidx,
                   const int **diag_ptr);
int jv_get_csc(jv_handle h, const int **colptr, const int **rowidx,
               const int **csc2csr, const int **cdiag);
int jv_get_perm(jv_handle h, const int **perm, const int **iperm,
                const int **vmap);

/* Synchronise the handle's stream, return the accumulated device status and
 * clear it.  bad_row (host, may be NULL) receives the row of the error. */
int jv_status_sync(jv_handle h, int *bad_row);

/* Krylov drivers (Sec. I: CG / GMRES preconditioned by the ILU factors).
 * All vectors are FP64; the preconditioner M = LU is applied with the factor
 * lu of dtype lu_t (FP32 factors run FP32 solves, reading the FP64 residual
 * and writing an FP64 preconditioned vector).  x holds x0 on entry. */
typedef struct {
    double tol;        /* stop when ||b - A x|| / ||b|| <= tol (default 1e-8) */
    int maxit;         /* PCG iteration limit (default 10000) */
    int restart;       /* FGMRES restart length m (default 30) */
    int max_restarts;  /* FGMRES cycle limit (default 200) */
} jv_krylov_opts;

typedef struct {
    int iters;           /* iterations (PCG) or inner Arnoldi steps (FGMRES) */
    int converged;       /* 1 when the tolerance was met */
    double relres;       /* recursive relative residual at exit */
    double true_relres;  /* ||b - A x|| / ||b|| recomputed at exit */
} jv_krylov_info;

void jv_default_krylov_opts(jv_krylov_opts *o);

/* Flexible (Polak-Ribiere) ILU(0)-preconditioned CG.  vals: A in FP64.
 * Returns JV_OK, JV_ERR_NOT_CONVERGED, or an error.  info: host. */
int jv_pcg(jv_handle h, const double *vals, jv_dtype lu_t, const void *lu,
           const double *b, double *x, const jv_krylov_opts *o,
           jv_krylov_info *info);

/* Right-preconditioned flexible GMRES(m), modified Gram-Schmidt Arnoldi. */
int jv_fgmres(jv_handle h, const double *vals, jv_dtype lu_t, const void *lu,
              const double *b, double *x, const jv_krylov_opts *o,
              jv_krylov_info *info);

/* Forward substitution x = L^-1 b that allocates no device memory (the paper
 * has no counterpart: this is a convenience for callers that cannot call
 * cudaMalloc -- code running under an allocator or memory budget it does not
 * own, code that must avoid the synchronisation cudaMalloc/cudaFree imply, or
 * code with no place to keep a jv_handle).  Same arithmetic and result as
 * jv_lsolve with FP64 factor and vectors and one right-hand side.
 *   n <= 2097152 (2^21) rows, else JV_ERR_ARG (the scratch is fixed-size).
 *   rowptr[n+1], colidx[], diag[n]: a valid CSR pattern of the factor and the
 *   position of every diagonal entry (e.g. from jv_get_pattern; they are
 *   trusted); lu[]: the factor from jv_ilu0_factor; order[n]: the rows in an
 *   order in which every row comes after all rows it depends on (the level
 *   sets of jv_get_levels for JV_LOWER, or simply 0..n-1); b[n] in, x[n] out
 *   (x must not alias b).  stream: cudaStream_t (NULL = legacy default
 *   stream).
 * Synchronous: waits for its own work on the stream and returns JV_OK,
 * JV_ERR_ARG (also when an entry of order lies outside [0, n) or a strictly
 * lower entry of a row names a column outside [0, row): such a row writes
 * nothing) or JV_ERR_TIMEOUT (a wait gave up: order is not
 * dependency-respecting -- a bad order may time out, or may still finish if
 * the rows it waits on happen to be processed first).  After a failed call x
 * is unspecified.
 * Its scratch (8 MB of per-row flags plus a few words) is one file-scope
 * device array that every GPU loading the library holds until the process
 * exits; each call looks its device address up with the caller's device
 * current.  All calls share the array and each call clears it before use, so
 * calls that overlap on the GPU race. */
int jv_lsolve_noalloc(int n, const int *rowptr, const int *colidx, const int *diag,
                      const int *order, const double *lu, const double *b, double *x,
                      void *stream);

/* ILU(k) symbolic factorisation (the level-of-fill pattern that ILU(k)
 * factors on: Javelin runs its up-looking numeric sweep on A's pattern
 * widened by the requested fill, Sec. II / Sec. V).  Entry (i, j) is kept when its level
 * of fill is <= level, where every entry of A has level 0 and, row by row,
 * lev(i,j) = min over the columns k < i of row i (ascending, fill included)
 * of lev(i,k) + lev(k,j) + 1, for j in row k's filled pattern.  ILU(k) is
 * then: this pattern, A's values placed on it (jv_scatter_values), and
 * jv_analyze + jv_ilu0_factor on the filled pattern.
 * n, nnz, rowptr[n+1], colidx[nnz]: A's device CSR pattern (valid: sorted
 * columns, diagonal present -- not re-checked here).  level >= 0.
 * Call it twice: with fill_colidx == NULL it writes fill_rowptr[n+1]
 * (device) and *fill_nnz (host); then, with fill_colidx (device, *fill_nnz
 * ints) and optionally fill_level (device, *fill_nnz ints, or NULL), it
 * writes the columns (ascending in every row) and their levels.  Each call
 * recomputes the pattern on the GPU: every row on its own through the
 * fill-path characterisation (the level of (i,j) is one less than the length
 * of the shortest path i -> j in A's graph through vertices numbered below
 * min(i,j)); a row whose search outgrows shared memory is redone by the
 * row-by-row sweep above, rows claimed in order and each waiting
 * point-to-point on the rows it reads.  Synchronous; allocates and frees
 * its own device scratch.  JV_ERR_NOMEM if a filled row exceeds 1024 entries
 * (*bad_row, host, receives it) or the pattern exceeds 2^31 - 1 entries;
 * JV_ERR_TIMEOUT if a wait expired. */
int jv_iluk_symbolic(int n, int nnz, const int *rowptr, const int *colidx, int level,
                     int *fill_rowptr, int *fill_colidx, int *fill_level, long long *fill_nnz,
                     int *bad_row, void *stream);

/* A's values on a pattern that contains A's (e.g. the ILU(k) pattern):
 * fill_vals[q] = a_ij for the entry q = (i, j) of A, 0 elsewhere.  t: the
 * dtype of vals and fill_vals.  All arrays device; async on stream. */
int jv_scatter_values(int n, const int *rowptr, const int *colidx, jv_dtype t, const void *vals,
                      const int *fill_rowptr, const int *fill_colidx, void *fill_vals,
                      void *stream);

/* Measured latency of one dependency hop, in microseconds: a value stored by
 * one SM (relaxed store, gpu scope) and seen by another SM polling it
 * (relaxed load).  In the point-to-point schedule of Sec. III-A (Fig. 4)
 * every level of the dependency DAG costs at least one such hop, so
 * levels x hop is the critical-path bound of the sync-free kernels.
 * Launches a cooperative grid of one 32-thread CTA per SM on `stream`
 * (cudaStream_t or NULL) in which CTA 0 and a partner CTA exchange `rounds`
 * round trips (> 0); repeated for `npartners` (> 0) partners spread over the
 * grid (both dies); *out_us (host) receives the median one-way time.
 * Synchronous; allocates and frees 272 bytes of device memory.  Every wait
 * is bounded (0.2 s per partner): JV_ERR_TIMEOUT if one expired,
 * JV_ERR_CUDA if cooperative launch is unsupported or a CUDA call failed. */
int jv_hop_latency(int rounds, int npartners, double *out_us, void *stream);

/* Number of kernels this library has launched in the process so far. */
unsigned long long jv_launch_count(void);

/* Static English text for a status code. */
const char *jv_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* JV_H */
