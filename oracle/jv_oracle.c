/*
 * jv_oracle.c -- plain, serial, slow-but-obviously-correct CPU oracle for the
 * Javelin hot path (Booth & Bolet, "Javelin: A Scalable Implementation for
 * Sparse Incomplete LU Factorization", arXiv 1812.06160).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Conventions (all readings of the paper are listed with the design notes):
 *   - CSR, 0-based, int32 indices, strictly ascending columns in every row,
 *     diagonal present (Sec. III, Fig. 1 divides by a_{col,col}).
 *   - L is unit lower triangular and stored strictly below the diagonal;
 *     U carries the diagonal; both live in A's own pattern (Fig. 1: "L and U
 *     are stored in A").
 *   - Every update of the form s <- s -/+ a*b is one fused multiply-add
 *     (C99 fma / fmaf: the exact a*b added to s, rounded once); every other
 *     statement is a separate IEEE operation (the file is compiled with
 *     -ffp-contract=off, so nothing else is fused).
 *   - Multi-right-hand-side vectors are row-major n x nrhs.
 *
 * Status codes (numbers chosen to read the same as the library's, by
 * convention only): 0 ok, -1 bad argument, -2 bad pattern (column out of
 * range, unsorted or duplicate), -3 missing diagonal, -4 zero or non-finite
 * pivot.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define JVO_OK 0
#define JVO_ERR_ARG (-1)
#define JVO_ERR_PATTERN (-2)
#define JVO_ERR_NO_DIAG (-3)
#define JVO_ERR_ZERO_PIVOT (-4)

/* ------------------------------------------------------------------------ */
/* Validation and diagonal positions (Sec. III, Fig. 1: the column loop must */
/* visit columns in ascending order and a_{col,col} must exist).             */
/* ------------------------------------------------------------------------ */
int jvo_validate(int n, int nnz, const int *rowptr, const int *colidx,
                 int *diag, int *bad_row)
{
    *bad_row = -1;
    if (n <= 0 || nnz < 0) return JVO_ERR_ARG;
    if (rowptr[0] != 0 || rowptr[n] != nnz) { *bad_row = 0; return JVO_ERR_PATTERN; }
    for (int i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) { *bad_row = i; return JVO_ERR_PATTERN; }
    }
    for (int i = 0; i < n; ++i) {
        int d = -1;
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int c = colidx[p];
            if (c < 0 || c >= n) { *bad_row = i; return JVO_ERR_PATTERN; }
            if (p > rowptr[i] && colidx[p - 1] >= c) { *bad_row = i; return JVO_ERR_PATTERN; }
            if (c == i) d = p;
        }
        if (d < 0) { *bad_row = i; return JVO_ERR_NO_DIAG; }
        diag[i] = d;
    }
    return JVO_OK;
}

/* ------------------------------------------------------------------------ */
/* Levels, route (a): longest path in the DAG (Sec. II "level scheduling",   */
/* Sec. III-A).  For the lower pattern, row i depends on every j < i in row  */
/* i; visiting rows in ascending order finalises every j before i, so        */
/* lev[i] = 0 without dependencies, else 1 + max lev[j].  upper != 0 mirrors */
/* this for the backward (U) solve: dependencies are j > i, rows descending. */
/* Returns the number of levels.                                              */
/* ------------------------------------------------------------------------ */
int jvo_levels_longest_path(int n, const int *rowptr, const int *colidx,
                            int upper, int *lev)
{
    int nlev = 0;
    for (int t = 0; t < n; ++t) {
        int i = upper ? (n - 1 - t) : t;
        int best = -1;
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int j = colidx[p];
            int is_dep = upper ? (j > i) : (j < i);
            if (is_dep && lev[j] > best) best = lev[j];
        }
        lev[i] = best + 1;
        if (lev[i] + 1 > nlev) nlev = lev[i] + 1;
    }
    return nlev;
}

/* ------------------------------------------------------------------------ */
/* Levels, route (b): peeling, literally as Sec. II describes level          */
/* scheduling -- the vertices with no incoming edge form a level, they and   */
/* their outgoing edges are removed, repeat.  Edge j -> i for every          */
/* dependency j of row i.                                                     */
/* ------------------------------------------------------------------------ */
int jvo_levels_peel(int n, const int *rowptr, const int *colidx, int upper,
                    int *lev)
{
    int *indeg = (int *)calloc((size_t)n, sizeof(int));
    int *cur = (int *)malloc((size_t)n * sizeof(int));
    int *nxt = (int *)malloc((size_t)n * sizeof(int));
    /* outgoing edges: dependents of j.  Build them by a counting pass. */
    int *optr = (int *)calloc((size_t)n + 1, sizeof(int));
    int nedge = 0;
    for (int i = 0; i < n; ++i)
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int j = colidx[p];
            if (upper ? (j > i) : (j < i)) { optr[j + 1]++; indeg[i]++; nedge++; }
        }
    for (int j = 0; j < n; ++j) optr[j + 1] += optr[j];
    int *oidx = (int *)malloc((size_t)(nedge > 0 ? nedge : 1) * sizeof(int));
    int *fill = (int *)malloc((size_t)n * sizeof(int));
    for (int j = 0; j < n; ++j) fill[j] = optr[j];
    for (int i = 0; i < n; ++i)
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int j = colidx[p];
            if (upper ? (j > i) : (j < i)) oidx[fill[j]++] = i;
        }
    int ncur = 0;
    for (int i = 0; i < n; ++i) if (indeg[i] == 0) cur[ncur++] = i;
    int level = 0, seen = 0;
    while (ncur > 0) {
        int nnext = 0;
        for (int t = 0; t < ncur; ++t) {
            int j = cur[t];
            lev[j] = level;
            seen++;
            for (int e = optr[j]; e < optr[j + 1]; ++e) {
                int i = oidx[e];
                if (--indeg[i] == 0) nxt[nnext++] = i;
            }
        }
        int *tmp = cur; cur = nxt; nxt = tmp;
        ncur = nnext;
        level++;
    }
    free(indeg); free(cur); free(nxt); free(optr); free(oidx); free(fill);
    return seen == n ? level : -1;
}

/* ------------------------------------------------------------------------ */
/* Level sets: rows grouped by level, ascending row index inside a level     */
/* (Sec. III-A; the tie order is this implementation's reading).  A stable   */
/* counting sort.                                                             */
/* ------------------------------------------------------------------------ */
void jvo_bucket_levels(int n, const int *lev, int nlev, int *level_ptr,
                       int *level_rows)
{
    for (int l = 0; l <= nlev; ++l) level_ptr[l] = 0;
    for (int i = 0; i < n; ++i) level_ptr[lev[i] + 1]++;
    for (int l = 0; l < nlev; ++l) level_ptr[l + 1] += level_ptr[l];
    int *fill = (int *)malloc((size_t)(nlev > 0 ? nlev : 1) * sizeof(int));
    for (int l = 0; l < nlev; ++l) fill[l] = level_ptr[l];
    for (int i = 0; i < n; ++i) level_rows[fill[lev[i]]++] = i;
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* Transpose of the pattern (CSC of A): colptr, row indices ascending inside */
/* each column, and csc2csr[q] = CSR position of CSC entry q.  Needed by the */
/* adjoint's transposed solves (not part of the paper).                      */
/* ------------------------------------------------------------------------ */
void jvo_transpose(int n, const int *rowptr, const int *colidx, int *colptr,
                   int *rowidx, int *csc2csr)
{
    for (int j = 0; j <= n; ++j) colptr[j] = 0;
    for (int p = 0; p < rowptr[n]; ++p) colptr[colidx[p] + 1]++;
    for (int j = 0; j < n; ++j) colptr[j + 1] += colptr[j];
    int *fill = (int *)malloc((size_t)n * sizeof(int));
    for (int j = 0; j < n; ++j) fill[j] = colptr[j];
    for (int i = 0; i < n; ++i)
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int q = fill[colidx[p]]++;
            rowidx[q] = i;
            csc2csr[q] = p;
        }
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* Symmetric permutation B = P A P^T (Sec. III: the nonzeros are permuted    */
/* into the level order while copying A into the CSR of L and U).  Row r of  */
/* B is row perm[r] of A; column c of A becomes iperm[c]; columns are        */
/* re-sorted ascending; vmap[t] = position in A of B's entry t.              */
/* ------------------------------------------------------------------------ */
void jvo_permute(int n, const int *rowptr, const int *colidx, const int *perm,
                 int *iperm, int *browptr, int *bcolidx, int *vmap)
{
    for (int r = 0; r < n; ++r) iperm[perm[r]] = r;
    browptr[0] = 0;
    for (int r = 0; r < n; ++r) {
        int i = perm[r];
        int len = rowptr[i + 1] - rowptr[i];
        int base = browptr[r];
        browptr[r + 1] = base + len;
        /* insertion sort of the mapped columns: plain and obviously right */
        for (int t = 0; t < len; ++t) {
            int p = rowptr[i] + t;
            int c = iperm[colidx[p]];
            int s = base + t;
            while (s > base && bcolidx[s - 1] > c) {
                bcolidx[s] = bcolidx[s - 1];
                vmap[s] = vmap[s - 1];
                s--;
            }
            bcolidx[s] = c;
            vmap[s] = p;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* ILU(0), up-looking (row-wise left-looking, "IKJ") on A's own pattern --   */
/* Sec. III, Fig. 1.  For every row i, for every col k < i of row i in       */
/* ascending order: a_ik <- a_ik / a_kk, then for every update column j > k  */
/* of row k that is also in row i: a_ij <- a_ij - a_ik * a_kj (one fused     */
/* multiply-add, rounded once).  No pivoting                                 */
/* (Sec. III).  Membership of j in row i is found through a dense scatter of */
/* row i.  A zero or non-finite pivot a_ii stops the factorisation with      */
/* bad_row = i.  In place on a[].                                             */
/* ------------------------------------------------------------------------ */
int jvo_ilu0(int n, const int *rowptr, const int *colidx, const int *diag,
             double *a, int *bad_row)
{
    *bad_row = -1;
    int *pos = (int *)malloc((size_t)n * sizeof(int));
    for (int j = 0; j < n; ++j) pos[j] = -1;
    for (int i = 0; i < n; ++i) {
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) pos[colidx[p]] = p;
        for (int p = rowptr[i]; p < diag[i]; ++p) {
            int k = colidx[p];
            double lik = a[p] / a[diag[k]];
            a[p] = lik;
            for (int q = diag[k] + 1; q < rowptr[k + 1]; ++q) {
                int j = colidx[q];
                if (pos[j] >= 0) {
                    a[pos[j]] = fma(-lik, a[q], a[pos[j]]);
                }
            }
        }
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) pos[colidx[p]] = -1;
        double piv = a[diag[i]];
        if (piv == 0.0 || !isfinite(piv)) {
            *bad_row = i;
            free(pos);
            return JVO_ERR_ZERO_PIVOT;
        }
    }
    free(pos);
    return JVO_OK;
}

/* The same algorithm with every value and every operation in binary32 --   */
/* the single-precision twin used to check a single-precision factor.  The  */
/* pivot test is done on the value promoted to binary64.                     */
int jvo_ilu0_f32(int n, const int *rowptr, const int *colidx, const int *diag,
                 float *a, int *bad_row)
{
    *bad_row = -1;
    int *pos = (int *)malloc((size_t)n * sizeof(int));
    for (int j = 0; j < n; ++j) pos[j] = -1;
    for (int i = 0; i < n; ++i) {
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) pos[colidx[p]] = p;
        for (int p = rowptr[i]; p < diag[i]; ++p) {
            int k = colidx[p];
            float lik = a[p] / a[diag[k]];
            a[p] = lik;
            for (int q = diag[k] + 1; q < rowptr[k + 1]; ++q) {
                int j = colidx[q];
                if (pos[j] >= 0) {
                    a[pos[j]] = fmaf(-lik, a[q], a[pos[j]]);
                }
            }
        }
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) pos[colidx[p]] = -1;
        double piv = (double)a[diag[i]];
        if (piv == 0.0 || !isfinite(piv)) {
            *bad_row = i;
            free(pos);
            return JVO_ERR_ZERO_PIVOT;
        }
    }
    free(pos);
    return JVO_OK;
}

/* ------------------------------------------------------------------------ */
/* Modified ILU(0) (MILU, which the up-looking design of Sec. I / Sec. III   */
/* is said to support): the same IKJ sweep, but an update a_ij -= a_ik a_kj  */
/* whose column j is not in row i's pattern is not dropped -- it is applied  */
/* to the diagonal a_ii instead, at the moment it occurs (same k, same j     */
/* order), so the diagonal absorbs every dropped fill-in and the row sums of */
/* L U equal those of A in exact arithmetic.                                 */
/* ------------------------------------------------------------------------ */
int jvo_milu0(int n, const int *rowptr, const int *colidx, const int *diag,
              double *a, int *bad_row)
{
    *bad_row = -1;
    int *pos = (int *)malloc((size_t)n * sizeof(int));
    for (int j = 0; j < n; ++j) pos[j] = -1;
    for (int i = 0; i < n; ++i) {
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) pos[colidx[p]] = p;
        for (int p = rowptr[i]; p < diag[i]; ++p) {
            int k = colidx[p];
            double lik = a[p] / a[diag[k]];
            a[p] = lik;
            for (int q = diag[k] + 1; q < rowptr[k + 1]; ++q) {
                int j = colidx[q];
                int t = pos[j] >= 0 ? pos[j] : diag[i];     /* dropped: onto a_ii */
                a[t] = fma(-lik, a[q], a[t]);
            }
        }
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) pos[colidx[p]] = -1;
        double piv = a[diag[i]];
        if (piv == 0.0 || !isfinite(piv)) {
            *bad_row = i;
            free(pos);
            return JVO_ERR_ZERO_PIVOT;
        }
    }
    free(pos);
    return JVO_OK;
}

/* MILU in binary32 (every value and operation single precision). */
int jvo_milu0_f32(int n, const int *rowptr, const int *colidx, const int *diag,
                  float *a, int *bad_row)
{
    *bad_row = -1;
    int *pos = (int *)malloc((size_t)n * sizeof(int));
    for (int j = 0; j < n; ++j) pos[j] = -1;
    for (int i = 0; i < n; ++i) {
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) pos[colidx[p]] = p;
        for (int p = rowptr[i]; p < diag[i]; ++p) {
            int k = colidx[p];
            float lik = a[p] / a[diag[k]];
            a[p] = lik;
            for (int q = diag[k] + 1; q < rowptr[k + 1]; ++q) {
                int j = colidx[q];
                int t = pos[j] >= 0 ? pos[j] : diag[i];
                a[t] = fmaf(-lik, a[q], a[t]);
            }
        }
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) pos[colidx[p]] = -1;
        double piv = (double)a[diag[i]];
        if (piv == 0.0 || !isfinite(piv)) {
            *bad_row = i;
            free(pos);
            return JVO_ERR_ZERO_PIVOT;
        }
    }
    free(pos);
    return JVO_OK;
}

/* ------------------------------------------------------------------------ */
/* ILU(k) symbolic factorisation -- the level-of-fill pattern that ILU(k)     */
/* factors on (Sec. II, and Sec. V "Incomplete levels": Javelin runs the     */
/* same up-looking numeric sweep on a pattern widened by the fill the user    */
/* asks for).  Row by row, i ascending: lev(i,j) = 0 for every entry of A's row  */
/* i, otherwise unset; then for every column k < i of the row, in ascending   */
/* order (fill columns included as they appear): for every column j > k of   */
/* row k's filled pattern, lev(i,j) <- min(lev(i,j), lev(i,k) + lev(k,j) + 1) */
/* if that is <= K.  Row i's pattern is every j with a level <= K.            */
/* The next k is taken from a binary min-heap of the row's columns < i.       */
/* cap bounds the output; returns the filled nnz, or -1 when cap is too      */
/* small (the caller retries with more).                                     */
/* ------------------------------------------------------------------------ */
static void heap_push(int *h, int *m, int v)
{
    int c = (*m)++;
    h[c] = v;
    while (c > 0 && h[(c - 1) / 2] > h[c]) {
        int p = (c - 1) / 2, t = h[p];
        h[p] = h[c];
        h[c] = t;
        c = p;
    }
}

static int heap_pop(int *h, int *m)
{
    int top = h[0];
    h[0] = h[--(*m)];
    int c = 0;
    for (;;) {
        int l = 2 * c + 1, r = l + 1, s = c;
        if (l < *m && h[l] < h[s]) s = l;
        if (r < *m && h[r] < h[s]) s = r;
        if (s == c) break;
        int t = h[s];
        h[s] = h[c];
        h[c] = t;
        c = s;
    }
    return top;
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

long long jvo_iluk_symbolic(int n, const int *rowptr, const int *colidx, int K, long long cap,
                            int *out_rowptr, int *out_colidx, int *out_lev)
{
    const int UNSET = -1;
    int *lev = (int *)malloc((size_t)n * sizeof(int));
    int *touched = (int *)malloc((size_t)n * sizeof(int));
    int *heap = (int *)malloc((size_t)n * sizeof(int));
    for (int j = 0; j < n; ++j) lev[j] = UNSET;
    long long nz = 0;
    out_rowptr[0] = 0;
    for (int i = 0; i < n; ++i) {
        int nt = 0, hm = 0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int j = colidx[p];
            lev[j] = 0;
            touched[nt++] = j;
            if (j < i) heap_push(heap, &hm, j);
        }
        int last = -1;
        while (hm > 0) {
            int k = heap_pop(heap, &hm);
            if (k == last) continue;           /* a column pushed twice */
            last = k;
            int lik = lev[k];
            for (int q = out_rowptr[k]; q < out_rowptr[k + 1]; ++q) {
                int j = out_colidx[q];
                if (j <= k) continue;          /* row k's filled upper part */
                int l = lik + out_lev[q] + 1;
                if (l > K) continue;
                if (lev[j] == UNSET) {
                    lev[j] = l;
                    touched[nt++] = j;
                    if (j < i) heap_push(heap, &hm, j);
                } else if (l < lev[j]) {
                    lev[j] = l;
                }
            }
        }
        if (nz + nt > cap) {
            free(lev);
            free(touched);
            free(heap);
            return -1;
        }
        qsort(touched, (size_t)nt, sizeof(int), cmp_int);
        for (int t = 0; t < nt; ++t) {
            out_colidx[nz + t] = touched[t];
            out_lev[nz + t] = lev[touched[t]];
            lev[touched[t]] = UNSET;
        }
        nz += nt;
        out_rowptr[i + 1] = (int)nz;
    }
    free(lev);
    free(touched);
    free(heap);
    return nz;
}

/* ------------------------------------------------------------------------ */
/* Triangular solves (Sec. VI: forward and backward stri).                  */
/* L x = b, L unit lower: x_i = b_i - sum_{j<i} l_ij x_j, rows ascending,   */
/* the sum taken in ascending column order.                                 */
/* ------------------------------------------------------------------------ */
void jvo_lsolve(int n, const int *rowptr, const int *colidx, const int *diag,
                const double *lu, const double *b, double *x, int nrhs)
{
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < nrhs; ++c) {
            double s = b[(size_t)i * nrhs + c];
            for (int p = rowptr[i]; p < diag[i]; ++p) {
                s = fma(-lu[p], x[(size_t)colidx[p] * nrhs + c], s);
            }
            x[(size_t)i * nrhs + c] = s;
        }
}

/* U x = b: x_i = (b_i - sum_{j>i} u_ij x_j) / u_ii, rows descending. */
void jvo_usolve(int n, const int *rowptr, const int *colidx, const int *diag,
                const double *lu, const double *b, double *x, int nrhs)
{
    for (int i = n - 1; i >= 0; --i)
        for (int c = 0; c < nrhs; ++c) {
            double s = b[(size_t)i * nrhs + c];
            for (int p = diag[i] + 1; p < rowptr[i + 1]; ++p) {
                s = fma(-lu[p], x[(size_t)colidx[p] * nrhs + c], s);
            }
            x[(size_t)i * nrhs + c] = s / lu[diag[i]];
        }
}

/* U^T x = b (forward, column sweep on U's rows): once x_i is final, row i  */
/* of U scatters -u_ij x_i into every later equation j.                      */
void jvo_usolve_t(int n, const int *rowptr, const int *colidx, const int *diag,
                  const double *lu, const double *b, double *x, int nrhs)
{
    size_t len = (size_t)n * nrhs;
    double *g = (double *)malloc(len * sizeof(double));
    memcpy(g, b, len * sizeof(double));
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < nrhs; ++c) {
            double xi = g[(size_t)i * nrhs + c] / lu[diag[i]];
            x[(size_t)i * nrhs + c] = xi;
            for (int p = diag[i] + 1; p < rowptr[i + 1]; ++p) {
                size_t o = (size_t)colidx[p] * nrhs + c;
                g[o] = fma(-lu[p], xi, g[o]);
            }
        }
    free(g);
}

/* L^T x = b (backward, unit diagonal): once x_i is final, row i of L       */
/* scatters -l_ij x_i into every earlier equation j.                         */
void jvo_lsolve_t(int n, const int *rowptr, const int *colidx, const int *diag,
                  const double *lu, const double *b, double *x, int nrhs)
{
    size_t len = (size_t)n * nrhs;
    double *g = (double *)malloc(len * sizeof(double));
    memcpy(g, b, len * sizeof(double));
    for (int i = n - 1; i >= 0; --i)
        for (int c = 0; c < nrhs; ++c) {
            double xi = g[(size_t)i * nrhs + c];
            x[(size_t)i * nrhs + c] = xi;
            for (int p = rowptr[i]; p < diag[i]; ++p) {
                size_t o = (size_t)colidx[p] * nrhs + c;
                g[o] = fma(-lu[p], xi, g[o]);
            }
        }
    free(g);
}

/* Gradient of z = U^-1 L^-1 r with respect to the stored factor values,    */
/* restricted to the pattern: g_p = alpha * sum_c a[i,c] * b[j,c] for every */
/* entry p = (i, j) of the chosen part (0: strictly lower, 1: upper with     */
/* the diagonal).  Entries outside the part are left untouched.              */
void jvo_masked_outer(int n, const int *rowptr, const int *colidx,
                      const int *diag, int which, const double *a,
                      const double *b, int nrhs, double alpha, double *g)
{
    for (int i = 0; i < n; ++i) {
        int lo = which == 0 ? rowptr[i] : diag[i];
        int hi = which == 0 ? diag[i] : rowptr[i + 1];
        for (int p = lo; p < hi; ++p) {
            int j = colidx[p];
            double s = 0.0;
            for (int c = 0; c < nrhs; ++c) {
                s = fma(a[(size_t)i * nrhs + c], b[(size_t)j * nrhs + c], s);
            }
            g[p] = alpha * s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* spmv (Sec. I, Sec. VI): y = alpha * A x + beta * y, ascending columns.   */
/* beta == 0 ignores the old y entirely.                                     */
/* ------------------------------------------------------------------------ */
void jvo_spmv(int n, const int *rowptr, const int *colidx, const double *a,
              const double *x, double *y, double alpha, double beta)
{
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            s = fma(a[p], x[colidx[p]], s);
        }
        double v = alpha * s;
        if (beta != 0.0) v = fma(beta, y[i], v);
        y[i] = v;
    }
}

/* ------------------------------------------------------------------------ */
/* Krylov drivers (Sec. I: CG / GMRES preconditioned by the ILU factors).   */
/* ------------------------------------------------------------------------ */
static double dot(int n, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) { double prod = a[i] * b[i]; s = s + prod; }
    return s;
}

static void apply_prec(int n, const int *rowptr, const int *colidx,
                       const int *diag, const double *lu, const double *r,
                       double *tmp, double *z)
{
    jvo_lsolve(n, rowptr, colidx, diag, lu, r, tmp, 1);
    jvo_usolve(n, rowptr, colidx, diag, lu, tmp, z, 1);
}

/* Flexible preconditioned CG (Polak-Ribiere beta, so a preconditioner that  */
/* is only approximately linear cannot stall it).  x holds x0 on entry.      */
/* Stops when ||b - A x_k|| / ||b|| <= tol (recursive residual), then        */
/* recomputes the true residual.  Returns the iteration count, or -1 when   */
/* maxit was reached.                                                        */
int jvo_pcg(int n, const int *rowptr, const int *colidx, const int *diag,
            const double *a, const double *lu, const double *b, double *x,
            double tol, int maxit, double *relres_out)
{
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *z = (double *)malloc((size_t)n * sizeof(double));
    double *zn = (double *)malloc((size_t)n * sizeof(double));
    double *p = (double *)malloc((size_t)n * sizeof(double));
    double *q = (double *)malloc((size_t)n * sizeof(double));
    double *t = (double *)malloc((size_t)n * sizeof(double));
    jvo_spmv(n, rowptr, colidx, a, x, r, 1.0, 0.0);
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) bnorm = 1.0;
    int it = 0, done = sqrt(dot(n, r, r)) / bnorm <= tol;
    apply_prec(n, rowptr, colidx, diag, lu, r, t, z);
    for (int i = 0; i < n; ++i) p[i] = z[i];
    double rz = dot(n, r, z);
    while (!done && it < maxit) {
        jvo_spmv(n, rowptr, colidx, a, p, q, 1.0, 0.0);
        double alpha = rz / dot(n, p, q);
        for (int i = 0; i < n; ++i) { double d = alpha * p[i]; x[i] = x[i] + d; }
        for (int i = 0; i < n; ++i) { double d = alpha * q[i]; r[i] = r[i] - d; }
        it++;
        if (sqrt(dot(n, r, r)) / bnorm <= tol) { done = 1; break; }
        apply_prec(n, rowptr, colidx, diag, lu, r, t, zn);
        double rzn = dot(n, r, zn);
        double rzo = dot(n, r, z);
        double beta = (rzn - rzo) / rz;
        rz = rzn;
        for (int i = 0; i < n; ++i) { double d = beta * p[i]; p[i] = zn[i] + d; }
        double *sw = z; z = zn; zn = sw;
    }
    jvo_spmv(n, rowptr, colidx, a, x, r, 1.0, 0.0);
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
    *relres_out = sqrt(dot(n, r, r)) / bnorm;
    free(r); free(z); free(zn); free(p); free(q); free(t);
    return done ? it : -1;
}

/* Flexible GMRES(m), right preconditioned (the preconditioned vectors z_j  */
/* are kept, so the outer solve tolerates a preconditioner applied in lower */
/* precision).  Arnoldi with modified Gram-Schmidt; Givens rotations on the */
/* (m+1) x m Hessenberg matrix.  Returns the total inner iteration count,   */
/* or -1 when max_restarts cycles did not converge.                         */
int jvo_fgmres(int n, const int *rowptr, const int *colidx, const int *diag,
               const double *a, const double *lu, const double *b, double *x,
               int m, double tol, int max_restarts, double *relres_out)
{
    double *V = (double *)malloc((size_t)(m + 1) * n * sizeof(double));
    double *Z = (double *)malloc((size_t)m * n * sizeof(double));
    double *w = (double *)malloc((size_t)n * sizeof(double));
    double *t = (double *)malloc((size_t)n * sizeof(double));
    double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double)); /* H[i*m+j] */
    double *cs = (double *)malloc((size_t)m * sizeof(double));
    double *sn = (double *)malloc((size_t)m * sizeof(double));
    double *g = (double *)malloc((size_t)(m + 1) * sizeof(double));
    double *y = (double *)malloc((size_t)m * sizeof(double));
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) bnorm = 1.0;
    int total = 0, converged = 0;
    for (int cycle = 0; cycle < max_restarts && !converged; ++cycle) {
        jvo_spmv(n, rowptr, colidx, a, x, w, 1.0, 0.0);
        for (int i = 0; i < n; ++i) w[i] = b[i] - w[i];
        double beta = sqrt(dot(n, w, w));
        if (beta / bnorm <= tol) { converged = 1; break; }
        for (int i = 0; i < n; ++i) V[i] = w[i] / beta;
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
            apply_prec(n, rowptr, colidx, diag, lu, vj, t, zj);
            jvo_spmv(n, rowptr, colidx, a, zj, w, 1.0, 0.0);
            for (int i = 0; i <= j; ++i) {
                double *vi = V + (size_t)i * n;
                double h = dot(n, w, vi);
                H[i * m + j] = h;
                for (int e = 0; e < n; ++e) { double d = h * vi[e]; w[e] = w[e] - d; }
            }
            double hn = sqrt(dot(n, w, w));
            H[(j + 1) * m + j] = hn;
            if (hn != 0.0) {
                double *vn = V + (size_t)(j + 1) * n;
                for (int e = 0; e < n; ++e) vn[e] = w[e] / hn;
            }
            /* apply the previous rotations to column j, then a new one */
            for (int i = 0; i < j; ++i) {
                double h0 = H[i * m + j], h1 = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * h0 + sn[i] * h1;
                H[(i + 1) * m + j] = -sn[i] * h0 + cs[i] * h1;
            }
            double h0 = H[j * m + j], h1 = H[(j + 1) * m + j];
            double rr = sqrt(h0 * h0 + h1 * h1);
            cs[j] = rr == 0.0 ? 1.0 : h0 / rr;
            sn[j] = rr == 0.0 ? 0.0 : h1 / rr;
            H[j * m + j] = rr;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            k = j + 1;
            total++;
            if (fabs(g[j + 1]) / bnorm <= tol || hn == 0.0) break;
        }
        /* back substitution H[0:k,0:k] y = g[0:k], then x += Z y */
        for (int i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int l = i + 1; l < k; ++l) s = s - H[i * m + l] * y[l];
            y[i] = s / H[i * m + i];
        }
        for (int j = 0; j < k; ++j) {
            double *zj = Z + (size_t)j * n;
            for (int e = 0; e < n; ++e) { double d = y[j] * zj[e]; x[e] = x[e] + d; }
        }
        jvo_spmv(n, rowptr, colidx, a, x, w, 1.0, 0.0);
        for (int i = 0; i < n; ++i) w[i] = b[i] - w[i];
        if (sqrt(dot(n, w, w)) / bnorm <= tol) converged = 1;
    }
    jvo_spmv(n, rowptr, colidx, a, x, w, 1.0, 0.0);
    for (int i = 0; i < n; ++i) w[i] = b[i] - w[i];
    *relres_out = sqrt(dot(n, w, w)) / bnorm;
    free(V); free(Z); free(w); free(t); free(H); free(cs); free(sn); free(g); free(y);
    return converged ? total : -1;
}
