// jv_analyze: dependency analysis on the GPU.
//
//  * validation + diag_ptr (Sec. III, Fig. 1 needs ascending columns and the
//    diagonal a_{col,col});
//  * CSC of the pattern (stable radix sort of the column indices), used for
//    the dependants lists and for the adjoint's transposed solves;
//  * levels of the four dependency DAGs by peeling (Sec. II: the vertices
//    without incoming edges form a level, they are removed with their
//    outgoing edges, repeat) -- one launch per level in batches, with the
//    frontier sizes kept on the device;
//  * level sets: rows grouped by level, ascending inside a level, by a stable
//    radix sort keyed on the level, so the result is unique and bit-exact;
//  * per-level work lists ("tasks") of up to 32/vw rows that never straddle a
//    level boundary, for the factor and solve kernels;
//  * optionally the symmetric permutation B = P A P^T into the level order
//    (Sec. III: the nonzeros are permuted into the level ordering).
#include <algorithm>

#include "jv_internal.cuh"

namespace jv {

int halloc(jv_handle h, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return JV_ERR_NOMEM;
    }
    h->allocs.push_back(*p);
    return JV_OK;
}

int ensure_buffer(jv_handle h, void **p, size_t *bytes, size_t need) {
    if (*bytes >= need && *p) return JV_OK;
    if (*p) {
        JV_CUDA(cudaStreamSynchronize(h->stream));
        cudaFree(*p);
        *p = nullptr;
        *bytes = 0;
    }
    if (cudaMalloc(p, need + 16) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return JV_ERR_NOMEM;
    }
    *bytes = need;
    return JV_OK;
}

namespace {

// Temporary device allocations released when the analysis returns.
struct Temp {
    std::vector<void *> ptrs;
    ~Temp() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T> int get(T **p, size_t count) {
        void *q = nullptr;
        if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) {
            cudaGetLastError();
            return JV_ERR_NOMEM;
        }
        ptrs.push_back(q);
        *p = (T *)q;
        return JV_OK;
    }
};

int bits_for(long long maxval) {
    int b = 1;
    while (b < 31 && (1ll << b) <= maxval) ++b;
    return b;
}

#define JV_TRY(x)                 \
    do {                          \
        int rc_ = (x);            \
        if (rc_ != JV_OK) return rc_; \
    } while (0)

// ------------------------------------------------------------- validation
__global__ void k_validate(int n, int nnz, const int *rowptr, const int *colidx, int *diag,
                           unsigned long long *st, int *nnz_lower) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0 && (rowptr[0] != 0 || rowptr[n] != nnz)) {
        report(st, JV_ERR_PATTERN, 0);
        return;
    }
    int s = rowptr[i], e = rowptr[i + 1];
    if (s < 0 || e > nnz || s > e) {
        report(st, JV_ERR_PATTERN, i);
        return;
    }
    int d = -1;
    for (int p = s; p < e; ++p) {
        int c = colidx[p];
        if (c < 0 || c >= n || (p > s && colidx[p - 1] >= c)) {
            report(st, JV_ERR_PATTERN, i);
            return;
        }
        if (c == i) d = p;
    }
    if (d < 0) {
        report(st, JV_ERR_NO_DIAG, i);
        return;
    }
    diag[i] = d;
    atomicAdd(nnz_lower, d - s);
}

__global__ void k_row_of(int n, const int *rowptr, int *row_of) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) row_of[p] = i;
}

__global__ void k_copy_u32(const int *src, unsigned *dst, int m) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) dst[i] = (unsigned)src[i];
}

__global__ void k_csc_finish(int nnz, const unsigned *col_sorted, const unsigned *pos_sorted,
                             const int *row_of, int *rowidx, int *csc2csr, int *cdiag) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nnz) return;
    int p = (int)pos_sorted[q];
    int r = row_of[p];
    rowidx[q] = r;
    csc2csr[q] = p;
    if ((unsigned)r == col_sorted[q]) cdiag[r] = q;
}

// -------------------------------------------------- symbolic factorisation
// For the strictly lower entry p = (r, k) of row r, Fig. 1 updates every
// a_rj with j > k, j in row k and in row r.  One warp per row, lanes over the
// row's lower entries; the pairs (t = position of (r, j), q = position of
// (k, j)) of one p are listed in ascending j, which is the order Fig. 1 applies
// them.  With MILU, a column j of row k that is not in row r gives the pair
// (t = position of (r, r), q): the update lands on the diagonal, in the same
// place of the order.  Pass 1 counts (cnt[p], zero off the lower part), pass
// 2 fills.
template <bool FILL, bool MILU>
__global__ void k_pairs(int n, const int *rowptr, const int *colidx, const int *diag, int *cnt,
                        const int *ptr, int2 *pairs) {
    const long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const int rs = rowptr[r], re = rowptr[r + 1], rd = diag[r];
    for (int p = rs + lane; p < rd; p += 32) {
        const int k = colidx[p];
        const int ke = rowptr[k + 1];
        int c = 0;
        const int base = FILL ? ptr[p] : 0;
        for (int q = diag[k] + 1; q < ke; ++q) {
            int t = find_col(colidx, p + 1, re, colidx[q]);
            if (MILU && t < 0) t = rd;        // modified ILU: dropped fill onto a_ii
            if (t >= 0) {
                if (FILL) pairs[base + c] = make_int2(t, q);
                ++c;
            }
        }
        if (!FILL) cnt[p] = c;
    }
    if (!FILL)
        for (int p = rd + lane; p < re; p += 32) cnt[p] = 0;
}

// step[j] = the lower entry p whose update pair j is (pairs of p: pair_ptr[p] .. pair_ptr[p+1]).
__global__ void k_pair_step(int nnz, const int *pair_ptr, unsigned *step) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    for (int j = pair_ptr[p]; j < pair_ptr[p + 1]; ++j) step[j] = (unsigned)p;
}
__global__ void k_pair_target(int np, const int2 *pairs, unsigned *key, unsigned *idx) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    key[j] = (unsigned)pairs[j].x;
    idx[j] = (unsigned)j;
}
__global__ void k_tpairs(int np, const unsigned *sorted_idx, const unsigned *step, const int2 *pairs,
                         const unsigned char *upd, int2 *tpairs) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const unsigned j = sorted_idx[s];
    const int q = pairs[j].y;
    tpairs[s] = make_int2((int)step[j], upd[q] ? ~q : q);   // ~q: an operand to await
}

// kpos[p] = the factor work-list position of row k, for every L entry
// p = (r, k): where the pivot the entry divides by is published.
__global__ void k_kpos(int n, const int *rowptr, const int *diag, const int *colidx,
                       const int *ipos, int *kpos) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int p = rowptr[r], e = diag[r]; p < e; ++p) kpos[p] = ipos[colidx[p]];
}

// For every row: the depth of the dependency chain among its L entries (an
// entry depends on the in-row entries whose steps update it) and whether the
// pull form pays -- its waves (= that depth) at most half the row's steps.
// depth[] is scratch over the row's positions.  One thread per row.
__global__ void k_row_pull(int n, const int *rowptr, const int *diag, const int *tpair_ptr,
                           const int2 *tpairs, int *depth, unsigned char *pull,
                           unsigned char *edepth) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int rs = rowptr[r], rd = diag[r];
    int most = 0;
    for (int p = rs; p < rd; ++p) {
        int d = 1;
        for (int k = tpair_ptr[p]; k < tpair_ptr[p + 1]; ++k) d = max(d, depth[tpairs[k].x] + 1);
        depth[p] = d;
        edepth[p] = (unsigned char)min(d, 255);
        most = max(most, d);
    }
    pull[r] = (unsigned char)(2 * most <= rd - rs ? 1 : 0);
}

// upd[t] = 1 for every entry some step of Fig. 1 updates (the target of a
// pair); the others keep A's value from start to end, so a row that reads one
// as an operand reads it from A's values and never waits for it.  cnt: pairs
// whose operand q is itself updated (operands that must be awaited).
__global__ void k_mark_targets(long long np, const int2 *pairs, unsigned char *upd) {
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j < np) upd[pairs[j].x] = 1;
}
__global__ void k_count_dynamic(long long np, const int2 *pairs, const unsigned char *upd,
                                unsigned long long *cnt) {
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool d = j < np && upd[pairs[j].y];
    const unsigned m = __ballot_sync(0xffffffffu, d);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(cnt, (unsigned long long)__popc(m));
}

__global__ void k_kdiag(int nnz, const int *colidx, const int *diag, int *kdiag) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) kdiag[p] = diag[colidx[p]];
}

// ---------------------------------------------------------------- peeling
struct Dag {
    Span cnt_beg, cnt_end;   // number of dependencies of v = cnt_end(v) - cnt_beg(v)
    Span dep_beg, dep_end;   // dependants of u: idx[dep_beg(u) .. dep_end(u))
    const int *idx;
    // optional second part (idx2 != null): the DAG is the union of both, a
    // dependency listed in both counted twice and removed twice -- e.g. the
    // levels of lower(A + A^T) from the row and the column lists of A,
    // without forming A + A^T
    Span cnt2_beg, cnt2_end, dep2_beg, dep2_end;
    const int *idx2;
};

__global__ void k_peel_init(int n, Dag g, int *cnt, int *lev, int *front, int *size) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = g.cnt_end.at(i) - g.cnt_beg.at(i);
    if (g.idx2) c += g.cnt2_end.at(i) - g.cnt2_beg.at(i);
    cnt[i] = c;
    if (c == 0) {
        lev[i] = 0;
        front[atomicAdd(size, 1)] = i;
    }
}

// One level: every dependant whose last dependency is removed joins the next
// frontier with the next level number.
__global__ void k_peel_round(Dag g, int *cnt, int *lev, int next_level, const int *fin,
                             const int *size_in, int *fout, int *size_out) {
    int size = *size_in;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < size; t += gridDim.x * blockDim.x) {
        int u = fin[t];
        for (int part = 0; part < (g.idx2 ? 2 : 1); ++part) {
            const int *idx = part ? g.idx2 : g.idx;
            const int e1 = part ? g.dep2_end.at(u) : g.dep_end.at(u);
            for (int e = part ? g.dep2_beg.at(u) : g.dep_beg.at(u); e < e1; ++e) {
                int v = idx[e];
                if (atomicSub(&cnt[v], 1) == 1) {
                    lev[v] = next_level;
                    fout[atomicAdd(size_out, 1)] = v;
                }
            }
        }
    }
}

constexpr int kPeelBatch = 32;

int peel_levels(jv_handle h, const Dag &g, int *lev, Temp &tmp, int *nlev_out,
                std::vector<int> &widths) {
    const int n = h->n;
    cudaStream_t s = h->stream;
    int *cnt, *fa, *fb, *sizes;
    JV_TRY(tmp.get(&cnt, n));
    JV_TRY(tmp.get(&fa, n));
    JV_TRY(tmp.get(&fb, n));
    JV_TRY(tmp.get(&sizes, kPeelBatch + 1));
    JV_CUDA(cudaMemsetAsync(sizes, 0, (kPeelBatch + 1) * sizeof(int), s));
    count_launch();
    k_peel_init<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, g, cnt, lev, fa, sizes);
    JV_CHECK_LAUNCH();
    widths.clear();
    int hs[kPeelBatch + 1];
    long long total = 0;
    const int grid = h->num_sms * 8;
    for (int level = 0;; level += kPeelBatch) {
        JV_CUDA(cudaMemsetAsync(sizes + 1, 0, kPeelBatch * sizeof(int), s));
        for (int b = 0; b < kPeelBatch; ++b) {
            int r = level + b;
            int *fin = (r % 2 == 0) ? fa : fb;
            int *fout = (r % 2 == 0) ? fb : fa;
            count_launch();
            k_peel_round<<<grid, kBlock, 0, s>>>(g, cnt, lev, r + 1, fin, sizes + b, fout,
                                                 sizes + b + 1);
            JV_CHECK_LAUNCH();
        }
        JV_CUDA(cudaMemcpyAsync(hs, sizes, sizeof(hs), cudaMemcpyDeviceToHost, s));
        JV_CUDA(cudaStreamSynchronize(s));
        for (int b = 0; b < kPeelBatch; ++b) {
            if (hs[b] == 0) {
                *nlev_out = level + b;
                return total == n ? JV_OK : JV_ERR_INTERNAL;
            }
            widths.push_back(hs[b]);
            total += hs[b];
            if (total > n) return JV_ERR_INTERNAL;
        }
        JV_CUDA(cudaMemcpyAsync(sizes, sizes + kPeelBatch, sizeof(int), cudaMemcpyDeviceToDevice, s));
    }
}

// Level sets of one DAG: level of every row, rows grouped by level.
int build_levelset(jv_handle h, int which, const Dag &g, Temp &tmp, unsigned *kbuf,
                   unsigned *vbuf, unsigned *kalt, unsigned *valt, int *rtmp) {
    const int n = h->n;
    cudaStream_t s = h->stream;
    LevelSet &L = h->ls[which];
    JV_TRY(halloc_n(h, &L.lev, n));
    JV_TRY(halloc_n(h, &L.rows, n));
    std::vector<int> widths;
    JV_TRY(peel_levels(h, g, L.lev, tmp, &L.nlev, widths));
    JV_TRY(halloc_n(h, &L.ptr, L.nlev + 1));
    // stable sort of (level, row): ascending rows inside every level
    count_launch();
    k_copy_u32<<<grid_for(n, kBlock), kBlock, 0, s>>>(L.lev, kbuf, n);
    JV_CHECK_LAUNCH();
    JV_TRY(iota_i32((int *)vbuf, n, s));
    JV_TRY(radix_sort_pairs(kbuf, vbuf, kalt, valt, n, bits_for(L.nlev - 1), rtmp, s));
    JV_CUDA(cudaMemcpyAsync(L.rows, vbuf, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    JV_TRY(keys_to_ptr(kbuf, n, L.ptr, L.nlev, s));
    L.h_ptr.resize(L.nlev + 1);
    JV_CUDA(cudaMemcpyAsync(L.h_ptr.data(), L.ptr, (L.nlev + 1) * sizeof(int),
                            cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaStreamSynchronize(s));
    for (int l = 0; l < L.nlev; ++l)
        if (L.h_ptr[l + 1] - L.h_ptr[l] != widths[l]) return JV_ERR_INTERNAL;
    return JV_OK;
}

// Per-row costs for the binning: dependencies of the four solves, and for
// the factor the shared-memory words a row needs (its values plus every U
// value it reads: one u_kk per lower entry and one u_kj per update pair).
__global__ void k_row_costs(int n, const int *rowptr, const int *diag, const int *colptr,
                            const int *cdiag, const int *pair_ptr, int *cost) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int rs = rowptr[i], re = rowptr[i + 1], rd = diag[i];
    cost[i] = rd - rs;
    cost[(size_t)n + i] = re - rd - 1;
    cost[2 * (size_t)n + i] = cdiag[i] - colptr[i];
    cost[3 * (size_t)n + i] = colptr[i + 1] - cdiag[i] - 1;
    cost[4 * (size_t)n + i] = (re - rs) + (rd - rs) + (pair_ptr[rd] - pair_ptr[rs]);
}

// Host-side binning of one level structure (see Bins).
// ops[r]: operands a one-lane row r awaits (sets the poll window).
// group[r] (factor only, may be null): 1 when a row above the threshold is
// run by kGroupLanes lanes, kWarp / kGroupLanes rows to a task.
int make_bins(jv_handle h, const LevelSet &L, const int *cost, int threshold, const int *ops,
              Bins &B, const unsigned char *group = nullptr) {
    const int n = h->n;
    cudaStream_t s = h->stream;
    std::vector<int> rows((size_t)n), brows, lo, hi;
    JV_CUDA(cudaMemcpyAsync(rows.data(), L.rows, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaStreamSynchronize(s));
    brows.reserve(n);
    // one-lane tasks of 32 rows where levels are wide; of 16 where they are
    // narrow (under 2,048 rows on average), so a level spreads over more warps
    const int per_task = (long long)n < 2048LL * L.nlev ? 16 : kWarp;
    B.h_task_ptr.assign(L.nlev + 1, 0);
    B.nlong = 0;
    B.ngroup = 0;
    for (int l = 0; l < L.nlev; ++l) {
        B.h_task_ptr[l] = (int)lo.size();
        const int a = L.h_ptr[l], e = L.h_ptr[l + 1];
        const int first = (int)brows.size();
        for (int t = a; t < e; ++t)
            if (cost[rows[t]] <= threshold) brows.push_back(rows[t]);
        const int nshort = (int)brows.size() - first;
        for (int t = 0; t < nshort; t += per_task) {
            lo.push_back(first + t);
            hi.push_back(first + std::min(t + per_task, nshort));
        }
        if (group) {
            const int gfirst = (int)brows.size();
            for (int t = a; t < e; ++t)
                if (cost[rows[t]] > threshold && group[rows[t]]) brows.push_back(rows[t]);
            const int ng = (int)brows.size() - gfirst;
            for (int t = 0; t < ng; t += kWarp / kGroupLanes) {
                lo.push_back(gfirst + t);
                hi.push_back((gfirst + std::min(t + kWarp / kGroupLanes, ng)) | kGroupBit);
                ++B.ngroup;
            }
        }
        for (int t = a; t < e; ++t)
            if (cost[rows[t]] > threshold && !(group && group[rows[t]])) {
                lo.push_back((int)brows.size());
                hi.push_back(((int)brows.size() + 1) | kLongBit);
                brows.push_back(rows[t]);
                ++B.nlong;
            }
    }
    B.ntasks = (int)lo.size();
    B.h_task_ptr[L.nlev] = B.ntasks;
    int most = 0;
    for (int t = 0; t < B.ntasks; ++t)
        if (!(hi[t] & (kLongBit | kGroupBit)))
            for (int p = lo[t]; p < hi[t]; ++p) most = std::max(most, ops[brows[p]]);
    // > 16: some row needs several windows of kPoll (the general poll loop)
    B.window = most <= 2 ? 2 : most <= 4 ? 4 : most <= 8 ? 8 : most <= 16 ? 16 : 17;
    std::vector<int> tlev((size_t)B.ntasks);
    for (int l = 0; l < L.nlev; ++l)
        for (int t = B.h_task_ptr[l]; t < B.h_task_ptr[l + 1]; ++t) tlev[t] = l;
    std::vector<int> ipos((size_t)n);
    for (int p = 0; p < n; ++p) ipos[brows[p]] = p;
    JV_TRY(halloc_n(h, &B.rows, n));
    JV_TRY(halloc_n(h, &B.ipos, n));
    JV_TRY(halloc_n(h, &B.task_lo, B.ntasks));
    JV_TRY(halloc_n(h, &B.task_hi, B.ntasks));
    JV_TRY(halloc_n(h, &B.task_lev, B.ntasks));
    JV_TRY(halloc_n(h, &B.task_ptr, L.nlev + 1));
    JV_CUDA(cudaMemcpyAsync(B.task_lev, tlev.data(), tlev.size() * 4, cudaMemcpyHostToDevice, s));
    JV_CUDA(cudaMemcpyAsync(B.task_ptr, B.h_task_ptr.data(), (size_t)(L.nlev + 1) * 4,
                            cudaMemcpyHostToDevice, s));
    JV_CUDA(cudaMemcpyAsync(B.rows, brows.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    JV_CUDA(cudaMemcpyAsync(B.ipos, ipos.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    JV_CUDA(cudaMemcpyAsync(B.task_lo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice, s));
    JV_CUDA(cudaMemcpyAsync(B.task_hi, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice, s));
    JV_CUDA(cudaStreamSynchronize(s));   // host vectors go out of scope
    return JV_OK;
}

// ---------------------------------------------------------- full structure
int build_all(jv_handle h, const int *rowptr_src, const int *colidx_src) {
    const int n = h->n, nnz = h->nnz;
    cudaStream_t s = h->stream;
    Temp tmp;
    JV_TRY(halloc_n(h, &h->rowptr, n + 1));
    JV_TRY(halloc_n(h, &h->colidx, nnz));
    JV_TRY(halloc_n(h, &h->diag, n));
    JV_CUDA(cudaMemcpyAsync(h->rowptr, rowptr_src, (size_t)(n + 1) * 4, cudaMemcpyDeviceToDevice, s));
    JV_CUDA(cudaMemcpyAsync(h->colidx, colidx_src, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s));
    int *cnt_l;
    JV_TRY(tmp.get(&cnt_l, 1));
    JV_CUDA(cudaMemsetAsync(cnt_l, 0, 4, s));
    JV_CUDA(cudaMemsetAsync(h->status, 0xff, 8, s));
    count_launch();
    k_validate<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, nnz, h->rowptr, h->colidx, h->diag,
                                                      h->status, cnt_l);
    JV_CHECK_LAUNCH();
    JV_CUDA(cudaMemcpyAsync(h->h_status, h->status, 8, cudaMemcpyDeviceToHost, s));
    int h_nl = 0;
    JV_CUDA(cudaMemcpyAsync(&h_nl, cnt_l, 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaStreamSynchronize(s));
    if (*h->h_status != ~0ull) return decode_status(*h->h_status, &h->bad_row);
    h->nnz_lower = h_nl;
    h->nnz_upper = nnz - n - h_nl;

    // scratch for sorts
    const int m = std::max(n, nnz);
    unsigned *kbuf, *vbuf, *kalt, *valt;
    int *rtmp, *row_of;
    JV_TRY(tmp.get(&kbuf, m));
    JV_TRY(tmp.get(&vbuf, m));
    JV_TRY(tmp.get(&kalt, m));
    JV_TRY(tmp.get(&valt, m));
    JV_TRY(tmp.get(&rtmp, radix_tmp_ints(m)));
    JV_TRY(tmp.get(&row_of, nnz));

    // CSC
    JV_TRY(halloc_n(h, &h->colptr, n + 1));
    JV_TRY(halloc_n(h, &h->rowidx, nnz));
    JV_TRY(halloc_n(h, &h->csc2csr, nnz));
    JV_TRY(halloc_n(h, &h->cdiag, n));
    count_launch();
    k_row_of<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, h->rowptr, row_of);
    JV_CHECK_LAUNCH();
    count_launch();
    k_copy_u32<<<grid_for(nnz, kBlock), kBlock, 0, s>>>(h->colidx, kbuf, nnz);
    JV_CHECK_LAUNCH();
    JV_TRY(iota_i32((int *)vbuf, nnz, s));
    JV_TRY(radix_sort_pairs(kbuf, vbuf, kalt, valt, nnz, bits_for(n - 1), rtmp, s));
    JV_TRY(keys_to_ptr(kbuf, nnz, h->colptr, n, s));
    count_launch();
    k_csc_finish<<<grid_for(nnz, kBlock), kBlock, 0, s>>>(nnz, kbuf, vbuf, row_of, h->rowidx,
                                                          h->csc2csr, h->cdiag);
    JV_CHECK_LAUNCH();

    // the four DAGs: lower(A) (factor, L solve), upper(A) (U solve), and the
    // two transposed ones for the adjoint
    const Span none{nullptr, 0, 0};
    Dag gl{{h->rowptr, 0, 0}, {h->diag, 0, 0}, {h->cdiag, 0, 1}, {h->colptr, 1, 0}, h->rowidx,
           none, none, none, none, nullptr};
    Dag gu{{h->diag, 0, 1}, {h->rowptr, 1, 0}, {h->colptr, 0, 0}, {h->cdiag, 0, 0}, h->rowidx,
           none, none, none, none, nullptr};
    Dag gut{{h->colptr, 0, 0}, {h->cdiag, 0, 0}, {h->diag, 0, 1}, {h->rowptr, 1, 0}, h->colidx,
            none, none, none, none, nullptr};
    Dag glt{{h->cdiag, 0, 1}, {h->colptr, 1, 0}, {h->rowptr, 0, 0}, {h->diag, 0, 0}, h->colidx,
            none, none, none, none, nullptr};
    if (h->opt.sym_levels) {
        // Sec. III: levels of lower(A + A^T) (and upper(A + A^T)), the union
        // of lower(A) and lower(A^T); every structure's dependencies are a
        // subset of one of the two, so the factor and all four solves run on
        // them, and the level-order permutation keeps A's triangular split
        gl.cnt2_beg = gut.cnt_beg; gl.cnt2_end = gut.cnt_end;
        gl.dep2_beg = gut.dep_beg; gl.dep2_end = gut.dep_end; gl.idx2 = gut.idx;
        gu.cnt2_beg = glt.cnt_beg; gu.cnt2_end = glt.cnt_end;
        gu.dep2_beg = glt.dep_beg; gu.dep2_end = glt.dep_end; gu.idx2 = glt.idx;
        JV_TRY(build_levelset(h, JV_LOWER, gl, tmp, kbuf, vbuf, kalt, valt, rtmp));
        JV_TRY(build_levelset(h, JV_UPPER, gu, tmp, kbuf, vbuf, kalt, valt, rtmp));
        h->ls[JV_UPPER_T] = h->ls[JV_LOWER];      // shares the device arrays
        h->ls[JV_LOWER_T] = h->ls[JV_UPPER];
    } else {
        JV_TRY(build_levelset(h, JV_LOWER, gl, tmp, kbuf, vbuf, kalt, valt, rtmp));
        JV_TRY(build_levelset(h, JV_UPPER, gu, tmp, kbuf, vbuf, kalt, valt, rtmp));
        JV_TRY(build_levelset(h, JV_UPPER_T, gut, tmp, kbuf, vbuf, kalt, valt, rtmp));
        JV_TRY(build_levelset(h, JV_LOWER_T, glt, tmp, kbuf, vbuf, kalt, valt, rtmp));
    }

    // symbolic factorisation: the update pairs of every strictly lower entry
    int *cnt = (int *)kbuf;   // nnz counts (kbuf is free again)
    JV_TRY(halloc_n(h, &h->pair_ptr, (size_t)nnz + 1));
    count_launch();
    if (h->opt.milu)
        k_pairs<false, true><<<grid_for(n, kWarpsPerBlock), kBlock, 0, s>>>(
            n, h->rowptr, h->colidx, h->diag, cnt, nullptr, nullptr);
    else
        k_pairs<false, false><<<grid_for(n, kWarpsPerBlock), kBlock, 0, s>>>(
            n, h->rowptr, h->colidx, h->diag, cnt, nullptr, nullptr);
    JV_CHECK_LAUNCH();
    JV_TRY(exclusive_scan_i32(cnt, h->pair_ptr, nnz, rtmp, s));
    int np = 0;
    JV_CUDA(cudaMemcpyAsync(&np, h->pair_ptr + nnz, 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaStreamSynchronize(s));
    h->npairs = np;
    JV_TRY(halloc_n(h, &h->pairs, (size_t)np + 1));
    count_launch();
    if (h->opt.milu)
        k_pairs<true, true><<<grid_for(n, kWarpsPerBlock), kBlock, 0, s>>>(
            n, h->rowptr, h->colidx, h->diag, nullptr, h->pair_ptr, h->pairs);
    else
        k_pairs<true, false><<<grid_for(n, kWarpsPerBlock), kBlock, 0, s>>>(
            n, h->rowptr, h->colidx, h->diag, nullptr, h->pair_ptr, h->pairs);
    JV_CHECK_LAUNCH();
    JV_TRY(halloc_n(h, &h->kdiag, nnz));
    count_launch();
    k_kdiag<<<grid_for(nnz, kBlock), kBlock, 0, s>>>(nnz, h->colidx, h->diag, h->kdiag);
    JV_CHECK_LAUNCH();
    // entries the factor updates, and the pairs whose operand it must await
    JV_TRY(halloc_n(h, &h->upd, nnz));
    JV_CUDA(cudaMemsetAsync(h->upd, 0, (size_t)nnz, s));
    {
        Temp ctmp;
        unsigned long long *dc;
        JV_TRY(ctmp.get(&dc, 1));
        JV_CUDA(cudaMemsetAsync(dc, 0, 8, s));
        if (np > 0) {
            count_launch();
            k_mark_targets<<<grid_for(np, kBlock), kBlock, 0, s>>>(np, h->pairs, h->upd);
            JV_CHECK_LAUNCH();
            count_launch();
            k_count_dynamic<<<grid_for(np, kBlock), kBlock, 0, s>>>(np, h->pairs, h->upd, dc);
            JV_CHECK_LAUNCH();
        }
        unsigned long long hc = 0;
        JV_CUDA(cudaMemcpyAsync(&hc, dc, 8, cudaMemcpyDeviceToHost, s));
        JV_CUDA(cudaStreamSynchronize(s));
        h->ndyn_pairs = (long long)hc;
    }

    // the same pairs grouped by target: every entry's updates in ascending
    // step (a stable sort of the step-ordered list by target), for the
    // one-warp-per-row factor, which pulls them per entry
    JV_TRY(halloc_n(h, &h->tpair_ptr, (size_t)nnz + 1));
    JV_TRY(halloc_n(h, &h->tpairs, (size_t)np + 1));
    if (np > 0) {
        Temp ptmp;
        unsigned *step, *pk, *pv, *pka, *pva;
        int *prt;
        JV_TRY(ptmp.get(&step, np));
        JV_TRY(ptmp.get(&pk, np));
        JV_TRY(ptmp.get(&pv, np));
        JV_TRY(ptmp.get(&pka, np));
        JV_TRY(ptmp.get(&pva, np));
        JV_TRY(ptmp.get(&prt, radix_tmp_ints(np)));
        count_launch();
        k_pair_step<<<grid_for(nnz, kBlock), kBlock, 0, s>>>(nnz, h->pair_ptr, step);
        JV_CHECK_LAUNCH();
        count_launch();
        k_pair_target<<<grid_for(np, kBlock), kBlock, 0, s>>>(np, h->pairs, pk, pv);
        JV_CHECK_LAUNCH();
        JV_TRY(radix_sort_pairs(pk, pv, pka, pva, np, bits_for(nnz - 1), prt, s));
        JV_TRY(keys_to_ptr(pk, np, h->tpair_ptr, nnz, s));
        count_launch();
        k_tpairs<<<grid_for(np, kBlock), kBlock, 0, s>>>(np, pv, step, h->pairs, h->upd, h->tpairs);
        JV_CHECK_LAUNCH();
        JV_CUDA(cudaStreamSynchronize(s));
    } else {
        JV_CUDA(cudaMemsetAsync(h->tpair_ptr, 0, ((size_t)nnz + 1) * 4, s));
    }
    JV_TRY(halloc_n(h, &h->row_pull, n));
    JV_TRY(halloc_n(h, &h->edepth, nnz));
    {
        Temp dtmp;
        int *depth;
        JV_TRY(dtmp.get(&depth, nnz));
        count_launch();
        k_row_pull<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, h->rowptr, h->diag, h->tpair_ptr,
                                                          h->tpairs, depth, h->row_pull, h->edepth);
        JV_CHECK_LAUNCH();
        JV_CUDA(cudaStreamSynchronize(s));
    }

    // spmv: rows by length, longest first (a stable counting sort), and the longest row
    std::vector<int> hrp((size_t)n + 1);
    JV_CUDA(cudaMemcpyAsync(hrp.data(), h->rowptr, hrp.size() * 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaStreamSynchronize(s));
    h->maxrow = 0;
    for (int r = 0; r < n; ++r) h->maxrow = std::max(h->maxrow, hrp[r + 1] - hrp[r]);
    {
        std::vector<int> start((size_t)h->maxrow + 2, 0), srows((size_t)n);
        for (int r = 0; r < n; ++r) ++start[h->maxrow - (hrp[r + 1] - hrp[r]) + 1];
        for (int L = 0; L <= h->maxrow; ++L) start[L + 1] += start[L];
        for (int r = 0; r < n; ++r) srows[start[h->maxrow - (hrp[r + 1] - hrp[r])]++] = r;
        JV_TRY(halloc_n(h, &h->spmv_rows, n));
        JV_CUDA(cudaMemcpyAsync(h->spmv_rows, srows.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
        JV_CUDA(cudaStreamSynchronize(s));
        // the rows that split their sum over a warp come first in this order
        const int wide = h->opt.spmv_long_row > 0 ? h->opt.spmv_long_row : kSpmvLongRow;
        h->spmv_wide = 0;
        if (!h->opt.exact)
            while (h->spmv_wide < n && hrp[srows[h->spmv_wide] + 1] - hrp[srows[h->spmv_wide]] > wide)
                ++h->spmv_wide;
    }

    // binned work lists: the four solves and the factor
    int *dcost;
    JV_TRY(tmp.get(&dcost, 5 * (size_t)n));
    count_launch();
    k_row_costs<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, h->rowptr, h->diag, h->colptr, h->cdiag,
                                                       h->pair_ptr, dcost);
    JV_CHECK_LAUNCH();
    std::vector<int> cost(5 * (size_t)n);
    JV_CUDA(cudaMemcpyAsync(cost.data(), dcost, cost.size() * 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaStreamSynchronize(s));
    const int long_deps = h->opt.long_row > 0 ? h->opt.long_row : kLongDeps;
    for (int k = 0; k < 4; ++k)
        JV_TRY(make_bins(h, h->ls[k], cost.data() + (size_t)k * n, long_deps,
                         cost.data() + (size_t)k * n, h->ls[k].bins));
    std::vector<int> fops((size_t)n);          // factor operands: cost minus the row's length
    for (int i = 0; i < n; ++i) fops[i] = cost[4 * (size_t)n + i] - (hrp[i + 1] - hrp[i]);
    // the factor's one-lane slot: the wide one when many rows need 17..32
    // words (e.g. the fill pairs of MILU), else the narrow one
    long long mid_rows = 0;
    for (int i = 0; i < n; ++i) {
        const int c = cost[4 * (size_t)n + i];
        mid_rows += (c > kLaneSlot && c <= kLaneSlotWide);
    }
    h->fslot = 4 * mid_rows >= n ? kLaneSlotWide : kLaneSlot;
    // rows above the one-lane slot that fit a group's share of the warp's
    // shared memory (values and operands at 8 bytes, targets and step ends at
    // 4), and whose L entries depend on each other: kGroupLanes lanes each,
    // four rows to a warp in lockstep.  Rows whose L entries are mostly
    // independent take the pull form on the whole warp: on the power-law
    // matrix four rows of unequal lengths per warp, in the step form or in the
    // pull form, measured 13.4 -> 18.1 ms (FP64 factor), the lockstep loops
    // running at the longest row's length.  Longer rows keep the whole warp.
    std::vector<unsigned char> pull((size_t)n);
    JV_CUDA(cudaMemcpyAsync(pull.data(), h->row_pull, (size_t)n, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaStreamSynchronize(s));
    std::vector<unsigned char> grp((size_t)n, 0);
    const long long gcap = (long long)factor_warp_smem(h->fslot) / (kWarp / kGroupLanes);
    for (int i = 0; i < n; ++i) {
        const long long c = cost[4 * (size_t)n + i], len = hrp[i + 1] - hrp[i];
        grp[i] = (unsigned char)(!pull[i] && c * 8 + (c - len) * 4 <= gcap);
    }
    JV_TRY(make_bins(h, h->ls[JV_LOWER], cost.data() + 4 * (size_t)n, h->fslot, fops.data(),
                     h->fbins, grp.data()));
    JV_TRY(halloc_n(h, &h->kpos, nnz));
    count_launch();
    k_kpos<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, h->rowptr, h->diag, h->colidx, h->fbins.ipos,
                                                  h->kpos);
    JV_CHECK_LAUNCH();
    return plan_bands(h);
}

// ------------------------------------------------------------- reordering
__global__ void k_inverse_perm(int n, const int *perm, int *iperm) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) iperm[perm[r]] = r;
}
__global__ void k_perm_lengths(int n, const int *rowptr, const int *perm, int *len) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) len[r] = rowptr[perm[r] + 1] - rowptr[perm[r]];
}
__global__ void k_perm_entries(int n, const int *rowptr, const int *colidx, const int *perm,
                               const int *iperm, const int *browptr, unsigned *bcol,
                               unsigned *brow, int *src) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int i = perm[r];
    int d = browptr[r];
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p, ++d) {
        bcol[d] = (unsigned)iperm[colidx[p]];
        brow[d] = (unsigned)r;
        src[d] = p;
    }
}
__global__ void k_gather_u32(int m, const unsigned *src, const unsigned *idx, unsigned *dst) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) dst[t] = src[idx[t]];
}
__global__ void k_perm_finish(int m, const unsigned *order, const unsigned *bcol, const int *src,
                              int *colidx_out, int *vmap_out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    unsigned o = order[t];
    colidx_out[t] = (int)bcol[o];
    vmap_out[t] = src[o];
}

}  // namespace

void free_all(jv_handle h) {
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
    for (auto &L : h->ls) L = LevelSet();
    h->fbins = Bins();
    for (auto &C : h->corner) C = CornerPlan();
    for (auto &S : h->scorner) S[0] = S[1] = SolveCorner();
}

int analyze(jv_handle h, const int *rowptr, const int *colidx) {
    const int n = h->n, nnz = h->nnz;
    cudaStream_t s = h->stream;
    int rc = build_all(h, rowptr, colidx);
    if (rc != JV_OK) return rc;
    if (!h->opt.reorder) return plan_stages(h);

    // B = P A P^T with P the level order of lower(A)
    Temp tmp;
    int *perm, *iperm, *browptr, *bcolidx, *vmap, *len, *src;
    unsigned *bcol, *brow, *kbuf, *vbuf, *kalt, *valt;
    int *rtmp;
    JV_TRY(tmp.get(&perm, n));
    JV_TRY(tmp.get(&iperm, n));
    JV_TRY(tmp.get(&browptr, n + 1));
    JV_TRY(tmp.get(&len, n));
    JV_TRY(tmp.get(&bcolidx, nnz));
    JV_TRY(tmp.get(&vmap, nnz));
    JV_TRY(tmp.get(&src, nnz));
    JV_TRY(tmp.get(&bcol, nnz));
    JV_TRY(tmp.get(&brow, nnz));
    JV_TRY(tmp.get(&kbuf, nnz));
    JV_TRY(tmp.get(&vbuf, nnz));
    JV_TRY(tmp.get(&kalt, nnz));
    JV_TRY(tmp.get(&valt, nnz));
    int m = std::max(n, nnz);
    JV_TRY(tmp.get(&rtmp, radix_tmp_ints(m) + scan_tmp_ints(n)));
    JV_CUDA(cudaMemcpyAsync(perm, h->ls[JV_LOWER].rows, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    count_launch();
    k_inverse_perm<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, perm, iperm);
    JV_CHECK_LAUNCH();
    count_launch();
    k_perm_lengths<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, h->rowptr, perm, len);
    JV_CHECK_LAUNCH();
    JV_TRY(exclusive_scan_i32(len, browptr, n, rtmp, s));
    count_launch();
    k_perm_entries<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, h->rowptr, h->colidx, perm, iperm,
                                                          browptr, bcol, brow, src);
    JV_CHECK_LAUNCH();
    // sort by (row, col): stable by column first, then stable by row
    JV_CUDA(cudaMemcpyAsync(kbuf, bcol, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s));
    JV_TRY(iota_i32((int *)vbuf, nnz, s));
    JV_TRY(radix_sort_pairs(kbuf, vbuf, kalt, valt, nnz, bits_for(n - 1), rtmp, s));
    count_launch();
    k_gather_u32<<<grid_for(nnz, kBlock), kBlock, 0, s>>>(nnz, brow, vbuf, kbuf);
    JV_CHECK_LAUNCH();
    JV_TRY(radix_sort_pairs(kbuf, vbuf, kalt, valt, nnz, bits_for(n - 1), rtmp, s));
    count_launch();
    k_perm_finish<<<grid_for(nnz, kBlock), kBlock, 0, s>>>(nnz, vbuf, bcol, src, bcolidx, vmap);
    JV_CHECK_LAUNCH();
    JV_CUDA(cudaStreamSynchronize(s));

    // rebuild every structure on B; keep perm / iperm / vmap
    free_all(h);
    JV_TRY(build_all(h, browptr, bcolidx));
    JV_TRY(halloc_n(h, &h->perm, n));
    JV_TRY(halloc_n(h, &h->iperm, n));
    JV_TRY(halloc_n(h, &h->vmap, nnz));
    JV_CUDA(cudaMemcpyAsync(h->perm, perm, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    JV_CUDA(cudaMemcpyAsync(h->iperm, iperm, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    JV_CUDA(cudaMemcpyAsync(h->vmap, vmap, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s));
    JV_CUDA(cudaStreamSynchronize(s));
    return plan_stages(h);
}

}  // namespace jv
