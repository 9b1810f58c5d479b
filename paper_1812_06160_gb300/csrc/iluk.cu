// ILU(k) symbolic factorisation on the GPU: the level-of-fill pattern that
// ILU(k) factors on.  Javelin takes the sparsity pattern "with desired
// fill-in" and runs its up-looking numeric sweep on it (Sec. II; Sec. V,
// "Incomplete levels"), so ILU(k) = this pattern + the ILU(0) kernels on it.
//
// Row i's pattern: lev(i,j) = 0 for the entries of A's row i; then, for every
// column k < i of the row in ascending order (fill columns included as they
// appear), for every column j > k of row k's FILLED pattern,
// lev(i,j) = min(lev(i,j), lev(i,k) + lev(k,j) + 1), kept when <= K.
//
// Two kernels.  The first computes every row on its own, from the fill-path
// characterisation (below), with no waits.  The second -- for the rows whose
// search outgrows the first one's tables -- runs the row sweep itself:
// row i needs the finished patterns of the rows k it meets, all k < i.  Rows
// are claimed in ascending order by a persistent grid, one warp per row, and
// a row waits (bounded) on a completion word of each row k it uses -- the
// point-to-point scheme of Sec. III-A applied to the symbolic phase.  A row's
// pattern is kept sorted in shared memory (at most kIlukCap entries); row k's
// upper part is merged into it 32 candidates at a time: a candidate already
// present lowers its level, the new ones are inserted by rank.  A finished row
// goes to a pool (one atomic bump per row), then publishes its offset, length
// and diagonal position and raises its completion word (release).
#include <algorithm>

#include "jv_internal.cuh"

#define JV_TRY(x)                     \
    do {                              \
        int rc_ = (x);                \
        if (rc_ != JV_OK) return rc_; \
    } while (0)

namespace jv {
namespace {

constexpr int kIlukCap = 1024;            // entries of one filled row (shared memory)
constexpr int kIlukWarps = 8;             // warps per CTA (two buffers of kIlukCap each)

struct IlukArgs {
    int n, K;
    const int *rowptr, *colidx;
    int *pool_col, *pool_lev;
    unsigned long long pool_cap;
    unsigned long long *pool_top;
    int *row_off, *row_cnt, *row_dpos;
    int *done;
    unsigned *ticket;                     // [0] next row, [1] finished CTAs, [2] abort
    unsigned long long *status;
    long long timeout;
};

__device__ __forceinline__ int ld_acquire_s32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// first position t in [0, c) with a[t] >= v (c if none)
__device__ __forceinline__ int lower_bound(const int *a, int c, int v) {
    int lo = 0, hi = c;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Bounded wait (lane 0) for row k's completion word; false if it gave up.
__device__ bool await_row(const IlukArgs &a, int k, int i) {
    bool ok = true;
    if ((threadIdx.x & 31) == 0) {
        const long long t0 = clock64();
        for (unsigned it = 0; ld_acquire_s32(a.done + k) == 0; ++it) {
            if ((it & 63u) == 63u) {
                if (sf_aborted(a.ticket)) { ok = false; break; }
                if (clock64() - t0 > a.timeout) {
                    report(a.status, JV_ERR_TIMEOUT, i);
                    sf_abort(a.ticket);
                    ok = false;
                    break;
                }
            }
        }
    }
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

__device__ void iluk_row(const IlukArgs &a, int i, int *buf) {
    const int lane = threadIdx.x & 31;
    if (ld_acquire_s32(a.done + i)) return;                   // computed by the path kernel
    int *col = buf, *lev = buf + kIlukCap;                    // current pattern
    int *col2 = buf + 2 * kIlukCap, *lev2 = buf + 3 * kIlukCap;  // merge target
    __shared__ int s_new[kIlukWarps][3][32];                  // (position, col, level) by rank
    int(*nw)[32] = s_new[threadIdx.x >> 5];
    const int rs = __ldg(a.rowptr + i);
    int c = __ldg(a.rowptr + i + 1) - rs;
    if (c > kIlukCap) {
        if (lane == 0) { report(a.status, JV_ERR_NOMEM, i); sf_abort(a.ticket); }
        return;
    }
    for (int t = lane; t < c; t += 32) {
        col[t] = __ldg(a.colidx + rs + t);
        lev[t] = 0;
    }
    __syncwarp();
    for (int p = 0; p < c && col[p] < i; ++p) {
        const int k = col[p];
        const int lik = lev[p];
        if (!await_row(a, k, i)) return;
        (void)ld_acquire_s32(a.done + k);           // every lane acquires what lane 0 saw
        const int kb = a.row_off[k];
        const int ub = kb + a.row_dpos[k] + 1, ue = kb + a.row_cnt[k];
        for (int base = ub; base < ue; base += 32) {
            const int q = base + lane;
            int j = 0, l = 0, pos = 0;
            bool valid = q < ue;
            if (valid) {
                j = a.pool_col[q];
                l = lik + a.pool_lev[q] + 1;
                valid = l <= a.K;
            }
            bool found = false;
            if (valid) {
                pos = lower_bound(col, c, j);
                found = pos < c && col[pos] == j;
                if (found && l < lev[pos]) lev[pos] = l;        // distinct j: distinct pos
            }
            const unsigned newm = __ballot_sync(0xffffffffu, valid && !found);
            const int nnew = __popc(newm);
            __syncwarp();                                       // level updates visible
            if (nnew == 0) continue;
            if (c + nnew > kIlukCap) {
                if (lane == 0) { report(a.status, JV_ERR_NOMEM, i); sf_abort(a.ticket); }
                return;
            }
            if (valid && !found) {                              // candidates are ascending in j
                const int rank = __popc(newm & ((1u << lane) - 1u));
                nw[0][rank] = pos;
                nw[1][rank] = j;
                nw[2][rank] = l;
            }
            __syncwarp();
            // old entry t moves right by the number of new entries placed at or before it
            for (int t = lane; t < c; t += 32) {
                int lo = 0, hi = nnew;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (nw[0][mid] <= t) lo = mid + 1; else hi = mid;
                }
                col2[t + lo] = col[t];
                lev2[t + lo] = lev[t];
            }
            if (lane < nnew) {
                col2[nw[0][lane] + lane] = nw[1][lane];
                lev2[nw[0][lane] + lane] = nw[2][lane];
            }
            __syncwarp();
            int *tc = col, *tl = lev;
            col = col2; lev = lev2; col2 = tc; lev2 = tl;
            c += nnew;
        }
    }
    // publish: pool slot, then offset / length / diagonal, then the completion word
    __syncwarp();
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(a.pool_top, (unsigned long long)c);
    off = __shfl_sync(0xffffffffu, off, 0);
    if (off + (unsigned long long)c > a.pool_cap) {
        // pool too small: the host retries with a larger one; the row stays
        // unpublished and the abort word releases every row waiting on it
        if (lane == 0) { report(a.status, JV_ERR_NOMEM, -1); sf_abort(a.ticket); }
        return;
    }
    for (int t = lane; t < c; t += 32) {
        a.pool_col[off + t] = col[t];
        a.pool_lev[off + t] = lev[t];
    }
    if (lane == 0) {
        a.row_off[i] = (int)off;
        a.row_cnt[i] = c;
        a.row_dpos[i] = lower_bound(col, c, i);
    }
    __syncwarp();
    __threadfence();
    if (lane == 0) st_release(a.done + i, 1);
}

__global__ void __launch_bounds__(kIlukWarps * 32, 1) k_iluk(IlukArgs a) {
    extern __shared__ __align__(16) int dyn_int[];
    int *buf = dyn_int + (size_t)(threadIdx.x >> 5) * 4 * kIlukCap;
    sf_for_each_task(a.ticket, 0, a.n, [&](int i) { iluk_row(a, i, buf); });
    sf_finish(a.ticket);
}

// ---------------------------------------------------- independent rows
// The level of fill of (i, j) is one less than the length of the shortest
// path i -> j in the graph of A whose intermediate vertices are all numbered
// below min(i, j) (the fill-path characterisation of ILU(k)).  So every row
// can be computed on its own, with no waits: a K + 1 layer dynamic program
// over path lengths keeps, for every vertex reached by a path of length L
// from i through vertices < i, the smallest largest-intermediate over such
// paths; (i, w) has level L - 1 at the first L where that is below w.  Per
// warp: three shared-memory hash tables (this layer, the next, the result),
// then a bitonic sort of the result.  A row whose tables overflow is left to
// the point-to-point kernel above (flagged in ovf).
constexpr int kPathSlots = 2048;          // slots of one hash table (power of two)
constexpr int kPathWarps = 4;             // warps per CTA: 3 tables x 2 x 8 KB each

__device__ __forceinline__ bool tab_insert(int *key, int *val, int w, int m) {
    unsigned h = ((unsigned)w * 2654435761u) >> (32 - 11);
    for (int probe = 0; probe < kPathSlots; ++probe, h = (h + 1) & (kPathSlots - 1)) {
        const int k = atomicCAS(key + h, -1, w);
        if (k == -1 || k == w) {
            atomicMin(val + h, m);
            return true;
        }
    }
    return false;
}

__device__ void iluk_row_paths(const IlukArgs &a, int i, int *sm, int *ovf) {
    const int lane = threadIdx.x & 31;
    int *ka = sm, *va = sm + kPathSlots;                      // layer L
    int *kb = sm + 2 * kPathSlots, *vb = sm + 3 * kPathSlots;  // layer L + 1
    int *kf = sm + 4 * kPathSlots, *vf = sm + 5 * kPathSlots;  // result: level of fill
    __shared__ int s_cnt[kPathWarps];
    const int wib = threadIdx.x >> 5;
    for (int t = lane; t < kPathSlots; t += 32) {
        ka[t] = -1; va[t] = 0x7fffffff;
        kf[t] = -1; vf[t] = 0x7fffffff;
    }
    __syncwarp();
    bool bad = false;
    const int rs = __ldg(a.rowptr + i), re = __ldg(a.rowptr + i + 1);
    for (int p = rs + lane; p < re; p += 32) {               // paths of length 1: A's row
        const int w = __ldg(a.colidx + p);
        bad |= !tab_insert(ka, va, w, -1);
        bad |= !tab_insert(kf, vf, w, 0);
    }
    __syncwarp();
    for (int L = 1; L <= a.K && !__any_sync(0xffffffffu, bad); ++L) {
        for (int t = lane; t < kPathSlots; t += 32) { kb[t] = -1; vb[t] = 0x7fffffff; }
        __syncwarp();
        for (int t = lane; t < kPathSlots; t += 32) {
            const int v = ka[t];
            if (v < 0 || v >= i) continue;                     // only vertices < i lie inside
            const int m = max(va[t], v);
            for (int q = __ldg(a.rowptr + v); q < __ldg(a.rowptr + v + 1); ++q)
                bad |= !tab_insert(kb, vb, __ldg(a.colidx + q), m);
        }
        __syncwarp();
        for (int t = lane; t < kPathSlots; t += 32) {
            const int w = kb[t];
            if (w >= 0 && vb[t] < w) bad |= !tab_insert(kf, vf, w, L);
        }
        __syncwarp();
        int *tk = ka, *tv = va;
        ka = kb; va = vb; kb = tk; vb = tv;
    }
    if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) atomicExch(ovf, 1);
        return;
    }
    // gather the result into the other two tables' space and sort it by column
    int *sk = ka, *sv = va;                                   // free now
    if (lane == 0) s_cnt[wib] = 0;
    __syncwarp();
    for (int t = lane; t < kPathSlots; t += 32)
        if (kf[t] >= 0) {
            const int d = atomicAdd(&s_cnt[wib], 1);
            sk[d] = kf[t];
            sv[d] = vf[t];
        }
    __syncwarp();
    const int c = s_cnt[wib];
    if (c > kIlukCap) {
        if (lane == 0) { report(a.status, JV_ERR_NOMEM, i); sf_abort(a.ticket); }
        return;
    }
    int np2 = 1;
    while (np2 < c) np2 <<= 1;
    for (int t = c + lane; t < np2; t += 32) { sk[t] = 0x7fffffff; sv[t] = 0; }
    __syncwarp();
    for (int k = 2; k <= np2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < np2; t += 32) {
                const int x = t ^ j;
                if (x > t && ((sk[t] > sk[x]) == ((t & k) == 0))) {
                    const int k0 = sk[t], v0 = sv[t];
                    sk[t] = sk[x]; sv[t] = sv[x];
                    sk[x] = k0; sv[x] = v0;
                }
            }
            __syncwarp();
        }
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(a.pool_top, (unsigned long long)c);
    off = __shfl_sync(0xffffffffu, off, 0);
    if (off + (unsigned long long)c > a.pool_cap) {
        if (lane == 0) { report(a.status, JV_ERR_NOMEM, -1); sf_abort(a.ticket); }
        return;
    }
    for (int t = lane; t < c; t += 32) {
        a.pool_col[off + t] = sk[t];
        a.pool_lev[off + t] = sv[t];
    }
    if (lane == 0) {
        a.row_off[i] = (int)off;
        a.row_cnt[i] = c;
        a.row_dpos[i] = lower_bound(sk, c, i);
        a.done[i] = 1;                                          // computed here
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kPathWarps * 32, 1) k_iluk_paths(IlukArgs a, int *ovf) {
    extern __shared__ __align__(16) int dyn_int[];
    int *sm = dyn_int + (size_t)(threadIdx.x >> 5) * 6 * kPathSlots;
    const long long nw = (long long)gridDim.x * kPathWarps;
    for (long long i = blockIdx.x * (long long)kPathWarps + (threadIdx.x >> 5); i < a.n; i += nw) {
        if (sf_aborted(a.ticket)) break;
        iluk_row_paths(a, (int)i, sm, ovf);
    }
}

// Row i of the output: copy its pool slot.
__global__ void k_iluk_gather(int n, const int *row_off, const int *row_cnt, const int *fill_rowptr,
                              const int *pool_col, const int *pool_lev, int *out_col, int *out_lev) {
    const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const int i = (int)w, off = row_off[i], cnt = row_cnt[i], dst = fill_rowptr[i];
    for (int t = lane; t < cnt; t += 32) {
        out_col[dst + t] = pool_col[off + t];
        if (out_lev) out_lev[dst + t] = pool_lev[off + t];
    }
}

// A's values on the filled pattern (zeros elsewhere); one warp per row.
template <class T>
__global__ void k_scatter(int n, const int *rowptr, const int *colidx, const T *vals,
                          const int *frowptr, const int *fcolidx, T *fvals) {
    const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const int i = (int)w;
    const int f0 = frowptr[i], f1 = frowptr[i + 1];
    for (int q = f0 + lane; q < f1; q += 32) fvals[q] = (T)0;
    __syncwarp();
    for (int p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) {
        const int t = find_col(fcolidx, f0, f1, colidx[p]);
        if (t >= 0) fvals[t] = vals[p];
    }
}

struct Dev {                                   // device allocations of one call
    std::vector<void *> ptrs;
    ~Dev() { for (void *p : ptrs) cudaFree(p); }
    template <class T> int get(T **p, size_t count) {
        if (cudaMalloc((void **)p, count * sizeof(T) + 16) != cudaSuccess) {
            cudaGetLastError();
            return JV_ERR_NOMEM;
        }
        ptrs.push_back(*p);
        return JV_OK;
    }
};

}  // namespace

int iluk_symbolic(int n, int nnz, const int *rowptr, const int *colidx, int level, int *fill_rowptr,
                  int *fill_colidx, int *fill_level, long long *fill_nnz, cudaStream_t s,
                  int *bad_row) {
    int dev = 0, nsm = 0;
    JV_CUDA(cudaGetDevice(&dev));
    JV_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    Dev d;
    IlukArgs a{};
    a.n = n;
    a.K = level;
    a.rowptr = rowptr;
    a.colidx = colidx;
    a.timeout = kDefaultSpin;
    JV_TRY(d.get(&a.row_off, n));
    JV_TRY(d.get(&a.row_cnt, n));
    JV_TRY(d.get(&a.row_dpos, n));
    JV_TRY(d.get(&a.done, n));
    JV_TRY(d.get(&a.ticket, 8));
    JV_TRY(d.get(&a.status, 1));
    JV_TRY(d.get(&a.pool_top, 1));
    int *ovf;
    JV_TRY(d.get(&ovf, 1));
    const size_t smem = (size_t)kIlukWarps * 4 * kIlukCap * sizeof(int);
    JV_CUDA(cudaFuncSetAttribute(k_iluk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const size_t psmem = (size_t)kPathWarps * 6 * kPathSlots * sizeof(int);
    JV_CUDA(cudaFuncSetAttribute(k_iluk_paths, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)psmem));
    unsigned long long cap = 4ull * nnz + 2ull * n;
    for (int attempt = 0;; ++attempt) {
        Dev pool;
        JV_TRY(pool.get(&a.pool_col, cap));
        JV_TRY(pool.get(&a.pool_lev, cap));
        a.pool_cap = cap;
        JV_CUDA(cudaMemsetAsync(a.done, 0, (size_t)n * 4, s));
        JV_CUDA(cudaMemsetAsync(a.ticket, 0, 8 * 4, s));
        JV_CUDA(cudaMemsetAsync(a.status, 0xff, 8, s));
        JV_CUDA(cudaMemsetAsync(a.pool_top, 0, 8, s));
        JV_CUDA(cudaMemsetAsync(ovf, 0, 4, s));
        // every row on its own; rows whose path tables overflow are left
        // for the point-to-point kernel, which skips the rows already done
        count_launch();
        k_iluk_paths<<<nsm, kPathWarps * 32, psmem, s>>>(a, ovf);
        JV_CHECK_LAUNCH();
        int h_ovf = 0;
        JV_CUDA(cudaMemcpyAsync(&h_ovf, ovf, 4, cudaMemcpyDeviceToHost, s));
        JV_CUDA(cudaStreamSynchronize(s));
        if (h_ovf) {
            JV_CUDA(cudaMemsetAsync(a.ticket, 0, 8 * 4, s));
            count_launch();
            k_iluk<<<nsm, kIlukWarps * 32, smem, s>>>(a);
            JV_CHECK_LAUNCH();
        }
        unsigned long long st = 0, top = 0;
        JV_CUDA(cudaMemcpyAsync(&st, a.status, 8, cudaMemcpyDeviceToHost, s));
        JV_CUDA(cudaMemcpyAsync(&top, a.pool_top, 8, cudaMemcpyDeviceToHost, s));
        JV_CUDA(cudaStreamSynchronize(s));
        int row = -1;
        const int rc = decode_status(st, &row);
        if (rc == JV_ERR_NOMEM && row < 0 && attempt < 8) {     // pool overflow: grow and redo
            cap = std::max(cap * 2, top + 1);
            continue;
        }
        if (rc != JV_OK) {
            if (bad_row) *bad_row = row;
            return rc;
        }
        // fill_rowptr = exclusive scan of the row lengths
        int *rtmp;
        JV_TRY(pool.get(&rtmp, scan_tmp_ints(n + 1)));
        JV_TRY(exclusive_scan_i32(a.row_cnt, fill_rowptr, n, rtmp, s));
        long long total = (long long)top;
        *fill_nnz = total;
        if (total > 0x7fffffffLL) return JV_ERR_NOMEM;
        if (fill_colidx) {
            count_launch();
            k_iluk_gather<<<grid_for((long long)n * 32, kBlock), kBlock, 0, s>>>(
                n, a.row_off, a.row_cnt, fill_rowptr, a.pool_col, a.pool_lev, fill_colidx,
                fill_level);
            JV_CHECK_LAUNCH();
        }
        JV_CUDA(cudaStreamSynchronize(s));
        return JV_OK;
    }
}

int scatter_values(int n, const int *rowptr, const int *colidx, jv_dtype t, const void *vals,
                   const int *frowptr, const int *fcolidx, void *fvals, cudaStream_t s) {
    count_launch();
    const int grid = grid_for((long long)n * 32, kBlock);
    if (t == JV_F64)
        k_scatter<double><<<grid, kBlock, 0, s>>>(n, rowptr, colidx, static_cast<const double *>(vals),
                                                  frowptr, fcolidx, static_cast<double *>(fvals));
    else
        k_scatter<float><<<grid, kBlock, 0, s>>>(n, rowptr, colidx, static_cast<const float *>(vals),
                                                 frowptr, fcolidx, static_cast<float *>(fvals));
    JV_CHECK_LAUNCH();
    return JV_OK;
}

}  // namespace jv
