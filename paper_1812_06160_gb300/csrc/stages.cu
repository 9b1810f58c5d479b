// Two-stage schedules (Sec. III-A, Fig. 2): the stage test that splits the
// levels of every dependency structure into upper-stage levels and
// second-stage material, the hybrid schedule built on it, and the Even-Rows
// corner of the factor (Sec. III-B, Fig. 8) with its one-CTA kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "jv_internal.cuh"

namespace jv {

#define JV_TRY(x)                 \
    do {                          \
        int rc_ = (x);            \
        if (rc_ != JV_OK) return rc_; \
    } while (0)

namespace {

size_t up16(size_t b) { return (b + 15) & ~(size_t)15; }

template <class T> struct RN;
template <> struct RN<double> {
    __device__ static double fms(double a, double b, double c) { return __fma_rn(-a, b, c); }
    __device__ static double div(double a, double b) { return __ddiv_rn(a, b); }
};
template <> struct RN<float> {
    __device__ static float fms(float a, float b, float c) { return __fmaf_rn(-a, b, c); }
    __device__ static float div(float a, float b) { return __fdiv_rn(a, b); }
};

// Per-level sums of a structure's dependency counts end(i) - beg(i) (the row
// density of the stage test).
__global__ void k_level_len(int n, Span beg, Span end, const int *lev, unsigned long long *sum) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    atomicAdd(sum + __ldg(lev + i), (unsigned long long)(end.at(i) - beg.at(i)));
}

// Per-level sums of what a corner row costs in shared memory: its entries,
// and a bound on its program words (3 + 3 per step + 2 per pair, counting the
// steps on rows above the corner too).
__global__ void k_corner_cost(int n, const int *rowptr, const int *diag, const int *pair_ptr,
                              const int *lev, unsigned long long *ent, unsigned long long *words) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int rs = __ldg(rowptr + i), rd = __ldg(diag + i);
    const int l = __ldg(lev + i);
    atomicAdd(ent + l, (unsigned long long)(__ldg(rowptr + i + 1) - rs));
    const long long np = (long long)__ldg(pair_ptr + rd) - __ldg(pair_ptr + rs);
    atomicAdd(words + l, (unsigned long long)(3 + 3ll * (rd - rs) + 2 * np));
}

void spans_of(jv_handle h, int s, Span *beg, Span *end) {
    switch (s) {
        case JV_LOWER:   *beg = {h->rowptr, 0, 0}; *end = {h->diag, 0, 0}; break;
        case JV_UPPER:   *beg = {h->diag, 0, 1};   *end = {h->rowptr, 1, 0}; break;
        case JV_UPPER_T: *beg = {h->colptr, 0, 0}; *end = {h->cdiag, 0, 0}; break;
        default:         *beg = {h->cdiag, 0, 1};  *end = {h->colptr, 1, 0}; break;
    }
}

struct Dev {
    std::vector<void *> p;
    ~Dev() { for (void *q : p) cudaFree(q); }
    template <class T> int get(T **q, size_t count) {
        void *v = nullptr;
        if (cudaMalloc(&v, count * sizeof(T) + 16) != cudaSuccess) {
            cudaGetLastError();
            return JV_ERR_NOMEM;
        }
        p.push_back(v);
        *q = (T *)v;
        return JV_OK;
    }
};

}  // namespace

// The stage test of Sec. III-A on the host: upper[l] = 1 when level l has at
// least stage_min_rows rows, a mean dependency count at most
// stage_max_density times the structure's mean (len = per-level sums; the
// mean is their total over n), and its first row before stage_position * n.
// Returns the first level of the tail of second-stage levels.
int stage_upper(int nlev, const int *level_ptr, const unsigned long long *len, int n,
                const jv_options &opt, unsigned char *upper) {
    unsigned long long total = 0;
    if (len)
        for (int l = 0; l < nlev; ++l) total += len[l];
    const double mean = n > 0 ? (double)total / n : 0.0;
    const int min_rows = opt.stage_min_rows > 0 ? opt.stage_min_rows : 1024;
    const double pos = opt.stage_position;
    for (int l = 0; l < nlev; ++l) {
        const int w = level_ptr[l + 1] - level_ptr[l];
        bool up = w >= min_rows;
        if (up && opt.stage_max_density > 0 && len)
            up = (double)len[l] / w <= opt.stage_max_density * mean;
        if (up && pos > 0 && pos < 1) up = (double)level_ptr[l] < pos * n;
        upper[l] = up ? 1 : 0;
    }
    int t = nlev;
    while (t > 0 && !upper[t - 1]) --t;
    return t;
}

namespace {

// The stage test of Sec. III-A on every level of structure s: at least
// stage_min_rows rows, mean dependency count at most stage_max_density times
// the structure's mean, first row before stage_position * n.  Fills the
// hybrid segments and the tail start of the level set.
int stage_test(jv_handle h, int s) {
    LevelSet &L = h->ls[s];
    const int n = h->n, nlev = L.nlev;
    L.segs.clear();
    L.tail = nlev;
    if (nlev == 0) return JV_OK;
    std::vector<unsigned long long> len(nlev, 0);
    if (h->opt.stage_max_density > 0) {
        Dev d;
        unsigned long long *dsum;
        JV_TRY(d.get(&dsum, nlev));
        JV_CUDA(cudaMemsetAsync(dsum, 0, (size_t)nlev * 8, h->stream));
        Span beg, end;
        spans_of(h, s, &beg, &end);
        count_launch();
        k_level_len<<<grid_for(n, kBlock), kBlock, 0, h->stream>>>(n, beg, end, L.lev, dsum);
        JV_CHECK_LAUNCH();
        JV_CUDA(cudaMemcpyAsync(len.data(), dsum, (size_t)nlev * 8, cudaMemcpyDeviceToHost, h->stream));
        JV_CUDA(cudaStreamSynchronize(h->stream));
    }
    std::vector<unsigned char> upper(nlev);
    L.tail = stage_upper(nlev, L.h_ptr.data(), len.data(), n, h->opt, upper.data());
    for (int l = 0; l < nlev;) {
        if (upper[l]) {
            L.segs.push_back({l, l + 1, false});
            ++l;
        } else {
            int e = l;
            while (e < nlev && !upper[e]) ++e;
            L.segs.push_back({l, e, true});
            l = e;
        }
    }
    return JV_OK;
}

// Build the corner program of the levels [K, nlev) of lower(A) (rows [c, n),
// checked to be the last rows of the handle's order) and upload it.
int build_corner(jv_handle h, int K, size_t tl, CornerPlan &C) {
    const LevelSet &L = h->ls[JV_LOWER];
    const int n = h->n, nnz = h->nnz, nlev = L.nlev;
    cudaStream_t s = h->stream;
    C = CornerPlan();
    const int R = n - L.h_ptr[K];
    if (R <= 0) return JV_OK;
    const int c = n - R;
    std::vector<int> order(R);
    JV_CUDA(cudaMemcpyAsync(order.data(), L.rows + L.h_ptr[K], (size_t)R * 4, cudaMemcpyDeviceToHost, s));
    std::vector<int> hrp(R + 1), hd(R);
    JV_CUDA(cudaMemcpyAsync(hrp.data(), h->rowptr + c, (size_t)(R + 1) * 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaMemcpyAsync(hd.data(), h->diag + c, (size_t)R * 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaStreamSynchronize(s));
    for (int r = 0; r < R; ++r)
        if (order[r] < c) return JV_ERR_ARG;    // the tail levels are not the last rows
    const int E0 = hrp[0], E = nnz - E0;
    if (E >= 65536 || R >= 65536) return JV_ERR_INTERNAL;
    std::vector<int> hcol(E), hkd(E), hpp(E + 1);
    JV_CUDA(cudaMemcpyAsync(hcol.data(), h->colidx + E0, (size_t)E * 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaMemcpyAsync(hkd.data(), h->kdiag + E0, (size_t)E * 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaMemcpyAsync(hpp.data(), h->pair_ptr + E0, (size_t)(E + 1) * 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaStreamSynchronize(s));
    const int P0 = hpp[0], NP = hpp[E] - P0;
    std::vector<int2> hpairs(NP > 0 ? NP : 1);
    if (NP > 0) {
        JV_CUDA(cudaMemcpyAsync(hpairs.data(), h->pairs + P0, (size_t)NP * sizeof(int2),
                                cudaMemcpyDeviceToHost, s));
        JV_CUDA(cudaStreamSynchronize(s));
    }
    std::vector<unsigned short> prog;
    std::vector<int> pptr(R + 1), lptr(nlev - K + 1);
    prog.reserve((size_t)R * 16);
    for (int r = 0; r < R; ++r) {
        const int i = order[r], rl = i - c;
        const int rs = hrp[rl] - E0, rd = hd[rl] - E0;
        int first = rs;                         // first step on a corner column
        while (first < rd && hcol[first] < c) ++first;
        pptr[r] = (int)prog.size();
        prog.push_back((unsigned short)rl);
        prog.push_back((unsigned short)(rd - first));
        prog.push_back((unsigned short)rd);
        for (int e = first; e < rd; ++e) {
            const int j0 = hpp[e] - P0, j1 = hpp[e + 1] - P0;
            prog.push_back((unsigned short)e);
            prog.push_back((unsigned short)(hkd[e] - E0));
            prog.push_back((unsigned short)(j1 - j0));
            for (int j = j0; j < j1; ++j) {
                prog.push_back((unsigned short)(hpairs[j].x - E0));
                prog.push_back((unsigned short)(hpairs[j].y - E0));
            }
        }
    }
    pptr[R] = (int)prog.size();
    if (prog.size() & 1) prog.push_back(0);
    for (int l = K; l <= nlev; ++l) lptr[l - K] = L.h_ptr[l] - L.h_ptr[K];
    C.K = K;
    C.nl = nlev - K;
    C.c = c;
    C.R = R;
    C.E0 = E0;
    C.E = E;
    C.words = (int)prog.size();
    C.smem = up16((size_t)E * tl) + up16((size_t)(R + 1) * 4) + up16((size_t)(C.nl + 1) * 4) +
             up16((size_t)C.words * 2);
    JV_TRY(halloc_n(h, &C.prog_ptr, R + 1));
    JV_TRY(halloc_n(h, &C.lvl_ptr, C.nl + 1));
    JV_TRY(halloc_n(h, &C.prog, prog.size()));
    JV_CUDA(cudaMemcpyAsync(C.prog_ptr, pptr.data(), (size_t)(R + 1) * 4, cudaMemcpyHostToDevice, s));
    JV_CUDA(cudaMemcpyAsync(C.lvl_ptr, lptr.data(), (size_t)(C.nl + 1) * 4, cudaMemcpyHostToDevice, s));
    JV_CUDA(cudaMemcpyAsync(C.prog, prog.data(), prog.size() * 2, cudaMemcpyHostToDevice, s));
    JV_CUDA(cudaStreamSynchronize(s));
    C.use = true;
    return JV_OK;
}

// The corner of each factor dtype: the tail of second-stage levels of
// lower(A), shortened from its top until its values and program fit one CTA's
// shared memory (and 16-bit offsets).
int plan_corner(jv_handle h) {
    const LevelSet &L = h->ls[JV_LOWER];
    const int n = h->n, nlev = L.nlev;
    if (nlev == 0) return JV_OK;
    int budget = 0;
    JV_CUDA(cudaDeviceGetAttribute(&budget, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    Dev d;
    unsigned long long *dent, *dwords;
    JV_TRY(d.get(&dent, nlev));
    JV_TRY(d.get(&dwords, nlev));
    JV_CUDA(cudaMemsetAsync(dent, 0, (size_t)nlev * 8, h->stream));
    JV_CUDA(cudaMemsetAsync(dwords, 0, (size_t)nlev * 8, h->stream));
    count_launch();
    k_corner_cost<<<grid_for(n, kBlock), kBlock, 0, h->stream>>>(n, h->rowptr, h->diag, h->pair_ptr,
                                                                 L.lev, dent, dwords);
    JV_CHECK_LAUNCH();
    std::vector<unsigned long long> ent(nlev), words(nlev);
    JV_CUDA(cudaMemcpyAsync(ent.data(), dent, (size_t)nlev * 8, cudaMemcpyDeviceToHost, h->stream));
    JV_CUDA(cudaMemcpyAsync(words.data(), dwords, (size_t)nlev * 8, cudaMemcpyDeviceToHost, h->stream));
    JV_CUDA(cudaStreamSynchronize(h->stream));
    for (int t = 0; t < 2; ++t) {
        const size_t tl = t == JV_F64 ? 8 : 4;
        unsigned long long E = 0, W = 0;
        int K = nlev;
        while (K > L.tail) {
            const unsigned long long E2 = E + ent[K - 1], W2 = W + words[K - 1];
            const long long R2 = n - L.h_ptr[K - 1];
            const unsigned long long need = E2 * tl + 16 + (R2 + 1) * 4 + 16 + (nlev - K + 2) * 4 + 16 +
                                            (W2 + 1) * 2 + 16;
            if (E2 >= 65536 || R2 >= 65536 || need > (unsigned long long)budget) break;
            E = E2;
            W = W2;
            --K;
        }
        JV_TRY(build_corner(h, K, tl, h->corner[t]));
    }
    return JV_OK;
}

// Staging loops of the one-CTA kernels: each thread keeps kStage loads in
// flight (a plain strided loop would wait for each load before the next).
constexpr int kStage = 8;
template <class Load, class Store>
__device__ __forceinline__ void stage(int count, Load load, Store store) {
    using T = decltype(load(0));
    const int nt = blockDim.x;
    for (int i0 = threadIdx.x; i0 < count; i0 += kStage * nt) {
        T v[kStage];
#pragma unroll
        for (int k = 0; k < kStage; ++k)
            if (i0 + k * nt < count) v[k] = load(i0 + k * nt);
#pragma unroll
        for (int k = 0; k < kStage; ++k)
            if (i0 + k * nt < count) store(i0 + k * nt, v[k]);
    }
}
// dst[i] = src[idx[i]]: the indices, then the values, kStage at a time
template <class T>
__device__ __forceinline__ void stage_gather(int count, const int *idx, const T *src, T *dst) {
    const int nt = blockDim.x;
    for (int i0 = threadIdx.x; i0 < count; i0 += kStage * nt) {
        int p[kStage];
#pragma unroll
        for (int k = 0; k < kStage; ++k) p[k] = i0 + k * nt < count ? __ldg(idx + i0 + k * nt) : -1;
        T v[kStage];
#pragma unroll
        for (int k = 0; k < kStage; ++k)
            if (p[k] >= 0) v[k] = src[p[k]];
#pragma unroll
        for (int k = 0; k < kStage; ++k)
            if (p[k] >= 0) dst[i0 + k * nt] = v[k];
    }
}

struct CornerArgs {
    const int *rowptr, *diag, *kdiag, *pair_ptr;
    const int2 *pairs;
    const int *prog_ptr, *lvl_ptr;
    const unsigned short *prog;
    const void *vals;
    void *lu;
    unsigned long long *status;
    int c, R, E0, E, nl, words;
    int off_pptr, off_lptr, off_prog;
};

// One CTA: the corner's values, program and level pointers in shared memory;
// FACTOR_L of every corner row at once (its steps on rows above the corner,
// whose factors the upper stage has written), then FACTOR_LU of the corner,
// its levels in order separated by __syncthreads, one thread per row; then
// the values back to lu.  Every row applies its steps in ascending column
// order and every step its updates in their stored order, as Fig. 1 does.
template <class TV, class TL>
__global__ void __launch_bounds__(kCornerThreads, 1) k_er_corner(CornerArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    TL *sv = reinterpret_cast<TL *>(smem);
    int *pptr = reinterpret_cast<int *>(smem + a.off_pptr);
    int *lptr = reinterpret_cast<int *>(smem + a.off_lptr);
    unsigned short *prog = reinterpret_cast<unsigned short *>(smem + a.off_prog);
    const int tid = threadIdx.x, nt = blockDim.x;
    const TV *vals = static_cast<const TV *>(a.vals) + a.E0;
    stage(a.E, [&](int e) { return (TL)__ldg(vals + e); }, [&](int e, TL v) { sv[e] = v; });
    stage(a.R + 1, [&](int r) { return __ldg(a.prog_ptr + r); }, [&](int r, int v) { pptr[r] = v; });
    stage(a.nl + 1, [&](int l) { return __ldg(a.lvl_ptr + l); }, [&](int l, int v) { lptr[l] = v; });
    {
        const unsigned *src = reinterpret_cast<const unsigned *>(a.prog);
        unsigned *dst = reinterpret_cast<unsigned *>(prog);
        stage(a.words >> 1, [&](int w) { return __ldg(src + w); }, [&](int w, unsigned v) { dst[w] = v; });
    }
    __syncthreads();
    const TL *lu = static_cast<const TL *>(a.lu);
    // FACTOR_L
    for (int r = tid; r < a.R; r += nt) {
        const int w = pptr[r];
        const int i = a.c + prog[w];
        const int rs = __ldg(a.rowptr + i), pe = __ldg(a.diag + i) - prog[w + 1];
        for (int p = rs; p < pe; ++p) {
            const int e = p - a.E0;
            const TL lik = RN<TL>::div(sv[e], lu[__ldg(a.kdiag + p)]);
            for (int j = __ldg(a.pair_ptr + p), je = __ldg(a.pair_ptr + p + 1); j < je; ++j) {
                const int2 tq = __ldg(a.pairs + j);
                sv[tq.x - a.E0] = RN<TL>::fms(lik, lu[tq.y], sv[tq.x - a.E0]);
            }
            sv[e] = lik;
        }
    }
    __syncthreads();
    // FACTOR_LU of the corner
    for (int l = 0; l < a.nl; ++l) {
        const int r1 = lptr[l + 1];
        for (int r = lptr[l] + tid; r < r1; r += nt) {
            int w = pptr[r];
            const int rl = prog[w], ns = prog[w + 1], dl = prog[w + 2];
            w += 3;
            for (int st = 0; st < ns; ++st) {
                const int e = prog[w], dk = prog[w + 1], np = prog[w + 2];
                w += 3;
                const TL lik = RN<TL>::div(sv[e], sv[dk]);
                for (int k = 0; k < np; ++k, w += 2) {
                    const int t = prog[w];
                    sv[t] = RN<TL>::fms(lik, sv[prog[w + 1]], sv[t]);
                }
                sv[e] = lik;
            }
            const double dd = (double)sv[dl];
            if (dd == 0.0 || !isfinite(dd)) report(a.status, JV_ERR_ZERO_PIVOT, a.c + rl);
        }
        __syncthreads();
    }
    TL *out = static_cast<TL *>(a.lu) + a.E0;
    for (int e = tid; e < a.E; e += nt) out[e] = sv[e];
}

// Build the solve corner of structure s over its levels [K, nlev), if its
// rows are the last rows (forward structures) or the first rows (backward
// ones) of the handle's order and its slots fit 16 bits.  Leaves C unused
// otherwise.
int build_solve_corner(jv_handle h, int s, int K, SolveCorner &C) {
    const LevelSet &L = h->ls[s];
    const int n = h->n, nlev = L.nlev;
    cudaStream_t st = h->stream;
    C = SolveCorner();
    const int R = n - L.h_ptr[K];
    if (R <= 0) return JV_OK;
    const bool forward = s == JV_LOWER || s == JV_UPPER_T;
    const bool unit = s == JV_LOWER || s == JV_LOWER_T;
    const bool reverse = s == JV_LOWER_T;
    const bool csc = s == JV_UPPER_T || s == JV_LOWER_T;
    const int c0 = forward ? n - R : 0, c1 = forward ? n : R;
    std::vector<int> order(R);
    JV_CUDA(cudaMemcpyAsync(order.data(), L.rows + L.h_ptr[K], (size_t)R * 4, cudaMemcpyDeviceToHost, st));
    // ptr[c0..c1], dg[c0..c1) of the CSR (L, U) or CSC (U^T, L^T); CSR diag for the pivots
    std::vector<int> hptr(R + 1), hdg(R), hdiag(R);
    JV_CUDA(cudaMemcpyAsync(hptr.data(), (csc ? h->colptr : h->rowptr) + c0, (size_t)(R + 1) * 4,
                            cudaMemcpyDeviceToHost, st));
    JV_CUDA(cudaMemcpyAsync(hdg.data(), (csc ? h->cdiag : h->diag) + c0, (size_t)R * 4,
                            cudaMemcpyDeviceToHost, st));
    JV_CUDA(cudaMemcpyAsync(hdiag.data(), h->diag + c0, (size_t)R * 4, cudaMemcpyDeviceToHost, st));
    JV_CUDA(cudaStreamSynchronize(st));
    for (int r = 0; r < R; ++r)
        if (order[r] < c0 || order[r] >= c1) return JV_OK;   // not a contiguous end: no corner
    const int q0 = hptr[0], q1 = hptr[R];
    std::vector<int> hidx(q1 - q0 + 1), hvmap(csc ? q1 - q0 + 1 : 1);
    if (q1 > q0) {
        JV_CUDA(cudaMemcpyAsync(hidx.data(), (csc ? h->rowidx : h->colidx) + q0, (size_t)(q1 - q0) * 4,
                                cudaMemcpyDeviceToHost, st));
        if (csc)
            JV_CUDA(cudaMemcpyAsync(hvmap.data(), h->csc2csr + q0, (size_t)(q1 - q0) * 4,
                                    cudaMemcpyDeviceToHost, st));
        JV_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<unsigned short> prog;
    std::vector<int> pptr(R + 1), lptr(nlev - K + 1), vpos, ext;
    std::vector<int> slot_of;                  // outside row -> slot, by binary search on ext
    std::vector<std::pair<int, int>> pending;  // (row, program word) of outside operands
    for (int r = 0; r < R; ++r) {
        const int i = order[r], rl = i - c0;
        int b, e;
        switch (s) {                            // the substitution's dependency range
            case JV_LOWER:   b = hptr[rl];        e = hdg[rl];          break;
            case JV_UPPER:   b = hdg[rl] + 1;     e = hptr[rl + 1];     break;
            case JV_UPPER_T: b = hptr[rl];        e = hdg[rl];          break;
            default:         b = hdg[rl] + 1;     e = hptr[rl + 1];     break;
        }
        const int ne = e - b;
        pptr[r] = (int)prog.size();
        prog.push_back((unsigned short)rl);
        prog.push_back((unsigned short)ne);
        for (int k = 0; k < ne; ++k) {
            const int q = reverse ? e - 1 - k : b + k;
            const int j = hidx[q - q0];
            if (j >= c0 && j < c1) {
                prog.push_back((unsigned short)(j - c0));
            } else {
                pending.push_back({j, (int)prog.size()});
                prog.push_back(0);
            }
            vpos.push_back(csc ? hvmap[q - q0] : q);
        }
        if (!unit) vpos.push_back(hdiag[rl]);
    }
    pptr[R] = (int)prog.size();
    for (auto &pw : pending) ext.push_back(pw.first);
    std::sort(ext.begin(), ext.end());
    ext.erase(std::unique(ext.begin(), ext.end()), ext.end());
    if ((long long)R + (long long)ext.size() >= 65536) return JV_OK;
    for (auto &pw : pending) {
        const int k = (int)(std::lower_bound(ext.begin(), ext.end(), pw.first) - ext.begin());
        prog[pw.second] = (unsigned short)(R + k);
    }
    if (prog.size() & 1) prog.push_back(0);
    for (int l = K; l <= nlev; ++l) lptr[l - K] = L.h_ptr[l] - L.h_ptr[K];
    C.K = K;
    C.nl = nlev - K;
    C.c0 = c0;
    C.R = R;
    C.next = (int)ext.size();
    C.nval = (int)vpos.size();
    C.words = (int)prog.size();
    JV_TRY(halloc_n(h, &C.prog_ptr, R + 1));
    JV_TRY(halloc_n(h, &C.lvl_ptr, C.nl + 1));
    JV_TRY(halloc_n(h, &C.vpos, vpos.size() + 1));
    JV_TRY(halloc_n(h, &C.ext, ext.size() + 1));
    JV_TRY(halloc_n(h, &C.prog, prog.size()));
    JV_CUDA(cudaMemcpyAsync(C.prog_ptr, pptr.data(), (size_t)(R + 1) * 4, cudaMemcpyHostToDevice, st));
    JV_CUDA(cudaMemcpyAsync(C.lvl_ptr, lptr.data(), (size_t)(C.nl + 1) * 4, cudaMemcpyHostToDevice, st));
    if (!vpos.empty())
        JV_CUDA(cudaMemcpyAsync(C.vpos, vpos.data(), vpos.size() * 4, cudaMemcpyHostToDevice, st));
    if (!ext.empty())
        JV_CUDA(cudaMemcpyAsync(C.ext, ext.data(), ext.size() * 4, cudaMemcpyHostToDevice, st));
    JV_CUDA(cudaMemcpyAsync(C.prog, prog.data(), prog.size() * 2, cudaMemcpyHostToDevice, st));
    JV_CUDA(cudaStreamSynchronize(st));
    C.use = true;
    return JV_OK;
}

// Shared memory of a solve corner: x and outside operands, values, program,
// row and level pointers.
size_t solve_corner_smem(const SolveCorner &C, size_t tl, size_t tx) {
    return up16((size_t)(C.R + C.next) * tx) + up16((size_t)C.nval * tl) + up16((size_t)C.words * 2) +
           up16((size_t)(C.R + 1) * 4) + up16((size_t)(C.nl + 1) * 4);
}

// The solve corners of every structure for both value-size classes: the
// tail of second-stage levels, shortened from its top until a bound on its
// shared memory fits one CTA.
int plan_solve_corners(jv_handle h) {
    const int n = h->n;
    int budget = 0;
    JV_CUDA(cudaDeviceGetAttribute(&budget, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    for (int s = 0; s < 4; ++s) {
        const LevelSet &L = h->ls[s];
        const int nlev = L.nlev;
        if (nlev == 0) continue;
        Dev d;
        unsigned long long *dsum;
        JV_TRY(d.get(&dsum, nlev));
        JV_CUDA(cudaMemsetAsync(dsum, 0, (size_t)nlev * 8, h->stream));
        Span beg, end;
        spans_of(h, s, &beg, &end);
        count_launch();
        k_level_len<<<grid_for(n, kBlock), kBlock, 0, h->stream>>>(n, beg, end, L.lev, dsum);
        JV_CHECK_LAUNCH();
        std::vector<unsigned long long> ent(nlev);
        JV_CUDA(cudaMemcpyAsync(ent.data(), dsum, (size_t)nlev * 8, cudaMemcpyDeviceToHost, h->stream));
        JV_CUDA(cudaStreamSynchronize(h->stream));
        for (int k = 0; k < 2; ++k) {
            const size_t tl = k == 0 ? 8 : 4, tx = tl;
            unsigned long long E = 0;
            int K = nlev;
            while (K > L.tail) {
                const unsigned long long E2 = E + ent[K - 1];
                const unsigned long long R2 = (unsigned long long)(n - L.h_ptr[K - 1]);
                const unsigned long long need = (R2 + E2) * tx + 16 + (E2 + R2) * tl + 16 +
                                                (2 * R2 + E2 + 1) * 2 + 16 + (R2 + 1) * 4 + 16 +
                                                (unsigned long long)(nlev - K + 2) * 4 + 16;
                if (R2 + E2 >= 65536 || need > (unsigned long long)budget) break;
                E = E2;
                --K;
            }
            JV_TRY(build_solve_corner(h, s, K, h->scorner[s][k]));
        }
    }
    return JV_OK;
}

struct SolveCornerArgs {
    const int *prog_ptr, *lvl_ptr, *vpos, *ext;
    const unsigned short *prog;
    const void *lu, *b;
    void *x;
    int c0, R, next, nval, words, nl, unit;
    int off_val, off_prog, off_pptr, off_lptr;
};

// One CTA: x of the corner rows (first b, cast as the substitution casts it)
// and the outside operands in shared memory, with the values and programs;
// then the corner's levels in order, separated by __syncthreads, one thread
// per row: s = b_r; s = s - t_rj x_j in the serial order; x_r = s [/ u_rr].
template <class TL, class TB, class TX>
__global__ void __launch_bounds__(kCornerThreads, 1) k_trsv_corner(SolveCornerArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    TX *X = reinterpret_cast<TX *>(smem);
    TL *val = reinterpret_cast<TL *>(smem + a.off_val);
    unsigned short *prog = reinterpret_cast<unsigned short *>(smem + a.off_prog);
    int *pptr = reinterpret_cast<int *>(smem + a.off_pptr);
    int *lptr = reinterpret_cast<int *>(smem + a.off_lptr);
    const int tid = threadIdx.x, nt = blockDim.x;
    const TB *b = static_cast<const TB *>(a.b) + a.c0;
    const TX *x = static_cast<const TX *>(a.x);
    const TL *lu = static_cast<const TL *>(a.lu);
    stage(a.R, [&](int l) { return (TX)(TL)b[l]; }, [&](int l, TX v) { X[l] = v; });
    stage_gather(a.next, a.ext, x, X + a.R);
    stage_gather(a.nval, a.vpos, lu, val);
    stage(a.R + 1, [&](int r) { return __ldg(a.prog_ptr + r); }, [&](int r, int v) { pptr[r] = v; });
    stage(a.nl + 1, [&](int l) { return __ldg(a.lvl_ptr + l); }, [&](int l, int v) { lptr[l] = v; });
    {
        const unsigned *src = reinterpret_cast<const unsigned *>(a.prog);
        unsigned *dst = reinterpret_cast<unsigned *>(prog);
        stage(a.words >> 1, [&](int w) { return __ldg(src + w); }, [&](int w, unsigned v) { dst[w] = v; });
    }
    __syncthreads();
    for (int l = 0; l < a.nl; ++l) {
        const int r1 = lptr[l + 1];
        for (int r = lptr[l] + tid; r < r1; r += nt) {
            const int w = pptr[r];
            const int rl = prog[w], ne = prog[w + 1];
            const int vb = w - 2 * r + (a.unit ? 0 : r);
            TL s = (TL)X[rl];
            for (int e = 0; e < ne; ++e) s = RN<TL>::fms(val[vb + e], (TL)X[prog[w + 2 + e]], s);
            if (!a.unit) s = RN<TL>::div(s, val[vb + ne]);
            X[rl] = (TX)s;
        }
        __syncthreads();
    }
    TX *out = static_cast<TX *>(a.x) + a.c0;
    for (int l = tid; l < a.R; l += nt) out[l] = X[l];
}

}  // namespace

int plan_stages(jv_handle h) {
    for (int s = 0; s < 4; ++s) JV_TRY(stage_test(h, s));
    for (auto &C : h->corner) C = CornerPlan();
    for (auto &S : h->scorner) S[0] = S[1] = SolveCorner();
    if (h->opt.er_corner) {
        JV_TRY(plan_corner(h));
        JV_TRY(plan_solve_corners(h));
    }
    return JV_OK;
}

const SolveCorner *solve_corner_of(jv_handle h, int structure, size_t tl, size_t tx) {
    const SolveCorner &C = h->scorner[structure][tl == 4 && tx == 4 ? 1 : 0];
    return C.use ? &C : nullptr;
}

int corner_solve(jv_handle h, int structure, const SolveCorner &C, jv_dtype lu_t, const void *lu,
                 jv_dtype b_t, const void *b, jv_dtype x_t, void *x, cudaStream_t s) {
    const size_t tl = lu_t == JV_F64 ? 8 : 4, tx = x_t == JV_F64 ? 8 : 4;
    SolveCornerArgs a{};
    a.prog_ptr = C.prog_ptr;
    a.lvl_ptr = C.lvl_ptr;
    a.vpos = C.vpos;
    a.ext = C.ext;
    a.prog = C.prog;
    a.lu = lu;
    a.b = b;
    a.x = x;
    a.c0 = C.c0;
    a.R = C.R;
    a.next = C.next;
    a.nval = C.nval;
    a.words = C.words;
    a.nl = C.nl;
    a.unit = structure == JV_LOWER || structure == JV_LOWER_T;
    a.off_val = (int)up16((size_t)(C.R + C.next) * tx);
    a.off_prog = a.off_val + (int)up16((size_t)C.nval * tl);
    a.off_pptr = a.off_prog + (int)up16((size_t)C.words * 2);
    a.off_lptr = a.off_pptr + (int)up16((size_t)(C.R + 1) * 4);
    const int smem = (int)solve_corner_smem(C, tl, tx);
#define JV_SCORNER(TL_, TB_, TX_)                                                            \
    JV_CUDA(cudaFuncSetAttribute(k_trsv_corner<TL_, TB_, TX_>,                                \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem));         \
    count_launch();                                                                          \
    k_trsv_corner<TL_, TB_, TX_><<<1, kCornerThreads, smem, s>>>(a);
    if (lu_t == JV_F64 && b_t == JV_F64 && x_t == JV_F64) { JV_SCORNER(double, double, double) }
    else if (lu_t == JV_F32 && b_t == JV_F32 && x_t == JV_F32) { JV_SCORNER(float, float, float) }
    else if (lu_t == JV_F32 && b_t == JV_F64 && x_t == JV_F32) { JV_SCORNER(float, double, float) }
    else if (lu_t == JV_F32 && b_t == JV_F32 && x_t == JV_F64) { JV_SCORNER(float, float, double) }
    else if (lu_t == JV_F32 && b_t == JV_F64 && x_t == JV_F64) { JV_SCORNER(float, double, double) }
    else return JV_ERR_ARG;
#undef JV_SCORNER
    JV_CHECK_LAUNCH();
    return JV_OK;
}

bool has_sync_free(jv_handle h, const LevelSet &L, int lend) {
    if (lend <= 0 || h->opt.mode == JV_MODE_LEVEL) return false;
    if (h->opt.mode == JV_MODE_SYNCFREE) return true;
    for (const Seg &g : L.segs)
        if (g.l0 < lend && g.sf) return true;
    return false;
}

int hybrid_launches(const LevelSet &L, int lend) {
    int k = 0;
    for (const Seg &g : L.segs) {
        if (g.l0 >= lend) break;
        const int l1 = std::min(g.l1, lend);
        k += g.sf ? 1 : l1 - g.l0;
    }
    return k;
}

int corner_factor(jv_handle h, jv_dtype vals_t, const void *vals, jv_dtype lu_t, void *lu,
                  cudaStream_t s) {
    const CornerPlan &C = h->corner[lu_t];
    if (!C.use) return JV_OK;
    const size_t tl = lu_t == JV_F64 ? 8 : 4;
    CornerArgs a{};
    a.rowptr = h->rowptr;
    a.diag = h->diag;
    a.kdiag = h->kdiag;
    a.pair_ptr = h->pair_ptr;
    a.pairs = h->pairs;
    a.prog_ptr = C.prog_ptr;
    a.lvl_ptr = C.lvl_ptr;
    a.prog = C.prog;
    a.vals = vals;
    a.lu = lu;
    a.status = h->status;
    a.c = C.c;
    a.R = C.R;
    a.E0 = C.E0;
    a.E = C.E;
    a.nl = C.nl;
    a.words = C.words;
    a.off_pptr = (int)up16((size_t)C.E * tl);
    a.off_lptr = a.off_pptr + (int)up16((size_t)(C.R + 1) * 4);
    a.off_prog = a.off_lptr + (int)up16((size_t)(C.nl + 1) * 4);
    const int smem = a.off_prog + (int)up16((size_t)C.words * 2);
#define JV_CORNER(TV_, TL_)                                                                   \
    JV_CUDA(cudaFuncSetAttribute(k_er_corner<TV_, TL_>,                                        \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem));          \
    count_launch();                                                                           \
    k_er_corner<TV_, TL_><<<1, kCornerThreads, smem, s>>>(a);
    if (lu_t == JV_F64 && vals_t == JV_F64) { JV_CORNER(double, double) }
    else if (lu_t == JV_F32 && vals_t == JV_F32) { JV_CORNER(float, float) }
    else if (lu_t == JV_F32 && vals_t == JV_F64) { JV_CORNER(double, float) }
    else return JV_ERR_ARG;
#undef JV_CORNER
    JV_CHECK_LAUNCH();
    return JV_OK;
}

}  // namespace jv
