// Sparse triangular solves ("stri", Sec. VI): forward substitution with the
// unit lower factor, backward substitution with U, and the two transposed
// solves of the adjoint, all reusing the level structure built by the
// analysis (Sec. III-A: the factor and the solves share one DAG).
//
// One row r computes x_r = (b_r - sum_j t_rj x_j) [/ u_rr], where the
// dependency entries t_rj are a sub-range of row r of the CSR (L, U) or of
// column r of the CSC (U^T, L^T; the value is fetched through csc2csr).
//
// Single right-hand side: a group of VW lanes per row, partial sums reduced
// by a fixed shuffle tree.  Several right-hand sides: one warp per row and
// one lane per right-hand side (row-major n x nrhs, so the lanes read one
// contiguous segment of every dependency row).
//
// LEVEL mode: one launch per level.  SYNCFREE mode: one launch; CTAs take
// tickets in level order and every dependency is awaited on its own output
// word -- the output vector is pre-filled with a sentinel bit pattern and a
// single relaxed store publishes a finished value (no fence, no flag).
#include "jv_internal.cuh"

namespace jv {
namespace {

struct TriArgs {
    Span beg, end;         // dependency range of row r: [beg(r), end(r))
    const int *idx;        // column (CSR) or row (CSC) index of every entry
    const int *vmap;       // CSC -> CSR value position, or nullptr
    const int *diag;
    int unit;              // 1: unit diagonal (L, L^T)
    const int *rows, *task_lo, *task_hi;
    int task_begin, task_end;
    const void *lu, *b;
    void *x;
    int nrhs;
    unsigned *ticket;
    unsigned long long *status;
    long long timeout;
    int fault_row;
};

__device__ __forceinline__ int take_task(const TriArgs &a, bool syncfree) {
    const int wib = threadIdx.x >> 5;
    if (syncfree) return sf_take_ticket(a.ticket) * kWarpsPerBlock + wib;
    return a.task_begin + blockIdx.x * kWarpsPerBlock + wib;
}

// Bounded wait until the dependency's output word no longer holds the
// sentinel; gives up after the cycle budget or when another wait of the
// launch has given up (the value is then a quiet NaN).
template <class TX>
__device__ __forceinline__ TX wait_x(const TX *p, const TriArgs &a, int r) {
    using B = Bits<TX>;
    using U = typename B::U;
    U u = ld_relaxed(reinterpret_cast<const U *>(p));
    if (u == B::kSent) {
        const long long t0 = clock64();
        unsigned it = 0;
        for (;;) {
            u = ld_relaxed(reinterpret_cast<const U *>(p));
            if (u != B::kSent) break;
            if ((++it & 31u) == 0) {
                if (sf_aborted(a.ticket)) {
                    u = B::kCanonNan;
                    break;
                }
                if (clock64() - t0 > a.timeout) {
                    report(a.status, JV_ERR_TIMEOUT, r);
                    sf_abort(a.ticket);
                    u = B::kCanonNan;
                    break;
                }
            }
        }
    }
    return B::from(u);
}

template <class TX>
__device__ __forceinline__ void publish(TX *p, TX v) {
    using B = Bits<TX>;
    typename B::U u = isnan(v) ? B::kCanonNan : B::to(v);
    st_relaxed(reinterpret_cast<typename B::U *>(p), u);
}

template <class TL>
__device__ __forceinline__ TL load_val(const TriArgs &a, int q) {
    const TL *lu = static_cast<const TL *>(a.lu);
    return a.vmap ? __ldg(lu + __ldg(a.vmap + q)) : __ldg(lu + q);
}

template <class TL, class TB, class TX, int VW, bool SF>
__global__ void __launch_bounds__(kBlock) k_trsv(TriArgs a) {
    const int task = take_task(a, SF);
    if (task < a.task_end) {
        const int lane = threadIdx.x & 31;
        const int g = lane / VW, sub = lane % VW;
        const int pos = a.task_lo[task] + g;
        const bool act = pos < a.task_hi[task];
        TX *x = static_cast<TX *>(a.x);
        TL acc = 0;
        int r = 0;
        if (act) {
            r = a.rows[pos];
            const int e = a.end.at(r);
            for (int q = a.beg.at(r) + sub; q < e; q += VW) {
                const int j = __ldg(a.idx + q);
                const TL v = load_val<TL>(a, q);
                const TL xj = SF ? (TL)wait_x<TX>(x + j, a, r) : (TL)x[j];
                acc = fma(v, xj, acc);
            }
        }
#pragma unroll
        for (int o = VW / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (act && sub == 0) {
            TL xr = (TL)static_cast<const TB *>(a.b)[r] - acc;
            if (!a.unit) xr = xr / static_cast<const TL *>(a.lu)[a.diag[r]];
            if (SF) {
                if (r != a.fault_row) publish<TX>(x + r, (TX)xr);
            } else {
                x[r] = (TX)xr;
            }
        }
    }
    if (SF) sf_finish(a.ticket);
}

template <class TL, class TB, class TX, bool SF>
__global__ void __launch_bounds__(kBlock) k_trsm(TriArgs a) {
    const int task = take_task(a, SF);
    if (task < a.task_end) {
        const int lane = threadIdx.x & 31;
        const int r = a.rows[task];
        const int s = a.beg.at(r), e = a.end.at(r);
        const size_t ld = (size_t)a.nrhs;
        TX *x = static_cast<TX *>(a.x);
        const TB *b = static_cast<const TB *>(a.b);
        const bool unit = a.unit;
        const TL d = unit ? (TL)1 : static_cast<const TL *>(a.lu)[a.diag[r]];
        for (int c0 = 0; c0 < a.nrhs; c0 += 32) {
            const int c = c0 + lane;
            const bool ok = c < a.nrhs;
            TL acc = 0;
            for (int q = s; q < e; ++q) {
                const int j = __ldg(a.idx + q);
                const TL v = load_val<TL>(a, q);
                if (ok) {
                    const TX *xp = x + (size_t)j * ld + c;
                    const TL xj = SF ? (TL)wait_x<TX>(xp, a, r) : (TL)*xp;
                    acc = fma(v, xj, acc);
                }
            }
            if (ok) {
                TL xr = (TL)b[(size_t)r * ld + c] - acc;
                if (!unit) xr = xr / d;
                if (SF) {
                    if (r != a.fault_row) publish<TX>(x + (size_t)r * ld + c, (TX)xr);
                } else {
                    x[(size_t)r * ld + c] = (TX)xr;
                }
            }
        }
    }
    if (SF) sf_finish(a.ticket);
}

template <class TL, class TB, class TX, bool SF>
int launch(int vw, bool multi, int grid, cudaStream_t s, const TriArgs &a) {
    count_launch();
    if (multi) {
        k_trsm<TL, TB, TX, SF><<<grid, kBlock, 0, s>>>(a);
    } else {
        switch (vw) {
            case 1: k_trsv<TL, TB, TX, 1, SF><<<grid, kBlock, 0, s>>>(a); break;
            case 2: k_trsv<TL, TB, TX, 2, SF><<<grid, kBlock, 0, s>>>(a); break;
            case 4: k_trsv<TL, TB, TX, 4, SF><<<grid, kBlock, 0, s>>>(a); break;
            case 8: k_trsv<TL, TB, TX, 8, SF><<<grid, kBlock, 0, s>>>(a); break;
            case 16: k_trsv<TL, TB, TX, 16, SF><<<grid, kBlock, 0, s>>>(a); break;
            default: k_trsv<TL, TB, TX, 32, SF><<<grid, kBlock, 0, s>>>(a); break;
        }
    }
    JV_CHECK_LAUNCH();
    return JV_OK;
}

template <class TL, class TB, class TX>
int run(jv_handle h, int structure, const void *lu, const void *b, void *x, int nrhs) {
    const LevelSet &L = h->ls[structure];
    cudaStream_t s = h->stream;
    TriArgs a{};
    switch (structure) {
        case JV_LOWER:
            a.beg = {h->rowptr, 0, 0}; a.end = {h->diag, 0, 0};
            a.idx = h->colidx; a.vmap = nullptr; a.unit = 1; break;
        case JV_UPPER:
            a.beg = {h->diag, 0, 1}; a.end = {h->rowptr, 1, 0};
            a.idx = h->colidx; a.vmap = nullptr; a.unit = 0; break;
        case JV_UPPER_T:
            a.beg = {h->colptr, 0, 0}; a.end = {h->cdiag, 0, 0};
            a.idx = h->rowidx; a.vmap = h->csc2csr; a.unit = 0; break;
        default:  // JV_LOWER_T
            a.beg = {h->cdiag, 0, 1}; a.end = {h->colptr, 1, 0};
            a.idx = h->rowidx; a.vmap = h->csc2csr; a.unit = 1; break;
    }
    a.diag = h->diag;
    a.rows = L.rows;
    a.task_lo = L.task_lo;
    a.task_hi = L.task_hi;
    a.lu = lu;
    a.b = b;
    a.x = x;
    a.nrhs = nrhs;
    a.ticket = h->ticket;
    a.status = h->status;
    a.timeout = h->opt.spin_timeout_cycles > 0 ? h->opt.spin_timeout_cycles : kDefaultSpin;
    a.fault_row = h->opt.fault_row;
    const bool multi = nrhs > 1;
    if (h->opt.mode == JV_MODE_SYNCFREE) {
        int rc = fill_u32(x, (size_t)h->n * nrhs * (sizeof(TX) / 4), ~0u, s);
        if (rc) return rc;
        a.task_begin = 0;
        a.task_end = multi ? h->n : L.ntasks;
        return launch<TL, TB, TX, true>(L.vw, multi, grid_for(a.task_end, kWarpsPerBlock), s, a);
    }
    for (int l = 0; l < L.nlev; ++l) {
        a.task_begin = multi ? L.h_ptr[l] : L.h_task_ptr[l];
        a.task_end = multi ? L.h_ptr[l + 1] : L.h_task_ptr[l + 1];
        int rc = launch<TL, TB, TX, false>(L.vw, multi,
                                           grid_for(a.task_end - a.task_begin, kWarpsPerBlock), s, a);
        if (rc) return rc;
    }
    return JV_OK;
}

}  // namespace

int tri_solve(jv_handle h, int structure, jv_dtype lu_t, const void *lu, jv_dtype b_t,
              const void *b, jv_dtype x_t, void *x, int nrhs) {
    if (lu_t == JV_F64 && b_t == JV_F64 && x_t == JV_F64)
        return run<double, double, double>(h, structure, lu, b, x, nrhs);
    if (lu_t == JV_F32 && b_t == JV_F32 && x_t == JV_F32)
        return run<float, float, float>(h, structure, lu, b, x, nrhs);
    if (lu_t == JV_F32 && b_t == JV_F64 && x_t == JV_F32)
        return run<float, double, float>(h, structure, lu, b, x, nrhs);
    if (lu_t == JV_F32 && b_t == JV_F32 && x_t == JV_F64)
        return run<float, float, double>(h, structure, lu, b, x, nrhs);
    if (lu_t == JV_F32 && b_t == JV_F64 && x_t == JV_F64)
        return run<float, double, double>(h, structure, lu, b, x, nrhs);
    return JV_ERR_ARG;
}

}  // namespace jv
