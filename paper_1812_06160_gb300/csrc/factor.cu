// Numeric ILU(0) on A's own pattern -- Sec. III, Fig. 1 (up-looking: row by
// row, every row "looks up" at the already-factored rows it depends on).
//
// A group of VW lanes owns one row r:
//   for every col k < r of row r, in ascending order:
//       wait until row k is final                     (sync-free mode only)
//       a_rk <- a_rk / a_kk
//       for every update column j > k of row k (split over the VW lanes):
//           if j is in row r (binary search in r's sorted columns):
//               a_rj <- a_rj - a_rk * a_kj
// then the pivot a_rr is tested and the row is published.  Each entry of the
// row receives its updates in ascending k and every product / difference /
// quotient is rounded separately (__dmul_rn etc.), so the result is the same
// IEEE sequence as the serial algorithm, bit for bit.
//
// LEVEL mode: one launch per level of lower(A) (rows of a level are
// independent -- Sec. III: up-looking ILU has the dependency structure of a
// triangular solve).  SYNCFREE mode: one launch; CTAs take tickets in level
// order, and a row waits on a per-row flag of each dependency (the
// point-to-point synchronisation of Sec. III-A, Fig. 4), released after the
// row's values are stored and fenced.
#include "jv_internal.cuh"

namespace jv {
namespace {

struct FactorArgs {
    const int *rowptr, *colidx, *diag;
    const int *rows, *task_lo, *task_hi;
    int task_begin, task_end;     // LEVEL: this level's tasks; SYNCFREE: all tasks
    const void *vals;
    void *lu;
    int *flags;
    unsigned *ticket;             // [0] next ticket, [1] finished CTAs
    unsigned long long *status;
    long long timeout;
    int fault_row;
};

template <class T> struct RN;
template <> struct RN<double> {
    __device__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ static double sub(double a, double b) { return __dsub_rn(a, b); }
    __device__ static double div(double a, double b) { return __ddiv_rn(a, b); }
};
template <> struct RN<float> {
    __device__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ static float sub(float a, float b) { return __fsub_rn(a, b); }
    __device__ static float div(float a, float b) { return __fdiv_rn(a, b); }
};

__device__ __forceinline__ int find_col(const int *__restrict__ col, int lo, int hi, int j) {
    int end = hi;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (__ldg(col + mid) < j) lo = mid + 1; else hi = mid;
    }
    return (lo < end && __ldg(col + lo) == j) ? lo : -1;
}

// Bounded wait on a per-row flag: relaxed polling, then one fence (the
// acquire half of the flag's release/acquire pair).  Gives up after the
// cycle budget, or as soon as another wait of the launch has given up.
__device__ __forceinline__ void wait_flag(const FactorArgs &a, int k, int r) {
    if (ld_relaxed_s32(a.flags + k) == 0) {
        const long long t0 = clock64();
        unsigned it = 0;
        while (ld_relaxed_s32(a.flags + k) == 0) {
            if ((++it & 31u) == 0) {
                if (sf_aborted(a.ticket)) break;
                if (clock64() - t0 > a.timeout) {
                    report(a.status, JV_ERR_TIMEOUT, r);
                    sf_abort(a.ticket);
                    break;
                }
            }
        }
    }
    __threadfence();
}

// Values of an already-published row written by another SM: in sync-free
// mode read them at L2 (relaxed, gpu scope) rather than from a possibly
// stale L1 line; in level mode a kernel boundary separates writer and reader.
template <class T, bool SF>
__device__ __forceinline__ T ld_row(const T *p) {
    if constexpr (SF) {
        using U = typename Bits<T>::U;
        return Bits<T>::from(ld_relaxed(reinterpret_cast<const U *>(p)));
    } else {
        return *p;
    }
}

__device__ __forceinline__ int take_task(const FactorArgs &a, bool syncfree) {
    const int wib = threadIdx.x >> 5;
    if (syncfree) return sf_take_ticket(a.ticket) * kWarpsPerBlock + wib;
    return a.task_begin + blockIdx.x * kWarpsPerBlock + wib;
}

template <class TV, class TL, int VW, bool SF>
__global__ void __launch_bounds__(kBlock) k_ilu0(FactorArgs a) {
    const int task = take_task(a, SF);
    if (task < a.task_end) {
        const int lane = threadIdx.x & 31;
        const int g = lane / VW, sub = lane % VW;
        const unsigned gmask = (VW == 32) ? 0xffffffffu : (((1u << VW) - 1u) << (g * VW));
        const int pos = a.task_lo[task] + g;
        if (pos < a.task_hi[task]) {
            const int r = a.rows[pos];
            const int rs = a.rowptr[r], re = a.rowptr[r + 1], rd = a.diag[r];
            TL *lu = static_cast<TL *>(a.lu);
            const TV *vals = static_cast<const TV *>(a.vals);
            if ((const void *)vals != (const void *)lu)
                for (int p = rs + sub; p < re; p += VW) lu[p] = (TL)vals[p];
            __syncwarp(gmask);
            for (int p = rs; p < rd; ++p) {
                const int k = __ldg(a.colidx + p);
                if (SF) wait_flag(a, k, r);
                const int kd = __ldg(a.diag + k), ke = __ldg(a.rowptr + k + 1);
                const TL lik = RN<TL>::div(lu[p], ld_row<TL, SF>(lu + kd));
                __syncwarp(gmask);
                if (sub == 0) lu[p] = lik;
                for (int q = kd + 1 + sub; q < ke; q += VW) {
                    const int t = find_col(a.colidx, p + 1, re, __ldg(a.colidx + q));
                    if (t >= 0) lu[t] = RN<TL>::sub(lu[t], RN<TL>::mul(lik, ld_row<TL, SF>(lu + q)));
                }
                __syncwarp(gmask);
            }
            if (sub == 0) {
                const double d = (double)lu[rd];
                if (d == 0.0 || !isfinite(d)) report(a.status, JV_ERR_ZERO_PIVOT, r);
            }
            if (SF) {
                __threadfence();
                __syncwarp(gmask);
                if (sub == 0 && r != a.fault_row) st_release(a.flags + r, 1);
            }
        }
    }
    if (SF) sf_finish(a.ticket);
}

template <class TV, class TL, bool SF>
int launch_vw(int vw, int grid, cudaStream_t s, const FactorArgs &a) {
    count_launch();
    switch (vw) {
        case 1: k_ilu0<TV, TL, 1, SF><<<grid, kBlock, 0, s>>>(a); break;
        case 2: k_ilu0<TV, TL, 2, SF><<<grid, kBlock, 0, s>>>(a); break;
        case 4: k_ilu0<TV, TL, 4, SF><<<grid, kBlock, 0, s>>>(a); break;
        case 8: k_ilu0<TV, TL, 8, SF><<<grid, kBlock, 0, s>>>(a); break;
        case 16: k_ilu0<TV, TL, 16, SF><<<grid, kBlock, 0, s>>>(a); break;
        default: k_ilu0<TV, TL, 32, SF><<<grid, kBlock, 0, s>>>(a); break;
    }
    JV_CHECK_LAUNCH();
    return JV_OK;
}

template <class TV, class TL>
int run(jv_handle h, const void *vals, void *lu) {
    const LevelSet &L = h->ls[JV_LOWER];
    cudaStream_t s = h->stream;
    FactorArgs a;
    a.rowptr = h->rowptr;
    a.colidx = h->colidx;
    a.diag = h->diag;
    a.rows = L.rows;
    a.task_lo = L.task_lo;
    a.task_hi = L.task_hi;
    a.vals = vals;
    a.lu = lu;
    a.flags = h->flags;
    a.ticket = h->ticket;
    a.status = h->status;
    a.timeout = h->opt.spin_timeout_cycles > 0 ? h->opt.spin_timeout_cycles : kDefaultSpin;
    a.fault_row = h->opt.fault_row;
    if (h->opt.mode == JV_MODE_SYNCFREE) {
        int rc = fill_u32(h->flags, (size_t)h->n, 0u, s);
        if (rc) return rc;
        a.task_begin = 0;
        a.task_end = L.ntasks;
        return launch_vw<TV, TL, true>(L.vw, grid_for(L.ntasks, kWarpsPerBlock), s, a);
    }
    for (int l = 0; l < L.nlev; ++l) {
        a.task_begin = L.h_task_ptr[l];
        a.task_end = L.h_task_ptr[l + 1];
        int rc = launch_vw<TV, TL, false>(L.vw, grid_for(a.task_end - a.task_begin, kWarpsPerBlock),
                                          s, a);
        if (rc) return rc;
    }
    return JV_OK;
}

}  // namespace

int ilu0_factor(jv_handle h, jv_dtype vals_t, const void *vals, jv_dtype lu_t, void *lu) {
    if (lu_t == JV_F64 && vals_t == JV_F64) return run<double, double>(h, vals, lu);
    if (lu_t == JV_F32 && vals_t == JV_F32) return run<float, float>(h, vals, lu);
    if (lu_t == JV_F32 && vals_t == JV_F64) return run<double, float>(h, vals, lu);
    return JV_ERR_ARG;
}

}  // namespace jv
