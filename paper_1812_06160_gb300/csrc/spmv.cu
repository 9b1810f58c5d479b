// CSR spmv (Sec. I: with stri the kernel a preconditioned Krylov method
// repeats; Sec. VI defers it), the pattern-restricted outer product used by
// the factor gradient, and the gathers that move values and vectors into the
// level order of a reordered handle (Sec. III).
#include <cstdint>

#include "jv_internal.cuh"

namespace jv {
namespace {

template <class T> struct RN;
template <> struct RN<double> {
    __device__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    __device__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
};
template <> struct RN<float> {
    __device__ static float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    __device__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
};

// One long row r summed by the whole warp (default mode): lane l takes the
// entries p0 + l, p0 + l + 32, ... in ascending order, U of them per step,
// the indices and values of step i+1 loading while the gathers of step i
// are in flight; then a butterfly of xor shuffles adds the 32 partial sums.
// Addition is commutative, so every lane of the butterfly ends with the same
// bits, and the shape of the tree is fixed: the result does not depend on
// timing.  Called by all 32 lanes.
template <class T, int U>
__device__ __forceinline__ void spmv_row_warp(int r, const int *__restrict__ rowptr,
                                              const int *__restrict__ colidx,
                                              const T *__restrict__ vals, const T *__restrict__ x,
                                              T *y, T alpha, T beta, int has_alpha, int has_beta) {
    const int lane = threadIdx.x & 31;
    const int p0 = __ldg(rowptr + r), p1 = __ldg(rowptr + r + 1);
    int j[U];
    T a[U];
#pragma unroll
    for (int k = 0; k < U; ++k)
        if (p0 + lane + 32 * k < p1) { j[k] = __ldg(colidx + p0 + lane + 32 * k); a[k] = __ldg(vals + p0 + lane + 32 * k); }
    T s = 0;
    for (int c = p0 + lane; c < p1; c += 32 * U) {
        T xv[U];
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (c + 32 * k < p1) xv[k] = __ldg(x + j[k]);
        int jn[U];
        T an[U];
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (c + 32 * (U + k) < p1) { jn[k] = __ldg(colidx + c + 32 * (U + k)); an[k] = __ldg(vals + c + 32 * (U + k)); }
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (c + 32 * k < p1) s = RN<T>::fma(a[k], xv[k], s);
#pragma unroll
        for (int k = 0; k < U; ++k) { j[k] = jn[k]; a[k] = an[k]; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = RN<T>::add(s, __shfl_xor_sync(0xffffffffu, s, o));
    if (lane != 0) return;
    T v = has_alpha ? RN<T>::mul(alpha, s) : s;
    if (has_beta) v = RN<T>::fma(beta, y[r], v);
    y[r] = v;
}

// One lane per row, in the serial order of every row (each product added
// with one fused multiply-add in ascending column order -- the serial spmv's
// sequence, so the result is identical to it).  A warp instruction of the
// FP64 pipe costs 64 cycles on this part whatever its active lanes, and a
// row's chain of fused multiply-adds cannot be split without changing the
// result, so the rows are taken in order of length, longest first (the
// analysis sorts them once): the 32 rows of a warp have about the same
// length, every FP64 instruction works on 32 rows, and the longest chains
// start first.  A lane streams its row in chunks of U entries through a
// three-stage pipeline -- indices and values of chunk c+2 loading, x of chunk
// c+1 being gathered, chunk c being summed -- so a long row's loads stay
// ahead of its chain.  Short rows take short chunks and more CTAs per SM
// (fewer registers, more warps to hide the gathers; see spmv() for the
// choice by the longest row); long rows take chunks of 4 and four CTAs per
// SM (the power-law matrix: 0.80 -> 0.62 ms).
// WIDE: the first nwide rows of the order (the longest, default mode) take a
// warp each (spmv_row_warp) and the remaining rows follow one per lane.
template <class T, int U, int MINB, bool WIDE>
__global__ void __launch_bounds__(kBlock, MINB) k_spmv(int n, int nwide, const int *__restrict__ srows,
                                                    const int *__restrict__ rowptr,
                                                    const int *__restrict__ colidx,
                                                    const T *__restrict__ vals,
                                                    const T *__restrict__ x, T *y, T alpha, T beta,
                                                    int has_alpha, int has_beta) {
    long long t = blockIdx.x * (long long)kBlock + threadIdx.x;
    if constexpr (WIDE) {
        if ((t >> 5) < nwide) {                            // warp-uniform
            spmv_row_warp<T, U>(__ldg(srows + (t >> 5)), rowptr, colidx, vals, x, y, alpha, beta,
                                has_alpha, has_beta);
            return;
        }
        t -= 31ll * nwide;                                 // position nwide + (t - 32 nwide)
    }
    // lanes past the last row take an empty row (they stay for the warp votes)
    const int r = t < n ? __ldg(srows + t) : -1;
    const int p0 = r >= 0 ? __ldg(rowptr + r) : 0, p1 = r >= 0 ? __ldg(rowptr + r + 1) : 0;
    int j2[U];
    T a1[U], x1[U], a2[U];
    // chunk 0: indices and values, then its gathers; chunk 1: indices and values
#pragma unroll
    for (int k = 0; k < U; ++k)
        if (p0 + k < p1) { j2[k] = __ldg(colidx + p0 + k); a1[k] = __ldg(vals + p0 + k); }
#pragma unroll
    for (int k = 0; k < U; ++k)
        if (p0 + k < p1) x1[k] = __ldg(x + j2[k]);
#pragma unroll
    for (int k = 0; k < U; ++k)
        if (p0 + U + k < p1) { j2[k] = __ldg(colidx + p0 + U + k); a2[k] = __ldg(vals + p0 + U + k); }
    T s = 0;
    // a warp-uniform trip count (the longest row of the warp): the warp votes
    // in the loop need every lane
    const int nch = __reduce_max_sync(0xffffffffu, (unsigned)((p1 - p0 + U - 1) / U));
    for (int ci = 0, c = p0; ci < nch; ++ci, c += U) {
        T x2[U];
#pragma unroll
        for (int k = 0; k < U; ++k)                       // gathers of chunk c+1
            if (c + U + k < p1) x2[k] = __ldg(x + j2[k]);
        T a3[U];
#pragma unroll
        for (int k = 0; k < U; ++k)                       // indices and values of chunk c+2
            if (c + 2 * U + k < p1) { j2[k] = __ldg(colidx + c + 2 * U + k); a3[k] = __ldg(vals + c + 2 * U + k); }
        // the chain of chunk c; the lanes' rows have about the same length, so
        // the tail test is made warp-uniform first: an FP64 instruction whose
        // lanes are all switched off still costs its 64 cycles of the pipe
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (__any_sync(0xffffffffu, c + k < p1) && c + k < p1) s = RN<T>::fma(a1[k], x1[k], s);
#pragma unroll
        for (int k = 0; k < U; ++k) {
            a1[k] = a2[k];
            x1[k] = x2[k];
            a2[k] = a3[k];
        }
    }
    if (r < 0) return;
    T v = has_alpha ? RN<T>::mul(alpha, s) : s;            // alpha = 1: the product is s exactly
    if (has_beta) v = RN<T>::fma(beta, y[r], v);
    y[r] = v;
}

// The same lane-per-row serial sums (bit for bit), with each lane's indices
// and values read a quad at a time: 16-byte loads of 4 indices, and of 4
// floats or 2 x 2 doubles, at positions that are multiples of 4.  A lane's
// chunks start at the quad holding its first entry, so entries of the
// neighbouring rows are loaded and skipped (a quad is loaded only when it
// holds an entry of the row, and read element by element where it would
// pass the end of the arrays).  A load instruction of 32 lanes on 32
// different rows is 32 L2 requests whatever its width, and on the power-law
// matrix the L2's request rate is what binds (tag lookups 80 % busy): quads
// cut the index and value requests from 2 to 0.75 per entry; the x gathers,
// one request per entry in any form, remain.  The chains may take up to 3
// more (skipped) steps than the row's length, since the lanes' rows start
// at different offsets within their quads.
template <class T, int U>
__device__ __forceinline__ void load_quads(const int *__restrict__ colidx, const T *__restrict__ vals,
                                           int nnz, int c, int p0, int p1, int (&j)[U], T (&v)[U]) {
#pragma unroll
    for (int q = 0; q < U / 4; ++q) {
        const int b = c + 4 * q;
        if (b >= p1 || b + 3 < p0) continue;             // no entry of the row in this quad
        if (b + 3 < nnz) {
            const int4 jj = __ldg(reinterpret_cast<const int4 *>(colidx + b));
            j[4 * q] = jj.x; j[4 * q + 1] = jj.y; j[4 * q + 2] = jj.z; j[4 * q + 3] = jj.w;
            if constexpr (sizeof(T) == 4) {
                const float4 vv = __ldg(reinterpret_cast<const float4 *>(vals + b));
                v[4 * q] = vv.x; v[4 * q + 1] = vv.y; v[4 * q + 2] = vv.z; v[4 * q + 3] = vv.w;
            } else {
                if (b + 1 >= p0) {
                    const double2 lo = __ldg(reinterpret_cast<const double2 *>(vals + b));
                    v[4 * q] = lo.x; v[4 * q + 1] = lo.y;
                }
                if (b + 2 < p1) {
                    const double2 hi = __ldg(reinterpret_cast<const double2 *>(vals + b + 2));
                    v[4 * q + 2] = hi.x; v[4 * q + 3] = hi.y;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (b + k >= p0 && b + k < p1) { j[4 * q + k] = __ldg(colidx + b + k); v[4 * q + k] = __ldg(vals + b + k); }
        }
    }
}

template <class T, int U, int MINB, bool WIDE>
__global__ void __launch_bounds__(kBlock, MINB) k_spmv_quad(int n, int nnz, int nwide,
                                                         const int *__restrict__ srows,
                                                         const int *__restrict__ rowptr,
                                                         const int *__restrict__ colidx,
                                                         const T *__restrict__ vals,
                                                         const T *__restrict__ x, T *y, T alpha,
                                                         T beta, int has_alpha, int has_beta) {
    long long t = blockIdx.x * (long long)kBlock + threadIdx.x;
    if constexpr (WIDE) {
        if ((t >> 5) < nwide) {                            // warp-uniform
            spmv_row_warp<T, U>(__ldg(srows + (t >> 5)), rowptr, colidx, vals, x, y, alpha, beta,
                                has_alpha, has_beta);
            return;
        }
        t -= 31ll * nwide;
    }
    const int r = t < n ? __ldg(srows + t) : -1;
    const int p0 = r >= 0 ? __ldg(rowptr + r) : 0, p1 = r >= 0 ? __ldg(rowptr + r + 1) : 0;
    const int a0 = p0 & ~3;                                // the quad holding the first entry
    int j2[U];
    T a1[U], x1[U], a2[U];
    load_quads<T, U>(colidx, vals, nnz, a0, p0, p1, j2, a1);
#pragma unroll
    for (int k = 0; k < U; ++k)
        if (a0 + k >= p0 && a0 + k < p1) x1[k] = __ldg(x + j2[k]);
    load_quads<T, U>(colidx, vals, nnz, a0 + U, p0, p1, j2, a2);
    T s = 0;
    const int nch = __reduce_max_sync(0xffffffffu, (unsigned)(p1 > p0 ? (p1 - a0 + U - 1) / U : 0));
    for (int ci = 0, c = a0; ci < nch; ++ci, c += U) {
        T x2[U];
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (c + U + k >= p0 && c + U + k < p1) x2[k] = __ldg(x + j2[k]);
        T a3[U];
        load_quads<T, U>(colidx, vals, nnz, c + 2 * U, p0, p1, j2, a3);
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const bool in = c + k >= p0 && c + k < p1;
            if (__any_sync(0xffffffffu, in) && in) s = RN<T>::fma(a1[k], x1[k], s);
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            a1[k] = a2[k];
            x1[k] = x2[k];
            a2[k] = a3[k];
        }
    }
    if (r < 0) return;
    T v = has_alpha ? RN<T>::mul(alpha, s) : s;
    if (has_beta) v = RN<T>::fma(beta, y[r], v);
    y[r] = v;
}

// 16-byte vector of T: four floats or two doubles
template <class T> struct Vec16;
template <> struct Vec16<float> {
    using V = float4;
    static constexpr int k = 4;
    __device__ static float at(const V &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
};
template <> struct Vec16<double> {
    using V = double2;
    static constexpr int k = 2;
    __device__ static double at(const V &v, int e) { return e == 0 ? v.x : v.y; }
};

// g[p] = alpha * sum_c a[i,c] b[j,c] over the entries p = (i, j) of one part of
// row i: one warp per row, one lane per entry, the sum over c in order.  VEC:
// the rows of a and b are 16-byte aligned and a whole number of 16-byte
// vectors long, so each lane reads them 16 bytes at a time (the kernel is
// bound by load instructions); the fused multiply-adds keep the order c.
template <class T, bool VEC>
__global__ void __launch_bounds__(kBlock) k_masked_outer(int n, const int *rowptr, const int *colidx,
                                                         const int *diag, int which, const T *A,
                                                         const T *B, int nrhs, T alpha, T *g) {
    const int lane = threadIdx.x & 31;
    const long long i = (blockIdx.x * (long long)kBlock + threadIdx.x) >> 5;
    if (i >= n) return;
    const int lo = which == 0 ? rowptr[i] : diag[i];
    const int hi = which == 0 ? diag[i] : rowptr[i + 1];
    const size_t ld = (size_t)nrhs;
    const T *ai = A + i * ld;
    for (int p = lo + lane; p < hi; p += 32) {
        const T *bj = B + (size_t)__ldg(colidx + p) * ld;
        T s = 0;
        if constexpr (VEC) {
            using W = Vec16<T>;
            const typename W::V *a4 = reinterpret_cast<const typename W::V *>(ai);
            const typename W::V *b4 = reinterpret_cast<const typename W::V *>(bj);
            for (int c = 0; c < nrhs / W::k; ++c) {
                const typename W::V x = __ldg(a4 + c), y = __ldg(b4 + c);
#pragma unroll
                for (int e = 0; e < W::k; ++e) s = RN<T>::fma(W::at(x, e), W::at(y, e), s);
            }
        } else {
            for (int c = 0; c < nrhs; ++c) s = RN<T>::fma(__ldg(ai + c), __ldg(bj + c), s);
        }
        g[p] = RN<T>::mul(alpha, s);
    }
}

template <class T>
__global__ void k_gather_vals(int m, const int *vmap, const T *in, T *out) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < m) out[t] = in[vmap[t]];
}

template <class T>
__global__ void k_permute_rows(int n, int nrhs, const int *perm, int inverse, const T *in, T *out) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * nrhs) return;
    const long long r = t / nrhs, c = t - r * nrhs;
    const long long o = (long long)perm[r] * nrhs + c;
    if (inverse) out[o] = in[t]; else out[t] = in[o];
}

}  // namespace

int spmv(jv_handle h, jv_dtype t, const void *vals, const void *x, void *y, double alpha,
         double beta) {
    const int nw = h->spmv_wide;
    const int grid = grid_for(32ll * nw + (h->n - nw), kBlock);
    const int hb = beta != 0.0, ha = alpha != 1.0;
    // quad loads need 16-byte aligned index and value arrays, and pay on long
    // rows only (7-point 128^3 FP32: 72 -> 79 us with them; power-law matrix
    // FP64: 238 -> 216 us, exact mode 650 -> 559 us)
    const bool quad = h->maxrow > 32 && (uintptr_t)vals % 16 == 0 && (uintptr_t)h->colidx % 16 == 0;
    count_launch();
#define JV_SPMV(K_, T_, U_, B_, W_)                                                               \
    K_<T_, U_, B_, W_><<<grid, kBlock, 0, h->stream>>>(h->n, ARGS_##K_ nw, h->spmv_rows,          \
                                                       h->rowptr, h->colidx, (const T_ *)vals,    \
                                                       (const T_ *)x, (T_ *)y, (T_)alpha,         \
                                                       (T_)beta, ha, hb);
#define ARGS_k_spmv
#define ARGS_k_spmv_quad h->nnz,
    // chunk and CTAs per SM by the longest row: stencils of at most 8 entries
    // take single-entry chunks and eight CTAs per SM (7-point 128^3 FP64 52 ->
    // 50 us) and, in FP32, chunks of 4 and six CTAs (46 -> 38 us); the
    // 27-point rows keep longer chunks (the single-entry form: 85 -> 140 us)
    if (t == JV_F64) {
        if (nw == 0 && h->maxrow <= 8) { JV_SPMV(k_spmv, double, 1, 8, false) }
        else if (nw == 0 && h->maxrow <= 32) { JV_SPMV(k_spmv, double, 2, 6, false) }
        else if (quad && nw > 0) { JV_SPMV(k_spmv_quad, double, 4, 4, true) }
        else if (quad) { JV_SPMV(k_spmv_quad, double, 4, 4, false) }
        else if (nw > 0) { JV_SPMV(k_spmv, double, 4, 4, true) }
        else { JV_SPMV(k_spmv, double, 4, 4, false) }
    } else if (t == JV_F32) {
        if (quad && nw > 0) { JV_SPMV(k_spmv_quad, float, 8, 4, true) }
        else if (quad) { JV_SPMV(k_spmv_quad, float, 8, 4, false) }
        else if (nw > 0) { JV_SPMV(k_spmv, float, 8, 4, true) }
        else if (h->maxrow <= 8) { JV_SPMV(k_spmv, float, 4, 6, false) }
        else { JV_SPMV(k_spmv, float, 8, 4, false) }
    } else
        return JV_ERR_ARG;
#undef ARGS_k_spmv
#undef ARGS_k_spmv_quad
#undef JV_SPMV
    JV_CHECK_LAUNCH();
    return JV_OK;
}

int masked_outer(jv_handle h, jv_dtype t, int which, const void *a, const void *b, int nrhs,
                 double alpha, void *g) {
    const int grid = grid_for(h->n, kWarpsPerBlock);
    const size_t row_bytes = (size_t)nrhs * (t == JV_F64 ? 8 : 4);
    const bool vec = row_bytes % 16 == 0 && (uintptr_t)a % 16 == 0 && (uintptr_t)b % 16 == 0;
    count_launch();
#define JV_OUTER(T_, V_)                                                                         \
    k_masked_outer<T_, V_><<<grid, kBlock, 0, h->stream>>>(h->n, h->rowptr, h->colidx, h->diag,  \
                                                           which, (const T_ *)a, (const T_ *)b,  \
                                                           nrhs, (T_)alpha, (T_ *)g);
    if (t == JV_F64) {
        if (vec) { JV_OUTER(double, true) } else { JV_OUTER(double, false) }
    } else {
        if (vec) { JV_OUTER(float, true) } else { JV_OUTER(float, false) }
    }
#undef JV_OUTER
    JV_CHECK_LAUNCH();
    return JV_OK;
}

int permute_values(jv_handle h, jv_dtype t, const void *in, void *out) {
    const int grid = grid_for(h->nnz, kBlock);
    count_launch();
    if (t == JV_F64)
        k_gather_vals<double><<<grid, kBlock, 0, h->stream>>>(h->nnz, h->vmap, (const double *)in, (double *)out);
    else
        k_gather_vals<float><<<grid, kBlock, 0, h->stream>>>(h->nnz, h->vmap, (const float *)in, (float *)out);
    JV_CHECK_LAUNCH();
    return JV_OK;
}

int permute_vector(jv_handle h, jv_dtype t, int inverse, const void *in, void *out, int nrhs) {
    const int grid = grid_for((long long)h->n * nrhs, kBlock);
    count_launch();
    if (t == JV_F64)
        k_permute_rows<double><<<grid, kBlock, 0, h->stream>>>(h->n, nrhs, h->perm, inverse, (const double *)in, (double *)out);
    else
        k_permute_rows<float><<<grid, kBlock, 0, h->stream>>>(h->n, nrhs, h->perm, inverse, (const float *)in, (float *)out);
    JV_CHECK_LAUNCH();
    return JV_OK;
}

}  // namespace jv
