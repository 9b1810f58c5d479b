// CSR spmv (Sec. I: with stri the kernel a preconditioned Krylov method
// repeats; Sec. VI defers it), the pattern-restricted outer product used by
// the factor gradient, and the gathers that move values and vectors into the
// level order of a reordered handle (Sec. III).
#include "jv_internal.cuh"

namespace jv {
namespace {

// A group of VW lanes per row; consecutive groups take consecutive rows, so a
// warp reads one contiguous stretch of colidx / vals.
template <class T, int VW>
__global__ void __launch_bounds__(kBlock) k_spmv(int n, const int *__restrict__ rowptr,
                                                 const int *__restrict__ colidx,
                                                 const T *__restrict__ vals,
                                                 const T *__restrict__ x, T *y, T alpha, T beta) {
    constexpr int R = kWarp / VW;
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)kBlock + threadIdx.x) >> 5;
    const long long r = warp * R + lane / VW;
    const int sub = lane % VW;
    T acc = 0;
    if (r < n) {
        const int e = __ldg(rowptr + r + 1);
        for (int q = __ldg(rowptr + r) + sub; q < e; q += VW)
            acc = fma(__ldg(vals + q), __ldg(x + __ldg(colidx + q)), acc);
    }
#pragma unroll
    for (int o = VW / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (r < n && sub == 0) {
        T v = alpha * acc;
        if (beta != (T)0) v = fma(beta, y[r], v);
        y[r] = v;
    }
}

template <class T>
int spmv_t(jv_handle h, const void *vals, const void *x, void *y, double alpha, double beta) {
    const int vw = h->spmv_vw;
    const long long rows_per_block = (long long)kWarpsPerBlock * (kWarp / vw);
    const int grid = grid_for(h->n, (int)rows_per_block);
    cudaStream_t s = h->stream;
    const T *v = static_cast<const T *>(vals);
    const T *xx = static_cast<const T *>(x);
    T *yy = static_cast<T *>(y);
    count_launch();
    switch (vw) {
        case 1: k_spmv<T, 1><<<grid, kBlock, 0, s>>>(h->n, h->rowptr, h->colidx, v, xx, yy, (T)alpha, (T)beta); break;
        case 2: k_spmv<T, 2><<<grid, kBlock, 0, s>>>(h->n, h->rowptr, h->colidx, v, xx, yy, (T)alpha, (T)beta); break;
        case 4: k_spmv<T, 4><<<grid, kBlock, 0, s>>>(h->n, h->rowptr, h->colidx, v, xx, yy, (T)alpha, (T)beta); break;
        case 8: k_spmv<T, 8><<<grid, kBlock, 0, s>>>(h->n, h->rowptr, h->colidx, v, xx, yy, (T)alpha, (T)beta); break;
        case 16: k_spmv<T, 16><<<grid, kBlock, 0, s>>>(h->n, h->rowptr, h->colidx, v, xx, yy, (T)alpha, (T)beta); break;
        default: k_spmv<T, 32><<<grid, kBlock, 0, s>>>(h->n, h->rowptr, h->colidx, v, xx, yy, (T)alpha, (T)beta); break;
    }
    JV_CHECK_LAUNCH();
    return JV_OK;
}

// g[p] = alpha * sum_c a[i,c] b[j,c] for the entries p = (i, j) of one part of
// row i; one warp per row, lanes over the right-hand sides.
template <class T>
__global__ void __launch_bounds__(kBlock) k_masked_outer(int n, const int *rowptr, const int *colidx,
                                                         const int *diag, int which, const T *A,
                                                         const T *B, int nrhs, T alpha, T *g) {
    const int lane = threadIdx.x & 31;
    const long long i = (blockIdx.x * (long long)kBlock + threadIdx.x) >> 5;
    if (i >= n) return;
    const int lo = which == 0 ? rowptr[i] : diag[i];
    const int hi = which == 0 ? diag[i] : rowptr[i + 1];
    const size_t ld = (size_t)nrhs;
    for (int p = lo; p < hi; ++p) {
        const int j = colidx[p];
        T s = 0;
        for (int c = lane; c < nrhs; c += 32) s = fma(A[i * ld + c], B[(size_t)j * ld + c], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) g[p] = alpha * s;
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
    if (t == JV_F64) return spmv_t<double>(h, vals, x, y, alpha, beta);
    if (t == JV_F32) return spmv_t<float>(h, vals, x, y, alpha, beta);
    return JV_ERR_ARG;
}

int masked_outer(jv_handle h, jv_dtype t, int which, const void *a, const void *b, int nrhs,
                 double alpha, void *g) {
    const int grid = grid_for(h->n, kWarpsPerBlock);
    count_launch();
    if (t == JV_F64)
        k_masked_outer<double><<<grid, kBlock, 0, h->stream>>>(
            h->n, h->rowptr, h->colidx, h->diag, which, (const double *)a, (const double *)b, nrhs,
            alpha, (double *)g);
    else
        k_masked_outer<float><<<grid, kBlock, 0, h->stream>>>(
            h->n, h->rowptr, h->colidx, h->diag, which, (const float *)a, (const float *)b, nrhs,
            (float)alpha, (float *)g);
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
