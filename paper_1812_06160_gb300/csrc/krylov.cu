// Krylov drivers (Sec. I: CG and GMRES preconditioned by the ILU factors;
// Sec. VI notes that the solves run many times over for one factor).  All vectors are
// FP64 on the device; the scalars of the recurrences (alpha, beta, the
// Hessenberg column) are produced and consumed on the device, and only one
// residual norm (PCG) or one Hessenberg column (FGMRES, for the Givens
// rotations) crosses to the host per iteration.
//
// Dot products are deterministic: a fixed grid, a fixed per-thread stride
// and fixed shuffle trees; the last CTA to finish sums the per-CTA partials
// in index order.
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "jv_internal.cuh"

namespace jv {

constexpr int kDotBlocks = 304;

struct Workspace {
    int n = 0, m = 0;
    double *r = nullptr, *z = nullptr, *zn = nullptr, *p = nullptr, *q = nullptr;
    double *tmp = nullptr;            // intermediate L^-1 r of the preconditioner (FP64 or FP32)
    double *V = nullptr, *Z = nullptr, *w = nullptr;
    double *sc = nullptr;             // device scalars
    double *partial = nullptr;        // [kDotBlocks]
    unsigned *counter = nullptr;
    double *h_sc = nullptr;           // pinned host mirror of sc
    std::vector<void *> allocs;
};

void free_workspace(jv_handle h) {
    if (!h->ws) return;
    for (void *p : h->ws->allocs) cudaFree(p);
    if (h->ws->h_sc) cudaFreeHost(h->ws->h_sc);
    delete h->ws;
    h->ws = nullptr;
}

namespace {

enum { SC_RZ0 = 0, SC_RZ1 = 1, SC_PQ = 2, SC_RR = 3, SC_RZO = 4, SC_BB = 5, SC_H = 8 };
constexpr int kScalars = 64 + 8;

int ws_get(Workspace *w, double **p, size_t count) {
    void *q = nullptr;
    if (cudaMalloc(&q, count * sizeof(double) + 16) != cudaSuccess) {
        cudaGetLastError();
        return JV_ERR_NOMEM;
    }
    w->allocs.push_back(q);
    *p = (double *)q;
    return JV_OK;
}

int ensure_ws(jv_handle h, int m) {
    Workspace *w = h->ws;
    if (w && w->m >= m) return JV_OK;
    free_workspace(h);
    w = new Workspace();
    h->ws = w;
    w->n = h->n;
    w->m = m;
    const size_t n = h->n;
    int rc = JV_OK;
    rc |= ws_get(w, &w->r, n);
    rc |= ws_get(w, &w->z, n);
    rc |= ws_get(w, &w->zn, n);
    rc |= ws_get(w, &w->p, n);
    rc |= ws_get(w, &w->q, n);
    rc |= ws_get(w, &w->tmp, n);
    rc |= ws_get(w, &w->w, n);
    if (m > 0) {
        rc |= ws_get(w, &w->V, (size_t)(m + 1) * n);
        rc |= ws_get(w, &w->Z, (size_t)m * n);
    }
    rc |= ws_get(w, &w->sc, kScalars + 2 * (size_t)(m + 2));
    rc |= ws_get(w, &w->partial, 2 * kDotBlocks);
    double *cnt;
    rc |= ws_get(w, &cnt, 1);
    if (rc) {
        free_workspace(h);
        return JV_ERR_NOMEM;
    }
    w->counter = (unsigned *)cnt;
    if (cudaMemset(w->counter, 0, sizeof(unsigned)) != cudaSuccess) return JV_ERR_CUDA;
    if (cudaMallocHost(&w->h_sc, (kScalars + 2 * (size_t)(m + 2)) * sizeof(double)) != cudaSuccess) {
        free_workspace(h);
        return JV_ERR_NOMEM;
    }
    return JV_OK;
}

// ------------------------------------------------------------- BLAS-1
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// out = x.y (op 0) or sqrt(x.y) (op 1); y2 != nullptr also computes x.y2 -> out2.
__global__ void __launch_bounds__(kBlock) k_dot(int n, const double *x, const double *y,
                                                const double *y2, double *partial,
                                                unsigned *counter, double *out, double *out2,
                                                int op) {
    __shared__ double sw[2][kWarpsPerBlock];
    __shared__ bool last;
    double s1 = 0, s2 = 0;
    for (long long i = blockIdx.x * (long long)kBlock + threadIdx.x; i < n;
         i += (long long)gridDim.x * kBlock) {
        s1 = fma(x[i], y[i], s1);
        if (y2) s2 = fma(x[i], y2[i], s2);
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sw[0][wid] = s1; sw[1][wid] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b1 = 0, b2 = 0;
        for (int k = 0; k < kWarpsPerBlock; ++k) { b1 += sw[0][k]; b2 += sw[1][k]; }
        partial[2 * blockIdx.x] = b1;
        partial[2 * blockIdx.x + 1] = b2;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && wid == 0) {
        __threadfence();
        double t1 = 0, t2 = 0;
        for (int k = lane; k < (int)gridDim.x; k += 32) {
            t1 += ld_relaxed_f64(partial + 2 * k);
            t2 += ld_relaxed_f64(partial + 2 * k + 1);
        }
        t1 = warp_sum(t1);
        t2 = warp_sum(t2);
        if (lane == 0) {
            *out = op == 1 ? sqrt(t1) : t1;
            if (out2) *out2 = t2;
            *counter = 0;
        }
    }
}

// y = a*x + b*y with a = sa * (*pa / *pb) when pa != nullptr (else a = sa), b = sb
__global__ void k_axpby(int n, double sa, const double *pa, const double *pb, const double *x,
                        double sb, double *y) {
    double a = sa;
    if (pa) a = sa * (*pa / (pb ? *pb : 1.0));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = fma(a, x[i], sb * y[i]);
}

// PCG step 1: alpha = rz / pq;  x += alpha p;  r -= alpha q
__global__ void k_cg_step1(int n, const double *rz, const double *pq, const double *p,
                           const double *q, double *x, double *r) {
    const double alpha = *rz / *pq;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        r[i] = fma(-alpha, q[i], r[i]);
    }
}

// PCG step 2 (Polak-Ribiere): beta = (rz_new - rz_cross) / rz_old;  p = zn + beta p
__global__ void k_cg_step2(int n, const double *rzn, const double *rzo, const double *rz,
                           const double *zn, double *p) {
    const double beta = (*rzn - *rzo) / *rz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], zn[i]);
}

// v = w / *nrm (0 when *nrm == 0)
__global__ void k_scale_inv(int n, const double *nrm, const double *w, double *v) {
    const double s = *nrm;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        v[i] = s != 0.0 ? w[i] / s : 0.0;
}

// x += sum_j y[j] Z[j]   (j ascending)
__global__ void k_update_x(int n, int k, const double *y, const double *Z, double *x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double s = x[i];
        for (int j = 0; j < k; ++j) s = fma(y[j], Z[(size_t)j * n + i], s);
        x[i] = s;
    }
}

constexpr int kVecGrid = 152 * 8;

struct Ctx {
    jv_handle h;
    Workspace *w;
    cudaStream_t s;
    int n;
};

int dot(const Ctx &c, const double *x, const double *y, double *out, int op = 0,
        const double *y2 = nullptr, double *out2 = nullptr) {
    count_launch();
    k_dot<<<kDotBlocks, kBlock, 0, c.s>>>(c.n, x, y, y2, c.w->partial, c.w->counter, out, out2, op);
    JV_CHECK_LAUNCH();
    return JV_OK;
}

int axpby(const Ctx &c, double sa, const double *pa, const double *pb, const double *x, double sb,
          double *y) {
    count_launch();
    k_axpby<<<kVecGrid, kBlock, 0, c.s>>>(c.n, sa, pa, pb, x, sb, y);
    JV_CHECK_LAUNCH();
    return JV_OK;
}

int read_scalars(const Ctx &c, int first, int count) {
    JV_CUDA(cudaMemcpyAsync(c.w->h_sc + first, c.w->sc + first, count * sizeof(double),
                            cudaMemcpyDeviceToHost, c.s));
    JV_CUDA(cudaStreamSynchronize(c.s));
    return JV_OK;
}

int precond(const Ctx &c, jv_dtype lu_t, const void *lu, const double *r, double *z) {
    int rc = tri_solve(c.h, JV_LOWER, lu_t, lu, JV_F64, r, lu_t, c.w->tmp, 1);
    if (rc) return rc;
    return tri_solve(c.h, JV_UPPER, lu_t, lu, lu_t, c.w->tmp, JV_F64, z, 1);
}

int residual(const Ctx &c, const double *vals, const double *b, const double *x, double *r) {
    JV_CUDA(cudaMemcpyAsync(r, b, (size_t)c.n * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
    return spmv(c.h, JV_F64, vals, x, r, -1.0, 1.0);
}

#define JV_TRY(x)                     \
    do {                              \
        int rc_ = (x);                \
        if (rc_ != JV_OK) return rc_; \
    } while (0)

}  // namespace

int pcg(jv_handle h, const double *vals, jv_dtype lu_t, const void *lu, const double *b,
        double *x, const jv_krylov_opts *o, jv_krylov_info *info) {
    JV_TRY(ensure_ws(h, 0));
    Ctx c{h, h->ws, h->stream, h->n};
    Workspace *w = h->ws;
    double *sc = w->sc, *hs = w->h_sc;
    double *z = w->z, *zn = w->zn;
    int ia = SC_RZ0, ib = SC_RZ1;
    JV_TRY(dot(c, b, b, sc + SC_BB, 1));
    JV_TRY(residual(c, vals, b, x, w->r));
    JV_TRY(dot(c, w->r, w->r, sc + SC_RR, 1));
    JV_TRY(read_scalars(c, 0, 8));
    const double bnorm = hs[SC_BB] > 0 ? hs[SC_BB] : 1.0;
    double rel = hs[SC_RR] / bnorm;
    int it = 0;
    bool done = rel <= o->tol;
    if (!done) {
        JV_TRY(precond(c, lu_t, lu, w->r, z));
        JV_CUDA(cudaMemcpyAsync(w->p, z, (size_t)c.n * 8, cudaMemcpyDeviceToDevice, c.s));
        JV_TRY(dot(c, w->r, z, sc + ia));
    }
    while (!done && it < o->maxit) {
        JV_TRY(spmv(h, JV_F64, vals, w->p, w->q, 1.0, 0.0));
        JV_TRY(dot(c, w->p, w->q, sc + SC_PQ));
        count_launch();
        k_cg_step1<<<kVecGrid, kBlock, 0, c.s>>>(c.n, sc + ia, sc + SC_PQ, w->p, w->q, x, w->r);
        JV_CHECK_LAUNCH();
        ++it;
        JV_TRY(dot(c, w->r, w->r, sc + SC_RR, 1));
        JV_TRY(read_scalars(c, SC_RR, 1));
        rel = hs[SC_RR] / bnorm;
        if (!(rel > o->tol)) { done = rel <= o->tol; break; }
        JV_TRY(precond(c, lu_t, lu, w->r, zn));
        JV_TRY(dot(c, w->r, zn, sc + ib, 0, z, sc + SC_RZO));
        count_launch();
        k_cg_step2<<<kVecGrid, kBlock, 0, c.s>>>(c.n, sc + ib, sc + SC_RZO, sc + ia, zn, w->p);
        JV_CHECK_LAUNCH();
        std::swap(z, zn);
        std::swap(ia, ib);
    }
    // true residual
    JV_TRY(residual(c, vals, b, x, w->r));
    JV_TRY(dot(c, w->r, w->r, sc + SC_RR, 1));
    JV_TRY(read_scalars(c, SC_RR, 1));
    JV_CUDA(cudaMemcpyAsync(h->h_status, h->status, 8, cudaMemcpyDeviceToHost, c.s));
    JV_CUDA(cudaStreamSynchronize(c.s));
    int row = -1;
    const int st = decode_status(*h->h_status, &row);
    if (st != JV_OK) JV_CUDA(cudaMemsetAsync(h->status, 0xff, 8, c.s));
    if (info) {
        info->iters = it;
        info->converged = done ? 1 : 0;
        info->relres = rel;
        info->true_relres = hs[SC_RR] / bnorm;
    }
    if (st != JV_OK) return st;
    return done ? JV_OK : JV_ERR_NOT_CONVERGED;
}

int fgmres(jv_handle h, const double *vals, jv_dtype lu_t, const void *lu, const double *b,
           double *x, const jv_krylov_opts *o, jv_krylov_info *info) {
    const int m = o->restart > 0 ? o->restart : 30;
    JV_TRY(ensure_ws(h, m));
    Ctx c{h, h->ws, h->stream, h->n};
    Workspace *w = h->ws;
    double *sc = w->sc, *hs = w->h_sc;
    double *hcol = sc + SC_H;                 // [m+2]
    double *ydev = sc + SC_H + (m + 2);       // [m]
    const size_t n = c.n;
    JV_TRY(dot(c, b, b, sc + SC_BB, 1));
    JV_TRY(read_scalars(c, SC_BB, 1));
    const double bnorm = hs[SC_BB] > 0 ? hs[SC_BB] : 1.0;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    int total = 0;
    bool converged = false;
    double rel = 1.0;
    for (int cycle = 0; cycle < o->max_restarts && !converged; ++cycle) {
        JV_TRY(residual(c, vals, b, x, w->w));
        JV_TRY(dot(c, w->w, w->w, sc + SC_RR, 1));
        JV_TRY(read_scalars(c, SC_RR, 1));
        const double beta = hs[SC_RR];
        rel = beta / bnorm;
        if (rel <= o->tol) { converged = true; break; }
        count_launch();
        k_scale_inv<<<kVecGrid, kBlock, 0, c.s>>>(c.n, sc + SC_RR, w->w, w->V);
        JV_CHECK_LAUNCH();
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double *vj = w->V + (size_t)j * n, *zj = w->Z + (size_t)j * n;
            JV_TRY(precond(c, lu_t, lu, vj, zj));
            JV_TRY(spmv(h, JV_F64, vals, zj, w->w, 1.0, 0.0));
            for (int i = 0; i <= j; ++i) {      // modified Gram-Schmidt
                const double *vi = w->V + (size_t)i * n;
                JV_TRY(dot(c, w->w, vi, hcol + i));
                JV_TRY(axpby(c, -1.0, hcol + i, nullptr, vi, 1.0, w->w));
            }
            JV_TRY(dot(c, w->w, w->w, hcol + j + 1, 1));
            count_launch();
            k_scale_inv<<<kVecGrid, kBlock, 0, c.s>>>(c.n, hcol + j + 1, w->w,
                                                      w->V + (size_t)(j + 1) * n);
            JV_CHECK_LAUNCH();
            JV_TRY(read_scalars(c, SC_H, j + 2));
            for (int i = 0; i <= j + 1; ++i) H[(size_t)i * m + j] = hs[SC_H + i];
            for (int i = 0; i < j; ++i) {
                const double h0 = H[(size_t)i * m + j], h1 = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * h0 + sn[i] * h1;
                H[(size_t)(i + 1) * m + j] = -sn[i] * h0 + cs[i] * h1;
            }
            const double h0 = H[(size_t)j * m + j], h1 = H[(size_t)(j + 1) * m + j];
            const double rr = std::sqrt(h0 * h0 + h1 * h1);
            cs[j] = rr == 0.0 ? 1.0 : h0 / rr;
            sn[j] = rr == 0.0 ? 0.0 : h1 / rr;
            H[(size_t)j * m + j] = rr;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            k = j + 1;
            ++total;
            rel = std::fabs(g[j + 1]) / bnorm;
            if (rel <= o->tol || hs[SC_H + j + 1] == 0.0) break;
        }
        for (int i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int l = i + 1; l < k; ++l) s -= H[(size_t)i * m + l] * y[l];
            y[i] = s / H[(size_t)i * m + i];
        }
        JV_CUDA(cudaMemcpyAsync(ydev, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, c.s));
        count_launch();
        k_update_x<<<kVecGrid, kBlock, 0, c.s>>>(c.n, k, ydev, w->Z, x);
        JV_CHECK_LAUNCH();
        JV_CUDA(cudaStreamSynchronize(c.s));   // y lives on the host stack frame
    }
    JV_TRY(residual(c, vals, b, x, w->w));
    JV_TRY(dot(c, w->w, w->w, sc + SC_RR, 1));
    JV_TRY(read_scalars(c, SC_RR, 1));
    const double true_rel = hs[SC_RR] / bnorm;
    if (!converged && true_rel <= o->tol) converged = true;
    JV_CUDA(cudaMemcpyAsync(h->h_status, h->status, 8, cudaMemcpyDeviceToHost, c.s));
    JV_CUDA(cudaStreamSynchronize(c.s));
    int row = -1;
    const int st = decode_status(*h->h_status, &row);
    if (st != JV_OK) JV_CUDA(cudaMemsetAsync(h->status, 0xff, 8, c.s));
    if (info) {
        info->iters = total;
        info->converged = converged ? 1 : 0;
        info->relres = rel;
        info->true_relres = true_rel;
    }
    if (st != JV_OK) return st;
    return converged ? JV_OK : JV_ERR_NOT_CONVERGED;
}

}  // namespace jv
