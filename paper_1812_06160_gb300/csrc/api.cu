// extern "C" entry points declared in include/jv.h: argument checks, the
// handle's life cycle and the status protocol.  All arithmetic is in the
// kernels of the other translation units.
#include <cstring>
#include <vector>

#include "jv_internal.cuh"

namespace jv {
void free_all(jv_handle h);
int stage_upper(int nlev, const int *level_ptr, const unsigned long long *len, int n,
                const jv_options &opt, unsigned char *upper);
}

namespace {

thread_local int t_last_bad_row = -1;

size_t dtype_size(jv_dtype t) { return t == JV_F64 ? 8 : (t == JV_F32 ? 4 : 0); }

bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    const char *pa = static_cast<const char *>(a), *pb = static_cast<const char *>(b);
    return pa < pb + nb && pb < pa + na;
}

// After work has been enqueued: in check mode synchronise, read the device
// status word, clear it and return it.
int finish(jv_handle h, int rc, int *bad_row = nullptr) {
    if (bad_row) *bad_row = -1;
    if (rc != JV_OK) return rc;
    if (!h->opt.check) return JV_OK;
    JV_CUDA(cudaMemcpyAsync(h->h_status, h->status, 8, cudaMemcpyDeviceToHost, h->stream));
    JV_CUDA(cudaStreamSynchronize(h->stream));
    const unsigned long long key = *h->h_status;
    if (key != ~0ull) JV_CUDA(cudaMemsetAsync(h->status, 0xff, 8, h->stream));
    int row = -1;
    int st = jv::decode_status(key, &row);
    if (bad_row) *bad_row = row;
    return st;
}

int enter(jv_handle h) {
    if (!h) return JV_ERR_ARG;
    JV_CUDA(cudaSetDevice(h->device));
    return JV_OK;
}

void destroy_handle(jv_handle h) {
    if (!h) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    jv::free_workspace(h);
    jv::free_graphs(h);
    jv::free_all(h);
    if (h->fscratch) cudaFree(h->fscratch);
    if (h->xscratch) cudaFree(h->xscratch);
    if (h->pscratch) cudaFree(h->pscratch);
    if (h->piv) cudaFree(h->piv);
    if (h->xpos) cudaFree(h->xpos);
    if (h->ticket) cudaFree(h->ticket);
    if (h->status) cudaFree(h->status);
    if (h->h_status) cudaFreeHost(h->h_status);
    cudaSetDevice(cur);
    delete h;
}

int solve_common(jv_handle h, int structure, jv_dtype lu_t, const void *lu, jv_dtype b_t,
                 const void *b, jv_dtype x_t, void *x, int nrhs) {
    int rc = enter(h);
    if (rc) return rc;
    if (!lu || !b || !x || nrhs < 1) return JV_ERR_ARG;
    if (!dtype_size(lu_t) || !dtype_size(b_t) || !dtype_size(x_t)) return JV_ERR_ARG;
    const size_t nb = (size_t)h->n * nrhs;
    if (overlaps(b, nb * dtype_size(b_t), x, nb * dtype_size(x_t))) return JV_ERR_ARG;
    if (overlaps(lu, (size_t)h->nnz * dtype_size(lu_t), x, nb * dtype_size(x_t))) return JV_ERR_ARG;
    return finish(h, jv::tri_solve(h, structure, lu_t, lu, b_t, b, x_t, x, nrhs));
}

}  // namespace

extern "C" {

void jv_default_options(jv_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->mode = JV_MODE_SYNCFREE;
    opt->reorder = 0;
    opt->check = 1;
    opt->long_row = 0;
    opt->spin_timeout_cycles = 0;
    opt->fault_row = -1;
    opt->sf_ctas_per_sm = 0;
    opt->sf_backoff_ns = 0;
    opt->sf_gate_levels = -1;
    opt->milu = 0;
    opt->sym_levels = 0;
    opt->stage_min_rows = 0;
    opt->stage_max_density = 0.0;
    opt->stage_position = 0.0;
    opt->er_corner = 0;
    opt->no_graphs = 0;
    opt->exact = 0;
    opt->spmv_long_row = 0;
}

void jv_default_krylov_opts(jv_krylov_opts *o) {
    if (!o) return;
    o->tol = 1e-8;
    o->maxit = 10000;
    o->restart = 30;
    o->max_restarts = 200;
}

int jv_analyze(int n, int nnz, const int *rowptr, const int *colidx, const jv_options *opt,
               void *stream, jv_handle *out) {
    t_last_bad_row = -1;
    if (!out) return JV_ERR_ARG;
    *out = nullptr;
    if (n < 1 || nnz < n || !rowptr || !colidx) return JV_ERR_ARG;
    jv_handle h = new jv_handle_s();
    if (opt) h->opt = *opt; else jv_default_options(&h->opt);
    if (h->opt.mode != JV_MODE_LEVEL && h->opt.mode != JV_MODE_SYNCFREE && h->opt.mode != JV_MODE_HYBRID) {
        delete h;
        return JV_ERR_ARG;
    }
    if (h->opt.long_row < 0 || h->opt.sf_ctas_per_sm < 0 || h->opt.spmv_long_row < 0) {
        delete h;
        return JV_ERR_ARG;
    }
    if ((h->opt.milu || h->opt.sym_levels || h->opt.er_corner) && h->opt.band_rows > 0) {
        delete h;
        return JV_ERR_ARG;
    }
    if (h->opt.stage_min_rows < 0 || h->opt.stage_max_density < 0 || h->opt.stage_position < 0 ||
        h->opt.stage_position > 1 || !(h->opt.stage_max_density == h->opt.stage_max_density) ||
        !(h->opt.stage_position == h->opt.stage_position)) {
        delete h;
        return JV_ERR_ARG;
    }
    h->n = n;
    h->nnz = nnz;
    h->stream = static_cast<cudaStream_t>(stream);
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        delete h;
        return JV_ERR_CUDA;
    }
    if (cudaMalloc(&h->ticket, 8 * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&h->status, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&h->h_status, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        destroy_handle(h);
        return JV_ERR_NOMEM;
    }
    if (cudaMemsetAsync(h->ticket, 0, 8 * sizeof(unsigned), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->status, 0xff, 8, h->stream) != cudaSuccess) {
        destroy_handle(h);
        return JV_ERR_CUDA;
    }
    int rc = jv::analyze(h, rowptr, colidx);
    if (rc == JV_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = JV_ERR_CUDA;
    if (rc == JV_OK && cudaMemsetAsync(h->status, 0xff, 8, h->stream) != cudaSuccess) rc = JV_ERR_CUDA;
    if (rc != JV_OK) {
        t_last_bad_row = h->bad_row;
        destroy_handle(h);
        return rc;
    }
    *out = h;
    return JV_OK;
}

int jv_last_bad_row(void) { return t_last_bad_row; }

void jv_destroy(jv_handle h) { destroy_handle(h); }

int jv_set_stream(jv_handle h, void *stream) {
    if (!h) return JV_ERR_ARG;
    h->stream = static_cast<cudaStream_t>(stream);
    return JV_OK;
}

int jv_set_mode(jv_handle h, int mode) {
    if (!h || (mode != JV_MODE_LEVEL && mode != JV_MODE_SYNCFREE && mode != JV_MODE_HYBRID))
        return JV_ERR_ARG;
    h->opt.mode = mode;
    return JV_OK;
}

int jv_set_check(jv_handle h, int check) {
    if (!h) return JV_ERR_ARG;
    h->opt.check = check ? 1 : 0;
    return JV_OK;
}

int jv_ilu0_factor(jv_handle h, jv_dtype vals_t, const void *vals, jv_dtype lu_t, void *lu,
                   int *bad_row) {
    if (bad_row) *bad_row = -1;
    int rc = enter(h);
    if (rc) return rc;
    if (!vals || !lu || !dtype_size(vals_t) || !dtype_size(lu_t)) return JV_ERR_ARG;
    if (vals == lu && vals_t != lu_t) return JV_ERR_ARG;
    if (vals != lu && overlaps(vals, (size_t)h->nnz * dtype_size(vals_t), lu,
                               (size_t)h->nnz * dtype_size(lu_t)))
        return JV_ERR_ARG;
    return finish(h, jv::ilu0_factor(h, vals_t, vals, lu_t, lu), bad_row);
}

int jv_lsolve(jv_handle h, jv_dtype lu_t, const void *lu, jv_dtype b_t, const void *b,
              jv_dtype x_t, void *x, int nrhs) {
    return solve_common(h, JV_LOWER, lu_t, lu, b_t, b, x_t, x, nrhs);
}
int jv_usolve(jv_handle h, jv_dtype lu_t, const void *lu, jv_dtype b_t, const void *b,
              jv_dtype x_t, void *x, int nrhs) {
    return solve_common(h, JV_UPPER, lu_t, lu, b_t, b, x_t, x, nrhs);
}
int jv_lsolve_t(jv_handle h, jv_dtype lu_t, const void *lu, jv_dtype b_t, const void *b,
                jv_dtype x_t, void *x, int nrhs) {
    return solve_common(h, JV_LOWER_T, lu_t, lu, b_t, b, x_t, x, nrhs);
}
int jv_usolve_t(jv_handle h, jv_dtype lu_t, const void *lu, jv_dtype b_t, const void *b,
                jv_dtype x_t, void *x, int nrhs) {
    return solve_common(h, JV_UPPER_T, lu_t, lu, b_t, b, x_t, x, nrhs);
}

int jv_spmv(jv_handle h, jv_dtype t, const void *vals, const void *x, void *y, double alpha,
            double beta) {
    int rc = enter(h);
    if (rc) return rc;
    if (!vals || !x || !y || !dtype_size(t)) return JV_ERR_ARG;
    if (overlaps(x, (size_t)h->n * dtype_size(t), y, (size_t)h->n * dtype_size(t))) return JV_ERR_ARG;
    return finish(h, jv::spmv(h, t, vals, x, y, alpha, beta));
}

int jv_masked_outer(jv_handle h, jv_dtype t, int which, const void *a, const void *b, int nrhs,
                    double alpha, void *g) {
    int rc = enter(h);
    if (rc) return rc;
    if (!a || !b || !g || nrhs < 1 || !dtype_size(t) || (which != 0 && which != 1)) return JV_ERR_ARG;
    return finish(h, jv::masked_outer(h, t, which, a, b, nrhs, alpha, g));
}

int jv_permute_values(jv_handle h, jv_dtype t, const void *in, void *out) {
    int rc = enter(h);
    if (rc) return rc;
    if (!h->vmap || !in || !out || in == out || !dtype_size(t)) return JV_ERR_ARG;
    return finish(h, jv::permute_values(h, t, in, out));
}

int jv_permute_vector(jv_handle h, jv_dtype t, int inverse, const void *in, void *out, int nrhs) {
    int rc = enter(h);
    if (rc) return rc;
    if (!h->perm || !in || !out || in == out || nrhs < 1 || !dtype_size(t)) return JV_ERR_ARG;
    return finish(h, jv::permute_vector(h, t, inverse ? 1 : 0, in, out, nrhs));
}

int jv_stage_plan(int nlev, const int *level_ptr, const long long *dep_sum, int n,
                  const jv_options *opt, unsigned char *upper, int *tail) {
    if (nlev < 0 || n < 0 || !level_ptr || (nlev > 0 && !upper)) return JV_ERR_ARG;
    jv_options o;
    if (opt) o = *opt; else jv_default_options(&o);
    if (o.stage_min_rows < 0 || !(o.stage_max_density >= 0) || !(o.stage_position >= 0) ||
        o.stage_position > 1)
        return JV_ERR_ARG;
    if (level_ptr[0] != 0) return JV_ERR_ARG;
    for (int l = 0; l < nlev; ++l)
        if (level_ptr[l + 1] <= level_ptr[l]) return JV_ERR_ARG;   // levels are never empty
    if (level_ptr[nlev] != n) return JV_ERR_ARG;
    std::vector<unsigned long long> len;
    if (dep_sum) {
        len.resize(nlev);
        for (int l = 0; l < nlev; ++l) {
            if (dep_sum[l] < 0) return JV_ERR_ARG;
            len[l] = (unsigned long long)dep_sum[l];
        }
    } else if (o.stage_max_density > 0) {
        return JV_ERR_ARG;
    }
    const int t = jv::stage_upper(nlev, level_ptr, dep_sum ? len.data() : nullptr, n, o, upper);
    if (tail) *tail = t;
    return JV_OK;
}

int jv_get_info(jv_handle h, jv_info *info) {
    if (!h || !info) return JV_ERR_ARG;
    info->n = h->n;
    info->nnz = h->nnz;
    info->nnz_lower = h->nnz_lower;
    info->nnz_upper = h->nnz_upper;
    for (int k = 0; k < 4; ++k) {
        info->nlev[k] = h->ls[k].nlev;
        info->nlong[k] = h->ls[k].bins.nlong;
    }
    info->nlong_factor = h->fbins.nlong;
    for (int k = 0; k < 4; ++k) {
        info->band_rows[k] = h->ls[k].band.use ? h->ls[k].band.B : 0;
        info->nband_levels[k] = h->ls[k].band.use ? h->ls[k].band.nll_total : 0;
    }
    info->npairs = h->npairs;
    info->mode = h->opt.mode;
    info->reorder = h->opt.reorder;
    for (int k = 0; k < 4; ++k) info->hybrid_launches[k] = jv::hybrid_launches(h->ls[k], h->ls[k].nlev);
    info->hybrid_launches_factor = jv::hybrid_launches(h->ls[JV_LOWER], h->corner[JV_F64].use
                                                                            ? h->corner[JV_F64].K
                                                                            : h->ls[JV_LOWER].nlev);
    for (int t = 0; t < 2; ++t) {
        info->corner_rows[t] = h->corner[t].use ? h->corner[t].R : 0;
        info->corner_levels[t] = h->corner[t].use ? h->corner[t].nl : 0;
        for (int k = 0; k < 4; ++k)
            info->solve_corner_rows[k][t] = h->scorner[k][t].use ? h->scorner[k][t].R : 0;
    }
    info->spmv_wide_rows = h->spmv_wide;
    return JV_OK;
}

int jv_get_levels(jv_handle h, int which, int *nlev, const int **level_ptr,
                  const int **level_rows, const int **lev) {
    if (!h || which < 0 || which > 3) return JV_ERR_ARG;
    const jv::LevelSet &L = h->ls[which];
    if (nlev) *nlev = L.nlev;
    if (level_ptr) *level_ptr = L.ptr;
    if (level_rows) *level_rows = L.rows;
    if (lev) *lev = L.lev;
    return JV_OK;
}

int jv_get_pattern(jv_handle h, const int **rowptr, const int **colidx, const int **diag_ptr) {
    if (!h) return JV_ERR_ARG;
    if (rowptr) *rowptr = h->rowptr;
    if (colidx) *colidx = h->colidx;
    if (diag_ptr) *diag_ptr = h->diag;
    return JV_OK;
}

int jv_get_csc(jv_handle h, const int **colptr, const int **rowidx, const int **csc2csr,
               const int **cdiag) {
    if (!h) return JV_ERR_ARG;
    if (colptr) *colptr = h->colptr;
    if (rowidx) *rowidx = h->rowidx;
    if (csc2csr) *csc2csr = h->csc2csr;
    if (cdiag) *cdiag = h->cdiag;
    return JV_OK;
}

int jv_get_perm(jv_handle h, const int **perm, const int **iperm, const int **vmap) {
    if (!h) return JV_ERR_ARG;
    if (perm) *perm = h->perm;
    if (iperm) *iperm = h->iperm;
    if (vmap) *vmap = h->vmap;
    return JV_OK;
}

int jv_status_sync(jv_handle h, int *bad_row) {
    if (bad_row) *bad_row = -1;
    int rc = enter(h);
    if (rc) return rc;
    JV_CUDA(cudaMemcpyAsync(h->h_status, h->status, 8, cudaMemcpyDeviceToHost, h->stream));
    JV_CUDA(cudaStreamSynchronize(h->stream));
    const unsigned long long key = *h->h_status;
    JV_CUDA(cudaMemsetAsync(h->status, 0xff, 8, h->stream));
    JV_CUDA(cudaStreamSynchronize(h->stream));
    return jv::decode_status(key, bad_row);
}

int jv_pcg(jv_handle h, const double *vals, jv_dtype lu_t, const void *lu, const double *b,
           double *x, const jv_krylov_opts *o, jv_krylov_info *info) {
    int rc = enter(h);
    if (rc) return rc;
    if (!vals || !lu || !b || !x || !dtype_size(lu_t)) return JV_ERR_ARG;
    jv_krylov_opts d;
    jv_default_krylov_opts(&d);
    return jv::pcg(h, vals, lu_t, lu, b, x, o ? o : &d, info);
}

int jv_fgmres(jv_handle h, const double *vals, jv_dtype lu_t, const void *lu, const double *b,
              double *x, const jv_krylov_opts *o, jv_krylov_info *info) {
    int rc = enter(h);
    if (rc) return rc;
    if (!vals || !lu || !b || !x || !dtype_size(lu_t)) return JV_ERR_ARG;
    jv_krylov_opts d;
    jv_default_krylov_opts(&d);
    return jv::fgmres(h, vals, lu_t, lu, b, x, o ? o : &d, info);
}

int jv_iluk_symbolic(int n, int nnz, const int *rowptr, const int *colidx, int level,
                     int *fill_rowptr, int *fill_colidx, int *fill_level, long long *fill_nnz,
                     int *bad_row, void *stream) {
    if (bad_row) *bad_row = -1;
    if (n < 1 || nnz < n || !rowptr || !colidx || level < 0 || !fill_rowptr || !fill_nnz)
        return JV_ERR_ARG;
    return jv::iluk_symbolic(n, nnz, rowptr, colidx, level, fill_rowptr, fill_colidx, fill_level,
                             fill_nnz, static_cast<cudaStream_t>(stream), bad_row);
}

int jv_scatter_values(int n, const int *rowptr, const int *colidx, jv_dtype t, const void *vals,
                      const int *fill_rowptr, const int *fill_colidx, void *fill_vals,
                      void *stream) {
    if (n < 1 || !rowptr || !colidx || !vals || !fill_rowptr || !fill_colidx || !fill_vals ||
        (t != JV_F64 && t != JV_F32))
        return JV_ERR_ARG;
    return jv::scatter_values(n, rowptr, colidx, t, vals, fill_rowptr, fill_colidx, fill_vals,
                              static_cast<cudaStream_t>(stream));
}

int jv_hop_latency(int rounds, int npartners, double *out_us, void *stream) {
    if (rounds <= 0 || npartners <= 0 || !out_us) return JV_ERR_ARG;
    return jv::hop_latency(rounds, npartners, out_us, static_cast<cudaStream_t>(stream));
}

unsigned long long jv_launch_count(void) { return jv::g_launches.load(); }

const char *jv_status_string(int status) {
    switch (status) {
        case JV_OK: return "ok";
        case JV_ERR_ARG: return "invalid argument";
        case JV_ERR_PATTERN: return "invalid sparsity pattern (index out of range, unsorted or duplicate column, or bad row pointer)";
        case JV_ERR_NO_DIAG: return "a row has no stored diagonal entry";
        case JV_ERR_ZERO_PIVOT: return "zero or non-finite pivot";
        case JV_ERR_TIMEOUT: return "a sync-free wait timed out";
        case JV_ERR_CUDA: return "CUDA runtime error";
        case JV_ERR_NOMEM: return "device allocation failed";
        case JV_ERR_INTERNAL: return "internal analysis error";
        case JV_ERR_NOT_CONVERGED: return "Krylov iteration did not converge";
        default: return "unknown status";
    }
}

}  // extern "C"
