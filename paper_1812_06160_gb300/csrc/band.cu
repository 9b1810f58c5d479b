// Band schedule for the sync-free factor and solves (see BandPlan).
//
// The level-ordered sync-free schedule pays one cross-SM hop per level of the
// DAG (a publish -> observe round through L2 costs about 0.3-0.45 us on
// GB300, plus the poll rounds).  When most dependencies are short -- stencil
// and banded matrices in natural order -- most hops can instead stay inside
// one SM: the rows are split into contiguous bands, one CTA runs a band, and
// inside it the rows step through their *local* levels (longest path through
// dependencies inside the band) separated by __syncthreads, reading in-band
// values from shared memory.  Only dependencies on other bands are awaited
// on the published output words.
//
// Which band size helps depends on the matrix (a band boundary across the
// slow direction of a stencil serialises consecutive bands), so the planner
// evaluates a few candidate sizes with a small critical-path model, on the
// host, and keeps the level-ordered schedule when no band size wins:
//     F(band, k) = max(F(band, k-1), latest external dependency of the band's
//                  rows at local level k + hop) + step * ceil(rows / threads)
// with bands started in dependency order and at most G resident at once.
#include <algorithm>
#include <cmath>
#include <vector>

#include "jv_internal.cuh"

namespace jv {

namespace {

#define JV_TRY(x)                     \
    do {                              \
        int rc_ = (x);                \
        if (rc_ != JV_OK) return rc_; \
    } while (0)

constexpr double kStepUs = 0.10;    // one local level inside a CTA
constexpr double kHopUs = 0.50;     // a dependency across SMs
constexpr double kLevelUs = 2.0;    // one level of the level-ordered schedule (measured)
constexpr int kMaxBand = 16384;     // band values must fit in shared memory (FP64)

struct HostPattern {
    std::vector<int> rowptr, colidx, diag;
};

// Model one band size for a forward (L) or backward (U) structure.  llev
// receives the local levels.
double model_bands(const HostPattern &P, int n, bool forward, int B, int G, std::vector<int> &llev,
                   long long *internal, long long *total) {
    const int nb = (n + B - 1) / B;
    llev.assign(n, 0);
    std::vector<std::vector<double>> F(nb);
    std::vector<double> done(nb, 0.0);
    std::vector<int> order(nb);
    std::vector<double> E;
    std::vector<int> W;
    long long nin = 0, nall = 0;
    double finish = 0.0;
    for (int t = 0; t < nb; ++t) {
        const int b = forward ? t : nb - 1 - t;
        order[t] = b;
        const int R0 = b * B, R1 = std::min(R0 + B, n);
        E.assign(1, -1.0);
        W.assign(1, 0);
        for (int k = 0; k < R1 - R0; ++k) {
            const int i = forward ? R0 + k : R1 - 1 - k;
            const int qb = forward ? P.rowptr[i] : P.diag[i] + 1;
            const int qe = forward ? P.diag[i] : P.rowptr[i + 1];
            int m = -1;
            double e = -1.0;
            for (int q = qb; q < qe; ++q) {
                const int j = P.colidx[q];
                if (j >= R0 && j < R1) {
                    m = std::max(m, llev[j]);
                    ++nin;
                } else {
                    e = std::max(e, F[j / B][llev[j]] + kHopUs);
                }
                ++nall;
            }
            const int l = m + 1;
            llev[i] = l;
            if ((int)E.size() <= l) {
                E.resize(l + 1, -1.0);
                W.resize(l + 1, 0);
            }
            E[l] = std::max(E[l], e);
            W[l]++;
        }
        double cur = t >= G ? done[order[t - G]] : 0.0;
        F[b].resize(E.size());
        for (size_t k = 0; k < E.size(); ++k) {
            cur = std::max(cur, E[k]) + kStepUs * std::ceil(W[k] / (double)kBlock);
            F[b][k] = cur;
        }
        done[b] = cur;
        finish = std::max(finish, cur);
    }
    if (internal) *internal = nin;
    if (total) *total = nall;
    return finish;
}

int upload_plan(jv_handle h, BandPlan &bp, int B, const std::vector<int> &llev) {
    const int n = h->n;
    cudaStream_t s = h->stream;
    const int nb = (n + B - 1) / B;
    std::vector<int> rows((size_t)n), bl_ptr((size_t)nb + 1), ll_ptr;
    std::vector<int> cnt;
    ll_ptr.reserve((size_t)n + 1);
    int pos = 0, nll_max = 0;
    for (int b = 0; b < nb; ++b) {
        const int R0 = b * B, R1 = std::min(R0 + B, n);
        int nll = 0;
        for (int i = R0; i < R1; ++i) nll = std::max(nll, llev[i] + 1);
        nll_max = std::max(nll_max, nll);
        cnt.assign((size_t)nll + 1, 0);
        for (int i = R0; i < R1; ++i) cnt[llev[i] + 1]++;
        for (int l = 0; l < nll; ++l) cnt[l + 1] += cnt[l];
        bl_ptr[b] = (int)ll_ptr.size();
        for (int l = 0; l < nll; ++l) ll_ptr.push_back(pos + cnt[l]);
        for (int i = R0; i < R1; ++i) rows[pos + cnt[llev[i]]++] = i;   // ascending rows per level
        pos += R1 - R0;
    }
    bl_ptr[nb] = (int)ll_ptr.size();
    ll_ptr.push_back(n);
    bp.use = true;
    bp.B = B;
    bp.nb = nb;
    bp.nll_total = (int)ll_ptr.size() - 1;
    bp.nll_max = nll_max;
    JV_TRY(halloc_n(h, &bp.rows, n));
    JV_TRY(halloc_n(h, &bp.bl_ptr, nb + 1));
    JV_TRY(halloc_n(h, &bp.ll_ptr, ll_ptr.size()));
    JV_CUDA(cudaMemcpyAsync(bp.rows, rows.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    JV_CUDA(cudaMemcpyAsync(bp.bl_ptr, bl_ptr.data(), bl_ptr.size() * 4, cudaMemcpyHostToDevice, s));
    JV_CUDA(cudaMemcpyAsync(bp.ll_ptr, ll_ptr.data(), ll_ptr.size() * 4, cudaMemcpyHostToDevice, s));
    JV_CUDA(cudaStreamSynchronize(s));
    return JV_OK;
}

}  // namespace

int plan_bands(jv_handle h) {
    // Automatic selection stays off: measured on GB300, the band kernels lose
    // to the level-ordered schedule on every workload here (each local level
    // starts with a chain of dependent row-data loads that nothing overlaps),
    // so bands are built only on request (band_rows > 0).
    if (h->opt.band_rows <= 0) return JV_OK;
    const int n = h->n;
    if (n < 2) return JV_OK;
    cudaStream_t s = h->stream;
    HostPattern P;
    P.rowptr.resize((size_t)n + 1);
    P.colidx.resize((size_t)h->nnz);
    P.diag.resize((size_t)n);
    JV_CUDA(cudaMemcpyAsync(P.rowptr.data(), h->rowptr, P.rowptr.size() * 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaMemcpyAsync(P.colidx.data(), h->colidx, P.colidx.size() * 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaMemcpyAsync(P.diag.data(), h->diag, P.diag.size() * 4, cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaStreamSynchronize(s));
    for (int which : {JV_LOWER, JV_UPPER}) {
        const bool forward = which == JV_LOWER;
        BandPlan &bp = h->ls[which].band;
        std::vector<int> llev, best_llev;
        long long nin = 0, nall = 0;
        int best_B = 0;
        double best_t = 1e300;
        std::vector<int> cands;
        if (h->opt.band_rows > 0) {
            cands.push_back(std::min(h->opt.band_rows, n));
        } else {
            for (int B : {256, 512})
                if (B < n) cands.push_back(B);
            for (int k = 1; k <= kMaxBand / 1024; ++k)
                if (1024 * k < n) cands.push_back(1024 * k);
        }
        for (int B : cands) {
            const int per_sm = B * 8 > 100 * 1024 ? 1 : 2;
            const double t = model_bands(P, n, forward, B, h->num_sms * per_sm, llev, &nin, &nall);
            if (t < best_t) {
                best_t = t;
                best_B = B;
                best_llev.swap(llev);
                bp.internal_frac = nall ? (double)nin / nall : 0.0;
            }
        }
        const double level_t = h->ls[which].nlev * kLevelUs;
        const bool take = h->opt.band_rows > 0 ||
                          (best_B > 0 && best_t < 0.7 * level_t && bp.internal_frac >= 0.2);
        if (take && best_B > 0) {
            int rc = upload_plan(h, bp, best_B, best_llev);
            if (rc) return rc;
        }
    }
    return JV_OK;
}

// ---------------------------------------------------------------- kernels
namespace {

template <class T> struct RN;
template <> struct RN<double> {
    __device__ static double fms(double a, double b, double c) { return __fma_rn(-a, b, c); }
    __device__ static double div(double a, double b) { return __ddiv_rn(a, b); }
};
template <> struct RN<float> {
    __device__ static float fms(float a, float b, float c) { return __fmaf_rn(-a, b, c); }
    __device__ static float div(float a, float b) { return __fdiv_rn(a, b); }
};

struct BandSolveArgs {
    Span beg, end;
    const int *idx, *vmap, *diag;
    int unit, forward, reverse;
    const int *rows, *bl_ptr, *ll_ptr;
    int n, B, nb;
    const void *lu, *b;
    void *x;
    unsigned *ticket;
    unsigned long long *status;
    long long timeout;
    int fault_row;
};

template <class TX>
__device__ __forceinline__ typename Bits<TX>::U band_settle(const TX *p, typename Bits<TX>::U u,
                                                            unsigned *ticket,
                                                            unsigned long long *status,
                                                            long long timeout, int r) {
    using B = Bits<TX>;
    using U = typename B::U;
    if (u != B::kSent) return u;
    const long long t0 = clock64();
    unsigned it = 0;
    for (;;) {
        u = ld_relaxed(reinterpret_cast<const U *>(p));
        if (u != B::kSent) return u;
        if ((++it & 15u) == 0) {
            if (sf_aborted(ticket) || clock64() - t0 > timeout) {
                report(status, JV_ERR_TIMEOUT, r);
                sf_abort(ticket);
                return B::kCanonNan;
            }
        }
    }
}

template <class TX>
__device__ __forceinline__ void band_publish(TX *p, TX v) {
    using B = Bits<TX>;
    typename B::U u = isnan(v) ? B::kCanonNan : B::to(v);
    st_relaxed(reinterpret_cast<typename B::U *>(p), u);
}

// Claim the next band (block-uniform), or -1.
__device__ __forceinline__ int claim_band(unsigned *ticket, int nb, bool forward) {
    __shared__ int s_t;
    __syncthreads();
    if (threadIdx.x == 0) s_t = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int t = s_t;
    if (t >= nb) return -1;
    return forward ? t : nb - 1 - t;
}

// One thread per row of the current local level; in-band values from shared
// memory, others awaited on their published words; the ordered FMA chain.
template <class TL, class TB, class TX>
__global__ void __launch_bounds__(kBlock) k_band_trsv(BandSolveArgs a) {
    using B = Bits<TX>;
    using U = typename B::U;
    extern __shared__ __align__(16) unsigned char smem[];
    TL *xs = reinterpret_cast<TL *>(smem);
    const TL *lu = static_cast<const TL *>(a.lu);
    TX *x = static_cast<TX *>(a.x);
    for (int band; (band = claim_band(a.ticket, a.nb, a.forward)) >= 0;) {
        const int R0 = band * a.B, R1 = min(R0 + a.B, a.n);
        const int k1 = __ldg(a.bl_ptr + band + 1);
        for (int k = __ldg(a.bl_ptr + band); k < k1; ++k) {
            const int p1 = __ldg(a.ll_ptr + k + 1);
            for (int p = __ldg(a.ll_ptr + k) + threadIdx.x; p < p1; p += kBlock) {
                const int r = __ldg(a.rows + p);
                const int qb = a.beg.at(r), len = a.end.at(r) - qb;
                TL s = (TL)__ldg(static_cast<const TB *>(a.b) + r);
                const TL d = a.unit ? (TL)1 : __ldg(lu + __ldg(a.diag + r));
                for (int e0 = 0; e0 < len; e0 += kPoll) {
                    int jj[kPoll];
                    TL vv[kPoll], xv[kPoll];
                    U uu[kPoll];
#pragma unroll
                    for (int t = 0; t < kPoll; ++t) {
                        jj[t] = -1;
                        if (e0 + t < len) {
                            const int q = a.reverse ? qb + len - 1 - (e0 + t) : qb + e0 + t;
                            jj[t] = __ldg(a.idx + q);
                            vv[t] = a.vmap ? __ldg(lu + __ldg(a.vmap + q)) : __ldg(lu + q);
                        }
                    }
#pragma unroll
                    for (int t = 0; t < kPoll; ++t) {
                        const int j = jj[t];
                        if (j >= 0) {
                            if (j >= R0 && j < R1) xv[t] = xs[j - R0];
                            else uu[t] = ld_relaxed(reinterpret_cast<const U *>(x + j));
                        }
                    }
#pragma unroll
                    for (int t = 0; t < kPoll; ++t) {
                        const int j = jj[t];
                        if (j >= 0) {
                            if (!(j >= R0 && j < R1))
                                xv[t] = (TL)B::from(band_settle<TX>(x + j, uu[t], a.ticket, a.status,
                                                                     a.timeout, r));
                            s = RN<TL>::fms(vv[t], xv[t], s);
                        }
                    }
                }
                const TL xr = a.unit ? s : RN<TL>::div(s, d);
                xs[r - R0] = xr;
                if (r != a.fault_row) band_publish<TX>(x + r, (TX)xr);
            }
            __syncthreads();
        }
    }
    sf_finish(a.ticket);
}


struct BandFactorArgs {
    const int *rowptr, *colidx, *diag, *kdiag, *pair_ptr;
    const int2 *pairs;
    const int *rows, *bl_ptr, *ll_ptr;
    int n, B, nb;
    const void *vals;
    void *lu;
    void *scratch;
    unsigned *ticket;
    unsigned long long *status;
    long long timeout;
    int fault_row;
};

// One U operand of row r's factorisation: from a row of this band (written by
// this CTA at an earlier local level) or awaited on its published word.
template <class TL>
__device__ __forceinline__ TL band_operand(const BandFactorArgs &a, const TL *lu, int q, bool inside,
                                           int r) {
    using B = Bits<TL>;
    using U = typename B::U;
    if (inside) return lu[q];
    const U u = ld_relaxed(reinterpret_cast<const U *>(lu + q));
    return B::from(band_settle<TL>(lu + q, u, a.ticket, a.status, a.timeout, r));
}

// One thread per row of the current local level.  Rows whose values and
// operands fit kLaneSlot words work in shared memory (entry e of thread t at
// word e * kBlock + t), the others in the global scratch area.
template <class TV, class TL>
__global__ void __launch_bounds__(kBlock) k_band_ilu0(BandFactorArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    TL *lu = static_cast<TL *>(a.lu);
    const TV *vals = static_cast<const TV *>(a.vals);
    TL *sbase = reinterpret_cast<TL *>(smem) + threadIdx.x;
    for (int band; (band = claim_band(a.ticket, a.nb, true)) >= 0;) {
        const int R0 = band * a.B, R1 = min(R0 + a.B, a.n);
        const int P0 = __ldg(a.rowptr + R0), P1 = __ldg(a.rowptr + R1);   // band's CSR range
        const int k1 = __ldg(a.bl_ptr + band + 1);
        for (int k = __ldg(a.bl_ptr + band); k < k1; ++k) {
            const int p1 = __ldg(a.ll_ptr + k + 1);
            for (int p = __ldg(a.ll_ptr + k) + threadIdx.x; p < p1; p += kBlock) {
                const int r = __ldg(a.rows + p);
                const int rs = __ldg(a.rowptr + r), len = __ldg(a.rowptr + r + 1) - rs;
                const int nl = __ldg(a.diag + r) - rs;
                const int j0 = __ldg(a.pair_ptr + rs);
                const int np = __ldg(a.pair_ptr + rs + nl) - j0;
                const bool fast = len + nl + np <= kLaneSlot;
                TL *const wp = fast ? sbase : static_cast<TL *>(a.scratch) + rs;
                const int ws = fast ? kBlock : 1;
                auto W = [&](int e) -> TL & { return wp[e * ws]; };
                if (fast) {
                    TL v[kLaneSlot];
#pragma unroll
                    for (int e = 0; e < kLaneSlot; ++e)
                        if (e < len) v[e] = (TL)__ldg(vals + rs + e);
#pragma unroll
                    for (int e = 0; e < kLaneSlot; ++e)
                        if (e < len) W(e) = v[e];
                } else {
                    for (int e = 0; e < len; ++e) W(e) = (TL)__ldg(vals + rs + e);
                }
                if (fast) {
                    // every operand in one batch of independent loads: u_kk of each
                    // step, then u_kq of each pair; an operand lies in this band iff
                    // its position lies in the band's contiguous CSR range [P0, P1)
                    using U = typename Bits<TL>::U;
                    const int m = nl + np;
                    int oq[kLaneSlot];
                    U ou[kLaneSlot];
#pragma unroll
                    for (int e = 0; e < kLaneSlot; ++e)
                        if (e < m) oq[e] = e < nl ? __ldg(a.kdiag + rs + e) : __ldg(a.pairs + j0 + e - nl).y;
#pragma unroll
                    for (int e = 0; e < kLaneSlot; ++e)
                        if (e < m) {
                            if (oq[e] >= P0 && oq[e] < P1)
                                ou[e] = Bits<TL>::to(lu[oq[e]]);
                            else
                                ou[e] = ld_relaxed(reinterpret_cast<const U *>(lu + oq[e]));
                        }
#pragma unroll
                    for (int e = 0; e < kLaneSlot; ++e)
                        if (e < m) {
                            if (!(oq[e] >= P0 && oq[e] < P1))
                                ou[e] = band_settle<TL>(lu + oq[e], ou[e], a.ticket, a.status, a.timeout, r);
                            W(len + e) = Bits<TL>::from(ou[e]);
                        }
                }
                int j = j0;
                for (int st = 0; st < nl; ++st) {
                    const int qd = __ldg(a.kdiag + rs + st);
                    const TL ukk = fast ? W(len + st)
                                        : band_operand<TL>(a, lu, qd, qd >= P0 && qd < P1, r);
                    const TL lik = RN<TL>::div(W(st), ukk);
                    for (const int je = __ldg(a.pair_ptr + rs + st + 1); j < je; ++j) {
                        const int2 tq = __ldg(a.pairs + j);
                        const TL uq = fast ? W(len + nl + j - j0)
                                           : band_operand<TL>(a, lu, tq.y, tq.y >= P0 && tq.y < P1, r);
                        W(tq.x - rs) = RN<TL>::fms(lik, uq, W(tq.x - rs));
                    }
                    W(st) = lik;
                }
                const double dd = (double)W(nl);
                if (dd == 0.0 || !isfinite(dd)) report(a.status, JV_ERR_ZERO_PIVOT, r);
                for (int e = 0; e < len; ++e) {
                    const TL v = W(e);
                    if (e < nl) lu[rs + e] = v;
                    else if (r != a.fault_row) band_publish<TL>(lu + rs + e, v);
                }
            }
            __syncthreads();
        }
    }
    sf_finish(a.ticket);
}

}  // namespace

int band_solve(jv_handle h, int structure, jv_dtype lu_t, const void *lu, jv_dtype b_t,
               const void *b, jv_dtype x_t, void *x) {
    const BandPlan &bp = h->ls[structure].band;
    BandSolveArgs a{};
    switch (structure) {
        case JV_LOWER:
            a.beg = {h->rowptr, 0, 0}; a.end = {h->diag, 0, 0}; a.idx = h->colidx; a.vmap = nullptr;
            a.unit = 1; a.forward = 1; a.reverse = 0; break;
        case JV_UPPER:
            a.beg = {h->diag, 0, 1}; a.end = {h->rowptr, 1, 0}; a.idx = h->colidx; a.vmap = nullptr;
            a.unit = 0; a.forward = 0; a.reverse = 0; break;
        default:
            return JV_ERR_INTERNAL;
    }
    a.diag = h->diag;
    a.rows = bp.rows;
    a.bl_ptr = bp.bl_ptr;
    a.ll_ptr = bp.ll_ptr;
    a.n = h->n;
    a.B = bp.B;
    a.nb = bp.nb;
    a.lu = lu;
    a.b = b;
    a.x = x;
    a.ticket = h->ticket;
    a.status = h->status;
    a.timeout = h->opt.spin_timeout_cycles > 0 ? h->opt.spin_timeout_cycles : kDefaultSpin;
    a.fault_row = h->opt.fault_row;
    cudaStream_t s = h->stream;
    const size_t tx = x_t == JV_F64 ? 8 : 4;
    int rc = fill_u32(x, (size_t)h->n * (tx / 4), ~0u, s);
    if (rc) return rc;
    const int grid = std::min(bp.nb, h->num_sms * (bp.B * 8 > 100 * 1024 ? 1 : 2));
    size_t smem;
#define JV_BAND_SOLVE(TL_, TB_, TX_)                                                         \
    smem = (size_t)bp.B * sizeof(TL_);                                                     \
    JV_CUDA(cudaFuncSetAttribute(k_band_trsv<TL_, TB_, TX_>,                              \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    count_launch();                                                                        \
    k_band_trsv<TL_, TB_, TX_><<<grid, kBlock, smem, s>>>(a);
    if (lu_t == JV_F64 && b_t == JV_F64 && x_t == JV_F64) { JV_BAND_SOLVE(double, double, double) }
    else if (lu_t == JV_F32 && b_t == JV_F32 && x_t == JV_F32) { JV_BAND_SOLVE(float, float, float) }
    else if (lu_t == JV_F32 && b_t == JV_F64 && x_t == JV_F32) { JV_BAND_SOLVE(float, double, float) }
    else if (lu_t == JV_F32 && b_t == JV_F32 && x_t == JV_F64) { JV_BAND_SOLVE(float, float, double) }
    else if (lu_t == JV_F32 && b_t == JV_F64 && x_t == JV_F64) { JV_BAND_SOLVE(float, double, double) }
    else return JV_ERR_ARG;
#undef JV_BAND_SOLVE
    JV_CHECK_LAUNCH();
    return JV_OK;
}

int band_factor(jv_handle h, jv_dtype vals_t, const void *vals, jv_dtype lu_t, void *lu,
                void *scratch) {
    const BandPlan &bp = h->ls[JV_LOWER].band;
    BandFactorArgs a{};
    a.rowptr = h->rowptr;
    a.colidx = h->colidx;
    a.diag = h->diag;
    a.kdiag = h->kdiag;
    a.pair_ptr = h->pair_ptr;
    a.pairs = h->pairs;
    a.rows = bp.rows;
    a.bl_ptr = bp.bl_ptr;
    a.ll_ptr = bp.ll_ptr;
    a.n = h->n;
    a.B = bp.B;
    a.nb = bp.nb;
    a.vals = vals;
    a.lu = lu;
    a.scratch = scratch;
    a.ticket = h->ticket;
    a.status = h->status;
    a.timeout = h->opt.spin_timeout_cycles > 0 ? h->opt.spin_timeout_cycles : kDefaultSpin;
    a.fault_row = h->opt.fault_row;
    cudaStream_t s = h->stream;
    const size_t tl = lu_t == JV_F64 ? 8 : 4;
    int rc = fill_u32(lu, (size_t)h->nnz * (tl / 4), ~0u, s);
    if (rc) return rc;
    const int grid = std::min(bp.nb, h->num_sms * 2);
    const size_t smem = (size_t)kBlock * kLaneSlot * tl;
    if (lu_t == JV_F64 && vals_t == JV_F64) {
        count_launch();
        k_band_ilu0<double, double><<<grid, kBlock, smem, s>>>(a);
    } else if (lu_t == JV_F32 && vals_t == JV_F32) {
        count_launch();
        k_band_ilu0<float, float><<<grid, kBlock, smem, s>>>(a);
    } else if (lu_t == JV_F32 && vals_t == JV_F64) {
        count_launch();
        k_band_ilu0<double, float><<<grid, kBlock, smem, s>>>(a);
    } else {
        return JV_ERR_ARG;
    }
    JV_CHECK_LAUNCH();
    return JV_OK;
}

}  // namespace jv
