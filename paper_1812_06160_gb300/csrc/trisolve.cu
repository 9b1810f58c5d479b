// Sparse triangular solves ("stri", Sec. VI): forward substitution with the
// unit lower factor, backward substitution with U, and the two transposed
// solves of the adjoint, all on the level structure built by the analysis
// (Sec. III-A: the factor and the solves share one DAG).
//
// Row r computes s = b_r; s = s - t_rj x_j over its dependency entries in a
// fixed order; x_r = s [/ u_rr].  The entries are a sub-range of row r of the
// CSR (L, U) or of column r of the CSC (U^T, L^T, values fetched through
// csc2csr).  The order is the one the serial substitution uses (ascending
// columns; descending rows for L^T) and every update is one fused
// multiply-add, so the result equals the serial solve bit for bit; only the
// loads run in parallel.  (FP64 U and U^T solves form s / u_rr from 1/u_rr,
// computed while the row waits, and one correction -- the same quotient as
// the division, with a third of its instructions after the last operand
// arrives -- unless jv_options.exact asks for the division itself.)
//
// Work list (see Bins): a short task holds up to 32 rows of one level, one
// lane per row.  Every lane polls the next W dependencies of its own row (a
// window of 2, 4, 8 or 16, the smallest that holds the longest such row: every
// slot is an unrolled step of the poll loop, and its instructions are on the
// critical path of every level),
// consumes the ready prefix in order and publishes its row the moment the
// last one arrives, so no lane waits for another lane's dependencies.  A
// long task is one row with many dependencies; the whole warp loads 32 x
// kUnroll of them at a time and replays the ordered chain through shuffles
// (jv_options.exact), or, by default, every lane sums its own share in
// ascending order and a fixed tree combines the 32 shares: a chain about a
// 32nd as long (a 2,000-entry row of the power-law matrix was a chain of
// 2,000 dependent FP64 operations), deterministic, but not the serial order.
// Several right-hand sides: one warp per row, one lane per right-hand side
// (row-major n x nrhs: the lanes read one contiguous segment of every
// dependency row).
//
// LEVEL mode: one launch per level.  SYNCFREE mode: one persistent launch
// over all levels (see sf_next_chunk); the output vector is pre-filled with a
// sentinel bit pattern and one relaxed store publishes a finished value, so
// each dependency is awaited on its own output word (no flags, no fences).
#include <algorithm>

#include "jv_internal.cuh"

namespace jv {
namespace {

struct TriArgs {
    Span beg, end;         // dependency range of row r: [beg(r), end(r))
    const int *idx;        // column (CSR) or row (CSC) index of every entry
    const int *vmap;       // CSC -> CSR value position, or nullptr
    const int *diag;
    int unit;              // 1: unit diagonal (L, L^T)
    int rcp;               // FP64 U, U^T: divide through 1/u_rr (rcp_newton, computed before
                           // the row's operands arrive) and one correction (div_rcp)
    int tree;              // long rows: lanes sum their shares, then a fixed tree (not the
                           // serial order; jv_options.exact = 0)
    int reverse;           // 1: walk the range from its end (L^T)
    const int *rows, *task_lo, *task_hi;
    int task_begin, task_end;
    const void *lu, *b;
    void *x;
    void *xp;              // one-column solves: x at every row's work-list position (the word
                           // dependants poll; sentinel-filled in SYNCFREE mode)
    const int *ipos;       // work-list position of every row
    int nrhs;
    unsigned *ticket;
    unsigned long long *status;
    long long timeout;
    unsigned backoff_ns;
    int fault_row;
};

template <class T> struct RN;
template <> struct RN<double> {
    __device__ static double fms(double a, double b, double c) { return __fma_rn(-a, b, c); }
    __device__ static double div(double a, double b) { return __ddiv_rn(a, b); }
};
template <> struct RN<float> {
    __device__ static float fms(float a, float b, float c) { return __fmaf_rn(-a, b, c); }
    __device__ static float div(float a, float b) { return __fdiv_rn(a, b); }
};

// Spin (bounded) until *p no longer holds the sentinel; `u` is a first read.
template <class TX>
__device__ __forceinline__ typename Bits<TX>::U settle(const TX *p, typename Bits<TX>::U u,
                                                       const TriArgs &a, int r,
                                                       bool &fail) {
    using B = Bits<TX>;
    using U = typename B::U;
    if (u != B::kSent) return u;
    const long long t0 = clock64();
    unsigned it = 0;
    for (;;) {
        sf_pause(it, a.backoff_ns);
        u = ld_relaxed(reinterpret_cast<const U *>(p));
        if (u != B::kSent) return u;
        if ((++it & 15u) == 0) {
            if (sf_aborted(a.ticket)) {           // another wait gave up: so does this row
                fail = true;                      // (silently: that wait has reported)
                return B::kCanonNan;
            }
            if (clock64() - t0 > a.timeout) {
                report(a.status, JV_ERR_TIMEOUT, r);
                sf_abort(a.ticket);
                fail = true;
                return B::kCanonNan;
            }
        }
    }
}

template <class TX>
__device__ __forceinline__ void publish(TX *p, TX v) {
    using B = Bits<TX>;
    typename B::U u = B::to(v);
    st_relaxed(reinterpret_cast<typename B::U *>(p), B::nan_bits(u) ? B::kCanonNan : u);
}

template <class TX, bool SF>
__device__ __forceinline__ typename Bits<TX>::U first_read(const TX *p) {
    using U = typename Bits<TX>::U;
    if constexpr (SF) return ld_relaxed(reinterpret_cast<const U *>(p));
    else return *reinterpret_cast<const U *>(p);
}

template <class TL>
__device__ __forceinline__ TL load_val(const TriArgs &a, int q) {
    const TL *lu = static_cast<const TL *>(a.lu);
    return a.vmap ? __ldg(lu + __ldg(a.vmap + q)) : __ldg(lu + q);
}

// The diagonal a row finishes with, u_rr, and (FP64 with rcp) its reciprocal
// y, computed while the row waits for its operands.
template <class TL>
__device__ __forceinline__ TL load_diag(const TriArgs &a, int r, TL &y) {
    const TL d = __ldg(static_cast<const TL *>(a.lu) + __ldg(a.diag + r));
    y = (TL)1;
    if constexpr (sizeof(TL) == 8) {
        if (a.rcp) y = rcp_newton(d);
    }
    return d;
}
// x_r = s / u_rr from the finished sum (the same quotient either way)
template <class TL>
__device__ __forceinline__ TL finish_row(const TriArgs &a, TL s, TL d, TL y) {
    if (a.unit) return s;
    if constexpr (sizeof(TL) == 8) {
        if (a.rcp) return div_rcp(s, d, y);
    }
    return RN<TL>::div(s, d);
}

// A one-column row's result: published at its work-list position (the word
// its dependants poll: the rows of a task are consecutive there, and so are
// the rows their dependants' tasks read, whatever the matrix ordering), and
// stored at row r of x.
template <class TL, class TX>
__device__ __forceinline__ void store_xp(const TriArgs &a, bool sf, int pos, int r, TL v) {
    TX *xp = static_cast<TX *>(a.xp);
    if (sf) {
        if (r != a.fault_row) publish<TX>(xp + pos, (TX)v);
    } else {
        xp[pos] = (TX)v;
    }
    static_cast<TX *>(a.x)[r] = (TX)v;
}

template <class TL, class TX>
__device__ __forceinline__ void store_x(const TriArgs &a, bool sf, TX *p, int r, TL v) {
    if (sf) {
        if (r != a.fault_row) publish<TX>(p, (TX)v);
    } else {
        *p = (TX)v;
    }
}

// Short task: rows[lo..hi) of one level, one lane per row, polled independently.
// The indices and values of the next W dependencies (a window) are loaded
// once; every poll round then re-reads only the x words still missing.
template <class TL, class TB, class TX, bool SF, int W, bool ONE>
__device__ __forceinline__ void trsv_lanes(const TriArgs &a, int lo, int hi) {
    using B = Bits<TX>;
    using U = typename B::U;
    const int lane = threadIdx.x & 31;
    const int pos = lo + lane;
    const TX *x = static_cast<const TX *>(a.xp);           // polled by work-list position
    bool done = pos >= hi;
    int r = 0, qb = 0, len = 0, e = 0, wb = 0, wend = 0;
    TL s = 0, d = 1, dy = 1;
    int jw[W];
    TL vw[W];
    if (!done) {
        r = __ldg(a.rows + pos);
        qb = a.beg.at(r);
        len = a.end.at(r) - qb;
        s = (TL)__ldg(static_cast<const TB *>(a.b) + r);
        if (!a.unit) d = load_diag<TL>(a, r, dy);
        if (len > 0) {               // first window: indices and values
            wend = min(W, len);
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (k < wend) {
                    const int q = a.reverse ? qb + len - 1 - k : qb + k;
                    jw[k] = __ldg(a.ipos + __ldg(a.idx + q));
                    vw[k] = load_val<TL>(a, q);
                }
        }
    }
    U u[W];
    long long t0 = 0;
    unsigned rounds = 0;
    if constexpr (SF && ONE) {
        // Every row of the work list fits one window (len <= W): each round
        // polls only the words not seen yet, and a row finishes -- its
        // ordered chain, then its store -- in the round its last word arrives.
        // Wide windows (8, 16) consume the ready prefix in chunks of 4 as it
        // grows, each chunk issued only when some lane needs it, so that only
        // the last chunk's fused multiply-adds (64 cycles per FP64 warp
        // instruction) follow the last arrival; narrow ones chain at the end.
        unsigned seen = 0u;
        const unsigned need = (1u << len) - 1u;
        if (sizeof(TL) == 8 && W < 8 && hi - lo > 16) {
            // FP64 in a task of more than 16 rows (wide levels): a warp
            // instruction of the chain costs the same with 1 or 32 lanes, so
            // the warp polls until all its rows are ready, then chains and
            // stores them together (C2 L and U solves 0.68 -> 0.63 ms; tasks
            // of 16 rows, on narrow levels, lost 2 % this way and keep the
            // per-row finish below)
            // (for at most kHoldRounds rounds: then the rows finish one by
            // one below, so that a row held for a slow warp-mate never holds
            // up its own dependants for long)
            bool ready = done || len == 0;
            bool together = true;
            for (unsigned held = 0;; ++held) {
#pragma unroll
                for (int k = 0; k < W; ++k)
                    if (!ready && k < len && !((seen >> k) & 1u)) u[k] = ld_relaxed(reinterpret_cast<const U *>(x + jw[k]));
#pragma unroll
                for (int k = 0; k < W; ++k)
                    if (!ready && k < len && !((seen >> k) & 1u) && u[k] != B::kSent) seen |= 1u << k;
                ready = ready || seen == need;
                if (__all_sync(0xffffffffu, ready)) break;
                if (held >= kHoldRounds) {
                    together = false;
                    break;
                }
                if (!ready) {
                    if (rounds++ == 0) t0 = clock64();
                    if ((rounds & 15u) == 0) {
                        if (sf_aborted(a.ticket)) {
                            ready = done = true;          // another wait gave up and reported
                        } else if (clock64() - t0 > a.timeout) {
                            report(a.status, JV_ERR_TIMEOUT, r);
                            sf_abort(a.ticket);
                            ready = done = true;
                        }
                    }
                }
            }
            if (together) {
                if (!done) {
#pragma unroll
                    for (int k = 0; k < W; ++k)
                        if (k < len) s = RN<TL>::fms(vw[k], (TL)B::from(u[k]), s);
                    store_xp<TL, TX>(a, SF, pos, r, finish_row<TL>(a, s, d, dy));
                }
                return;
            }
        }
        int e = 0;                                       // entries consumed (wide windows)
        while (__any_sync(0xffffffffu, !done)) {
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (!done && k < len && !((seen >> k) & 1u)) u[k] = ld_relaxed(reinterpret_cast<const U *>(x + jw[k]));
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (!done && k < len && !((seen >> k) & 1u) && u[k] != B::kSent) seen |= 1u << k;
            if constexpr (W >= 8) {
                const int p = done ? e : __ffs(~seen) - 1;   // ready prefix [0, p)
#pragma unroll
                for (int q = 0; q < W; q += 4)
                    if (__any_sync(0xffffffffu, e < q + 4 && p > q)) {
#pragma unroll
                        for (int k = q; k < q + 4; ++k)
                            if (k >= e && k < p) s = RN<TL>::fms(vw[k], (TL)B::from(u[k]), s);
                    }
                e = p;
            }
            if (!done && seen == need) {
                if constexpr (W < 8) {
#pragma unroll
                    for (int k = 0; k < W; ++k)
                        if (k < len) s = RN<TL>::fms(vw[k], (TL)B::from(u[k]), s);
                }
                store_xp<TL, TX>(a, SF, pos, r, finish_row<TL>(a, s, d, dy));
                done = true;
            } else if (!done) {
                if (rounds++ == 0) t0 = clock64();
                if ((rounds & 15u) == 0) {
                    if (sf_aborted(a.ticket)) {
                        done = true;                  // another wait gave up and reported
                    } else if (clock64() - t0 > a.timeout) {
                        report(a.status, JV_ERR_TIMEOUT, r);
                        sf_abort(a.ticket);
                        done = true;
                    }
                }
            }
        }
        return;
    }
    // The loop body is warp-uniform (finished lanes only mask their work),
    // so the consume step -- FP64 fused multiply-adds, slow on this part's
    // narrow FP64 pipe even when predicated off -- is skipped outright in
    // the common round where no lane's next dependency has arrived.
    while (__any_sync(0xffffffffu, !done)) {
        if (!done && e == wend && e < len) {
            // next window [wb, wend): indices, values and a first read of every x
            wb = e;
            wend = min(e + W, len);
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (wb + k < wend) {
                    const int q = a.reverse ? qb + len - 1 - (wb + k) : qb + wb + k;
                    jw[k] = __ldg(a.ipos + __ldg(a.idx + q));
                    vw[k] = load_val<TL>(a, q);
                }
        }
        // (re-)read every entry of the window not consumed yet; dependencies
        // tend to arrive together, so they are all polled in the same round
        bool progress = !done && e == len;
#pragma unroll
        for (int k = 0; k < W; ++k)
            if (!done && wb + k >= e && wb + k < wend) {
                u[k] = first_read<TX, SF>(x + jw[k]);
                if (wb + k == e) progress = !SF || u[k] != B::kSent;
            }
        if (__any_sync(0xffffffffu, progress) && !done) {
            // consume the ready prefix, in order
            bool ok = true;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (wb + k < e) continue;
                if (ok && wb + k < wend && (!SF || u[k] != B::kSent)) {
                    s = RN<TL>::fms(vw[k], (TL)B::from(u[k]), s);
                    ++e;
                } else {
                    ok = false;
                }
            }
            if (e == len) {
                store_xp<TL, TX>(a, SF, pos, r, finish_row<TL>(a, s, d, dy));
                done = true;
            }
        }
        if (SF && !done && !progress) {
            if (rounds++ == 0) t0 = clock64();
            if ((rounds & 15u) == 0) {
                if (sf_aborted(a.ticket)) {
                    done = true;                  // another wait gave up and reported
                } else if (clock64() - t0 > a.timeout) {
                    report(a.status, JV_ERR_TIMEOUT, r);
                    sf_abort(a.ticket);
                    done = true;
                }
            }
        }
    }
}

// Long task: one row, the whole warp loads its dependencies.
template <class TL, class TB, class TX, bool SF>
__device__ __forceinline__ void trsv_warp(const TriArgs &a, int pos) {
    using B = Bits<TX>;
    using U = typename B::U;
    constexpr int CH = kWarp * kUnroll;
    const int lane = threadIdx.x & 31;
    const TX *x = static_cast<const TX *>(a.xp);           // polled by work-list position
    const int r = __ldg(a.rows + pos);
    const int qb = a.beg.at(r);
    const int len = a.end.at(r) - qb;
    TL s = (TL)__ldg(static_cast<const TB *>(a.b) + r);
    TL dy = 1;
    const TL d = a.unit ? (TL)1 : load_diag<TL>(a, r, dy);
    bool fail = false;                 // a wait gave up: publish nothing
    TL part = 0;                       // tree: this lane's share of the sum
    for (int c0 = 0; c0 < len; c0 += CH) {
        int q[kUnroll];
        TL v[kUnroll];
        U u[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const int e = c0 + k * kWarp + lane;
            q[k] = -1;
            if (e < len) {
                q[k] = a.reverse ? qb + len - 1 - e : qb + e;
                v[k] = load_val<TL>(a, q[k]);
                u[k] = first_read<TX, SF>(x + __ldg(a.ipos + __ldg(a.idx + q[k])));
            }
        }
        TL xv[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            xv[k] = 0;
            if (q[k] >= 0) {
                if (SF) u[k] = settle<TX>(x + __ldg(a.ipos + __ldg(a.idx + q[k])), u[k], a, r, fail);
                xv[k] = (TL)B::from(u[k]);
            } else {
                v[k] = 0;
            }
        }
        if (a.tree) {
            // each lane's share, in ascending order (absent entries are 0 * 0)
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) part = RN<TL>::fms(v[k], xv[k], part);
        } else {
            // the ordered chain: entry c0 + k*32 + l is held by lane l
#pragma unroll
            for (int k = 0; k < kUnroll; ++k)
                for (int l = 0; l < kWarp; ++l) {
                    const TL vl = __shfl_sync(0xffffffffu, v[k], l);
                    const TL xl = __shfl_sync(0xffffffffu, xv[k], l);
                    if (c0 + k * kWarp + l < len) s = RN<TL>::fms(vl, xl, s);
                }
        }
    }
    if (a.tree) {                      // the lanes' shares combined by a fixed tree
#pragma unroll
        for (int off = kWarp / 2; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        s += part;
    }
    if (SF && __any_sync(0xffffffffu, fail)) return;
    if (lane == 0) store_xp<TL, TX>(a, SF, pos, r, finish_row<TL>(a, s, d, dy));
}

template <class TL, class TB, class TX, bool SF, int W, bool ONE>
__device__ __forceinline__ void trsv_task(const TriArgs &a, int task) {
    const int lo = __ldg(a.task_lo + task), hi = __ldg(a.task_hi + task);
    if (hi & kLongBit) trsv_warp<TL, TB, TX, SF>(a, lo);
    else trsv_lanes<TL, TB, TX, SF, W, ONE>(a, lo, hi);
}

template <class TL, class TB, class TX, bool SF, int W, bool ONE>
__global__ void __launch_bounds__(kBlock, 1) k_trsv(TriArgs a) {
    const int wib = threadIdx.x >> 5;
    if (SF) {
        sf_for_each_task(a.ticket, a.task_begin, a.task_end,
                         [&](int task) { trsv_task<TL, TB, TX, SF, W, ONE>(a, task); });
        sf_finish(a.ticket);
    } else {
        const int task = a.task_begin + blockIdx.x * kWarpsPerBlock + wib;
        if (task < a.task_end) trsv_task<TL, TB, TX, SF, W, ONE>(a, task);
    }
}

// Several right-hand sides: one warp per row (rows[task]), one lane per column.
template <class TL, class TB, class TX, bool SF>
__device__ __forceinline__ void trsm_task(const TriArgs &a, int task) {
    using B = Bits<TX>;
    using U = typename B::U;
    const int lane = threadIdx.x & 31;
    const int r = __ldg(a.rows + task);
    const int qb = a.beg.at(r), len = a.end.at(r) - qb;
    const size_t ld = (size_t)a.nrhs;
    TX *x = static_cast<TX *>(a.x);
    const TB *b = static_cast<const TB *>(a.b);
    TL dy = 1;
    const TL d = a.unit ? (TL)1 : load_diag<TL>(a, r, dy);
    for (int c0 = 0; c0 < a.nrhs; c0 += 32) {
        const int c = c0 + lane;
        const bool ok = c < a.nrhs;
        TL s = ok ? (TL)b[(size_t)r * ld + c] : (TL)0;
        bool fail = false;             // a wait gave up: publish nothing
        for (int e0 = 0; e0 < len; e0 += kUnroll) {
            int j[kUnroll];
            TL v[kUnroll];
            U u[kUnroll];
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                const int e = e0 + k;
                j[k] = -1;
                if (e < len) {
                    const int q = a.reverse ? qb + len - 1 - e : qb + e;
                    j[k] = __ldg(a.idx + q);
                    v[k] = load_val<TL>(a, q);
                    if (ok) u[k] = first_read<TX, SF>(x + (size_t)j[k] * ld + c);
                }
            }
            if (ok) {
#pragma unroll
                for (int k = 0; k < kUnroll; ++k) {
                    if (j[k] >= 0) {
                        if (SF) u[k] = settle<TX>(x + (size_t)j[k] * ld + c, u[k], a, r, fail);
                        s = RN<TL>::fms(v[k], (TL)B::from(u[k]), s);
                    }
                }
            }
        }
        if (ok && !fail) store_x<TL, TX>(a, SF, x + (size_t)r * ld + c, r, finish_row<TL>(a, s, d, dy));
    }
}

template <class TL, class TB, class TX, bool SF>
__global__ void __launch_bounds__(kBlock) k_trsm(TriArgs a) {
    const int wib = threadIdx.x >> 5;
    if (SF) {
        sf_for_each_task(a.ticket, a.task_begin, a.task_end, [&](int task) { trsm_task<TL, TB, TX, SF>(a, task); });
        sf_finish(a.ticket);
    } else {
        const int task = a.task_begin + blockIdx.x * kWarpsPerBlock + wib;
        if (task < a.task_end) trsm_task<TL, TB, TX, SF>(a, task);
    }
}

template <class TL, class TB, class TX, bool SF>
int launch(bool multi, int window, int grid, cudaStream_t s, const TriArgs &a) {
    count_launch();
    if (multi) k_trsm<TL, TB, TX, SF><<<grid, kBlock, 0, s>>>(a);
    else if (window <= 2) k_trsv<TL, TB, TX, SF, 2, true><<<grid, kBlock, 0, s>>>(a);
    else if (window <= 4) k_trsv<TL, TB, TX, SF, 4, true><<<grid, kBlock, 0, s>>>(a);
    else if (window <= 8) k_trsv<TL, TB, TX, SF, 8, true><<<grid, kBlock, 0, s>>>(a);
    else if (window <= 16) k_trsv<TL, TB, TX, SF, 16, true><<<grid, kBlock, 0, s>>>(a);
    else k_trsv<TL, TB, TX, SF, kPoll, false><<<grid, kBlock, 0, s>>>(a);
    JV_CHECK_LAUNCH();
    return JV_OK;
}

template <class T> constexpr jv_dtype dt() { return sizeof(T) == 8 ? JV_F64 : JV_F32; }

template <class TL, class TB, class TX>
int run(jv_handle h, int structure, const void *lu, const void *b, void *x, int nrhs) {
    const LevelSet &L = h->ls[structure];
    if (h->opt.mode == JV_MODE_SYNCFREE && nrhs == 1 && L.band.use)
        return band_solve(h, structure, dt<TL>(), lu, dt<TB>(), b, dt<TX>(), x);
    const Bins &W = L.bins;
    cudaStream_t s = h->stream;
    TriArgs a{};
    switch (structure) {
        case JV_LOWER:
            a.beg = {h->rowptr, 0, 0}; a.end = {h->diag, 0, 0};
            a.idx = h->colidx; a.vmap = nullptr; a.unit = 1; a.reverse = 0; break;
        case JV_UPPER:
            a.beg = {h->diag, 0, 1}; a.end = {h->rowptr, 1, 0};
            a.idx = h->colidx; a.vmap = nullptr; a.unit = 0; a.reverse = 0; break;
        case JV_UPPER_T:
            a.beg = {h->colptr, 0, 0}; a.end = {h->cdiag, 0, 0};
            a.idx = h->rowidx; a.vmap = h->csc2csr; a.unit = 0; a.reverse = 0; break;
        default:  // JV_LOWER_T
            a.beg = {h->cdiag, 0, 1}; a.end = {h->colptr, 1, 0};
            a.idx = h->rowidx; a.vmap = h->csc2csr; a.unit = 1; a.reverse = 1; break;
    }
    const bool multi = nrhs > 1;
    if (!multi) {                       // the polled copy of x, by work-list position
        const int rc = ensure_buffer(h, &h->xpos, &h->xpos_bytes, (size_t)h->n * sizeof(TX));
        if (rc) return rc;
        a.xp = h->xpos;
        a.ipos = W.ipos;
    }
    a.diag = h->diag;
    a.rows = multi ? L.rows : W.rows;
    a.task_lo = W.task_lo;
    a.task_hi = W.task_hi;
    a.lu = lu;
    a.b = b;
    a.x = x;
    a.nrhs = nrhs;
    a.ticket = h->ticket;
    a.status = h->status;
    a.timeout = h->opt.spin_timeout_cycles > 0 ? h->opt.spin_timeout_cycles : kDefaultSpin;
    a.fault_row = h->opt.fault_row;
    a.backoff_ns = sf_backoff(h);
    a.rcp = sizeof(TL) == 8 && !h->opt.exact;
    a.tree = !h->opt.exact;
    // a one-column solve may end in an Even-Rows corner: the upper stage
    // then runs the levels above it
    const SolveCorner *C = multi ? nullptr : solve_corner_of(h, structure, sizeof(TL), sizeof(TX));
    const int lend = C ? C->K : L.nlev;
    // tasks of levels [l0, l1): rows (several right-hand sides) or work-list tasks
    auto tasks = [&](int l0, int l1) {
        a.task_begin = multi ? L.h_ptr[l0] : W.h_task_ptr[l0];
        a.task_end = multi ? L.h_ptr[l1] : W.h_task_ptr[l1];
    };
    // the launch sequence on stream s (the handle's, or a capture stream)
    auto seq = [&](cudaStream_t s) -> int {
        auto one_level = [&](int l) {
            tasks(l, l + 1);
            return launch<TL, TB, TX, false>(multi, W.window,
                                             grid_for(a.task_end - a.task_begin, kWarpsPerBlock), s, a);
        };
        auto sync_free = [&](int l0, int l1) {
            tasks(l0, l1);
            if (a.task_end <= a.task_begin) return (int)JV_OK;
            // several right-hand sides: one row per task, so one CTA per SM
            // would claim little more than one level ahead of the dependency
            // front; two per SM (32-45 registers a thread) measured 18 %
            // faster on 32 columns, while one-column solves lost with two
            return launch<TL, TB, TX, true>(multi, W.window,
                                            sf_grid(h, a.task_end - a.task_begin, multi ? 2 : 1), s, a);
        };
        int rc = JV_OK;
        if (has_sync_free(h, L, lend)) {
            rc = fill_u32(multi ? x : h->xpos, (size_t)h->n * nrhs * (sizeof(TX) / 4), ~0u, s);
            if (rc) return rc;
        }
        if (h->opt.mode == JV_MODE_SYNCFREE) {
            rc = sync_free(0, lend);
        } else if (h->opt.mode == JV_MODE_LEVEL) {
            for (int l = 0; l < lend && rc == JV_OK; ++l) rc = one_level(l);
        } else {
            // hybrid: upper-stage levels one launch each, second-stage runs sync-free
            for (const Seg &g : L.segs) {
                if (g.l0 >= lend || rc != JV_OK) break;
                const int l1 = std::min(g.l1, lend);
                if (g.sf) rc = sync_free(g.l0, l1);
                else for (int l = g.l0; l < l1 && rc == JV_OK; ++l) rc = one_level(l);
            }
        }
        if (rc != JV_OK || !C) return rc;
        return corner_solve(h, structure, *C, dt<TL>(), lu, dt<TB>(), b, dt<TX>(), x, s);
    };
    if (h->opt.mode == JV_MODE_SYNCFREE) return seq(s);
    const std::vector<unsigned long long> key = {
        2, (unsigned long long)structure, sizeof(TL), sizeof(TB), sizeof(TX),
        (unsigned long long)h->opt.mode, (unsigned long long)(uintptr_t)lu,
        (unsigned long long)(uintptr_t)b, (unsigned long long)(uintptr_t)x, (unsigned long long)nrhs,
        (unsigned long long)(uintptr_t)a.xp};
    return graph_run(h, key, seq);
}

__global__ void k_widen(size_t m, const float *in, double *out) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < m) out[i] = (double)in[i];
}

// An FP32 factor's solve into an FP64 x (the preconditioner of the FP64
// Krylov drivers writes z this way) runs into an FP32 scratch vector, then
// widens it in one pass.  Widening is exact, and every dependant read the
// FP32 value either way, so x is the same bit for bit; the solve itself
// then polls 4-byte words and converts nothing per row (the conversions go
// to the narrow FP64 pipe: C2 U solve 0.545 -> 0.44 ms).
template <class TB>
int run_widened(jv_handle h, int structure, const void *lu, const void *b, void *x, int nrhs) {
    const size_t m = (size_t)h->n * nrhs;
    if (h->xscratch_bytes < m * sizeof(float)) {
        if (h->xscratch) {
            JV_CUDA(cudaStreamSynchronize(h->stream));
            cudaFree(h->xscratch);
            h->xscratch = nullptr;
            h->xscratch_bytes = 0;
        }
        if (cudaMalloc(&h->xscratch, m * sizeof(float) + 16) != cudaSuccess) {
            cudaGetLastError();
            h->xscratch = nullptr;
            return JV_ERR_NOMEM;
        }
        h->xscratch_bytes = m * sizeof(float);
    }
    int rc = run<float, TB, float>(h, structure, lu, b, h->xscratch, nrhs);
    if (rc) return rc;
    if (m == 0) return JV_OK;
    count_launch();
    k_widen<<<grid_for((long long)m, kBlock), kBlock, 0, h->stream>>>(
        m, static_cast<const float *>(h->xscratch), static_cast<double *>(x));
    JV_CHECK_LAUNCH();
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
        return run_widened<float>(h, structure, lu, b, x, nrhs);
    if (lu_t == JV_F32 && b_t == JV_F64 && x_t == JV_F64)
        return run_widened<double>(h, structure, lu, b, x, nrhs);
    return JV_ERR_ARG;
}

}  // namespace jv
