// Numeric ILU(0) on A's own pattern -- Sec. III, Fig. 1 (up-looking: row by
// row, every row "looks up" at the already-factored rows it depends on):
//
//   for every col k < r of row r, in ascending order (entry p = (r, k)):
//       l_rk = a_rk / u_kk
//       for every precomputed pair (t, q) of p:      (t = (r, j), q = (k, j), j > k)
//           a_rt = a_rt - l_rk * u_kq                (one fused multiply-add)
//
// Every entry receives its updates in ascending k, with the same IEEE
// operations as the serial algorithm, so the factor equals it bit for bit.
// The pairs come from the symbolic pass of the analysis (the update
// structure of Fig. 1 depends only on the pattern).
//
// A row's U operands are u_kk for each lower entry, then u_kq for each pair,
// in the order the steps consume them.  A task first loads, in one batch of
// independent loads, everything the row needs that does not depend on other
// rows: its values, the positions of its operands, its pair targets and step
// boundaries -- into shared memory.  After that, waiting costs one memory
// round trip per poll and the arithmetic touches shared memory only.
//
// Work list (see Bins): a short task holds up to 32 rows of one level, one
// lane per row (a per-lane slot interleaved across the warp's shared memory);
// every lane polls its next W operands (4 or 8), keeps the ready prefix, and
// factors and publishes its row as soon as the last one arrives -- no lane
// waits for another's dependencies.  A long task is one row run by the whole
// warp (operands prefetched, pairs split over the lanes, steps in order);
// rows too large for the warp's shared memory work in a global scratch area
// and await each operand when they use it.
//
// Pivots: a finished row k publishes its pivot in a separate array, at the
// row's position in the work list (tasks hold consecutive positions, and the
// rows of consecutive tasks of one level depend on consecutive positions of
// earlier levels, so a warp's polls of its 32 rows' pivots touch a few
// sectors instead of one sector per row, whatever the matrix ordering).  An
// operand u_kq that no step updates keeps A's value throughout, so it is read
// from A's values when the task starts and never awaited; only pivots and
// updated u_kq are polled (for a 5- or 7-point stencil, only the pivots, and
// lu then needs no sentinel fill).
//
// Reciprocal pivots (RCP, FP64 unless jv_options.exact): the pivot
// a row publishes is y_k = 1/u_kk (Newton's iteration, rcp_newton), and a
// dependant forms l_rk = a_rk * y_k.  On this part a warp instruction of the FP64 pipe costs
// 64 cycles whatever its active lanes, and the three correctly rounded
// divisions of a 7-point row were the longest run of FP64 work on the
// critical path of every level; one reciprocal per row (five instructions)
// and one multiply per step replace them.  Each multiplier is then within a
// few units in the last place of the quotient instead of equal to it.
//
// LEVEL mode: one launch per level of lower(A) (Sec. III-A: up-looking ILU has
// the dependency structure of a triangular solve).  SYNCFREE mode (the
// point-to-point synchronisation of Sec. III-A, Fig. 4): one persistent
// launch; the output array is the synchronisation -- lu is first filled with
// a sentinel bit pattern, a finished row publishes each U value with one
// store, and a dependant polls only the U values it reads.
#include <algorithm>
#include <cmath>

#include "jv_internal.cuh"

namespace jv {
namespace {

// Shared memory per warp.  Lane layout: S (the slot, 16 or 32) values (8 B), operand
// positions (4 B) and pair targets / step ends (1 B each) per lane, each
// interleaved across the 32 lanes.
template <int S> __host__ __device__ constexpr int val_bytes() { return kWarp * S * 8; }
template <int S> __host__ __device__ constexpr int warp_smem() {
    return val_bytes<S>() + kWarp * S * (4 + 1 + 1);
}

struct FactorArgs {
    const int *rowptr, *diag, *kdiag, *pair_ptr;
    const int2 *pairs;
    const int *rows, *task_lo, *task_hi;
    const int *task_lev, *task_ptr;   // level gate (SYNCFREE)
    int gate_levels;
    int task_begin, task_end;     // LEVEL: this level's tasks; SYNCFREE: all tasks
    const void *vals;             // A's values (TV)
    void *lu;                     // factor (TL); sentinel-filled in SYNCFREE mode
    void *scratch;                // TL[nnz] work area for long rows that overflow the slot
    unsigned *ticket;
    unsigned long long *status;
    long long timeout;
    unsigned backoff_ns;
    int fault_row;
    int milu;                     // several pairs of one step may target the diagonal
    const int *tpair_ptr;         // pairs by target (one-warp-per-row rows, pull form), or null
    const int2 *tpairs;           // (step p, operand q), q as ~q when it is awaited
    const int *kpos;              // L entries: the work-list position of their pivot row
    void *pscratch;               // operands of rows too long for shared memory
    long long npairs_total;       // offset of the u_kk area in pscratch
    const unsigned char *row_pull; // per row: take the pull form
    const unsigned char *edepth;  // per L entry: depth of its in-row chain (255: 255 or more)
    const unsigned char *upd;     // 1: some step updates the entry (a pair operand to await)
    void *piv;                    // pivot of every row at its work-list position: u_kk, or
                                  // 1/u_kk with RCP (sentinel-filled in SYNCFREE mode)
    int tree;                     // pull form: a U entry with more than kTreePairs updates
                                  // sums them over the warp's lanes and a fixed tree
};

// a U entry of a pull-form row with more updates than this (a hub row's
// diagonal: one update per L entry) sums them over the warp in tree mode
constexpr int kTreePairs = 32;

template <class T> struct RN;
template <> struct RN<double> {
    __device__ static double fms(double a, double b, double c) { return __fma_rn(-a, b, c); }
    __device__ static double div(double a, double b) { return __ddiv_rn(a, b); }
};
template <> struct RN<float> {
    __device__ static float fms(float a, float b, float c) { return __fmaf_rn(-a, b, c); }
    __device__ static float div(float a, float b) { return __fdiv_rn(a, b); }
};

// Bounded spin until the U value at p is published; `u` is a first read.
template <class T>
__device__ __forceinline__ typename Bits<T>::U settle(const T *p, typename Bits<T>::U u,
                                                      const FactorArgs &a, int r,
                                                      bool &fail) {
    using B = Bits<T>;
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

template <class T, bool SF>
__device__ __forceinline__ typename Bits<T>::U first_read(const T *p) {
    using U = typename Bits<T>::U;
    if constexpr (SF) return ld_relaxed(reinterpret_cast<const U *>(p));
    else return *reinterpret_cast<const U *>(p);
}

template <class T>
__device__ __forceinline__ void publish(T *p, T v) {
    using B = Bits<T>;
    typename B::U u = B::to(v);
    st_relaxed(reinterpret_cast<typename B::U *>(p), B::nan_bits(u) ? B::kCanonNan : u);
}

template <class T>
__device__ __forceinline__ void pivot_check(const FactorArgs &a, int r, T d) {
    if (Bits<T>::zero_or_nonfinite_bits(Bits<T>::to(d))) report(a.status, JV_ERR_ZERO_PIVOT, r);
}

// u_kq at lu position q: from A's values when no step updates it, else
// awaited (bounded) on its own word.
template <class TV, class TL, bool SF>
__device__ __forceinline__ TL pair_operand(const FactorArgs &a, int q, int r, bool &fail) {
    if (!__ldg(a.upd + q)) return (TL)__ldg(static_cast<const TV *>(a.vals) + q);
    const TL *src = static_cast<const TL *>(a.lu) + q;
    return Bits<TL>::from(SF ? settle<TL>(src, first_read<TL, SF>(src), a, r, fail)
                             : first_read<TL, SF>(src));
}

// ------------------------------------------------------- one lane per row
template <class TV, class TL, bool SF, int W, int S, bool RCP>
__device__ __forceinline__ void factor_lanes(const FactorArgs &a, int lo, int hi, unsigned gate,
                                             unsigned char *smem) {
    using B = Bits<TL>;
    using U = typename B::U;
    const int lane = threadIdx.x & 31;
    TL *vb = reinterpret_cast<TL *>(smem) + lane;
    int *ob = reinterpret_cast<int *>(smem + val_bytes<S>()) + lane;
    unsigned char *tb = smem + val_bytes<S>() + kWarp * S * 4 + lane;
    unsigned char *eb = tb + kWarp * S;
    auto V = [&](int e) -> TL & { return vb[e * kWarp]; };           // values, then operands
    auto OPOS = [&](int e) -> int & { return ob[e * kWarp]; };       // operand positions
    auto TGT = [&](int i) -> unsigned char & { return tb[i * kWarp]; };
    auto STEP_END = [&](int p) -> unsigned char & { return eb[p * kWarp]; };
    const int pos = lo + lane;
    bool done = pos >= hi;
    int r = 0, rs = 0, len = 0, nl = 0, m = 0, got = 0;
    unsigned tmask = 0;                 // row-local entries some step of the row updates
    unsigned smask = 0;                 // operands final from the start (read from A's values)
    TL *lu = static_cast<TL *>(a.lu);
    TL *piv = static_cast<TL *>(a.piv);
    // where operand e of the row is awaited: the pivot of a step (in piv, at
    // the pivot row's work-list position), or u_kq of a pair (in lu)
    auto src = [&](int e, int pos_) -> const TL * { return (e < nl ? piv : lu) + pos_; };
    if (!done) {
        r = __ldg(a.rows + pos);
        rs = __ldg(a.rowptr + r);
        len = __ldg(a.rowptr + r + 1) - rs;
        nl = __ldg(a.diag + r) - rs;
        const int j0 = __ldg(a.pair_ptr + rs);
        const int np = __ldg(a.pair_ptr + rs + nl) - j0;
        m = nl + np;
        const TV *vals = static_cast<const TV *>(a.vals);
        if constexpr (S <= kLaneSlot) {
            TL v[S];
            int kd[S], se[S];
            int2 pr[S];
#pragma unroll
            for (int e = 0; e < S; ++e) {
                if (e < len) v[e] = (TL)__ldg(vals + rs + e);
                if (e < nl) kd[e] = __ldg(a.kpos + rs + e);       // the pivot's position
                if (e < nl) se[e] = __ldg(a.pair_ptr + rs + e + 1);
                if (e < np) pr[e] = __ldg(a.pairs + j0 + e);
            }
            // the narrow slot: the update flags, then the final-from-the-start
            // operands, as two more batches of loads
            unsigned char up[S];
            TL sv[S];
#pragma unroll
            for (int e = 0; e < S; ++e) {
                if (e < np) up[e] = __ldg(a.upd + pr[e].y);
            }
#pragma unroll
            for (int e = 0; e < S; ++e)
                if (e < np && !up[e]) sv[e] = (TL)__ldg(vals + pr[e].y);  // u_kq = a_kq throughout
#pragma unroll
            for (int e = 0; e < S; ++e) {
                if (e < len) V(e) = v[e];
                if (e < nl) { OPOS(e) = kd[e]; STEP_END(e) = (unsigned char)(se[e] - j0); }
                if (e < np) {
                    OPOS(nl + e) = pr[e].y;
                    TGT(e) = (unsigned char)(pr[e].x - rs);
                    tmask |= 1u << (pr[e].x - rs);
                    if (!up[e]) {
                        V(len + nl + e) = sv[e];
                        smask |= 1u << (nl + e);
                    }
                }
            }
        } else {
            // the wide slot: sixteen entries at a time through shared memory,
            // and the dependent loads read the arrays back, which keeps the
            // registers of the whole kernel (its poll loop included) in bounds
            for (int h0 = 0; h0 < S; h0 += 16) {
                TL v[16];
                int kd[16], se[16];
                int2 pr[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int e = h0 + i;
                    if (e < len) v[i] = (TL)__ldg(vals + rs + e);
                    if (e < nl) kd[i] = __ldg(a.kpos + rs + e);
                    if (e < nl) se[i] = __ldg(a.pair_ptr + rs + e + 1);
                    if (e < np) pr[i] = __ldg(a.pairs + j0 + e);
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int e = h0 + i;
                    if (e < len) V(e) = v[i];
                    if (e < nl) { OPOS(e) = kd[i]; STEP_END(e) = (unsigned char)(se[i] - j0); }
                    if (e < np) {                          // pair slots lie above every step slot
                        OPOS(nl + e) = pr[i].y;
                        TGT(e) = (unsigned char)(pr[i].x - rs);
                        tmask |= 1u << (pr[i].x - rs);
                    }
                }
            }
#pragma unroll 8
            for (int e = 0; e < S; ++e) {
                if (e < np && !__ldg(a.upd + OPOS(nl + e))) smask |= 1u << (nl + e);
            }
#pragma unroll 8
            for (int e = 0; e < S; ++e)
                if (e < np && ((smask >> (nl + e)) & 1u))
                    V(len + nl + e) = (TL)__ldg(vals + OPOS(nl + e));
        }
        // a U entry no step updates is final already: store it now, so that
        // only the updated ones (for a stencil, the diagonal) follow the steps
        // (no row awaits it: a reader takes it from A's values)
#pragma unroll
        for (int e = 0; e < S; ++e)
            if (e >= nl && e < len && !((tmask >> e) & 1u)) lu[rs + e] = V(e);
        if (SF && gate) {               // bring the awaited operands' lines into L2 before sleeping
#pragma unroll
            for (int e = 0; e < S; ++e)
                if (e < m && !((smask >> e) & 1u)) prefetch_l2(src(e, OPOS(e)));
        }
    }
    if (SF && gate) sf_gate_wait(a.ticket, gate, a.timeout);
    // factor the row from its operands in shared memory and publish it
    auto finish = [&]() {
        int j = 0;
        for (int p = 0; p < nl; ++p) {
            const TL lik = RCP ? V(p) * V(len + p) : RN<TL>::div(V(p), V(len + p));
            for (const int j1 = STEP_END(p); j < j1; ++j) {
                const int t = TGT(j);
                V(t) = RN<TL>::fms(lik, V(len + nl + j), V(t));
            }
            V(p) = lik;
        }
        // the pivot (its reciprocal with RCP) first: the word the dependants
        // of a stencil row wait on; then the updated U entries, then the L part
        if (!SF || r != a.fault_row) {
            const TL pv = RCP ? rcp_newton(V(nl)) : V(nl);
            if (SF) publish<TL>(piv + pos, pv);
            else piv[pos] = pv;
            for (int e = nl; e < len; ++e)
                if ((tmask >> e) & 1u) {
                    if (SF) publish<TL>(lu + rs + e, V(e));
                    else lu[rs + e] = V(e);
                }
        }
        pivot_check<TL>(a, r, V(nl));
        for (int e = 0; e < nl; ++e) lu[rs + e] = V(e);
    };
    long long t0 = 0;
    unsigned rounds = 0;
    unsigned held = 0;                  // FP64: rounds the warp's ready rows have waited
    U u[W];
    // operands past the window that must be awaited (the rest were read from
    // A's values): none for MILU's 7-point rows, whose 9 pair operands all are
    const unsigned need = m >= 32 ? 0xffffffffu : (1u << m) - 1u;
    const unsigned late = W >= 32 ? 0u : ((need & ~smask) >> W);
    if (SF && __all_sync(0xffffffffu, done || late == 0u)) {
        // every awaited operand of the row fits the window: each round polls
        // only the operands not seen yet (a bit mask); the row is factored the
        // round its last operand arrives
        int op[W];
#pragma unroll
        for (int k = 0; k < W; ++k) op[k] = k < m ? OPOS(k) : 0;
        unsigned seen = smask;
        while (__any_sync(0xffffffffu, !done)) {
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (!done && k < m && !((seen >> k) & 1u))
                    u[k] = ld_relaxed(reinterpret_cast<const U *>(src(k, op[k])));
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (!done && k < m && !((seen >> k) & 1u) && u[k] != B::kSent) {
                    seen |= 1u << k;
                    V(len + k) = B::from(u[k]);
                }
            const bool ready = !done && seen == need;
            bool go = ready;
            if constexpr (sizeof(TL) == 8) {
                // FP64: every warp instruction of the finish (divisions and
                // fused multiply-adds) costs the same with 1 or 32 lanes, so
                // the rows wait until all rows of the warp are ready and
                // finish together (C2 factor 1.50 -> 1.29 ms, C5 3.94 -> 3.72)
                // -- for at most kHoldRounds rounds, so that a row held for
                // a slow warp-mate never holds up its own dependants for long
                if (!__all_sync(0xffffffffu, done || ready) && ++held <= kHoldRounds) go = false;
            }
            if (go) {
                finish();
                done = true;
            } else if (!done && !ready) {
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
    int wb = 0, wend = 0;
    while (__any_sync(0xffffffffu, !done)) {
        bool ready = false;
        if (!done) {
            if (got == wend) {              // next window of operands [wb, wend)
                wb = got;
                wend = min(got + W, m);
            }
            // (re-)read every awaited operand of the window not taken yet; they
            // tend to be published together, so they are all polled in the same round
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (wb + k >= got && wb + k < wend && !((smask >> (wb + k)) & 1u))
                    u[k] = first_read<TL, SF>(src(wb + k, OPOS(wb + k)));
            bool ok = true;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (wb + k < got) continue;
                const bool fixed = (smask >> (wb + k)) & 1u;     // already in V
                if (ok && wb + k < wend && (fixed || !SF || u[k] != B::kSent)) {
                    if (!fixed) V(len + wb + k) = B::from(u[k]);
                    ++got;
                } else {
                    ok = false;
                }
            }
            ready = got == m;
        }
        bool go = ready;
        if constexpr (sizeof(TL) == 8) {
            // FP64: finish the warp's rows together, as in the single-window
            // loop (C2 MILU(0) factor 3.12 -> 2.21 ms), for a bounded time
            if (!__all_sync(0xffffffffu, done || ready) && ++held <= kHoldRounds) go = false;
        }
        if (go) {
            finish();
            done = true;
        } else if (SF && !done && !ready && got < wend) {
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

// ----------------------------------------- G lanes per row (G = 8 or 32)
// The row at work-list position pos, run by a group of G lanes: the whole
// warp (a long task) or a quarter of it (a medium task of four rows: the
// four groups run the same steps in lockstep when their rows have the same
// shape, as the interior rows of a stencil do, so each FP64 warp instruction
// serves four rows).  smem_bytes: the group's share of the warp's shared
// memory; a row that does not fit works in the global scratch area.
template <class TV, class TL, bool SF, bool RCP, int G>
__device__ __forceinline__ void factor_warp(const FactorArgs &a, int pos, unsigned gate,
                                            unsigned char *smem, int smem_bytes) {
    using B = Bits<TL>;
    using U = typename B::U;
    const int lane = threadIdx.x & (G - 1);
    const unsigned gmask = G == kWarp ? 0xffffffffu
                                      : ((1u << G) - 1u) << ((threadIdx.x & (kWarp - 1)) & ~(G - 1));
    const int r = __ldg(a.rows + pos);
    const int rs = __ldg(a.rowptr + r), re = __ldg(a.rowptr + r + 1), rd = __ldg(a.diag + r);
    const int len = re - rs, nl = rd - rs;
    const int j0 = __ldg(a.pair_ptr + rs);
    const int np = __ldg(a.pair_ptr + rd) - j0;
    const int m = nl + np;
    bool fail = false;                 // a wait gave up: publish nothing
    TL *lu = static_cast<TL *>(a.lu);
    TL *piv = static_cast<TL *>(a.piv);
    const TV *vals = static_cast<const TV *>(a.vals);
    const size_t need = (size_t)(len + m) * sizeof(TL) + (size_t)(np + nl) * sizeof(int);
    const bool fast = need <= (size_t)smem_bytes;
    TL *w = fast ? reinterpret_cast<TL *>(smem) : static_cast<TL *>(a.scratch) + rs;
    TL *uv = w + len;
    int *tgt = reinterpret_cast<int *>(uv + m);                // fast path only
    int *send = tgt + np;
    for (int e = lane; e < len; e += G) w[e] = (TL)__ldg(vals + rs + e);
    if (SF && gate) sf_gate_wait(a.ticket, gate, a.timeout);
    if (fast) {
        for (int e = lane; e < np; e += G) tgt[e] = __ldg(a.pairs + j0 + e).x - rs;
        for (int e = lane; e < nl; e += G) send[e] = __ldg(a.pair_ptr + rs + e + 1) - j0;
        // the operands in two passes that keep no per-operand registers: the
        // first issues every first read (independent loads, all in flight
        // together) and parks the value in shared memory; the second polls, in
        // rounds, the words that still held the sentinel
        auto where = [&](int e, bool &fixed) -> const TL * {
            fixed = false;
            if (e < nl) return piv + __ldg(a.kpos + rs + e);   // pivot of step e
            const int q = __ldg(a.pairs + j0 + e - nl).y;                       // u_kq of a pair
            if (__ldg(a.upd + q)) return lu + q;
            fixed = true;                                  // final from the start: A's value
            return reinterpret_cast<const TL *>(vals + q);
        };
#pragma unroll 4
        for (int e = lane; e < m; e += G) {
            bool fixed;
            const TL *p = where(e, fixed);
            uv[e] = fixed ? (TL)__ldg(reinterpret_cast<const TV *>(p)) : B::from(first_read<TL, SF>(p));
        }
        if (SF) {
            // rounds: every lane re-reads all its words still missing, the
            // loads of a round in flight together, until the group has them all
            // (bounded like every wait: the abort word, then the cycle budget)
            long long t0 = 0;
            unsigned rounds = 0;
            // pivots first: the pair operands a producer updates follow its
            // pivot within a few hundred cycles, so while the row waits only the
            // pivots are polled (13 words of a 27-point row instead of 114)
            for (int ph = 0; ph < 2; ++ph) {
                bool pending = !fail;
                while (__any_sync(gmask, pending)) {
                    if (pending) {
                        pending = false;
#pragma unroll 4
                        for (int e = lane; e < (ph ? m : nl); e += G) {
                            if (B::to(uv[e]) != B::kSent) continue;
                            bool fixed;
                            const U u = ld_relaxed(reinterpret_cast<const U *>(where(e, fixed)));
                            if (u != B::kSent) uv[e] = B::from(u);
                            else pending = true;
                        }
                        if (pending) {
                            if (rounds++ == 0) t0 = clock64();
                            if ((rounds & 15u) == 0) {
                                if (sf_aborted(a.ticket)) {            // another wait gave up
                                    fail = true;
                                    pending = false;
                                } else if (clock64() - t0 > a.timeout) {
                                    report(a.status, JV_ERR_TIMEOUT, r);
                                    sf_abort(a.ticket);
                                    fail = true;
                                    pending = false;
                                }
                            }
                        }
                    }
                }
            }
        }
    }
    __syncwarp(gmask);
    int jb = 0;
    for (int p = 0; p < nl; ++p) {
        TL ukk;
        if (fast) {
            ukk = uv[p];
        } else {
            const TL *src = piv + __ldg(a.kpos + rs + p);
            ukk = B::from(SF ? settle<TL>(src, first_read<TL, SF>(src), a, r, fail) : first_read<TL, SF>(src));
        }
        const TL lik = RCP ? w[p] * ukk : RN<TL>::div(w[p], ukk);
        const int je = fast ? send[p] : __ldg(a.pair_ptr + rs + p + 1) - j0;
        // the targets of one step are distinct -- except, with MILU, the
        // diagonal, which lane 0 then updates alone, in the listed order
        for (int j = jb + lane; j < je; j += G) {
            int t;
            TL uq;
            if (fast) {
                t = tgt[j];
                uq = uv[nl + j];
            } else {
                const int2 tq = __ldg(a.pairs + j0 + j);
                t = tq.x - rs;
                uq = pair_operand<TV, TL, SF>(a, tq.y, r, fail);
            }
            if (!a.milu || t != nl) w[t] = RN<TL>::fms(lik, uq, w[t]);
        }
        if (a.milu && lane == 0) {
            for (int j = jb; j < je; ++j) {
                int t;
                TL uq;
                if (fast) {
                    t = tgt[j];
                    uq = uv[nl + j];
                } else {
                    const int2 tq = __ldg(a.pairs + j0 + j);
                    t = tq.x - rs;
                    if (t != nl) continue;
                    uq = pair_operand<TV, TL, SF>(a, tq.y, r, fail);
                }
                if (t == nl) w[nl] = RN<TL>::fms(lik, uq, w[nl]);
            }
        }
        jb = je;
        __syncwarp(gmask);
        if (lane == 0) w[p] = lik;
    }
    __syncwarp(gmask);
    if (SF && __any_sync(gmask, fail)) return;
    if (lane == 0) pivot_check<TL>(a, r, w[nl]);
    if (lane == 0 && (!SF || r != a.fault_row)) {
        const TL pv = RCP ? rcp_newton(w[nl]) : w[nl];
        if (SF) publish<TL>(piv + pos, pv);
        else piv[pos] = pv;
    }
    for (int e = lane; e < len; e += G) {
        const TL v = w[e];
        if (!SF || e < nl) lu[rs + e] = v;
        else if (r != a.fault_row) publish<TL>(lu + rs + e, v);
    }
    __syncwarp(gmask);                                         // shared memory reusable
}

// ------------------------------------------------- four rows per warp
// The medium rows of a task (up to kWarp / kGroupLanes of one level), one
// group of kGroupLanes lanes each, in lockstep: every loop runs the warp's
// largest trip count and every barrier spans the warp, so the groups never
// diverge and each FP64 warp instruction of the step loop serves all four
// rows (groups whose row has fewer steps, or no row, sit the extra
// iterations out).  Every row of such a task fits its group's share of the
// warp's shared memory (the analysis checks it).
template <class TV, class TL, bool SF, bool RCP>
__device__ __forceinline__ void factor_group(const FactorArgs &a, int lo, int hi, unsigned gate,
                                             unsigned char *smem, int share) {
    using B = Bits<TL>;
    using U = typename B::U;
    constexpr int G = kGroupLanes;
    const int lane = threadIdx.x & (G - 1);
    const int g = (threadIdx.x & (kWarp - 1)) / G;
    const unsigned gmask = ((1u << G) - 1u) << (g * G);
    const int pos = lo + g;
    const bool has = pos < hi;
    int r = 0, rs = 0, len = 0, nl = 0, j0 = 0, np = 0;
    if (has) {
        r = __ldg(a.rows + pos);
        rs = __ldg(a.rowptr + r);
        len = __ldg(a.rowptr + r + 1) - rs;
        const int rd = __ldg(a.diag + r);
        nl = rd - rs;
        j0 = __ldg(a.pair_ptr + rs);
        np = __ldg(a.pair_ptr + rd) - j0;
    }
    const int m = nl + np;
    bool fail = false;
    TL *lu = static_cast<TL *>(a.lu);
    TL *piv = static_cast<TL *>(a.piv);
    const TV *vals = static_cast<const TV *>(a.vals);
    TL *w = reinterpret_cast<TL *>(smem + g * share);
    TL *uv = w + len;
    int *tgt = reinterpret_cast<int *>(uv + m);
    int *send = tgt + np;
    for (int e = lane; e < len; e += G) w[e] = (TL)__ldg(vals + rs + e);
    if (SF && gate) sf_gate_wait(a.ticket, gate, a.timeout);
    for (int e = lane; e < np; e += G) tgt[e] = __ldg(a.pairs + j0 + e).x - rs;
    for (int e = lane; e < nl; e += G) send[e] = __ldg(a.pair_ptr + rs + e + 1) - j0;
    // operands: all first reads in flight together, then rounds over the
    // words still missing (see factor_warp)
    auto where = [&](int e, bool &fixed) -> const TL * {
        fixed = false;
        if (e < nl) return piv + __ldg(a.kpos + rs + e);
        const int q = __ldg(a.pairs + j0 + e - nl).y;
        if (__ldg(a.upd + q)) return lu + q;
        fixed = true;
        return reinterpret_cast<const TL *>(vals + q);
    };
#pragma unroll 4
    for (int e = lane; e < m; e += G) {
        bool fixed;
        const TL *p = where(e, fixed);
        uv[e] = fixed ? (TL)__ldg(reinterpret_cast<const TV *>(p)) : B::from(first_read<TL, SF>(p));
    }
    if (SF) {
        long long t0 = 0;
        unsigned rounds = 0;
        // pivots first: the pair operands a producer updates follow its
        // pivot within a few hundred cycles, so while the row waits only the
        // pivots are polled (13 words of a 27-point row instead of 114)
        for (int ph = 0; ph < 2; ++ph) {
            bool pending = !fail;
            while (__any_sync(0xffffffffu, pending)) {
                if (pending) {
                    pending = false;
#pragma unroll 4
                    for (int e = lane; e < (ph ? m : nl); e += G) {
                        if (B::to(uv[e]) != B::kSent) continue;
                        bool fixed;
                        const U u = ld_relaxed(reinterpret_cast<const U *>(where(e, fixed)));
                        if (u != B::kSent) uv[e] = B::from(u);
                        else pending = true;
                    }
                    if (pending) {
                        if (rounds++ == 0) t0 = clock64();
                        if ((rounds & 15u) == 0) {
                            if (sf_aborted(a.ticket)) {
                                fail = true;
                                pending = false;
                            } else if (clock64() - t0 > a.timeout) {
                                report(a.status, JV_ERR_TIMEOUT, r);
                                sf_abort(a.ticket);
                                fail = true;
                                pending = false;
                            }
                        }
                    }
                }
            }
        }
    }
    __syncwarp();
    // the steps, in lockstep across the groups
    const int nlmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)nl);
    int jb = 0;
    for (int p = 0; p < nlmax; ++p) {
        TL lik = 0;
        int je = jb;
        if (p < nl) {
            lik = RCP ? w[p] * uv[p] : RN<TL>::div(w[p], uv[p]);
            je = send[p];
        }
        const int cmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)(je - jb));
        for (int c = 0; c < cmax; c += G) {
            const int j = jb + c + lane;
            if (j < je) {
                const int t = tgt[j];
                if (!a.milu || t != nl) w[t] = RN<TL>::fms(lik, uv[nl + j], w[t]);
            }
        }
        // MILU: several pairs of one step may target the diagonal (lane 0, in order)
        if (a.milu && lane == 0)
            for (int j = jb; j < je; ++j)
                if (tgt[j] == nl) w[nl] = RN<TL>::fms(lik, uv[nl + j], w[nl]);
        jb = je;
        __syncwarp();
        if (lane == 0 && p < nl) w[p] = lik;
    }
    __syncwarp();
    const unsigned failed = __ballot_sync(0xffffffffu, fail);
    if (has && !(SF && (failed & gmask))) {
        if (lane == 0) pivot_check<TL>(a, r, w[nl]);
        if (lane == 0 && (!SF || r != a.fault_row)) {
            const TL pv = RCP ? rcp_newton(w[nl]) : w[nl];
            if (SF) publish<TL>(piv + pos, pv);
            else piv[pos] = pv;
        }
        for (int e = lane; e < len; e += G) {
            const TL v = w[e];
            if (!SF || e < nl) lu[rs + e] = v;
            else if (r != a.fault_row) publish<TL>(lu + rs + e, v);
        }
    }
    __syncwarp();                                              // shared memory reusable
}

// ------------------------------------------- one warp per row, pull form
// Fig. 1's arithmetic regrouped by target: entry t of row r receives its
// updates a_t -= l_p u_q (ascending step p, one fused multiply-add each) --
// exactly the sequence the step-by-step sweep applies to it -- and an L entry
// then divides by its u_kk.  So the L entries whose in-row producers are all
// final can be finished together: the warp takes them 32 at a time and
// finishes, wave after wave, every lane whose producers in the chunk are done
// (one division sequence per wave instead of one per step); then every U
// entry pulls its updates at once.  The row's operands (every u_q, every
// u_kk) are read first, in parallel, each through its bounded wait, into
// shared memory (or the operand scratch for a row too long for it).
template <class TV, class TL, bool SF, int S, bool RCP>
__device__ __forceinline__ void factor_warp_pull(const FactorArgs &a, int pos, unsigned gate,
                                                 unsigned char *smem) {
    using B = Bits<TL>;
    const int lane = threadIdx.x & 31;
    const int r = __ldg(a.rows + pos);
    const int rs = __ldg(a.rowptr + r), re = __ldg(a.rowptr + r + 1), rd = __ldg(a.diag + r);
    const int len = re - rs, nl = rd - rs;
    const int s0 = __ldg(a.tpair_ptr + rs);
    const int nq = __ldg(a.tpair_ptr + re) - s0;             // the row's update operands
    TL *lu = static_cast<TL *>(a.lu);
    const TV *vals = static_cast<const TV *>(a.vals);
    bool fail = false;
    const bool fast = (size_t)(len + nl + nq) * sizeof(TL) <= (size_t)warp_smem<S>();
    TL *w, *ukk, *uq;
    if (fast) {
        w = reinterpret_cast<TL *>(smem);
        ukk = w + len;
        uq = ukk + nl;
    } else {
        w = static_cast<TL *>(a.scratch) + rs;
        uq = static_cast<TL *>(a.pscratch) + s0;
        ukk = static_cast<TL *>(a.pscratch) + a.npairs_total + rs;
    }
#pragma unroll 4
    for (int e = lane; e < len; e += kWarp) w[e] = (TL)__ldg(vals + rs + e);
    if (SF && gate) sf_gate_wait(a.ticket, gate, a.timeout);
    TL *piv = static_cast<TL *>(a.piv);
    // the operands, kUnroll per lane at a time: the loads of a batch are issued
    // together, then each is awaited (most are final long before: a long row
    // reads rows of many earlier levels)
    for (int e0 = 0; e0 < nl + nq; e0 += kWarp * kUnroll) {
        const TL *src[kUnroll];
        typename B::U u[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const int e = e0 + k * kWarp + lane;
            src[k] = nullptr;
            if (e < nl) {                                  // u_kk, or its reciprocal (RCP)
                src[k] = piv + __ldg(a.kpos + rs + e);
            } else if (e < nl + nq) {                      // u_kq
                const int q = __ldg(a.tpairs + s0 + e - nl).y;
                if (q < 0) src[k] = static_cast<const TL *>(a.lu) + ~q;
                else u[k] = B::to((TL)__ldg(vals + q));   // final from the start
            }
            if (src[k]) u[k] = first_read<TL, SF>(src[k]);
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            const int e = e0 + k * kWarp + lane;
            if (e >= nl + nq) continue;
            if (SF && src[k]) u[k] = settle<TL>(src[k], u[k], a, r, fail);
            if (e < nl) ukk[e] = B::from(u[k]);
            else uq[e - nl] = B::from(u[k]);
        }
    }
    __syncwarp();
    // one L entry: its updates in ascending step, then the division
    auto finish_l = [&](int e) {
        const int t0 = __ldg(a.tpair_ptr + rs + e) - s0, t1 = __ldg(a.tpair_ptr + rs + e + 1) - s0;
        TL acc = w[e];
        for (int k = t0; k < t1; ++k) acc = RN<TL>::fms(w[__ldg(a.tpairs + s0 + k).x - rs], uq[k], acc);
        w[e] = RCP ? acc * ukk[e] : RN<TL>::div(acc, ukk[e]);
    };
    // L entries by depth of their in-row chain (the analysis's edepth: an
    // entry's producers all have smaller depth), every entry of one depth at
    // once, lane-strided with four entries in flight per lane; a row whose
    // chain is 255 deep or more takes chunks of 32 with waves inside a chunk
    int dmax = 0;
#pragma unroll 8
    for (int e = lane; e < nl; e += kWarp) dmax = max(dmax, (int)__ldg(a.edepth + rs + e));
    dmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)dmax);
    if (dmax == 1) {
        // no step of the row updates an L entry (the power-law rows): every
        // l_rk from a_rk alone, without looking up the (empty) update lists
#pragma unroll 4
        for (int e = lane; e < nl; e += kWarp) w[e] = RCP ? w[e] * ukk[e] : RN<TL>::div(w[e], ukk[e]);
        __syncwarp();
    } else if (dmax < 255) {
        for (int d = 1; d <= dmax; ++d) {
#pragma unroll 4
            for (int e = lane; e < nl; e += kWarp)
                if (dmax == 1 || __ldg(a.edepth + rs + e) == d) finish_l(e);
            __syncwarp();
        }
    } else {
        for (int c0 = 0; c0 < nl; c0 += kWarp) {
            const int e = c0 + lane;
            int t0 = 0, t1 = 0;
            bool done = e >= nl;
            if (!done) {
                t0 = __ldg(a.tpair_ptr + rs + e) - s0;
                t1 = __ldg(a.tpair_ptr + rs + e + 1) - s0;
            }
            for (unsigned dm = __ballot_sync(0xffffffffu, done); dm != 0xffffffffu;
                 dm = __ballot_sync(0xffffffffu, done)) {
                bool ready = !done;
                for (int k = t0; k < t1 && ready; ++k) {
                    const int pp = __ldg(a.tpairs + s0 + k).x - rs - c0;
                    if (pp >= 0) ready = (dm >> pp) & 1u;      // a producer in this chunk
                }
                if (ready) {
                    finish_l(e);
                    done = true;
                }
                __syncwarp();
            }
        }
    }
    // U entries (the diagonal included): every one pulls its updates
    if (!a.tree) {
#pragma unroll 4
        for (int e = nl + lane; e < len; e += kWarp) {
            const int t0 = __ldg(a.tpair_ptr + rs + e) - s0, t1 = __ldg(a.tpair_ptr + rs + e + 1) - s0;
            TL acc = w[e];
            for (int k = t0; k < t1; ++k)
                acc = RN<TL>::fms(w[__ldg(a.tpairs + s0 + k).x - rs], uq[k], acc);
            w[e] = acc;
        }
    } else {
        // tree mode: an entry with more than kTreePairs updates (a hub row's
        // diagonal takes one per L entry: a chain of 1,000 dependent FP64
        // operations on the power-law matrix) is summed by the whole warp --
        // every lane its share in ascending step order, then a fixed
        // butterfly, then added to a_q -- after the lane-strided pass over the
        // others; deterministic, but not the serial order
        for (int e0 = nl; e0 < len; e0 += kWarp) {
            const int e = e0 + lane;
            int t0 = 0, t1 = 0;
            if (e < len) {
                t0 = __ldg(a.tpair_ptr + rs + e) - s0;
                t1 = __ldg(a.tpair_ptr + rs + e + 1) - s0;
            }
            const bool wide = t1 - t0 > kTreePairs;
            if (e < len && !wide) {
                TL acc = w[e];
                for (int k = t0; k < t1; ++k)
                    acc = RN<TL>::fms(w[__ldg(a.tpairs + s0 + k).x - rs], uq[k], acc);
                w[e] = acc;
            }
            for (unsigned wm = __ballot_sync(0xffffffffu, wide); wm != 0u; wm &= wm - 1u) {
                const int src = __ffs(wm) - 1;
                const int k0 = __shfl_sync(0xffffffffu, t0, src), k1 = __shfl_sync(0xffffffffu, t1, src);
                TL part = 0;
                // the lane's share in ascending order, four entries' loads in flight
                for (int k = k0 + lane; k < k1; k += 4 * kWarp) {
                    int st[4];
                    TL uv[4], lv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (k + i * kWarp < k1) {
                            st[i] = __ldg(a.tpairs + s0 + k + i * kWarp).x - rs;
                            uv[i] = uq[k + i * kWarp];
                        }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (k + i * kWarp < k1) lv[i] = w[st[i]];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (k + i * kWarp < k1) part = RN<TL>::fms(lv[i], uv[i], part);
                }
#pragma unroll
                for (int off = kWarp / 2; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
                if (lane == 0) w[e0 + src] += part;
            }
        }
    }
    __syncwarp();
    if (SF && __any_sync(0xffffffffu, fail)) return;
    if (lane == 0) pivot_check<TL>(a, r, w[nl]);
    if (lane == 0 && (!SF || r != a.fault_row)) {
        const TL pv = RCP ? rcp_newton(w[nl]) : w[nl];
        if (SF) publish<TL>(piv + pos, pv);
        else piv[pos] = pv;
    }
    for (int e = lane; e < len; e += kWarp) {
        const TL v = w[e];
        if (!SF || e < nl) lu[rs + e] = v;
        else if (r != a.fault_row) publish<TL>(lu + rs + e, v);
    }
    __syncwarp();                                              // shared memory reusable
}

template <class TV, class TL, bool SF, int W, int S, bool RCP>
__device__ __forceinline__ void factor_task(const FactorArgs &a, int task, unsigned char *smem) {
    const int lo = __ldg(a.task_lo + task), hi = __ldg(a.task_hi + task);
    const unsigned gate = SF ? sf_gate_of(a.task_lev, a.task_ptr, a.gate_levels, a.task_begin, task) : 0u;
    if (hi & kLongBit) {
        if (a.tpairs && __ldg(a.row_pull + __ldg(a.rows + lo)))
            factor_warp_pull<TV, TL, SF, S, RCP>(a, lo, gate, smem);
        else
            factor_warp<TV, TL, SF, RCP, kWarp>(a, lo, gate, smem, warp_smem<S>());
    } else if (hi & kGroupBit) {                 // kWarp / kGroupLanes rows in lockstep
        factor_group<TV, TL, SF, RCP>(a, lo, hi & ~kGroupBit, gate, smem,
                                      warp_smem<S>() / (kWarp / kGroupLanes));
    }
    else factor_lanes<TV, TL, SF, W, S, RCP>(a, lo, hi, gate, smem);
    __syncwarp();
}

template <class TV, class TL, bool SF, int W, int S, bool RCP>
__global__ void __launch_bounds__(kBlock, 1) k_ilu0(FactorArgs a) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const int wib = threadIdx.x >> 5;
    unsigned char *smem = dyn_smem + (size_t)wib * warp_smem<S>();
    if (SF) {
        sf_for_each_task(a.ticket, a.task_begin, a.task_end,
                         [&](int task) { factor_task<TV, TL, SF, W, S, RCP>(a, task, smem); });
        sf_finish(a.ticket);
    } else {
        const int task = a.task_begin + blockIdx.x * kWarpsPerBlock + wib;
        if (task < a.task_end) factor_task<TV, TL, SF, W, S, RCP>(a, task, smem);
    }
}

template <int S> constexpr int block_smem() { return kWarpsPerBlock * warp_smem<S>(); }

}  // namespace

int factor_warp_smem(int slot) {
    return slot > kLaneSlot ? warp_smem<kLaneSlotWide>() : warp_smem<kLaneSlot>();
}

namespace {

// Scratch: [0, nnz) work area for long rows, [nnz, 2 nnz) copy of the input
// for in-place calls (8-byte elements, enough for either dtype).
int ensure_scratch(jv_handle h) {
    const size_t need = 2 * (size_t)h->nnz * sizeof(double) + 64;
    if (h->fscratch_bytes >= need) return JV_OK;
    if (h->fscratch) {
        JV_CUDA(cudaStreamSynchronize(h->stream));
        cudaFree(h->fscratch);
        h->fscratch = nullptr;
        h->fscratch_bytes = 0;
    }
    if (cudaMalloc(&h->fscratch, need) != cudaSuccess) {
        cudaGetLastError();
        h->fscratch = nullptr;
        return JV_ERR_NOMEM;
    }
    h->fscratch_bytes = need;
    return JV_OK;
}

template <class TV, class TL, bool SF, int W, int S, bool RCP>
int launch_w(int grid, cudaStream_t s, const FactorArgs &a) {
    JV_CUDA(cudaFuncSetAttribute(k_ilu0<TV, TL, SF, W, S, RCP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, block_smem<S>()));
    count_launch();
    k_ilu0<TV, TL, SF, W, S, RCP><<<grid, kBlock, block_smem<S>(), s>>>(a);
    JV_CHECK_LAUNCH();
    return JV_OK;
}
template <class TV, class TL, bool SF, bool RCP>
int launch_r(int window, int slot, int grid, cudaStream_t s, const FactorArgs &a) {
    if (slot > kLaneSlot)
        return window <= 4 ? launch_w<TV, TL, SF, 4, kLaneSlotWide, RCP>(grid, s, a)
                           : launch_w<TV, TL, SF, kPoll, kLaneSlotWide, RCP>(grid, s, a);
    return window <= 4 ? launch_w<TV, TL, SF, 4, kLaneSlot, RCP>(grid, s, a)
                       : launch_w<TV, TL, SF, kPoll, kLaneSlot, RCP>(grid, s, a);
}
// reciprocal pivots for an FP64 factor unless exact division is asked for
template <class TV, class TL, bool SF>
int launch(bool rcp, int window, int slot, int grid, cudaStream_t s, const FactorArgs &a) {
    if constexpr (sizeof(TL) == 8) {
        if (rcp) return launch_r<TV, TL, SF, true>(window, slot, grid, s, a);
    }
    return launch_r<TV, TL, SF, false>(window, slot, grid, s, a);
}

template <class TV, class TL>
int run(jv_handle h, const void *vals, void *lu) {
    const Bins &W = h->fbins;
    const LevelSet &L = h->ls[JV_LOWER];
    cudaStream_t s = h->stream;
    const bool inplace = vals == lu;
    // the work area: rows of the warp and group forms, and rows of the band
    // schedule over its kLaneSlot words (which the work list's one-lane slot,
    // when it is the wide one, does not imply), that do not fit shared memory
    if (inplace || W.nlong > 0 || W.ngroup > 0 || L.band.use) {
        int rc = ensure_scratch(h);
        if (rc) return rc;
    }
    if (W.nlong > 0) {                  // operand area of the one-warp-per-row rows
        const size_t need = ((size_t)h->npairs + h->nnz) * sizeof(double) + 64;
        if (h->pscratch_bytes < need) {
            if (h->pscratch) {
                JV_CUDA(cudaStreamSynchronize(s));
                cudaFree(h->pscratch);
                h->pscratch = nullptr;
                h->pscratch_bytes = 0;
            }
            if (cudaMalloc(&h->pscratch, need) != cudaSuccess) {
                cudaGetLastError();
                h->pscratch = nullptr;
                return JV_ERR_NOMEM;
            }
            h->pscratch_bytes = need;
        }
    }
    // reciprocal pivots: FP64 factors unless exact division is asked for
    const bool rcp = sizeof(TL) == 8 && !h->opt.exact;
    if (h->piv_bytes < (size_t)h->n * sizeof(TL)) {          // the pivot array
        if (h->piv) {
            JV_CUDA(cudaStreamSynchronize(s));
            cudaFree(h->piv);
            h->piv = nullptr;
            h->piv_bytes = 0;
        }
        if (cudaMalloc(&h->piv, (size_t)h->n * sizeof(double) + 16) != cudaSuccess) {
            cudaGetLastError();
            h->piv = nullptr;
            return JV_ERR_NOMEM;
        }
        h->piv_bytes = (size_t)h->n * sizeof(double);
    }
    const void *const user_vals = vals;
    void *const copy = inplace ? static_cast<char *>(h->fscratch) + (size_t)h->nnz * sizeof(double)
                               : nullptr;
    if (inplace) vals = copy;
    if (h->opt.mode == JV_MODE_SYNCFREE && L.band.use) {
        if (inplace)
            JV_CUDA(cudaMemcpyAsync(copy, user_vals, (size_t)h->nnz * sizeof(TV),
                                    cudaMemcpyDeviceToDevice, s));
        return band_factor(h, sizeof(TV) == 8 ? JV_F64 : JV_F32, vals,
                           sizeof(TL) == 8 ? JV_F64 : JV_F32, lu, h->fscratch);
    }
    FactorArgs a;
    a.rowptr = h->rowptr;
    a.diag = h->diag;
    a.kdiag = h->kdiag;
    a.pair_ptr = h->pair_ptr;
    a.pairs = h->pairs;
    a.rows = W.rows;
    a.task_lo = W.task_lo;
    a.task_hi = W.task_hi;
    a.task_lev = W.task_lev;
    a.task_ptr = W.task_ptr;
    if (h->opt.sf_gate_levels >= 0) {
        a.gate_levels = h->opt.sf_gate_levels;
    } else {                            // automatic: about 64 tasks' worth of levels
        const double per_level = (double)W.ntasks / (L.nlev > 0 ? L.nlev : 1);
        a.gate_levels = (int)std::min(64.0, std::max(1.0, std::ceil(64.0 / per_level)));
    }
    a.vals = vals;
    a.lu = lu;
    a.scratch = h->fscratch;
    a.ticket = h->ticket;
    a.status = h->status;
    a.timeout = h->opt.spin_timeout_cycles > 0 ? h->opt.spin_timeout_cycles : kDefaultSpin;
    a.fault_row = h->opt.fault_row;
    a.milu = h->opt.milu;
    a.tpair_ptr = h->tpair_ptr;
    a.tpairs = h->tpairs;
    a.kpos = h->kpos;
    a.pscratch = h->pscratch;
    a.npairs_total = h->npairs;
    a.row_pull = h->row_pull;
    a.edepth = h->edepth;
    a.upd = h->upd;
    a.piv = h->piv;
    a.tree = sizeof(TL) == 8 && !h->opt.exact;
    a.backoff_ns = sf_backoff(h);
    // the upper stage: levels [0, lend), above the Even-Rows corner if any
    const jv_dtype lu_t = sizeof(TL) == 8 ? JV_F64 : JV_F32;
    const CornerPlan &C = h->corner[lu_t];
    const int lend = C.use ? C.K : L.nlev;
    // the launch sequence on stream s (the handle's, or a capture stream)
    auto seq = [&](cudaStream_t s) -> int {
        if (inplace)
            JV_CUDA(cudaMemcpyAsync(copy, user_vals, (size_t)h->nnz * sizeof(TV), cudaMemcpyDeviceToDevice, s));
        auto one_level = [&](int l) {
            a.task_begin = W.h_task_ptr[l];
            a.task_end = W.h_task_ptr[l + 1];
            return launch<TV, TL, false>(rcp, W.window, h->fslot,
                                         grid_for(a.task_end - a.task_begin, kWarpsPerBlock), s, a);
        };
        auto sync_free = [&](int l0, int l1) {
            a.task_begin = W.h_task_ptr[l0];
            a.task_end = W.h_task_ptr[l1];
            if (a.task_end <= a.task_begin) return (int)JV_OK;
            return launch<TV, TL, true>(rcp, W.window, h->fslot, sf_grid(h, a.task_end - a.task_begin), s, a);
        };
        int rc = JV_OK;
        if (has_sync_free(h, L, lend)) {
            // the awaited words carry the sentinel until they are published:
            // every pivot, and lu too when some pair operand is an entry the
            // steps update (none for the 5- and 7-point stencils)
            rc = h->ndyn_pairs > 0 ? fill2_u32(lu, (size_t)h->nnz * sizeof(TL) / 4, h->piv,
                                               (size_t)h->n * sizeof(TL) / 4, ~0u, s)
                                   : fill_u32(h->piv, (size_t)h->n * sizeof(TL) / 4, ~0u, s);
            if (rc) return rc;
        }
        if (h->opt.mode == JV_MODE_SYNCFREE) {
            rc = sync_free(0, lend);
        } else if (h->opt.mode == JV_MODE_LEVEL) {
            for (int l = 0; l < lend && rc == JV_OK; ++l) rc = one_level(l);
        } else {
            for (const Seg &g : L.segs) {
                if (g.l0 >= lend || rc != JV_OK) break;
                const int l1 = std::min(g.l1, lend);
                if (g.sf) rc = sync_free(g.l0, l1);
                else for (int l = g.l0; l < l1 && rc == JV_OK; ++l) rc = one_level(l);
            }
        }
        if (rc) return rc;
        // the second stage: Even-Rows corner
        return corner_factor(h, sizeof(TV) == 8 ? JV_F64 : JV_F32, vals, lu_t, lu, s);
    };
    if (h->opt.mode == JV_MODE_SYNCFREE) return seq(s);
    const std::vector<unsigned long long> key = {
        1, sizeof(TV), sizeof(TL), (unsigned long long)h->opt.mode, (unsigned long long)(uintptr_t)user_vals,
        (unsigned long long)(uintptr_t)lu, (unsigned long long)(uintptr_t)h->fscratch,
        (unsigned long long)(uintptr_t)h->pscratch, (unsigned long long)(uintptr_t)h->piv};
    return graph_run(h, key, seq);
}

}  // namespace

int ilu0_factor(jv_handle h, jv_dtype vals_t, const void *vals, jv_dtype lu_t, void *lu) {
    if (lu_t == JV_F64 && vals_t == JV_F64) return run<double, double>(h, vals, lu);
    if (lu_t == JV_F32 && vals_t == JV_F32) return run<float, float>(h, vals, lu);
    if (lu_t == JV_F32 && vals_t == JV_F64) return run<double, float>(h, vals, lu);
    return JV_ERR_ARG;
}

}  // namespace jv
