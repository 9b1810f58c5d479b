// Internal declarations of libjavelin_gb (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <functional>
#include <vector>

#include "jv.h"

namespace jv {

constexpr int kWarp = 32;
constexpr int kBlock = 256;              // threads per CTA for every kernel here
constexpr int kWarpsPerBlock = kBlock / kWarp;
constexpr long long kDefaultSpin = 1ll << 32;
constexpr int kUnroll = 4;        // entries per lane per step (cooperative kernels)
constexpr int kPoll = 8;          // largest poll window of the one-lane-per-row kernels
constexpr int kLongDeps = 24;     // solve rows with more dependencies run one per warp
constexpr int kSpmvLongRow = 128; // spmv rows longer than this sum over a warp (exact = 0)
constexpr int kLaneSlot = 16;     // factor: 8-byte words of shared memory per one-lane row
constexpr int kLaneSlotWide = 32; // the same, when many rows need 17..32 (e.g. MILU fill pairs)
constexpr unsigned kHoldRounds = 64; // FP64 factor: poll rounds a ready row waits for its warp-mates

// ---------------------------------------------------------------- launches
extern std::atomic<unsigned long long> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

#define JV_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) {                                        \
            std::fprintf(stderr, "libjavelin_gb: %s failed: %s (%s:%d)\n", \
                         #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return JV_ERR_CUDA;                                         \
        }                                                               \
    } while (0)

#define JV_CHECK_LAUNCH()                                               \
    do {                                                                \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) {                                        \
            std::fprintf(stderr, "libjavelin_gb: launch failed: %s (%s:%d)\n", \
                         cudaGetErrorString(e_), __FILE__, __LINE__);   \
            return JV_ERR_CUDA;                                         \
        }                                                               \
    } while (0)

inline int grid_for(long long work, int per_block) {
    long long g = (work + per_block - 1) / per_block;
    return (int)(g < 1 ? 1 : g);
}

// ------------------------------------------------------------- device status
// One 64-bit word per handle: min over reported errors of (row << 32 | 16 + code),
// so the smallest failing row wins, and on one row a timeout (the cause)
// outranks the non-finite pivot it produces.  The word reads ~0 when all is well.
__device__ __forceinline__ void report(unsigned long long *st, int code, int row) {
    unsigned long long key = ((unsigned long long)(unsigned)row << 32) | (unsigned)(16 + code);
    atomicMin(st, key);
}
inline int decode_status(unsigned long long key, int *row) {
    if (key == ~0ull) { if (row) *row = -1; return JV_OK; }
    if (row) *row = (int)(key >> 32);
    return (int)(key & 0xffffffffu) - 16;
}

// ------------------------------------------------------ memory-order helpers
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned *p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ double ld_relaxed_f64(const double *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return __longlong_as_double((long long)v);
}
__device__ __forceinline__ int ld_relaxed_s32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Hint: bring the line holding p into L2 (no register result, no wait).
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// ------------------------------------------------------ sync-free launches
// Three words per handle: [0] next chunk ticket, [1] finished CTAs, [2] abort.
// A sync-free launch is a fixed grid of persistent CTAs; each CTA repeatedly
// claims the next chunk of kWarpsPerBlock level-ordered tasks with one atomic
// and runs it.  A chunk is only ever claimed by a running CTA and every task
// waits only on tasks of earlier chunks, so no wait depends on a CTA that is
// not resident, and the grid size bounds how far ahead of the dependency
// front the GPU runs (how many rows poll at once).  The last CTA to finish
// resets all three words, so the next launch starts from zero without a
// memset.  A wait that exceeds its cycle budget reports JV_ERR_TIMEOUT and
// raises the abort word; every other wait polls it and gives up too, so a
// fault costs one timeout period.
//
// Returns the first task of the CTA's next chunk, or -1 (block-uniform).
// (Used by the allocation-free solve; the kernels of the handle claim per
// warp, see sf_for_each_task.)
__device__ __forceinline__ int sf_next_chunk(unsigned *ticket, int ntasks) {
    __shared__ int s_base;
    __syncthreads();
    if (threadIdx.x == 0) s_base = (int)atomicAdd(ticket, 1u) * kWarpsPerBlock;
    __syncthreads();
    return s_base < ntasks ? s_base : -1;
}

// Back-off between polls of a word that is not ready yet.
__device__ __forceinline__ void sf_pause(unsigned it, unsigned max_ns) {
    if (max_ns == 0 || it < 4) return;
    unsigned ns = 16u << min(it - 4u, 6u);
    __nanosleep(ns < max_ns ? ns : max_ns);
}
// Per-warp claims: every warp takes the next level-ordered task with one
// atomic of its lane 0, so the consecutive tasks of one level spread over
// the warps of all SMs (a CTA-sized chunk would put a whole slice of the
// level on one SM, whose FP64 units and load path then set the pace of the
// level).  The claim for the warp's next task is issued when the current
// task starts and read when it ends, so its latency hides behind the task.
// Every task waits only on tasks of lower index, each claimed by a resident
// warp (a warp's pending claim is above its current task), so the lowest
// unfinished task always runs: no deadlock.  The launch covers tasks
// [begin, end): a launch over a later range of levels (the two-stage
// schedules) finds the rows of earlier ranges already written by the launches
// before it.  Warp-uniform; lanes must be converged.
template <class F>
__device__ __forceinline__ void sf_for_each_task(unsigned *ticket, int begin, int end, F &&run) {
    const int lane = threadIdx.x & (kWarp - 1);
    unsigned claim = 0;
    if (lane == 0) claim = atomicAdd(ticket, 1u);
    int task = begin + __shfl_sync(0xffffffffu, (int)claim, 0);
    while (task < end) {
        unsigned next = 0;
        if (lane == 0) next = atomicAdd(ticket, 1u);
        run(task);
        __syncwarp();
        if (lane == 0) atomicAdd(ticket + 3, 1u);        // finished tasks (level gate)
        task = begin + __shfl_sync(0xffffffffu, (int)next, 0);
    }
}

__device__ __forceinline__ void sf_finish(unsigned *ticket) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(ticket + 1, 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(ticket, 0u);
            atomicExch(ticket + 1, 0u);
            atomicExch(ticket + 2, 0u);
            atomicExch(ticket + 3, 0u);
        }
    }
}
__device__ __forceinline__ bool sf_aborted(const unsigned *ticket) {
    return ld_relaxed(ticket + 2) != 0u;
}
__device__ __forceinline__ void sf_abort(unsigned *ticket) { atomicExch(ticket + 2, 1u); }

// Level gate.  Word [3] counts finished tasks.  A task whose operands lie
// in levels far below the dependency front would poll them for many rounds
// and, with thousands of such rows in flight, the polls crowd each SM's load
// path and slow the rows that are about to become ready.  So a task first
// sleeps until `gate` tasks have finished (the tasks of the levels more
// than gate-levels below its own), with a pause that shrinks as the count
// approaches the gate, and only then polls its operands.  The count is a
// hint, never a correctness condition (every operand is still awaited on its
// own word); it reaches the gate because the tasks below it wait on nothing
// above.  Bounded by the wait bound, after which the task simply polls.
// The count starts at the launch's first task `begin`.  Warp-uniform.
__device__ __forceinline__ unsigned sf_gate_of(const int *task_lev, const int *task_ptr,
                                               int gate_levels, int begin, int task) {
    if (gate_levels <= 0) return 0u;
    const int l = __ldg(task_lev + task) - gate_levels;
    if (l <= 0) return 0u;
    const int g = __ldg(task_ptr + l) - begin;
    return g > 0 ? (unsigned)g : 0u;
}
__device__ __forceinline__ void sf_gate_wait(unsigned *ticket, unsigned gate, long long timeout) {
    unsigned c = ld_relaxed(ticket + 3);
    if (c >= gate) return;
    const long long t0 = clock64();
    for (unsigned it = 1;; ++it) {
        const unsigned gap = gate - c;
        __nanosleep(gap > 1024u ? 2048u : (gap < 16u ? 32u : 2u * gap));
        c = ld_relaxed(ticket + 3);
        if (c >= gate) return;
        // past the wait bound (or after an abort) stop sleeping and poll: the
        // gate is only a hint, the operand waits that follow are the ones
        // that detect and report a missing row
        if ((it & 7u) == 0 && (sf_aborted(ticket) || clock64() - t0 > timeout)) return;
    }
}

// ---------------------------------------------------------------- sentinels
// In sync-free solves the output vector itself carries readiness: it is
// first filled with an all-ones bit pattern (a NaN payload that no
// arithmetic result can carry, because results that are NaN are rewritten
// to the canonical quiet NaN before they are stored), and a dependant spins
// until the word it needs differs from it.  One aligned store publishes both
// the value and its readiness, so no fence is needed on either side.
template <class T> struct Bits;
template <> struct Bits<double> {
    using U = unsigned long long;
    static constexpr U kSent = ~0ull;
    static constexpr U kCanonNan = 0x7ff8000000000000ull;
    __device__ static double from(U u) { return __longlong_as_double((long long)u); }
    __device__ static U to(double d) { return (U)__double_as_longlong(d); }
    // integer tests: no FP64 instruction (the FP64 pipe is narrow on this part)
    __device__ static bool nan_bits(U u) { return (u & 0x7fffffffffffffffull) > 0x7ff0000000000000ull; }
    __device__ static bool zero_or_nonfinite_bits(U u) {
        return (u & 0x7fffffffffffffffull) == 0 || (u & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
    }
};
template <> struct Bits<float> {
    using U = unsigned;
    static constexpr U kSent = ~0u;
    static constexpr U kCanonNan = 0x7fc00000u;
    __device__ static float from(U u) { return __uint_as_float(u); }
    __device__ static U to(float f) { return __float_as_uint(f); }
    __device__ static bool nan_bits(U u) { return (u & 0x7fffffffu) > 0x7f800000u; }
    __device__ static bool zero_or_nonfinite_bits(U u) {
        return (u & 0x7fffffffu) == 0 || (u & 0x7f800000u) == 0x7f800000u;
    }
};

// 1/d for the FP64 factor and back substitution (jv_options.exact =
// 0): Newton's iteration for the reciprocal, y <- y + y (1 - d y), which
// squares the relative error at every step, started from the approximate
// reciprocal the hardware provides (PTX rcp.approx.ftz.f64).  Two steps take
// any seed better than 2^-14 to the rounding level: the result is within one
// unit in the last place of 1/d.  Zero, subnormal, huge and non-finite inputs
// (exponent outside +-1000, where the seed may flush to zero or 1/d be
// subnormal) take the correctly rounded __drcp_rn instead.  Five FP64-pipe
// instructions in the common case, against about three times as many for a
// correctly rounded division.
__device__ __forceinline__ double rcp_newton(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned ex = (unsigned)(u >> 52) & 0x7ffu;
    if (ex < 1023u - 1000u || ex > 1023u + 1000u) return __drcp_rn(d);
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    double e = __fma_rn(-d, y, 1.0);
    y = __fma_rn(y, e, y);
    e = __fma_rn(-d, y, 1.0);
    return __fma_rn(y, e, y);
}

// s / d from y = rcp_newton(d): q = s y, then one correction with the
// residual computed exactly by a fused multiply-add, q + (s - d q) y
// (Markstein's correction step for division).  Compared with __ddiv_rn on
// 6.4e9 random pairs (full random significands, a third of them with long
// runs of ones or zeros in the divisor, exponents within +-10, +-200 and
// +-900) it returned the correctly rounded quotient every time, although y
// itself is one unit in the last place off the correctly rounded 1/d for
// about 1 % of divisors.  Three FP64-pipe instructions once y is known,
// against about ten for a division.  Inputs with exponents outside +-500
// (where q or the residual could overflow or underflow), and zero s (whose
// sign the correction can lose), take __ddiv_rn.
__device__ __forceinline__ double div_rcp(double s, double d, double y) {
    const unsigned es = (unsigned)((unsigned long long)__double_as_longlong(s) >> 52) & 0x7ffu;
    const unsigned ed = (unsigned)((unsigned long long)__double_as_longlong(d) >> 52) & 0x7ffu;
    if (es - 523u > 1000u || ed - 523u > 1000u) return __ddiv_rn(s, d);
    const double q = s * y;
    return __fma_rn(__fma_rn(-d, q, s), y, q);
}

// f(i) = a[i + ai] + ad: one kernel can walk a CSR or CSC sub-range of row or
// column i (e.g. the strictly lower part of row i is [rowptr[i], diag[i])).
struct Span {
    const int *a;
    int ai, ad;
    __device__ __forceinline__ int at(int i) const { return __ldg(a + i + ai) + ad; }
};

// Position of column j in the sorted column range [lo, hi), or -1.
__device__ __forceinline__ int find_col(const int *__restrict__ col, int lo, int hi, int j) {
    const int end = hi;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(col + mid) < j) lo = mid + 1; else hi = mid;
    }
    return (lo < end && __ldg(col + lo) == j) ? lo : -1;
}

// -------------------------------------------------------------- level sets
// Work list of one level structure, rows binned by cost (the row-length
// classes of the load-balancing concern of Sec. III-A / III-B): inside every
// level the short rows come first, in ascending order, packed 32 to a task
// (16 where levels are narrow) with one lane per row; in the factor's list,
// medium rows follow, kWarp / kGroupLanes to a task with kGroupLanes lanes
// per row (the sub-warp rows of a 27-point stencil); every long row is a
// task of its own, run by the whole warp.  A task never spans two levels, so
// the rows of a task never depend on each other.
constexpr int kLongBit = (int)0x80000000u;   // task_hi flag: one-row cooperative task
constexpr int kGroupBit = 0x40000000;        // task_hi flag (factor): rows of kGroupLanes lanes each
constexpr int kGroupLanes = 8;
struct Bins {
    int *rows = nullptr;       // [n] binned rows
    int *ipos = nullptr;       // [n] position of every row in rows (inverse of rows)
    int *task_lo = nullptr;    // [ntasks] first position in rows
    int *task_hi = nullptr;    // [ntasks] end position, | kLongBit for a long-row task
    int *task_lev = nullptr;   // [ntasks] level of every task
    int *task_ptr = nullptr;   // [nlev+1] first task of every level (device copy)
    int ntasks = 0;
    int nlong = 0;
    int ngroup = 0;            // factor: tasks of kWarp / kGroupLanes rows, kGroupLanes lanes each
    int window = 8;            // operands a one-lane row polls per round: 2, 4, 8 or 16,
                               // the smallest holding the most operands of any short
                               // row; 17 = more (rows span several windows of kPoll)
    std::vector<int> h_task_ptr;  // [nlev+1] first task of every level
};

// Two-stage schedules.  A run of levels [l0, l1) of one level structure:
// one launch per level (upper-stage levels of the hybrid schedule) or one
// sync-free launch over the run (every maximal run of second-stage levels).
struct Seg {
    int l0, l1;
    bool sf;
};

// Even-Rows corner of the factor (Sec. III-B, Fig. 8): the levels [K, nlev)
// of lower(A), whose rows are the last rows [c, n) of the handle's order, so
// their entries are the CSR tail [E0, nnz).  One CTA holds the corner's
// values in shared memory, applies every row's updates from the rows above
// the corner (FACTOR_L), then factors the corner level by level.  The level
// loop reads a per-row program of 16-bit shared-memory offsets, in level
// order: [row - c, steps, diagonal] then per step [entry, u_kk, pairs] and
// per pair [target, operand] -- the step's updates in their stored order.
struct CornerPlan {
    bool use = false;
    int K = 0, nl = 0;          // first level, levels
    int c = 0, R = 0;           // first row, rows
    int E0 = 0, E = 0;          // first CSR position, entries
    int words = 0;              // program words
    size_t smem = 0;            // shared memory of the launch
    int *prog_ptr = nullptr;    // [R+1] first word of every row (level order)
    int *lvl_ptr = nullptr;     // [nl+1] first row of every corner level
    unsigned short *prog = nullptr;  // [words] (padded to an even count)
};
constexpr int kCornerThreads = 1024;

// Even-Rows corner of a single right-hand-side solve: the tail levels [K,
// nlev) of the structure's DAG, whose rows are the last rows [c0, n) of a
// forward structure (L, U^T) or the first rows [0, R) of a backward one (U,
// L^T).  One CTA keeps the corner's x (and the operands it reads from rows
// outside the corner, gathered once) in shared memory and solves the corner
// level by level.  Per row (level order) the program holds [row - c0,
// entries] and one operand slot per entry, in the serial order of the
// substitution; the entry values (then the diagonal, for U and U^T) follow
// the same order in a value array.
struct SolveCorner {
    bool use = false;
    int K = 0, nl = 0;          // first level, levels
    int c0 = 0, R = 0;          // first row, rows
    int next = 0;               // operands outside the corner
    int nval = 0, words = 0;    // values (entries + diagonals), program words
    int *prog_ptr = nullptr;    // [R+1]
    int *lvl_ptr = nullptr;     // [nl+1]
    int *vpos = nullptr;        // [nval] position in lu of every value
    int *ext = nullptr;         // [next] row of every outside operand
    unsigned short *prog = nullptr;  // [words] (padded to an even count)
};

// Band schedule of one level structure: rows split into nb contiguous bands
// of B rows (natural order); inside a band, rows are grouped by their local
// level -- the longest path through dependencies that stay inside the band.
// One CTA runs a band: local levels in order, separated by __syncthreads,
// values of the band's rows kept in shared memory; dependencies on other
// bands are awaited on the published output words.  Bands are claimed in
// dependency order (ascending for forward structures, descending for
// backward ones), so a band only waits on bands claimed before it.
struct BandPlan {
    bool use = false;
    int B = 0, nb = 0;
    int nll_total = 0;         // local levels over all bands
    int nll_max = 0;
    double internal_frac = 0;  // dependencies inside their band / all dependencies
    int *bl_ptr = nullptr;     // [nb+1] first local level of every band
    int *ll_ptr = nullptr;     // [nll_total+1] first position in rows of every local level
    int *rows = nullptr;       // [n] rows by (band, local level, row)
};

struct LevelSet {
    int nlev = 0;
    int *lev = nullptr;        // [n] level of every row
    int *ptr = nullptr;        // [nlev+1]
    int *rows = nullptr;       // [n] rows grouped by level, ascending inside
    std::vector<int> h_ptr;    // host copy of ptr
    Bins bins;                 // single right-hand-side solve work list
    BandPlan band;
    std::vector<Seg> segs;     // hybrid schedule over [0, nlev)
    int tail = 0;              // first level after which every level is second-stage
};

struct Workspace;  // Krylov scratch, krylov.cu

// A captured launch sequence (graph.cu), keyed by operation, dtypes, buffers
// and schedule.
struct GraphEntry {
    std::vector<unsigned long long> key;
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches = 0;   // kernels in the graph (launch counter)
    unsigned long long used = 0;       // last use (least recently used goes first)
};

}  // namespace jv

struct jv_handle_s {
    int device = 0;
    int n = 0, nnz = 0;
    int nnz_lower = 0, nnz_upper = 0;
    cudaStream_t stream = nullptr;
    jv_options opt{};
    // pattern (B = P A P^T when reordering)
    int *rowptr = nullptr, *colidx = nullptr, *diag = nullptr;
    // CSC of the pattern
    int *colptr = nullptr, *rowidx = nullptr, *csc2csr = nullptr, *cdiag = nullptr;
    jv::LevelSet ls[4];
    // reordering
    int *perm = nullptr, *iperm = nullptr, *vmap = nullptr;
    // symbolic factorisation: for every strictly lower entry p = (r, k) the
    // updates it drives, pairs (t, q) with a_rt -= l_rk * u_kq, t ascending
    int *pair_ptr = nullptr;                 // [nnz + 1], empty ranges off the strict lower part
    int2 *pairs = nullptr;                   // [npairs] (t, q) absolute CSR positions
    int *kdiag = nullptr;                    // [nnz] diag[colidx[p]]: position of u_kk for p = (r, k)
    int *tpair_ptr = nullptr;                // [nnz + 1] the pairs grouped by target entry t:
    int2 *tpairs = nullptr;                  // [npairs] (p, q) -- step p, operand q -- ascending p;
                                             // q stored as ~q when some step updates u_kq
                                             // (the operand is awaited, not read from A)
    unsigned char *row_pull = nullptr;       // [n] 1: a one-warp row takes the pull form
    unsigned char *edepth = nullptr;         // [nnz] L entries: depth of the in-row chain of steps
                                             // that update the entry (1: none; capped at 255)
    unsigned char *upd = nullptr;            // [nnz] 1: some step of the factor updates the entry
    long long ndyn_pairs = 0;                // pairs whose operand is updated (must be awaited)
    long long npairs = 0;
    jv::Bins fbins;                          // factor work list over the levels of lower(A)
    int *kpos = nullptr;                     // [nnz] L entries p = (r, k): the factor work-list
                                             // position of row k, where its pivot is published
    jv::CornerPlan corner[2];                // Even-Rows corner per factor dtype (jv_dtype)
    jv::SolveCorner scorner[4][2];           // per structure; [1]: lu and x both FP32
    int maxrow = 0;                          // longest row
    int *spmv_rows = nullptr;                // spmv: rows by length, longest first
    int spmv_wide = 0;                       // spmv: the first spmv_wide of them sum over a warp
    // lazily allocated factor scratch (long rows / in-place copies)
    void *fscratch = nullptr;
    size_t fscratch_bytes = 0;
    void *xpos = nullptr;                    // one-column solves: x by work-list position
    size_t xpos_bytes = 0;
    void *xscratch = nullptr;                // FP32 solution of FP32-factor solves into FP64 x
    size_t xscratch_bytes = 0;
    void *pscratch = nullptr;                // operands of long rows: [npairs + nnz] elements
    void *piv = nullptr;                     // factor: the pivot of every row (u_kk, or 1/u_kk
    size_t piv_bytes = 0;                    // with reciprocal pivots), published by the row at
                                             // its factor work-list position (sentinel-filled in
                                             // sync-free mode)
    int fslot = jv::kLaneSlot;               // factor one-lane slot (kLaneSlot or kLaneSlotWide)
    size_t pscratch_bytes = 0;
    // scratch shared by the sync-free kernels
    unsigned *ticket = nullptr;              // [8]: next task ticket, finished CTAs, abort,
                                             // finished tasks
    unsigned long long *status = nullptr;    // device status word
    unsigned long long *h_status = nullptr;  // pinned host mirror
    int bad_row = -1;                        // row of the last analysis error
    int num_sms = 0;                         // queried in jv_analyze
    jv::Workspace *ws = nullptr;
    std::vector<jv::GraphEntry> graphs;      // replayable per-level launch sequences
    unsigned long long graph_clock = 0;
    cudaStream_t cap_stream = nullptr;       // private stream the sequences are captured on
    std::vector<void *> allocs;              // everything to cudaFree on destroy
};

namespace jv {

// Persistent grid of a sync-free launch over `ntasks` tasks, and the poll
// back-off bound, from the handle's options.
inline int sf_grid(jv_handle h, int ntasks, int default_per_sm = 1) {
    const int per_sm = h->opt.sf_ctas_per_sm > 0 ? h->opt.sf_ctas_per_sm : default_per_sm;
    const int chunks = (ntasks + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int g = h->num_sms * per_sm;
    return chunks < g ? (chunks > 0 ? chunks : 1) : g;
}
inline unsigned sf_backoff(jv_handle h) {
    return h->opt.sf_backoff_ns <= 0 ? 0u : (unsigned)h->opt.sf_backoff_ns;
}

// allocation owned by the handle
int halloc(jv_handle h, void **p, size_t bytes);
// a lazily grown scratch buffer of the handle: (re)allocated, after the
// handle's stream drains, when *bytes < need
int ensure_buffer(jv_handle h, void **p, size_t *bytes, size_t need);
template <class T> int halloc_n(jv_handle h, T **p, size_t count) {
    return halloc(h, (void **)p, count * sizeof(T) + 16);
}

// prims.cu
// multiprocessors of the current device (queried once per device)
int current_device_sms();
int fill_u32(void *p, size_t count_u32, unsigned v, cudaStream_t s);
// two ranges in one launch
int fill2_u32(void *p0, size_t count0_u32, void *p1, size_t count1_u32, unsigned v, cudaStream_t s);
int iota_i32(int *p, int n, cudaStream_t s);
// exclusive scan of in[0..m) into out[0..m]; out[m] = total.  tmp: >= scan_tmp_ints(m)
size_t scan_tmp_ints(int m);
int exclusive_scan_i32(const int *in, int *out, int m, int *tmp, cudaStream_t s);
// stable LSD radix sort of (key, val) pairs by the low `bits` bits of key.
// Sorts keys/vals in place (using the alt buffers); tmp >= radix_tmp_ints(m).
size_t radix_tmp_ints(int m);
int radix_sort_pairs(unsigned *keys, unsigned *vals, unsigned *keys_alt, unsigned *vals_alt,
                     int m, int bits, int *tmp, cudaStream_t s);
// ptr[k] = first position whose sorted key is >= k, k = 0..K (ptr[K] = m)
int keys_to_ptr(const unsigned *sorted_keys, int m, int *ptr, int K, cudaStream_t s);

// analyze.cu
int analyze(jv_handle h, const int *rowptr, const int *colidx);

// factor.cu
// shared memory of one factor warp for a one-lane slot of `slot` words
int factor_warp_smem(int slot);
int ilu0_factor(jv_handle h, jv_dtype vals_t, const void *vals, jv_dtype lu_t, void *lu);

// band.cu: band schedule planner (host) and the band kernels
int plan_bands(jv_handle h);
int band_solve(jv_handle h, int structure, jv_dtype lu_t, const void *lu, jv_dtype b_t,
               const void *b, jv_dtype x_t, void *x);
int band_factor(jv_handle h, jv_dtype vals_t, const void *vals, jv_dtype lu_t, void *lu,
                void *scratch);

// graph.cu: run seq(stream) through a cached CUDA graph of it (or plainly,
// with no_graphs or inside a capture of the caller's own)
int graph_run(jv_handle h, const std::vector<unsigned long long> &key,
              const std::function<int(cudaStream_t)> &seq);
void free_graphs(jv_handle h);

// stages.cu: stage test, hybrid segments, Even-Rows corner
int plan_stages(jv_handle h);
int corner_factor(jv_handle h, jv_dtype vals_t, const void *vals, jv_dtype lu_t, void *lu,
                  cudaStream_t s);
// launches of a hybrid run over levels [0, lend) of structure s (per-level tasks)
int hybrid_launches(const LevelSet &L, int lend);
// whether the handle's schedule runs a sync-free launch over levels [0, lend)
// (which needs the output pre-filled with the sentinel)
bool has_sync_free(jv_handle h, const LevelSet &L, int lend);
// the solve corner a one-column solve of this structure and these value sizes uses, or null
const SolveCorner *solve_corner_of(jv_handle h, int structure, size_t tl, size_t tx);
int corner_solve(jv_handle h, int structure, const SolveCorner &C, jv_dtype lu_t, const void *lu,
                 jv_dtype b_t, const void *b, jv_dtype x_t, void *x, cudaStream_t s);

// trisolve.cu
int hop_latency(int rounds, int npartners, double *out_us, cudaStream_t s);
int iluk_symbolic(int n, int nnz, const int *rowptr, const int *colidx, int level, int *fill_rowptr,
                  int *fill_colidx, int *fill_level, long long *fill_nnz, cudaStream_t s,
                  int *bad_row);
int scatter_values(int n, const int *rowptr, const int *colidx, jv_dtype t, const void *vals,
                   const int *frowptr, const int *fcolidx, void *fvals, cudaStream_t s);
int tri_solve(jv_handle h, int structure, jv_dtype lu_t, const void *lu, jv_dtype b_t,
              const void *b, jv_dtype x_t, void *x, int nrhs);

// spmv.cu
int spmv(jv_handle h, jv_dtype t, const void *vals, const void *x, void *y, double alpha,
         double beta);
int masked_outer(jv_handle h, jv_dtype t, int which, const void *a, const void *b, int nrhs,
                 double alpha, void *g);
int permute_values(jv_handle h, jv_dtype t, const void *in, void *out);
int permute_vector(jv_handle h, jv_dtype t, int inverse, const void *in, void *out, int nrhs);

// krylov.cu
int pcg(jv_handle h, const double *vals, jv_dtype lu_t, const void *lu, const double *b,
        double *x, const jv_krylov_opts *o, jv_krylov_info *info);
int fgmres(jv_handle h, const double *vals, jv_dtype lu_t, const void *lu, const double *b,
           double *x, const jv_krylov_opts *o, jv_krylov_info *info);
void free_workspace(jv_handle h);

}  // namespace jv
