// jv_lsolve_noalloc: a forward substitution x = L^-1 b (unit lower factor,
// FP64, one right-hand side) that allocates no device memory at all.
//
// The regular entry points keep their scratch (chunk tickets, status word,
// per-row state) in memory that jv_analyze obtains with cudaMalloc.  Some
// callers cannot allocate: code that runs under an allocator it does not own
// (a framework's caching pool, a memory budget that must not grow), code that
// must not trigger the implicit synchronisation cudaMalloc/cudaFree imply, or
// code that has no place to keep a handle.  For them this variant keeps its
// scratch in one file-scope __device__ array of fixed size, which the CUDA
// runtime creates when the library's module is loaded on a device and keeps
// until the process exits (every GPU that loads the library holds it).
//
// Host code cannot use the array's name as a device address (in host code
// it names a host-side stand-in): every call looks the device address up
// with cudaGetSymbolAddress, with the caller's device current, so that a new
// context on that device (after cudaDeviceReset, say) is never handed the
// address of the old one.  All calls share the one array, which keeps what
// the last call left in it: each call clears the words that must start at
// zero before it uses them, and calls that overlap on the GPU (two streams,
// two threads) race on the array.  The call is synchronous: it waits for its
// own work to finish and reads the status word back.
//
// The schedule is a persistent sync-free sweep: CTAs claim chunks of
// kWarpsPerBlock rows of the caller's row order, one warp per row; a row waits
// (bounded) on an acquire-load of the ready flag of every row it reads, then
// replays the ordered chain s = fma(-l_rj, x_j, s) in ascending column order
// -- the serial forward substitution.  A row whose wait gave up, or that
// names a row or column outside the matrix, stores nothing and raises no
// flag.
#include "jv_internal.cuh"

namespace jv {
namespace {

constexpr int kNoAllocMaxRows = 1 << 21;             // 2,097,152 rows
constexpr size_t kNoAllocHeader = 256;               // ticket words + status word
constexpr size_t kNoAllocBytes = kNoAllocHeader + sizeof(int) * (size_t)kNoAllocMaxRows;

// Bytes [0, 16): four words -- ticket, finished CTAs, abort, unused;
// [16, 24): status word; [256, ...): the ready flag of every row.
constexpr size_t kStatusOffset = 16;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array in the current device's context.
int scratch_address(unsigned char **out) {
    void *p = nullptr;
    JV_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    *out = static_cast<unsigned char *>(p);
    return JV_OK;
}

__global__ void k_noalloc_clear(unsigned char *scratch, int n) {
    unsigned *words = reinterpret_cast<unsigned *>(scratch);
    int *flags = reinterpret_cast<int *>(scratch + kNoAllocHeader);
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < 4) words[i] = 0u;
    if (i == 0) *reinterpret_cast<unsigned long long *>(scratch + kStatusOffset) = ~0ull;
    for (long long t = i; t < n; t += (long long)gridDim.x * blockDim.x) flags[t] = 0;
}

__device__ __forceinline__ int ld_acquire_s32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(kBlock) k_lsolve_noalloc(int n, const int *rowptr,
                                                           const int *colidx, const int *diag,
                                                           const int *order, const double *lu,
                                                           const double *b, double *x,
                                                           unsigned char *scratch,
                                                           long long timeout) {
    unsigned *ticket = reinterpret_cast<unsigned *>(scratch);
    unsigned long long *status = reinterpret_cast<unsigned long long *>(scratch + kStatusOffset);
    int *flags = reinterpret_cast<int *>(scratch + kNoAllocHeader);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int base; (base = sf_next_chunk(ticket, n)) >= 0;) {
        const int t = base + wib;
        if (t >= n) continue;
        const int r = __ldg(order + t);
        if ((unsigned)r >= (unsigned)n) {              // not a row of the matrix
            if (lane == 0) {
                report(status, JV_ERR_ARG, t);
                sf_abort(ticket);
            }
            continue;
        }
        const int q0 = __ldg(rowptr + r), q1 = __ldg(diag + r);
        double s = __ldg(b + r);
        bool fail = false;                             // this lane gave up or saw a bad column
        for (int c0 = q0; c0 < q1; c0 += kWarp) {
            const int q = c0 + lane;
            double v = 0.0, xv = 0.0;
            if (q < q1) {
                const int j = __ldg(colidx + q);
                if ((unsigned)j >= (unsigned)r) {     // not a strictly lower column of row r
                    report(status, JV_ERR_ARG, r);
                    sf_abort(ticket);
                    fail = true;
                } else {
                    v = __ldg(lu + q);
                    if (ld_acquire_s32(flags + j) == 0) {
                        const long long t0 = clock64();
                        unsigned it = 0;
                        while (ld_acquire_s32(flags + j) == 0) {
                            if ((++it & 15u) == 0) {
                                if (sf_aborted(ticket)) {        // another wait gave up
                                    fail = true;
                                    break;
                                }
                                if (clock64() - t0 > timeout) {
                                    report(status, JV_ERR_TIMEOUT, r);
                                    sf_abort(ticket);
                                    fail = true;
                                    break;
                                }
                            }
                        }
                    }
                    if (!fail) xv = ld_relaxed_f64(x + j);
                }
            }
            const int cnt = min(kWarp, q1 - c0);
            for (int l = 0; l < cnt; ++l) {
                const double vl = __shfl_sync(0xffffffffu, v, l);
                const double xl = __shfl_sync(0xffffffffu, xv, l);
                s = __fma_rn(-vl, xl, s);
            }
        }
        // a row that lacks an operand publishes neither its value nor its flag
        if (!__any_sync(0xffffffffu, fail) && lane == 0) {
            x[r] = s;
            __threadfence();
            st_release(flags + r, 1);
        }
        __syncwarp();
    }
    sf_finish(ticket);
}

}  // namespace
}  // namespace jv

extern "C" int jv_lsolve_noalloc(int n, const int *rowptr, const int *colidx, const int *diag,
                                 const int *order, const double *lu, const double *b, double *x,
                                 void *stream) {
    using namespace jv;
    if (n < 1 || !rowptr || !colidx || !diag || !order || !lu || !b || !x) return JV_ERR_ARG;
    if (n > kNoAllocMaxRows) {
        std::fprintf(stderr, "jv_lsolve_noalloc: n = %d exceeds the fixed scratch of %d rows\n", n,
                     kNoAllocMaxRows);
        return JV_ERR_ARG;
    }
    if ((const void *)x == (const void *)b) return JV_ERR_ARG;
    unsigned char *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int sms = 0;
    int dev = 0;
    JV_CUDA(cudaGetDevice(&dev));
    JV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    count_launch();
    k_noalloc_clear<<<grid_for(n, kBlock) < 4 * sms ? grid_for(n, kBlock) : 4 * sms, kBlock, 0, s>>>(
        scratch, n);
    JV_CHECK_LAUNCH();
    const int chunks = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
    count_launch();
    k_lsolve_noalloc<<<chunks < sms ? chunks : sms, kBlock, 0, s>>>(n, rowptr, colidx, diag, order,
                                                                    lu, b, x, scratch, kDefaultSpin);
    JV_CHECK_LAUNCH();
    unsigned long long key = 0;
    JV_CUDA(cudaMemcpyAsync(&key, scratch + kStatusOffset, sizeof(key), cudaMemcpyDeviceToHost, s));
    JV_CUDA(cudaStreamSynchronize(s));
    return decode_status(key, nullptr);
}
