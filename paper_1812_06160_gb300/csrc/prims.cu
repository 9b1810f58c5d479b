// Device primitives used by the analysis: fill, iota, exclusive scan, stable
// LSD radix sort of (key, value) pairs, and sorted-key -> segment pointers.
// All are deterministic: integer results do not depend on scheduling, and the
// sort is stable (equal keys keep their input order), which is what makes the
// level sets and the CSC bit-exact run to run.
#include <mutex>

#include "jv_internal.cuh"

namespace jv {

std::atomic<unsigned long long> g_launches{0};

// ------------------------------------------------------------------- fill
__device__ __forceinline__ void fill_range(unsigned *p, size_t n, unsigned v, size_t i, size_t stride) {
    uintptr_t addr = (uintptr_t)p;
    size_t head = ((16 - (addr & 15)) & 15) / 4;
    if (head > n) head = n;
    for (size_t j = i; j < head; j += stride) p[j] = v;
    uint4 *q = reinterpret_cast<uint4 *>(p + head);
    size_t nv = (n - head) / 4;
    uint4 vv = make_uint4(v, v, v, v);
    for (size_t j = i; j < nv; j += stride) q[j] = vv;
    for (size_t j = head + nv * 4 + i; j < n; j += stride) p[j] = v;
}

__global__ void k_fill_u32(unsigned *p, size_t n, unsigned v) {
    fill_range(p, n, v, blockIdx.x * (size_t)blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

// two ranges in one launch: grid row y fills range y
__global__ void k_fill2_u32(unsigned *p0, size_t n0, unsigned *p1, size_t n1, unsigned v) {
    fill_range(blockIdx.y ? p1 : p0, blockIdx.y ? n1 : n0, v,
               blockIdx.x * (size_t)blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

int current_device_sms() {
    static std::mutex mu;
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 1; }
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev] == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
            cudaGetLastError();
            return 1;
        }
        cache[dev] = sms;
    }
    return cache[dev];
}

int fill_u32(void *p, size_t count, unsigned v, cudaStream_t s) {
    if (count == 0) return JV_OK;
    long long vec = (long long)(count / 4 + 1);
    int grid = grid_for(vec, kBlock);
    const int cap = current_device_sms() * 16;   // 16 CTAs per SM, grid-stride beyond
    if (grid > cap) grid = cap;
    count_launch();
    k_fill_u32<<<grid, kBlock, 0, s>>>((unsigned *)p, count, v);
    JV_CHECK_LAUNCH();
    return JV_OK;
}

int fill2_u32(void *p0, size_t count0, void *p1, size_t count1, unsigned v, cudaStream_t s) {
    const size_t big = count0 > count1 ? count0 : count1;
    if (big == 0) return JV_OK;
    int grid = grid_for((long long)(big / 4 + 1), kBlock);
    const int cap = current_device_sms() * 8;    // 2 x 8 CTAs per SM, grid-stride beyond
    if (grid > cap) grid = cap;
    count_launch();
    k_fill2_u32<<<dim3(grid, 2), kBlock, 0, s>>>((unsigned *)p0, count0, (unsigned *)p1, count1, v);
    JV_CHECK_LAUNCH();
    return JV_OK;
}

__global__ void k_iota(int *p, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

int iota_i32(int *p, int n, cudaStream_t s) {
    if (n <= 0) return JV_OK;
    count_launch();
    k_iota<<<grid_for(n, kBlock), kBlock, 0, s>>>(p, n);
    JV_CHECK_LAUNCH();
    return JV_OK;
}

// ------------------------------------------------------------------- scan
constexpr int kScanItems = 8;
constexpr int kScanTile = kBlock * kScanItems;   // 2048

// Exclusive scan of one value per thread across a block of NW warps.
template <int NW>
__device__ int block_exclusive_scan(int v, int *total) {
    __shared__ int wsum[NW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int w = lane < NW ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < NW) wsum[lane] = w;
    }
    __syncthreads();
    int pre = (wid > 0 ? wsum[wid - 1] : 0) + inc - v;
    *total = wsum[NW - 1];
    __syncthreads();
    return pre;
}

__global__ void k_scan_reduce(const int *in, int m, int *part) {
    size_t base = (size_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < (size_t)m) s += in[base + k];
    int total;
    block_exclusive_scan<kWarpsPerBlock>(s, &total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// One block of 1024 threads scans the tile sums in place; part[nt] = total.
__global__ void k_scan_part(int *part, int nt) {
    int chunk = (nt + 1023) / 1024;
    int lo = threadIdx.x * chunk;
    int hi = min(lo + chunk, nt);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += part[i];
    int total;
    int run = block_exclusive_scan<32>(s, &total);
    for (int i = lo; i < hi; ++i) {
        int v = part[i];
        part[i] = run;
        run += v;
    }
    if (threadIdx.x == 0) part[nt] = total;
}

__global__ void k_scan_down(const int *in, int *out, int m, const int *part, int nt) {
    size_t base = (size_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < (size_t)m) ? in[base + k] : 0;
        s += v[k];
    }
    int total;
    int run = block_exclusive_scan<kWarpsPerBlock>(s, &total) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < (size_t)m) out[base + k] = run;
        run += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[m] = part[nt];
}

size_t scan_tmp_ints(int m) { return (size_t)(m + kScanTile - 1) / kScanTile + 2; }

int exclusive_scan_i32(const int *in, int *out, int m, int *tmp, cudaStream_t s) {
    if (m <= 0) {
        JV_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
        return JV_OK;
    }
    int nt = (m + kScanTile - 1) / kScanTile;
    count_launch();
    k_scan_reduce<<<nt, kBlock, 0, s>>>(in, m, tmp);
    JV_CHECK_LAUNCH();
    count_launch();
    k_scan_part<<<1, 1024, 0, s>>>(tmp, nt);
    JV_CHECK_LAUNCH();
    count_launch();
    k_scan_down<<<nt, kBlock, 0, s>>>(in, out, m, tmp, nt);
    JV_CHECK_LAUNCH();
    return JV_OK;
}

// ------------------------------------------------------------- radix sort
constexpr int kRadixRounds = 16;                              // 32-key rounds per warp
constexpr int kRadixTile = kBlock * kRadixRounds;             // 4096 keys per CTA
constexpr int kRadixWarpChunk = kWarp * kRadixRounds;         // 512 keys per warp

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void k_rs_hist(const unsigned *keys, int m, int shift, int nt, int *counts) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    size_t base = (size_t)blockIdx.x * kRadixTile;
    for (int k = 0; k < kRadixRounds; ++k) {
        size_t idx = base + (size_t)k * kBlock + threadIdx.x;
        if (idx < (size_t)m) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * nt + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: the destination of a key is the global offset of its digit
// for this tile, plus the count of equal digits in earlier warps of the tile,
// in earlier rounds of this warp, and in lower lanes of this round.
__global__ void k_rs_scatter(const unsigned *kin, const unsigned *vin, unsigned *kout,
                             unsigned *vout, int m, int shift, int nt, const int *offs) {
    __shared__ int wh[kWarpsPerBlock][256];
    for (int i = threadIdx.x; i < kWarpsPerBlock * 256; i += kBlock) (&wh[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t base = (size_t)blockIdx.x * kRadixTile + (size_t)w * kRadixWarpChunk;
    for (int r = 0; r < kRadixRounds; ++r) {
        size_t idx = base + (size_t)r * kWarp + lane;
        bool valid = idx < (size_t)m;
        unsigned d = valid ? ((kin[idx] >> shift) & 255u) : 0u;
        unsigned act = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            unsigned peers = __match_any_sync(act, d);
            if (lane == __ffs(peers) - 1) wh[w][d] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    {
        int d = threadIdx.x;
        int run = offs[(size_t)d * nt + blockIdx.x];
        for (int ww = 0; ww < kWarpsPerBlock; ++ww) {
            int c = wh[ww][d];
            wh[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned lt = lanemask_lt();
    for (int r = 0; r < kRadixRounds; ++r) {
        size_t idx = base + (size_t)r * kWarp + lane;
        bool valid = idx < (size_t)m;
        unsigned key = valid ? kin[idx] : 0u;
        unsigned val = valid ? vin[idx] : 0u;
        unsigned d = (key >> shift) & 255u;
        unsigned act = __ballot_sync(0xffffffffu, valid);
        unsigned peers = 0;
        if (valid) {
            peers = __match_any_sync(act, d);
            int pos = wh[w][d] + __popc(peers & lt);
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wh[w][d] += __popc(peers);
        __syncwarp();
    }
}

size_t radix_tmp_ints(int m) {
    size_t nt = (size_t)(m + kRadixTile - 1) / kRadixTile;
    size_t nc = 256 * nt;
    return nc + 1 + scan_tmp_ints((int)nc) + 8;
}

int radix_sort_pairs(unsigned *keys, unsigned *vals, unsigned *keys_alt, unsigned *vals_alt,
                     int m, int bits, int *tmp, cudaStream_t s) {
    if (m <= 1) return JV_OK;
    if (bits < 1) bits = 1;
    int nt = (m + kRadixTile - 1) / kRadixTile;
    int nc = 256 * nt;
    int *counts = tmp;
    int *scan_tmp = tmp + nc + 1;
    unsigned *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        count_launch();
        k_rs_hist<<<nt, kBlock, 0, s>>>(ki, m, shift, nt, counts);
        JV_CHECK_LAUNCH();
        int rc = exclusive_scan_i32(counts, counts, nc, scan_tmp, s);
        if (rc) return rc;
        count_launch();
        k_rs_scatter<<<nt, kBlock, 0, s>>>(ki, vi, ko, vo, m, shift, nt, counts);
        JV_CHECK_LAUNCH();
        unsigned *t;
        t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    if (ki != keys) {
        JV_CUDA(cudaMemcpyAsync(keys, ki, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
        JV_CUDA(cudaMemcpyAsync(vals, vi, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
    }
    return JV_OK;
}

// ------------------------------------------------------- keys -> pointers
__global__ void k_keys_to_ptr(const unsigned *keys, int m, int *ptr, int K) {
    long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q > m) return;
    long long prev = (q == 0) ? -1 : (long long)keys[q - 1];
    long long cur = (q == m) ? (long long)K : (long long)keys[q];
    if (prev > K) prev = K;
    if (cur > K) cur = K;
    for (long long k = prev + 1; k <= cur; ++k) ptr[k] = (int)q;
}

int keys_to_ptr(const unsigned *sorted_keys, int m, int *ptr, int K, cudaStream_t s) {
    count_launch();
    k_keys_to_ptr<<<grid_for((long long)m + 1, kBlock), kBlock, 0, s>>>(sorted_keys, m, ptr, K);
    JV_CHECK_LAUNCH();
    return JV_OK;
}

}  // namespace jv
