// Hop latency: the unit step of the sync-free critical path.
//
// In the point-to-point schedule of Sec. III-A (Fig. 4) a row starts once
// the rows it depends on have published their results, so a chain of
// dependent rows costs, per link, one publication seen by another SM: a
// relaxed store at gpu scope that reaches the point of coherence (L2) and a
// relaxed load, polling there, that returns the new value.  This measures
// that link directly: CTA 0 and one partner CTA ping-pong a counter through
// two words; a round trip is two links.  The grid is one 32-thread CTA per
// SM launched cooperatively, so both CTAs are resident at once, and every
// wait is bounded by wall-clock time, so a missing partner ends in an error,
// never a hang.
#include <algorithm>

#include "jv_internal.cuh"

namespace jv {
namespace {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait (bounded) until *w == v; false on timeout.
__device__ __forceinline__ bool await_word(const unsigned *w, unsigned v, unsigned long long t_end) {
    for (unsigned it = 0;; ++it) {
        if (ld_relaxed(w) == v) return true;
        if ((it & 255u) == 0 && global_ns() > t_end) return false;
    }
}

// out[0] = elapsed ns of CTA 0's rounds, out[1] = number of sides that timed out.
__global__ void k_hop(unsigned *words, int partner, int rounds, unsigned long long limit_ns,
                      unsigned long long *out) {
    if (threadIdx.x != 0) return;
    const bool first = blockIdx.x == 0;
    if (!first && (int)blockIdx.x != partner) return;
    unsigned *ping = words, *pong = words + 32;          // 128 bytes apart
    const unsigned long long t0 = global_ns();
    const unsigned long long t_end = t0 + limit_ns;
    bool ok = true;
    for (int i = 1; i <= rounds && ok; ++i) {
        if (first) {
            st_relaxed(ping, (unsigned)i);
            ok = await_word(pong, (unsigned)i, t_end);
        } else {
            ok = await_word(ping, (unsigned)i, t_end);
            if (ok) st_relaxed(pong, (unsigned)i);
        }
    }
    if (first) out[0] = global_ns() - t0;
    if (!ok) atomicAdd(out + 1, 1ull);
}

}  // namespace

int hop_latency(int rounds, int npartners, double *out_us, cudaStream_t s) {
    int dev = 0, nsm = 0, coop = 0;
    JV_CUDA(cudaGetDevice(&dev));
    JV_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    JV_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop || nsm < 2) return JV_ERR_CUDA;
    unsigned *words = nullptr;
    unsigned long long *out = nullptr;
    JV_CUDA(cudaMalloc(&words, 256));
    if (cudaMalloc(&out, 16) != cudaSuccess) {
        cudaFree(words);
        return JV_ERR_NOMEM;
    }
    std::vector<double> hops;
    int rc = JV_OK;
    const unsigned long long limit_ns = 200ull * 1000 * 1000;   // 0.2 s per pair
    for (int k = 0; k < npartners && rc == JV_OK; ++k) {
        int partner = 1 + (int)((long long)k * (nsm - 1) / npartners);
        unsigned long long h_out[2] = {0, 0};
        if (cudaMemsetAsync(words, 0, 256, s) != cudaSuccess ||
            cudaMemsetAsync(out, 0, 16, s) != cudaSuccess) { rc = JV_ERR_CUDA; break; }
        void *args[] = {&words, &partner, &rounds, (void *)&limit_ns, &out};
        count_launch();
        if (cudaLaunchCooperativeKernel((void *)k_hop, dim3(nsm), dim3(32), args, 0, s) != cudaSuccess ||
            cudaMemcpyAsync(h_out, out, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { rc = JV_ERR_CUDA; break; }
        if (h_out[1] != 0) { rc = JV_ERR_TIMEOUT; break; }
        hops.push_back((double)h_out[0] * 1e-3 / (2.0 * rounds));
    }
    cudaFree(words);
    cudaFree(out);
    if (rc != JV_OK) return rc;
    std::sort(hops.begin(), hops.end());
    *out_us = hops[hops.size() / 2];
    return JV_OK;
}

}  // namespace jv
