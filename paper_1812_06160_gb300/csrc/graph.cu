// CUDA-graph replay of launch sequences.  The per-level schedules (mode LEVEL,
// and the upper-stage levels of HYBRID) issue one launch per level -- 382 on
// the 7-point 128^3 grid -- and one launch costs the host a few microseconds,
// more than a thin level's kernel takes on the GPU.  So the first call of a
// sequence captures it into a graph and later calls with the same operation,
// buffers and schedule replay it with one cudaGraphLaunch.  Capture runs on a
// private stream (the legacy default stream cannot be captured), which
// executes nothing; the graph is then launched on the handle's stream.
#include <cstdio>

#include "jv_internal.cuh"

namespace jv {

namespace {
constexpr size_t kMaxGraphs = 16;
}

int graph_run(jv_handle h, const std::vector<unsigned long long> &key,
              const std::function<int(cudaStream_t)> &seq) {
    if (h->opt.no_graphs) return seq(h->stream);
    // inside a capture of the caller's own: launch plainly into it
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (h->stream) JV_CUDA(cudaStreamIsCapturing(h->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone) return seq(h->stream);
    for (GraphEntry &g : h->graphs) {
        if (g.key != key) continue;
        g.used = ++h->graph_clock;
        g_launches.fetch_add(g.launches, std::memory_order_relaxed);
        JV_CUDA(cudaGraphLaunch(g.exec, h->stream));
        return JV_OK;
    }
    if (!h->cap_stream) JV_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const unsigned long long before = g_launches.load(std::memory_order_relaxed);
    JV_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
    const int rc = seq(h->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (rc != JV_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (rc != JV_OK) return rc;
        std::fprintf(stderr, "libjavelin_gb: graph capture failed: %s\n", cudaGetErrorString(e));
        return JV_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        std::fprintf(stderr, "libjavelin_gb: graph instantiation failed: %s\n", cudaGetErrorString(ei));
        return JV_ERR_CUDA;
    }
    if (h->graphs.size() >= kMaxGraphs) {          // drop the least recently used
        size_t lru = 0;
        for (size_t i = 1; i < h->graphs.size(); ++i)
            if (h->graphs[i].used < h->graphs[lru].used) lru = i;
        cudaGraphExecDestroy(h->graphs[lru].exec);
        h->graphs.erase(h->graphs.begin() + (long)lru);
    }
    GraphEntry g;
    g.key = key;
    g.exec = exec;
    g.launches = g_launches.load(std::memory_order_relaxed) - before;
    g.used = ++h->graph_clock;
    h->graphs.push_back(g);
    JV_CUDA(cudaGraphLaunch(exec, h->stream));
    return JV_OK;
}

void free_graphs(jv_handle h) {
    for (GraphEntry &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
}

}  // namespace jv
