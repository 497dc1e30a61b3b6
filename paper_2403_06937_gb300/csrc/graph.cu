// graph.cu -- see graph.cuh.
#include <mutex>

#include "graph.cuh"

namespace tc {
namespace {
struct GraphStream {
    cudaStream_t s = nullptr;
    cudaEvent_t before = nullptr, after = nullptr;
};
std::mutex g_mu;
GraphStream g_gs[64];

tc_status graph_stream(GraphStream** out) {
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TC_ERR_UNSUPPORTED_DEVICE, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    GraphStream& g = g_gs[dev];
    if (!g.s) {
        TC_CUDA(cudaStreamCreateWithFlags(&g.s, cudaStreamNonBlocking));
        TC_CUDA(cudaEventCreateWithFlags(&g.before, cudaEventDisableTiming));
        TC_CUDA(cudaEventCreateWithFlags(&g.after, cudaEventDisableTiming));
    }
    *out = &g;
    return TC_OK;
}
}  // namespace

tc_status run_captured(cudaStream_t user, const std::function<tc_status(cudaStream_t)>& first,
                       const std::function<tc_status(cudaStream_t)>& rest,
                       const std::function<tc_status(cudaStream_t)>& tail, bool capture) {
    if (capture) {
        // a caller already capturing `user` gets the launches in its own graph
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        TC_CUDA(cudaStreamIsCapturing(user, &cs));
        if (cs != cudaStreamCaptureStatusNone) capture = false;
    }
    if (!capture) {
        TC_TRY(first(user));
        TC_TRY(rest(user));
        return tail(user);
    }
    GraphStream* gs = nullptr;
    TC_TRY(graph_stream(&gs));
    cudaStream_t s = gs->s;
    TC_CUDA(cudaEventRecord(gs->before, user));
    TC_CUDA(cudaStreamWaitEvent(s, gs->before, 0));
    tc_status st = first(s);
    if (st == TC_OK) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        TC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        st = rest(s);
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (st == TC_OK && ce != cudaSuccess) st = fail(TC_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
        if (st == TC_OK) {
            ce = cudaGraphInstantiate(&exec, graph, 0);
            if (ce != cudaSuccess) st = fail(TC_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
        }
        if (st == TC_OK) {
            ce = cudaGraphLaunch(exec, s);
            if (ce != cudaSuccess) st = fail(TC_ERR_CUDA, "graph launch: %s", cudaGetErrorString(ce));
        }
        // an executable graph destroyed while in flight is freed when it completes
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
    if (st == TC_OK) st = tail(s);
    // order the caller's stream after everything enqueued here, also on failure
    cudaEventRecord(gs->after, s);
    cudaStreamWaitEvent(user, gs->after, 0);
    return st;
}

}  // namespace tc
