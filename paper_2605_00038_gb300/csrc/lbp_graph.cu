// lbp_graph_*: one lbp_decode call captured into a CUDA graph and replayed.
//
// A decode is a short chain of stream operations: a memset of the work
// counters, K_bp, K_osd_warp and K_osd.  At small batches the host cost of
// issuing them is a visible part of the latency.  lbp_graph_create issues the
// chain once into a capturing stream and instantiates the graph, and each
// lbp_graph_launch replays it with a single call.  Buffers, sizes and
// parameters are frozen at capture; new shots are decoded by writing their
// syndromes into the same device buffer before the launch.  The plan is the
// one lbp_decode would make for the call (the latency layouts of a batch of
// at most one shot per SM included).
#include <new>

#include "internal.h"
#include "timing.h"

struct lbp_graph {
    cudaGraphExec_t exec = nullptr;
    int device = 0;
};

extern "C" int lbp_graph_create(const lbp_code *code, const lbp_params *params, int64_t num_shots,
                                const uint64_t *syndromes, uint64_t *err_out, uint8_t *converged,
                                uint8_t *osd_out, int32_t *iters_out, float *llr_out, void *workspace,
                                size_t workspace_bytes, lbp_graph **out) {
    if (!out) return LBP_EINVAL;
    *out = nullptr;
    if (!code || !params || num_shots < 1 || num_shots > (1ll << 31) || !syndromes || !err_out || !converged ||
        !iters_out || !workspace)
        return LBP_EINVAL;
    const size_t need = lbp_workspace_size(code, params, num_shots);   // 0: invalid parameters
    if (need == 0) return LBP_EINVAL;
    if (workspace_bytes < need) return LBP_ENOMEM;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return LBP_EINVAL;
    if (lbp::timing_on()) return LBP_EINVAL;          // the timing hooks record events per call
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != code->device) return LBP_EINVAL;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return LBP_ECUDA;
    }
    int rc = LBP_OK;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        rc = LBP_ECUDA;
    } else {
        rc = lbp::decode_device(code, params, num_shots, syndromes, err_out, converged, osd_out, iters_out,
                                llr_out, workspace, workspace_bytes, cs);
        // The capture always ends, whether or not the chain was issued.
        if (cudaStreamEndCapture(cs, &graph) != cudaSuccess && rc == LBP_OK) rc = LBP_ECUDA;
    }
    lbp_graph *g = nullptr;
    if (rc == LBP_OK) {
        g = new (std::nothrow) lbp_graph();
        if (!g) rc = LBP_ENOMEM;
    }
    if (rc == LBP_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) rc = LBP_ECUDA;
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (rc != LBP_OK) {
        cudaGetLastError();
        delete g;
        return rc;
    }
    g->device = dev;
    *out = g;
    return LBP_OK;
}

extern "C" int lbp_graph_launch(lbp_graph *graph, void *stream) {
    if (!graph || !graph->exec) return LBP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != graph->device) return LBP_EINVAL;
    if (cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return LBP_ECUDA;
    }
    return LBP_OK;
}

extern "C" int lbp_graph_destroy(lbp_graph *graph) {
    if (!graph) return LBP_EINVAL;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    delete graph;
    return LBP_OK;
}
