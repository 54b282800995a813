// graph.h -- CUDA graphs with device-controlled loops:
//     while (W) { seg1; if (I) { seg_if; } seg2; }
// W and I are conditional handles the kernels set with cudaGraphSetConditional,
// so a whole solve runs from one graph launch with no host round trip.
// Segments are recorded by stream capture into the conditional bodies.
#pragma once

#include <vector>

#include "ctx.h"

namespace stag {

struct LoopGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle w = 0;   // while condition (default 1 at every launch)
    cudaGraphConditionalHandle i = 0;   // inner if condition (0 when there is none)
    void destroy()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
};

// Record the launches of seg(stream) into graph g after the nodes deps; the
// nodes left dangling at the end are returned in tail.
template <class Seg>
static int capture_into(cudaStream_t cap, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, Seg seg,
                        std::vector<cudaGraphNode_t>* tail)
{
    STAG_CUDA_TRY(cudaStreamBeginCaptureToGraph(cap, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                                cudaStreamCaptureModeThreadLocal));
    int rc = seg(cap);
    if (rc == STAG_OK && tail) {
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t* d = nullptr;
        size_t nd = 0;
        if (cudaStreamGetCaptureInfo(cap, &st, nullptr, nullptr, &d, nullptr, &nd) != cudaSuccess) rc = STAG_ECUDA;
        else tail->assign(d, d + nd);
    }
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &out);
    if (rc != STAG_OK) return rc;
    if (e != cudaSuccess) {
        set_error("graph capture failed: %s", cudaGetErrorString(e));
        return STAG_ECUDA;
    }
    return STAG_OK;
}

// Build and instantiate  while (W) { seg1; [if (I) { seg_if; }] seg2; }.
// The segments receive the handles through lg (set before they are called).
template <class S1, class SI, class S2>
int build_loop_graph(cudaStream_t cap, LoopGraph& lg, bool with_if, S1 seg1, SI seg_if, S2 seg2)
{
    lg.destroy();
    STAG_CUDA_TRY(cudaGraphCreate(&lg.graph, 0));
    STAG_CUDA_TRY(cudaGraphConditionalHandleCreate(&lg.w, lg.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = lg.w;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    STAG_CUDA_TRY(cudaGraphAddNode(&wnode, lg.graph, nullptr, nullptr, 0, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    std::vector<cudaGraphNode_t> tail;
    if (with_if) STAG_CUDA_TRY(cudaGraphConditionalHandleCreate(&lg.i, body, 0, 0));
    STAG_TRY(capture_into(cap, body, {}, seg1, &tail));
    if (with_if) {
        cudaGraphNodeParams ip = {};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = lg.i;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t inode;
        STAG_CUDA_TRY(cudaGraphAddNode(&inode, body, tail.data(), nullptr, tail.size(), &ip));
        STAG_TRY(capture_into(cap, ip.conditional.phGraph_out[0], {}, seg_if, nullptr));
        tail.assign(1, inode);
    }
    STAG_TRY(capture_into(cap, body, tail, seg2, nullptr));
    cudaError_t e = cudaGraphInstantiate(&lg.exec, lg.graph, 0);
    if (e != cudaSuccess) {
        set_error("graph instantiation failed: %s", cudaGetErrorString(e));
        lg.destroy();
        return STAG_ECUDA;
    }
    return STAG_OK;
}

}  // namespace stag
