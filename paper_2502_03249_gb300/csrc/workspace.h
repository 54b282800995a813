// workspace.h -- solver vectors, scalar records and CUDA graphs a context
// keeps between calls (allocated on first use, freed by stag_destroy).
#pragma once

#include "ctx.h"

namespace stag {

struct Workspace {
    // double-precision CG (even: x r p Ap b, odd: t), canonical layout
    double2 *x = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr, *b = nullptr, *t = nullptr;
    CgScalars* sc = nullptr;        // device scalar records
    CgScalars* sc_host = nullptr;   // pinned host mirror for the final read
    bool f64_ready = false;
    cudaGraph_t f64_graph = nullptr;
    cudaGraphExec_t f64_exec = nullptr;
};

int free_graph_pair(cudaGraph_t& g, cudaGraphExec_t& e);

}  // namespace stag
