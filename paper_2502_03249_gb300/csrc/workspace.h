// workspace.h -- solver vectors, scalar records and CUDA graphs a context
// keeps between calls (allocated on first use, freed by stag_destroy).
#pragma once

#include "ctx.h"
#include "graph.h"

namespace stag {

// Launch shapes of a CG plan's kernels, chosen by the autotuner (cg.cu).
struct CgShape {
    int hop = 128;                 // hop kernel block size
    int upd = vcfg(256, 1);        // update kernel (vcfg: block size, sites per thread)
    int pk = vcfg(256, 1);         // direction update kernel
    int mpdot_stage = 0;           // Mp_dot staging (STAGE_* bits, half 12-real)
};

// A hop-kernel candidate: the block size, with the STAGE_* bits of what the
// kernel stages in shared memory (dslash_site_staged) above HOP_STAGE_SHIFT.
constexpr int HOP_STAGE_SHIFT = 12;
constexpr int HOP_BS_MASK = (1 << HOP_STAGE_SHIFT) - 1;

// Buffers of one mixed-precision configuration (inner precision x compression).
struct MixedSlot {
    void *r = nullptr, *p = nullptr, *Ap = nullptr, *t = nullptr;   // inner precision
    void* xlo = nullptr;                                             // float accumulator of x
    CgScalars* sc = nullptr;
    // per link field [as uploaded, temporal gauge]: the loop graph (it holds
    // the link fields it was captured with), the double arithmetic of its
    // reliable update, and the inner kernels' launch shapes (autotuned once)
    LoopGraph lg[2];
    int Vh = 0;
    int graph_arith[2] = {-1, -1};
    bool ready = false;
    CgShape shape[2];
    bool tuned[2] = {false, false};
    template <class S> S spinor(void* buf) const;
};
template <> inline SpinorF32 MixedSlot::spinor<SpinorF32>(void* buf) const { return SpinorF32{(float2*)buf, Vh}; }
template <> inline SpinorF16 MixedSlot::spinor<SpinorF16>(void* buf) const
{
    return SpinorF16{(uint4*)buf, Vh};
}

// Buffers of one batched configuration (inner precision x compression), for
// up to cap systems: inner r p Ap t (S), xlo (F32 or F64), and the double
// vectors x_hi r_hi b t64, all n fields back to back.
struct BatchSlot {
    void *r = nullptr, *p = nullptr, *Ap = nullptr, *t = nullptr, *xlo = nullptr;
    double2 *x_hi = nullptr, *r_hi = nullptr, *b = nullptr, *t64 = nullptr;
    double2* x_df = nullptr;       // x_hi split into double-float pairs (double-float reliable updates)
    CgScalars* sc = nullptr;
    double* part = nullptr;
    double* shifts = nullptr;
    unsigned* cnt_sys = nullptr;   // per-system reduction counters, zero between kernels
    size_t s_stride = 0, sx_stride = 0, f64_stride = 0;
    int Vh = 0, cap = 0, nrhs = 0, gx = 0, prec = 0, graph_nb = 0, graph_arith = -1;
    int tg = 0, graph_tg = -1;     // temporal-gauge links (this solve's, and the graph's)
    bool ready = false;
    LoopGraph lg;
    template <class S> S spinor(void* buf) const;
    void release();
};
template <> inline SpinorF64 BatchSlot::spinor<SpinorF64>(void* buf) const { return SpinorF64{(double2*)buf}; }
template <> inline SpinorF32 BatchSlot::spinor<SpinorF32>(void* buf) const { return SpinorF32{(float2*)buf, Vh}; }
template <> inline SpinorF16 BatchSlot::spinor<SpinorF16>(void* buf) const
{
    return SpinorF16{(uint4*)buf, Vh};
}

// Buffers of the multi-shift Krylov phase (inner precision): p_i and x_i of
// every shift, r, Ap, t, the scalar records and the replicated source for the
// refinement.
struct MsSlot {
    void *P = nullptr, *X = nullptr, *r = nullptr, *Ap = nullptr, *t = nullptr;
    CgScalars* sc = nullptr;
    struct MsState* ms = nullptr;
    double* shifts = nullptr;
    double2* brep = nullptr;
    size_t stride = 0;
    int Vh = 0, cap = 0, nshift = 0, base = 0, graph_n = 0, graph_base = -1, graph_tg = -1;
    bool ready = false;
    LoopGraph lg;
    template <class S> S spinor(void* buf) const;
    void release();
};
template <> inline SpinorF64 MsSlot::spinor<SpinorF64>(void* buf) const { return SpinorF64{(double2*)buf}; }
template <> inline SpinorF32 MsSlot::spinor<SpinorF32>(void* buf) const { return SpinorF32{(float2*)buf, Vh}; }

struct Workspace {
    // double-precision CG (even: x r p Ap b, odd: t), canonical layout; the
    // mixed solver uses x, r, b, t as its double-precision vectors
    double2 *x = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr, *b = nullptr, *t = nullptr;
    CgScalars* sc = nullptr;        // device scalar records
    CgScalars* sc_host = nullptr;   // pinned host mirror for the final read
    bool f64_ready = false;
    // per plan [IEEE double, double-float, double-float in temporal gauge,
    // IEEE double in temporal gauge]
    cudaGraph_t f64_graph[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraphExec_t f64_exec[4] = {nullptr, nullptr, nullptr, nullptr};
    // double-float CG: 1 applies p = r + beta p inside the operator passes
    // (three launches per iteration), 0 as a pass of its own; -1 undecided
    int df_dir = -1;
    CgShape cg_shape[4];            // per plan, as f64_graph
    bool cg_tuned[4] = {false, false, false, false};
    MixedSlot mixed[2][2];          // [F32, F16][18, 12]
    BatchSlot batch[3][2];          // [F64, F32, F16][18, 12]
    MsSlot ms[2];                   // multi-shift [F64, F32]
};

int free_graph_pair(cudaGraph_t& g, cudaGraphExec_t& e);
void free_mixed(Workspace* ws);
void free_batches(Workspace* ws);

}  // namespace stag
