// cg.cu -- double-precision conjugate gradient on M = m^2 - D_eo D_oe
// (the inversion the paper benchmarks, Sec. 1 and Sec. 4.2), with the
// iteration running inside one CUDA graph whose while-loop condition is
// cleared on the device, so no host round trip happens per iteration.
#include <chrono>
#include <cstdlib>
#include <new>

#include "cg_df.cuh"
#include "tune.h"
#include "workspace.h"

namespace stag {

constexpr int HOP_BS = 128;
constexpr int BLAS_BS = 256;
constexpr int MAX_RESTARTS = 100;
// CG iterations per body of the graph's while loop: the conditional node costs
// a few microseconds per body execution, so the body holds several iterations
// (each kernel returns at once after the update kernel has set done, so at
// most GRAPH_UNROLL - 1 empty iterations run after convergence).
constexpr int GRAPH_UNROLL = 4;

typedef LinkField<double2, 18> LF64;

static inline int nblk(int n, int bs) { return (n + bs - 1) / bs; }

// ------------------------------------------------- tuned launch shapes
//
// The autotuner picks, per plan and lattice, the block size of the hop kernel
// (64, 128 or 256 threads, registers per thread unchanged) and the launch
// shape of the vector kernels (vcfg: 128 or 256 threads, one or two sites per
// thread).  Every shape computes the same bits (the reductions use fixed
// 128-site chunks, common.cuh).
#define STAG_VEC_SWITCH(cfg, CALL)                                   \
    switch (cfg) {                                                   \
    case vcfg(256, 1): { constexpr int BS = 256, SPT = 1; CALL; } break; \
    case vcfg(128, 1): { constexpr int BS = 128, SPT = 1; CALL; } break; \
    case vcfg(256, 2): { constexpr int BS = 256, SPT = 2; CALL; } break; \
    case vcfg(128, 2): { constexpr int BS = 128, SPT = 2; CALL; } break; \
    default: set_error("bad vector kernel shape %d", cfg); return STAG_EINVAL; \
    }
#define STAG_HOP_SWITCH(bs, CALL)                                    \
    switch (bs) {                                                    \
    case 128: { constexpr int BS = 128; CALL; } break;               \
    case 64: { constexpr int BS = 64; CALL; } break;                 \
    case 256: { constexpr int BS = 256; CALL; } break;               \
    default: set_error("bad hop block size %d", bs); return STAG_EINVAL; \
    }
static inline int vgrid(int Vh, int cfg) { return nblk(Vh, vcfg_BS(cfg) * vcfg_SPT(cfg)); }
static const std::vector<int> HOP_CANDS = {128, 64, 256};
static const std::vector<int> VEC_CANDS = {vcfg(256, 1), vcfg(128, 1), vcfg(256, 2), vcfg(128, 2)};

// -------------------------------------------------------------- M apply

int apply_M_f64(stag_ctx ctx, double2* out, const double2* in, double mass, double2* tmp_odd, cudaStream_t s)
{
    const void* lk = nullptr;
    STAG_TRY(ensure_links(ctx, STAG_F64, 18, &lk));
    LF64 U{(const double2*)lk, ctx->g.Vh};
    const int grid = nblk(ctx->g.Vh, HOP_BS);
    k_hop<LF64, SpinorF64, HOP_BS><<<grid, HOP_BS, 0, s>>>(ctx->g, 1, U, SpinorF64{(double2*)in}, SpinorF64{tmp_odd},
                                                           nullptr, 0);
    k_xpay_hop<LF64, SpinorF64, SpinorF64, HOP_BS><<<grid, HOP_BS, 0, s>>>(ctx->g, U, SpinorF64{tmp_odd}, SpinorF64{(double2*)in},
                                                                 SpinorF64{out}, mass * mass);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

// ------------------------------------------------------- start / residual

// Fresh start: x = 0, r = p = b, rr = rr0 = |b|^2, scalars reset.
template <int BS>
__global__ void __launch_bounds__(BS) k_cg_start_f64(int Vh, const double2* b, double2* x, double2* r, double2* p,
                                                     CgScalars* sc, double tol, int maxiter, double m2,
                                                     double sigma, double* part, unsigned* cnt)
{
    __shared__ double red[BS / 32];
    __shared__ bool last;
    const int h = blockIdx.x * BS + threadIdx.x;
    double d = 0.0;
    if (h < Vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 v = b[(size_t)h * 3 + c];
            x[(size_t)h * 3 + c] = make_double2(0.0, 0.0);
            r[(size_t)h * 3 + c] = v;
            p[(size_t)h * 3 + c] = v;
            d = fma(v.x, v.x, d);
            d = fma(v.y, v.y, d);
        }
    }
    const double bs = block_sum<BS>(d, red);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
    if (!arrive_last(cnt, &last)) return;
    const double bb = sum_partials<BS>(part, gridDim.x, red);
    if (threadIdx.x == 0) {
        *cnt = 0;
        CgScalars s = {};
        s.rr = s.rr0 = s.rr_true = bb;
        s.tol2 = tol * tol * bb;
        s.maxiter = maxiter;
        s.m2 = m2;
        s.sigma = sigma;
        s.done = (bb == 0.0) ? 1 : 0;
        *sc = s;
    }
}

// Restart from the true residual now held in r: p = r, rr = rr_true, beta = 0
// (the double-float iteration applies p = r + beta p when it next reads p).
template <int BS>
__global__ void __launch_bounds__(BS) k_cg_restart_f64(int Vh, const double2* r, double2* p, CgScalars* sc)
{
    const long long i = (long long)blockIdx.x * BS + threadIdx.x;
    if (i < 3LL * Vh) p[i] = r[i];
    if (i == 0) {
        sc->rr = sc->rr_true;
        sc->beta = 0.0;
        sc->done = 0;
        sc->status = 0;
    }
}

// ------------------------------------------------------------ workspace

int ensure_cg_f64(stag_ctx ctx)
{
    if (!ctx->ws) {
        ctx->ws = new (std::nothrow) Workspace();
        if (!ctx->ws) return STAG_ENOMEM;
    }
    Workspace* ws = ctx->ws;
    if (ws->f64_ready) return STAG_OK;
    const size_t n = (size_t)3 * ctx->g.Vh;
    double2** bufs[] = {&ws->x, &ws->r, &ws->p, &ws->Ap, &ws->b, &ws->t};
    for (auto b : bufs) {
        if (!*b) STAG_CUDA_TRY(cudaMalloc(b, n * sizeof(double2)));
    }
    if (!ws->sc) STAG_CUDA_TRY(cudaMalloc(&ws->sc, sizeof(CgScalars) * 64));
    if (!ws->sc_host) STAG_CUDA_TRY(cudaMallocHost(&ws->sc_host, sizeof(CgScalars) * 64));
    ws->f64_ready = true;
    return STAG_OK;
}

// Two double-precision CG plans share the driver below:
//   F64Plan   IEEE double (STAG_F64): double vectors, double links, FP64 BLAS;
//   DFPlan    double-float (STAG_F64X): the Krylov vectors as double-floats
//             (SpinorDF over the same buffers), double-float links, every
//             per-site operation on the FP32 pipe (cg_df.cuh).
// Each provides start / enqueue_iter / true_residual / restart / finish.
template <int SLOT>
struct F64PlanT {
    typedef LF64 LF;
    static constexpr int slot = SLOT;
    static constexpr int prec = STAG_F64;
    static int prepare(stag_ctx) { return STAG_OK; }
    static int start(stag_ctx ctx, const double2* b_in, double mass, double sigma, double tol, int maxiter)
    {
        Workspace* ws = ctx->ws;
        const int Vh = ctx->g.Vh;
        // b' = 2^-k b with its largest component in [1, 2); x = 2^k x' at the end
        STAG_TRY(normalise_fields(ctx, b_in, ws->b, 1, (size_t)3 * Vh, SLOT_SOLVE, ctx->stream));
        k_cg_start_f64<BLAS_BS><<<nblk(Vh, BLAS_BS), BLAS_BS, 0, ctx->stream>>>(
            Vh, ws->b, ws->x, ws->r, ws->p, ws->sc, tol, maxiter, mass * mass, sigma, ctx->partials, ctx->counters);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    static constexpr const char* name = SLOT == 0 ? "cg_f64" : "cg_f64_tg";
    static int launch_hop(stag_ctx ctx, const LF& U, int bs, cudaStream_t s, const CgScalars* sc)
    {
        Workspace* ws = ctx->ws;
        STAG_HOP_SWITCH(bs, (k_hop_guarded<LF, SpinorF64, BS><<<nblk(ctx->g.Vh, BS), BS, 0, s>>>(
                                ctx->g, 1, U, SpinorF64{ws->p}, SpinorF64{ws->t}, sc)));
        return STAG_OK;
    }
    static int launch_update(stag_ctx ctx, int cfg, cudaStream_t s, CgScalars* sc, cudaGraphConditionalHandle cond,
                             int use_cond)
    {
        Workspace* ws = ctx->ws;
        STAG_VEC_SWITCH(cfg, (k_cg_update<SpinorF64, BS, SPT><<<vgrid(ctx->g.Vh, cfg), BS, 0, s>>>(
                                 ctx->g.Vh, SpinorF64{ws->x}, SpinorF64{ws->r}, SpinorF64{ws->p}, SpinorF64{ws->Ap},
                                 sc, ctx->partials, ctx->counters, grid_sum_of(ctx), cond, use_cond)));
        return STAG_OK;
    }
    static int launch_p(stag_ctx ctx, int cfg, cudaStream_t s, const CgScalars* sc)
    {
        Workspace* ws = ctx->ws;
        STAG_VEC_SWITCH(cfg, (k_cg_p<SpinorF64, BS, SPT><<<vgrid(ctx->g.Vh, cfg), BS, 0, s>>>(
                                 ctx->g.Vh, SpinorF64{ws->r}, SpinorF64{ws->p}, sc)));
        return STAG_OK;
    }
    static bool has_p(stag_ctx) { return true; }
    // one CG iteration (four kernels) on stream s, in the tuned shapes
    static int enqueue_iter(stag_ctx ctx, const LF& U, cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond)
    {
        Workspace* ws = ctx->ws;
        const Geom g = ctx->g;
        const CgShape& sh = ws->cg_shape[slot];
        SpinorF64 p{ws->p}, Ap{ws->Ap}, t{ws->t};
        STAG_TRY(launch_hop(ctx, U, sh.hop, s, ws->sc));
        k_Mp_dot<LF, SpinorF64, SpinorF64, HOP_BS><<<nblk(g.Vh, HOP_BS), HOP_BS, 0, s>>>(g, U, t, p, Ap, ws->sc,
                                                                                       ctx->partials, ctx->counters,
                                                                                       grid_sum_of(ctx));
        STAG_TRY(launch_update(ctx, sh.upd, s, ws->sc, cond, use_cond));
        STAG_TRY(launch_p(ctx, sh.pk, s, ws->sc));
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    // r = b - M x in double precision
    static int true_residual(stag_ctx ctx, const LF& U)
    {
        Workspace* ws = ctx->ws;
        const Geom g = ctx->g;
        k_hop<LF, SpinorF64, HOP_BS><<<nblk(g.Vh, HOP_BS), HOP_BS, 0, ctx->stream>>>(g, 1, U, SpinorF64{ws->x},
                                                                                    SpinorF64{ws->t}, nullptr, 0);
        k_true_resid_f64<LF, SpinorF64, HOP_BS><<<nblk(g.Vh, HOP_BS), HOP_BS, 0, ctx->stream>>>(
            g, U, SpinorF64{ws->t}, ws->x, ws->b, ws->r, ws->sc, ctx->partials, ctx->counters, 0);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    static int finish(stag_ctx ctx, double2* x_out)
    {
        return scale_fields_out(ctx, ctx->ws->x, x_out, 1, (size_t)3 * ctx->g.Vh, SLOT_SOLVE, 1, ctx->stream);
    }
};

// Whether the double-float CG applies p = r + beta p inside its operator
// passes: when its five vectors (x r p Ap t, 48 bytes per site each) fit in
// half of L2, where the hop's second neighbour gather hits L2 (32^3 x 8: 5.62
// against 5.72 ms per solve); on larger lattices the separate pass is faster
// (48^3 x 12: 29.7 against 30.7 ms).  Environment STAG_CG_DIR=0 or 1 forces
// either arrangement (the two give the same bits).
static int decide_df_dir(stag_ctx ctx)
{
    Workspace* ws = ctx->ws;
    if (ws->df_dir >= 0) return STAG_OK;
    const char* e = getenv("STAG_CG_DIR");
    if (e && (e[0] == '0' || e[0] == '1')) {
        ws->df_dir = e[0] - '0';
        return STAG_OK;
    }
    int l2 = 0;
    STAG_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device));
    ws->df_dir = (5.0 * 48.0 * ctx->g.Vh <= 0.5 * (double)l2) ? 1 : 0;
    return STAG_OK;
}

template <class LFT, int SLOT>
struct DFPlanT {
    typedef LFT LF;
    static constexpr int slot = SLOT;
    static constexpr int prec = STAG_F64X;
    static SpinorDF v(double2* p) { return SpinorDF{reinterpret_cast<float4*>(p)}; }
    static int prepare(stag_ctx ctx) { return decide_df_dir(ctx); }
    static int start(stag_ctx ctx, const double2* b_in, double mass, double sigma, double tol, int maxiter)
    {
        Workspace* ws = ctx->ws;
        const int Vh = ctx->g.Vh;
        STAG_TRY(decide_df_dir(ctx));
        // b stays double (the true residual is formed against it), normalised to
        // b' = 2^-k b with its largest component in [1, 2): every vector of the
        // solve then lies well inside the double-float range
        STAG_TRY(normalise_fields(ctx, b_in, ws->b, 1, (size_t)3 * Vh, SLOT_SOLVE, ctx->stream));
        k_dfcg_start<BLAS_BS><<<nblk(Vh, BLAS_BS), BLAS_BS, 0, ctx->stream>>>(
            Vh, ws->b, v(ws->x), v(ws->r), v(ws->p), ws->sc, tol, maxiter, mass * mass, sigma, ctx->partials,
            ctx->counters);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    static constexpr const char* name = SLOT == 1 ? "cg_f64x" : "cg_f64x_tg";
    static int launch_hop(stag_ctx ctx, const LF& U, int bs, cudaStream_t s, const CgScalars* sc)
    {
        Workspace* ws = ctx->ws;
        const Geom g = ctx->g;
        if (ws->df_dir == 1)
            STAG_HOP_SWITCH(bs, (k_dfcg_hop<LF, BS><<<nblk(g.Vh, BS), BS, 0, s>>>(g, U, v(ws->r), v(ws->p),
                                                                                  v(ws->t), sc)))
        else
            STAG_HOP_SWITCH(bs, (k_hop_guarded<LF, SpinorDF, BS><<<nblk(g.Vh, BS), BS, 0, s>>>(
                                    g, 1, U, v(ws->p), v(ws->t), sc)))
        return STAG_OK;
    }
    static int launch_update(stag_ctx ctx, int cfg, cudaStream_t s, CgScalars* sc, cudaGraphConditionalHandle cond,
                             int use_cond)
    {
        Workspace* ws = ctx->ws;
        STAG_VEC_SWITCH(cfg, (k_dfcg_update<BS, SPT><<<vgrid(ctx->g.Vh, cfg), BS, 0, s>>>(
                                 ctx->g.Vh, v(ws->x), v(ws->r), v(ws->p), v(ws->Ap), sc, ctx->partials,
                                 ctx->counters, grid_sum_of(ctx), cond, use_cond)));
        return STAG_OK;
    }
    static int launch_p(stag_ctx ctx, int cfg, cudaStream_t s, const CgScalars* sc)
    {
        Workspace* ws = ctx->ws;
        STAG_VEC_SWITCH(cfg, (k_dfcg_p<BS, SPT><<<vgrid(ctx->g.Vh, cfg), BS, 0, s>>>(ctx->g.Vh, v(ws->r),
                                                                                      v(ws->p), sc)));
        return STAG_OK;
    }
    // the direction update runs as a pass of its own only without df_dir
    static bool has_p(stag_ctx ctx) { return ctx->ws->df_dir != 1; }
    static int enqueue_iter(stag_ctx ctx, const LF& U, cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond)
    {
        Workspace* ws = ctx->ws;
        const Geom g = ctx->g;
        const CgShape& sh = ws->cg_shape[slot];
        const int gh = nblk(g.Vh, HOP_BS);
        STAG_TRY(launch_hop(ctx, U, sh.hop, s, ws->sc));
        if (ws->df_dir == 1)
            k_dfcg_Mp_dot<LF, HOP_BS, true><<<gh, HOP_BS, 0, s>>>(g, U, v(ws->t), v(ws->r), v(ws->p), v(ws->Ap),
                                                                  ws->sc, ctx->partials, ctx->counters,
                                                                  grid_sum_of(ctx));
        else
            k_dfcg_Mp_dot<LF, HOP_BS, false><<<gh, HOP_BS, 0, s>>>(g, U, v(ws->t), v(ws->r), v(ws->p), v(ws->Ap),
                                                                   ws->sc, ctx->partials, ctx->counters,
                                                                   grid_sum_of(ctx));
        STAG_TRY(launch_update(ctx, sh.upd, s, ws->sc, cond, use_cond));
        if (ws->df_dir != 1) STAG_TRY(launch_p(ctx, sh.pk, s, ws->sc));
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    static int true_residual(stag_ctx ctx, const LF& U)
    {
        Workspace* ws = ctx->ws;
        const Geom g = ctx->g;
        k_hop<LF, SpinorDF, HOP_BS><<<nblk(g.Vh, HOP_BS), HOP_BS, 0, ctx->stream>>>(g, 1, U, v(ws->x), v(ws->t),
                                                                                   nullptr, 0);
        k_dfcg_true_resid<LF, HOP_BS><<<nblk(g.Vh, HOP_BS), HOP_BS, 0, ctx->stream>>>(
            g, U, v(ws->t), v(ws->x), ws->b, v(ws->r), ws->sc, ctx->partials, ctx->counters);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    static int finish(stag_ctx ctx, double2* x_out)
    {
        return join_fields_scaled(ctx, reinterpret_cast<const float4*>(ctx->ws->x), x_out, 1, (size_t)3 * ctx->g.Vh,
                                  SLOT_SOLVE, 1, 0, ctx->stream);
    }
};

// The plans by slot: IEEE double 0, double-float 1, and the same on
// temporal-gauge links (U.tg = 1, M' = g M g^dagger: tgauge.cu) 3 and 2.  A
// slot owns its graph, which holds the link field it was captured with.
typedef F64PlanT<0> F64Plan;
typedef F64PlanT<3> F64PlanTG;
typedef DFPlanT<LinkFieldDF<18>, 1> DFPlan;
typedef DFPlanT<LinkFieldDF<18>, 2> DFPlanTG;

// the graph  while (cond) { GRAPH_UNROLL CG iterations }, built once per context and plan
template <class Plan>
static int ensure_cg_graph(stag_ctx ctx, const typename Plan::LF& U)
{
    Workspace* ws = ctx->ws;
    const int slot = Plan::slot;
    if (ws->f64_exec[slot]) return STAG_OK;
    cudaGraph_t graph = nullptr;
    STAG_CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond;
    STAG_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    STAG_CUDA_TRY(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    STAG_CUDA_TRY(cudaStreamBeginCaptureToGraph(ctx->cap_stream, body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal));
    int rc = STAG_OK;
    for (int u = 0; u < GRAPH_UNROLL && rc == STAG_OK; ++u) rc = Plan::enqueue_iter(ctx, U, ctx->cap_stream, cond, 1);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &captured);
    if (rc != STAG_OK || e != cudaSuccess) {
        cudaGraphDestroy(graph);
        set_error("capturing the CG body failed: %s", cudaGetErrorString(e));
        return rc != STAG_OK ? rc : STAG_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        set_error("instantiating the CG graph failed: %s", cudaGetErrorString(e));
        return STAG_ECUDA;
    }
    ws->f64_graph[slot] = graph;
    ws->f64_exec[slot] = exec;
    return STAG_OK;
}

// run the iteration until the device says done: one graph launch, or a host
// loop that reads the done flag every check_every iterations
template <class Plan>
static int run_cg_loop(stag_ctx ctx, const typename Plan::LF& U, const stag_solver_params& prm)
{
    Workspace* ws = ctx->ws;
    if (prm.use_graph) {
        STAG_TRY(ensure_cg_graph<Plan>(ctx, U));
        STAG_CUDA_TRY(cudaGraphLaunch(ws->f64_exec[Plan::slot], ctx->stream));
        return STAG_OK;
    }
    const int every = prm.check_every > 0 ? prm.check_every : 25;
    for (;;) {
        for (int k = 0; k < every; ++k) STAG_TRY(Plan::enqueue_iter(ctx, U, ctx->stream, 0, 0));
        STAG_CUDA_TRY(cudaMemcpyAsync(ws->sc_host, ws->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, ctx->stream));
        STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        if (ws->sc_host->done) return STAG_OK;
    }
}

int free_graph_pair(cudaGraph_t& g, cudaGraphExec_t& e)
{
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
    e = nullptr;
    g = nullptr;
    return STAG_OK;
}

// Scalar record for timing the update kernel alone: never done (tol2 < 0,
// maxiter at its largest), a fixed alpha.
__global__ void k_update_time_init(CgScalars* sc)
{
    CgScalars s = {};
    s.rr = 1.0;
    s.alpha = 1e-3;
    s.tol2 = -1.0;
    s.maxiter = 0x7fffffff;
    *sc = s;
}

// Choose the plan's launch shapes (once per context and plan, before its
// graph is built): each candidate runs on the workspace vectors with a scalar
// record that never reports convergence; the solve then starts from scratch.
template <class Plan>
static int tune_cg_plan(stag_ctx ctx, const typename Plan::LF& U)
{
    Workspace* ws = ctx->ws;
    if (ws->cg_tuned[Plan::slot]) return STAG_OK;
    STAG_TRY(Plan::prepare(ctx));
    CgScalars* tsc = ws->sc + 61;   // spare records: 61 CG tuning, 62 mixed tuning, 63 the action
    k_update_time_init<<<1, 1, 0, ctx->stream>>>(tsc);
    STAG_CUDA_TRY(cudaGetLastError());
    CgShape sh;
    const int prec = Plan::prec;
    char kname[64];
    snprintf(kname, sizeof(kname), "%s_hop%s", Plan::name,
             ws->df_dir == 1 && Plan::prec == STAG_F64X ? "_dir" : "");
    STAG_TRY(tune_choice(ctx, tune_key(ctx, kname, prec, 18, 1), HOP_CANDS, &sh.hop,
                         [&](int c) { return Plan::launch_hop(ctx, U, c, ctx->stream, tsc); }));
    snprintf(kname, sizeof(kname), "%s_update", Plan::name);
    STAG_TRY(tune_choice(ctx, tune_key(ctx, kname, prec, 18, 1), VEC_CANDS, &sh.upd,
                         [&](int c) { return Plan::launch_update(ctx, c, ctx->stream, tsc, 0, 0); }));
    if (Plan::has_p(ctx)) {
        snprintf(kname, sizeof(kname), "%s_p", Plan::name);
        STAG_TRY(tune_choice(ctx, tune_key(ctx, kname, prec, 18, 1), VEC_CANDS, &sh.pk,
                             [&](int c) { return Plan::launch_p(ctx, c, ctx->stream, tsc); }));
    }
    ws->cg_shape[Plan::slot] = sh;
    ws->cg_tuned[Plan::slot] = true;
    return STAG_OK;
}

template <class Plan>
static int cg_solve_plan(stag_ctx ctx, const typename Plan::LF& U, double2* x_out, const double2* b_in, double mass,
                         double sigma, const stag_solver_params& prm, stag_solver_stats* st,
                         std::chrono::steady_clock::time_point t0)
{
    Workspace* ws = ctx->ws;
    const Geom g = ctx->g;
    const int maxiter = prm.maxiter > 0 ? prm.maxiter : 100000;
    STAG_TRY(tune_cg_plan<Plan>(ctx, U));
    STAG_TRY(Plan::start(ctx, b_in, mass, sigma, prm.tol, maxiter));
    int restarts = 0;
    CgScalars* hs = ws->sc_host;
    double prev_true = INFINITY;
    for (;;) {
        STAG_TRY(run_cg_loop<Plan>(ctx, U, prm));
        STAG_TRY(Plan::true_residual(ctx, U));
        STAG_CUDA_TRY(cudaMemcpyAsync(hs, ws->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, ctx->stream));
        STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        if (hs->rr0 == 0.0 || hs->rr_true <= hs->tol2 || hs->status == STAG_BREAKDOWN || hs->iter >= hs->maxiter)
            break;
        // A restart that did not halve the true residual norm means the
        // iteration sits at its rounding floor: stop (NOT_CONVERGED).
        if (!(hs->rr_true < 0.25 * prev_true) || restarts >= MAX_RESTARTS) break;
        prev_true = hs->rr_true;
        ++restarts;
        // p = r (16-byte elements: double or double-float vectors alike)
        k_cg_restart_f64<BLAS_BS><<<nblk(3 * g.Vh, BLAS_BS), BLAS_BS, 0, ctx->stream>>>(g.Vh, ws->r, ws->p, ws->sc);
        STAG_CUDA_TRY(cudaGetLastError());
    }
    STAG_TRY(Plan::finish(ctx, x_out));
    STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    int status = STAG_OK;
    if (hs->status == STAG_BREAKDOWN) status = STAG_BREAKDOWN;
    else if (hs->rr0 > 0.0 && hs->rr_true > hs->tol2) status = STAG_NOT_CONVERGED;
    if (st) {
        st->status = status;
        st->iters = hs->iter;
        st->restarts = restarts;
        st->reliable_updates = 0;
        st->true_rel_residual = hs->rr0 > 0 ? sqrt(hs->rr_true / hs->rr0) : 0.0;
        st->iter_rel_residual = hs->rr0 > 0 ? sqrt(hs->rr / hs->rr0) : 0.0;
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}

int cg_solve_f64(stag_ctx ctx, double2* x_out, const double2* b_in, double mass, double sigma,
                 const stag_solver_params& prm, stag_solver_stats* st)
{
    const auto t0 = std::chrono::steady_clock::now();
    STAG_TRY(ensure_cg_f64(ctx));
    int arith = STAG_F64;
    STAG_TRY(resolve_f64_arith(ctx, prm.f64_arith, &arith));
    if (prm.temporal_gauge) {
        // M x = b as M' x' = g b, x = g^dagger x' (same residual norm: g is unitary)
        const double2* G = nullptr;
        const void* lk = nullptr;
        double2* gb = nullptr;
        STAG_TRY(ensure_links_tg(ctx, arith, 18, &lk));
        STAG_TRY(ensure_tg_gauge(ctx, &G));
        STAG_TRY(ensure_tg_tmp(ctx, 1, &gb));
        STAG_TRY(tg_apply(ctx, G, b_in, gb, 1, 0));
        int rc;
        if (arith == STAG_F64X) {
            const LinkFieldDF<18> U{(const float4*)lk, ctx->g.Vh, 1};
            rc = cg_solve_plan<DFPlanTG>(ctx, U, x_out, gb, mass, sigma, prm, st, t0);
        } else {
            const LF64 U{(const double2*)lk, ctx->g.Vh, 1};
            rc = cg_solve_plan<F64PlanTG>(ctx, U, x_out, gb, mass, sigma, prm, st, t0);
        }
        if (rc < 0) return rc;
        STAG_TRY(tg_apply(ctx, G, x_out, x_out, 1, 1));
        STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        return rc;
    }
    if (arith == STAG_F64X) {
        const void* lk = nullptr;
        STAG_TRY(ensure_links(ctx, STAG_F64X, 18, &lk));
        const LinkFieldDF<18> U{(const float4*)lk, ctx->g.Vh};
        return cg_solve_plan<DFPlan>(ctx, U, x_out, b_in, mass, sigma, prm, st, t0);
    }
    // IEEE double: requested, or links outside the double-float range
    const void* lk = nullptr;
    STAG_TRY(ensure_links(ctx, STAG_F64, 18, &lk));
    const LF64 U{(const double2*)lk, ctx->g.Vh};
    return cg_solve_plan<F64Plan>(ctx, U, x_out, b_in, mass, sigma, prm, st, t0);
}

void free_workspace(stag_ctx ctx)
{
    Workspace* ws = ctx->ws;
    if (!ws) return;
    for (int i = 0; i < 4; ++i) free_graph_pair(ws->f64_graph[i], ws->f64_exec[i]);
    free_mixed(ws);
    free_batches(ws);
    for (auto& m : ws->ms) m.release();
    double2* bufs[] = {ws->x, ws->r, ws->p, ws->Ap, ws->b, ws->t};
    for (auto b : bufs)
        if (b) cudaFree(b);
    if (ws->sc) cudaFree(ws->sc);
    if (ws->sc_host) cudaFreeHost(ws->sc_host);
    delete ws;
    ctx->ws = nullptr;
}

int check_ctx(stag_ctx ctx);
int check_half_field(const void* p, const char* what);

}  // namespace stag

using namespace stag;

extern "C" {

int stag_cg_update_time(stag_ctx ctx, int f64_arith, int nrep, double* ms_per_launch)
{
    STAG_TRY(check_ctx(ctx));
    if (nrep < 1 || !ms_per_launch || (f64_arith != STAG_F64 && f64_arith != STAG_F64X)) {
        set_error("nrep must be >= 1, ms_per_launch non-NULL, f64_arith STAG_F64 or STAG_F64X");
        return STAG_EINVAL;
    }
    STAG_TRY(ensure_cg_f64(ctx));
    Workspace* ws = ctx->ws;
    const int Vh = ctx->g.Vh, gb = nblk(Vh, BLAS_BS);
    const size_t bytes = (size_t)3 * Vh * sizeof(double2);
    for (double2* v : {ws->x, ws->r, ws->p, ws->Ap}) STAG_CUDA_TRY(cudaMemsetAsync(v, 0, bytes, ctx->stream));
    k_update_time_init<<<1, 1, 0, ctx->stream>>>(ws->sc);
    auto launch = [&]() {
        if (f64_arith == STAG_F64X)
            k_dfcg_update<BLAS_BS, 1><<<gb, BLAS_BS, 0, ctx->stream>>>(Vh, DFPlan::v(ws->x), DFPlan::v(ws->r),
                                                                   DFPlan::v(ws->p), DFPlan::v(ws->Ap), ws->sc,
                                                                   ctx->partials, ctx->counters,
                                                                   grid_sum_of(ctx), 0, 0);
        else
            k_cg_update<SpinorF64, BLAS_BS, 1><<<gb, BLAS_BS, 0, ctx->stream>>>(
                Vh, SpinorF64{ws->x}, SpinorF64{ws->r}, SpinorF64{ws->p}, SpinorF64{ws->Ap}, ws->sc, ctx->partials,
                ctx->counters, grid_sum_of(ctx), 0, 0);
    };
    for (int k = 0; k < 2; ++k) launch();
    cudaEvent_t e0, e1;
    STAG_CUDA_TRY(cudaEventCreate(&e0));
    STAG_CUDA_TRY(cudaEventCreate(&e1));
    cudaEventRecord(e0, ctx->stream);
    for (int k = 0; k < nrep; ++k) launch();
    cudaEventRecord(e1, ctx->stream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    STAG_CUDA_TRY(e);
    *ms_per_launch = (double)ms / nrep;
    return STAG_OK;
}

void stag_solver_params_default(stag_solver_params* p)
{
    if (!p) return;
    p->tol = 1e-10;
    p->maxiter = 100000;
    p->use_graph = 1;
    p->check_every = 25;
    p->delta = DEFAULT_RELIABLE_DELTA;
    p->inner_prec = STAG_F32;
    p->inner_recon = STAG_RECON_12;
    p->rhs_block = 0;
    p->f64_arith = STAG_F64X;
    p->temporal_gauge = 0;
}

int stag_cg_solve(stag_ctx ctx, double* x_even, const double* b_even, double mass, const stag_solver_params* params,
                  stag_solver_stats* stats)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(x_even, "x_even"));
    STAG_TRY(check_half_field(b_even, "b_even"));
    stag_solver_params prm;
    stag_solver_params_default(&prm);
    if (params) prm = *params;
    if (!(prm.tol > 0.0)) {
        set_error("tol must be positive");
        return STAG_EINVAL;
    }
    if (!ctx->have_gauge) {
        set_error("no gauge field uploaded");
        return STAG_ENOGAUGE;
    }
    return cg_solve_f64(ctx, (double2*)x_even, (const double2*)b_even, mass, 0.0, prm, stats);
}

int stag_cg_solve_shifted(stag_ctx ctx, double* x_even, const double* b_even, double mass, double sigma,
                          const stag_solver_params* params, stag_solver_stats* stats)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(x_even, "x_even"));
    STAG_TRY(check_half_field(b_even, "b_even"));
    stag_solver_params prm;
    stag_solver_params_default(&prm);
    if (params) prm = *params;
    if (!(prm.tol > 0.0) || !(sigma >= 0.0) || !isfinite(sigma)) {
        set_error("tol must be positive and sigma finite and >= 0");
        return STAG_EINVAL;
    }
    if (!ctx->have_gauge) {
        set_error("no gauge field uploaded");
        return STAG_ENOGAUGE;
    }
    return cg_solve_f64(ctx, (double2*)x_even, (const double2*)b_even, mass, sigma, prm, stats);
}

}  // extern "C"
