// cg.cu -- double-precision conjugate gradient on M = m^2 - D_eo D_oe
// (the inversion the paper benchmarks, Sec. 1 and Sec. 4.2), with the
// iteration running inside one CUDA graph whose while-loop condition is
// cleared on the device, so no host round trip happens per iteration.
#include <chrono>
#include <new>

#include "cg_kernels.cuh"
#include "df64.cuh"
#include "workspace.h"

namespace stag {

constexpr int HOP_BS = 128;
constexpr int BLAS_BS = 256;
constexpr int MAX_RESTARTS = 100;

typedef LinkField<double2, 18> LF64;

static inline int nblk(int n, int bs) { return (n + bs - 1) / bs; }

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

// Restart from the true residual now held in r: p = r, rr = rr_true.
template <int BS>
__global__ void __launch_bounds__(BS) k_cg_restart_f64(int Vh, const double2* r, double2* p, CgScalars* sc)
{
    const long long i = (long long)blockIdx.x * BS + threadIdx.x;
    if (i < 3LL * Vh) p[i] = r[i];
    if (i == 0) {
        sc->rr = sc->rr_true;
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

// One double-precision CG plan per operator arithmetic: LF / SD are the link
// field and the spinor view the operator passes use (IEEE double: LinkField +
// SpinorF64; double-float: LinkFieldDF + SpinorF64asDF over the same double
// vectors).  The BLAS kernels always work on the double vectors.
template <class LF, class SD>
struct F64Plan {
    // one CG iteration (four kernels) on stream s
    static int enqueue_iter(stag_ctx ctx, const LF& U, cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond)
    {
        Workspace* ws = ctx->ws;
        const Geom g = ctx->g;
        const int gh = nblk(g.Vh, HOP_BS), gb = nblk(g.Vh, BLAS_BS);
        SpinorF64 p{ws->p}, Ap{ws->Ap}, x{ws->x}, r{ws->r};
        k_hop_guarded<LF, SD, HOP_BS><<<gh, HOP_BS, 0, s>>>(g, 1, U, SD{ws->p}, SD{ws->t}, ws->sc);
        k_Mp_dot<LF, SD, SpinorF64, HOP_BS><<<gh, HOP_BS, 0, s>>>(g, U, SD{ws->t}, p, Ap, ws->sc, ctx->partials,
                                                                  ctx->counters);
        k_cg_update<SpinorF64, BLAS_BS><<<gb, BLAS_BS, 0, s>>>(g.Vh, x, r, p, Ap, ws->sc, ctx->partials,
                                                              ctx->counters, cond, use_cond);
        k_cg_p<SpinorF64, BLAS_BS><<<gb, BLAS_BS, 0, s>>>(g.Vh, r, p, ws->sc);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }

    // the graph  while (cond) { one CG iteration }, built once per context
    static int ensure_graph(stag_ctx ctx, const LF& U, int slot)
    {
        Workspace* ws = ctx->ws;
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
        int rc = enqueue_iter(ctx, U, ctx->cap_stream, cond, 1);
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

    // run the iteration until the device says done: one graph launch, or a
    // host loop that reads the done flag every check_every iterations
    static int run_loop(stag_ctx ctx, const LF& U, const stag_solver_params& prm, int slot)
    {
        Workspace* ws = ctx->ws;
        if (prm.use_graph) {
            STAG_TRY(ensure_graph(ctx, U, slot));
            STAG_CUDA_TRY(cudaGraphLaunch(ws->f64_exec[slot], ctx->stream));
            return STAG_OK;
        }
        const int every = prm.check_every > 0 ? prm.check_every : 25;
        for (;;) {
            for (int k = 0; k < every; ++k) STAG_TRY(enqueue_iter(ctx, U, ctx->stream, 0, 0));
            STAG_CUDA_TRY(cudaMemcpyAsync(ws->sc_host, ws->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, ctx->stream));
            STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
            if (ws->sc_host->done) return STAG_OK;
        }
    }

    // r = b - M x in double precision (operator passes in this plan's arithmetic)
    static int true_residual(stag_ctx ctx, const LF& U)
    {
        Workspace* ws = ctx->ws;
        const Geom g = ctx->g;
        k_hop<LF, SD, HOP_BS><<<nblk(g.Vh, HOP_BS), HOP_BS, 0, ctx->stream>>>(g, 1, U, SD{ws->x}, SD{ws->t}, nullptr,
                                                                             0);
        k_true_resid_f64<LF, SD, HOP_BS><<<nblk(g.Vh, HOP_BS), HOP_BS, 0, ctx->stream>>>(
            g, U, ws->t, ws->x, ws->b, ws->r, ws->sc, ctx->partials, ctx->counters, 0);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
};

int free_graph_pair(cudaGraph_t& g, cudaGraphExec_t& e)
{
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
    e = nullptr;
    g = nullptr;
    return STAG_OK;
}

template <class LF, class SD>
static int cg_solve_plan(stag_ctx ctx, const LF& U, int slot, double2* x_out, const double2* b_in, double mass,
                         double sigma, const stag_solver_params& prm, stag_solver_stats* st,
                         std::chrono::steady_clock::time_point t0)
{
    typedef F64Plan<LF, SD> Plan;
    Workspace* ws = ctx->ws;
    const Geom g = ctx->g;
    const size_t bytes = (size_t)3 * g.Vh * sizeof(double2);
    const int maxiter = prm.maxiter > 0 ? prm.maxiter : 100000;
    STAG_CUDA_TRY(cudaMemcpyAsync(ws->b, b_in, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    k_cg_start_f64<BLAS_BS><<<nblk(g.Vh, BLAS_BS), BLAS_BS, 0, ctx->stream>>>(
        g.Vh, ws->b, ws->x, ws->r, ws->p, ws->sc, prm.tol, maxiter, mass * mass, sigma, ctx->partials, ctx->counters);
    STAG_CUDA_TRY(cudaGetLastError());
    int restarts = 0;
    CgScalars* hs = ws->sc_host;
    double prev_true = INFINITY;
    for (;;) {
        STAG_TRY(Plan::run_loop(ctx, U, prm, slot));
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
        k_cg_restart_f64<BLAS_BS><<<nblk(3 * g.Vh, BLAS_BS), BLAS_BS, 0, ctx->stream>>>(g.Vh, ws->r, ws->p, ws->sc);
        STAG_CUDA_TRY(cudaGetLastError());
    }
    STAG_CUDA_TRY(cudaMemcpyAsync(x_out, ws->x, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
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
    if (prm.f64_arith == STAG_F64X) {
        const void* lk = nullptr;
        STAG_TRY(ensure_links(ctx, STAG_F64X, 18, &lk));
        const LinkFieldDF<18> U{(const float4*)lk, ctx->g.Vh};
        return cg_solve_plan<LinkFieldDF<18>, SpinorF64asDF>(ctx, U, 1, x_out, b_in, mass, sigma, prm, st, t0);
    }
    if (prm.f64_arith != STAG_F64) {
        set_error("f64_arith must be STAG_F64 or STAG_F64X");
        return STAG_EINVAL;
    }
    const void* lk = nullptr;
    STAG_TRY(ensure_links(ctx, STAG_F64, 18, &lk));
    const LF64 U{(const double2*)lk, ctx->g.Vh};
    return cg_solve_plan<LF64, SpinorF64>(ctx, U, 0, x_out, b_in, mass, sigma, prm, st, t0);
}

void free_workspace(stag_ctx ctx)
{
    Workspace* ws = ctx->ws;
    if (!ws) return;
    for (int i = 0; i < 2; ++i) free_graph_pair(ws->f64_graph[i], ws->f64_exec[i]);
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

void stag_solver_params_default(stag_solver_params* p)
{
    if (!p) return;
    p->tol = 1e-10;
    p->maxiter = 100000;
    p->use_graph = 1;
    p->check_every = 25;
    p->delta = 0.1;
    p->inner_prec = STAG_F32;
    p->inner_recon = STAG_RECON_12;
    p->rhs_block = 0;
    p->f64_arith = STAG_F64X;
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
