// mixed.cu -- mixed-precision CG with reliable updates on M = m^2 - D_eo D_oe.
//
// The inner iteration runs in float or half storage (float arithmetic, 18- or
// 12-real links); the solution is accumulated and the true residual recomputed
// in double precision whenever the low-precision residual has fallen by a
// factor delta below its maximum since the last such "reliable update", and
// whenever the low-precision iteration believes it has converged.  After an
// update the low-precision residual is replaced by the double one and the
// search direction is kept, with beta = |r_true|^2 / |r_prev|^2.  The solve
// ends only on a double-precision true residual below tol.  (The paper only
// cites mixed-precision GPU solvers, bibliography entry of the QUDA
// collaboration; this is the standard reliable-update scheme.)
//
// Graph:  while (W) { hop; Mp_dot; update; if (I) { accum_x; hop64; resid64; finish } p }
#include <chrono>
#include <new>
#include <type_traits>

#include "cg_kernels.cuh"
#include "df64.cuh"
#include "graph.h"
#include "tune.h"
#include "workspace.h"

namespace stag {

constexpr int MHOP_BS = 128;
constexpr int MBLAS_BS = 256;

static inline int nblk_m(int n, int bs) { return (n + bs - 1) / bs; }

// x_hi = 0, r_hi = b, r = lo(b), p = r, xlo = 0; scalars from |b|^2.
template <class S, class SX, int BS>
__global__ void __launch_bounds__(BS) k_mixed_start(int Vh, const double2* b, double2* x_hi, double2* r_hi, S r,
                                                    S p, SX xlo, CgScalars* sc, double tol, int maxiter, double m2,
                                                    double delta, double* part, unsigned* cnt)
{
    __shared__ double red[BS / 32];
    __shared__ bool last;
    typedef typename S::real real;
    const int h = blockIdx.x * BS + threadIdx.x;
    double d = 0.0;
    if (h < Vh) {
        Vec3<real> v;
        Vec3<typename SX::real> z;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 bv = b[(size_t)h * 3 + c];
            x_hi[(size_t)h * 3 + c] = make_double2(0.0, 0.0);
            r_hi[(size_t)h * 3 + c] = bv;
            d = fma(bv.x, bv.x, d);
            d = fma(bv.y, bv.y, d);
            v.c[c].re = (real)bv.x;
            v.c[c].im = (real)bv.y;
            z.c[c].re = z.c[c].im = 0;
        }
        r.store(h, v);
        p.store(h, v);
        xlo.store(h, z);
    }
    const double bs = block_sum<BS>(d, red);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
    if (!arrive_last(cnt, &last)) return;
    const double bb = sum_partials<BS>(part, gridDim.x, red);
    if (threadIdx.x == 0) {
        *cnt = 0;
        CgScalars s = {};
        s.rr = s.rr0 = s.rr_true = s.rmax2 = bb;
        s.tol2 = tol * tol * bb;
        s.delta2 = delta * delta;
        s.maxiter = maxiter;
        s.m2 = m2;
        s.done = (bb == 0.0) ? 1 : 0;
        *sc = s;
    }
}

// xlo += alpha p, r -= alpha Ap, rr' = |r|^2 over SPT sites per thread
// (partials in 128-site chunks: every launch shape gives the same bits);
// decide whether a reliable update is due.
template <class S, class SX, int BS, int SPT>
__global__ void __launch_bounds__(BS) k_mixed_update(int Vh, SX x, S r, S p, S Ap, CgScalars* sc, double* part,
                                                     unsigned* cnt, GridSum gs, cudaGraphConditionalHandle wh,
                                                     cudaGraphConditionalHandle ih, int use_cond)
{
    __shared__ double red[BS / 32 * SPT];
    if (sc->done) {
        // iterations launched after convergence (host-driven loop) must not
        // repeat the final reliable update
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            sc->reliable = 0;
            if (use_cond) {
                cudaGraphSetConditional(ih, 0);
                cudaGraphSetConditional(wh, 0);
            }
        }
        return;
    }
    typedef typename S::real real;
    const real alpha = (real)sc->alpha;
    real d[SPT];
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int h = (blockIdx.x * SPT + j) * BS + threadIdx.x;
        d[j] = real(0);
        if (h < Vh) {
            Vec3<typename SX::real> xv = x.load_rw(h);
            Vec3<real> rv = r.load_rw(h);
            const Vec3<real> pv = p.load(h), av = Ap.load(h);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xv.c[c].re = fma(alpha, pv.c[c].re, xv.c[c].re);
                xv.c[c].im = fma(alpha, pv.c[c].im, xv.c[c].im);
                rv.c[c].re = fma(-alpha, av.c[c].re, rv.c[c].re);
                rv.c[c].im = fma(-alpha, av.c[c].im, rv.c[c].im);
            }
            x.store(h, xv);
            r.store(h, rv);
            d[j] = site_dot(rv, rv);
        }
    }
    const int nch = (Vh + RCHUNK - 1) / RCHUNK;
    chunk_partials<BS, SPT>(d, part, nch, red);
    constexpr int NCH = BS * SPT / RCHUNK;
    const int u0 = blockIdx.x * NCH;
    double rr_new;
    if (!grid_sum_finish<BS>(part, nch, u0, min(NCH, nch - u0), gs, cnt, red, &rr_new)) return;
    if (threadIdx.x == 0) {
        sc->rr_prev = sc->rr;
        sc->beta = rr_new / sc->rr;
        sc->rr = rr_new;
        sc->iter += 1;
        if (rr_new > sc->rmax2) sc->rmax2 = rr_new;
        const int rel = !isfinite(rr_new) || rr_new < sc->delta2 * sc->rmax2 || rr_new <= sc->tol2 ||
                        sc->iter >= sc->maxiter;
        sc->reliable = rel;
        if (use_cond) {
            cudaGraphSetConditional(ih, rel ? 1 : 0);
            cudaGraphSetConditional(wh, 1);
        }
    }
}

// x_hi += xlo (double), xlo = 0.
// x_df (double-float arithmetic only, else NULL) keeps x_hi split into
// double-float pairs, the storage the reliable update's operator reads.
template <class SX, int BS>
__global__ void __launch_bounds__(BS) k_accum_x(int Vh, double2* x_hi, SX xlo, const CgScalars* sc, int guard,
                                                float4* x_df)
{
    if (guard && !sc->reliable) return;
    const int h = blockIdx.x * BS + threadIdx.x;
    if (h >= Vh) return;
    const Vec3<typename SX::real> v = xlo.load_rw(h);
    Vec3<typename SX::real> z;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double2 xv = x_hi[(size_t)h * 3 + c];
        xv.x += (double)v.c[c].re;
        xv.y += (double)v.c[c].im;
        x_hi[(size_t)h * 3 + c] = xv;
        if (x_df) {
            const DF re = split_double(xv.x), im = split_double(xv.y);
            x_df[(size_t)h * 3 + c] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
        z.c[c].re = z.c[c].im = 0;
    }
    xlo.store(h, z);
}

// r = lo(r_hi); restart the low-precision recurrence from the true residual.
template <class S, int BS>
__global__ void __launch_bounds__(BS) k_reliable_finish(int Vh, const double2* r_hi, S r, CgScalars* sc,
                                                        cudaGraphConditionalHandle wh, int use_cond, int guard)
{
    if (guard && !sc->reliable) return;
    typedef typename S::real real;
    const int h = blockIdx.x * BS + threadIdx.x;
    if (h < Vh) {
        Vec3<real> v;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 q = r_hi[(size_t)h * 3 + c];
            v.c[c].re = (real)q.x;
            v.c[c].im = (real)q.y;
        }
        r.store(h, v);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double rt = sc->rr_true;
        sc->n_reliable += 1;
        if (!isfinite(rt)) {
            sc->status = STAG_BREAKDOWN;
            sc->done = 1;
        } else if (rt <= sc->tol2) {
            sc->done = 1;
        } else if (sc->iter >= sc->maxiter) {
            sc->status = STAG_NOT_CONVERGED;
            sc->done = 1;
        }
        sc->beta = rt / sc->rr_prev;
        sc->rr = rt;
        sc->rmax2 = rt;
        if (use_cond) cudaGraphSetConditional(wh, sc->done ? 0 : 1);
    }
}

// Scalar record for timing the inner kernels: never done, never due a
// reliable update, a fixed alpha and beta.
__global__ void k_mixed_time_init(CgScalars* sc)
{
    CgScalars s = {};
    s.rr = s.rmax2 = 1.0;
    s.alpha = 1e-3;
    s.beta = 0.5;
    s.tol2 = -1.0;
    s.delta2 = 0.0;
    s.maxiter = 0x7fffffff;
    *sc = s;
}

// ------------------------------------------------------------- driver

#define STAG_VEC_SWITCH(cfg, CALL)                                             \
    switch (cfg) {                                                             \
    case vcfg(256, 1): { constexpr int BS = 256, SPT = 1; CALL; } break;       \
    case vcfg(128, 1): { constexpr int BS = 128, SPT = 1; CALL; } break;       \
    case vcfg(256, 2): { constexpr int BS = 256, SPT = 2; CALL; } break;       \
    case vcfg(128, 2): { constexpr int BS = 128, SPT = 2; CALL; } break;       \
    default: set_error("bad vector kernel shape %d", cfg); return STAG_EINVAL; \
    }
#define STAG_HOP_SWITCH(bs, CALL)                                            \
    switch (bs) {                                                            \
    case 128: { constexpr int BS = 128; CALL; } break;                       \
    case 64: { constexpr int BS = 64; CALL; } break;                         \
    case 256: { constexpr int BS = 256; CALL; } break;                       \
    default: set_error("bad hop block size %d", bs); return STAG_EINVAL;     \
    }

template <class S, class SX, class LF, class LF64T, class SD64>
struct MixedPlan {
    // the inner iteration's kernels in the tuned launch shapes (m.shape)
    static int launch_hop(stag_ctx ctx, MixedSlot& m, const LF& U, int bs, cudaStream_t s, const CgScalars* sc)
    {
        const Geom g = ctx->g;
        S t = m.template spinor<S>(m.t), p = m.template spinor<S>(m.p);
        if constexpr (LinkStage<LF>::value) {
            switch (bs >> HOP_STAGE_SHIFT) {
            case STAGE_LINKS:
                STAG_HOP_SWITCH(bs & HOP_BS_MASK, (k_hop_guarded<LF, S, BS, STAGE_LINKS>
                                                   <<<nblk_m(g.Vh, BS), BS, 0, s>>>(g, 1, U, p, t, sc)));
                return STAG_OK;
            case STAGE_SPINORS:
                STAG_HOP_SWITCH(bs & HOP_BS_MASK, (k_hop_guarded<LF, S, BS, STAGE_SPINORS>
                                                   <<<nblk_m(g.Vh, BS), BS, 0, s>>>(g, 1, U, p, t, sc)));
                return STAG_OK;
            case STAGE_LINKS | STAGE_SPINORS:
                STAG_HOP_SWITCH(bs & HOP_BS_MASK, (k_hop_guarded<LF, S, BS, STAGE_LINKS | STAGE_SPINORS>
                                                   <<<nblk_m(g.Vh, BS), BS, 0, s>>>(g, 1, U, p, t, sc)));
                return STAG_OK;
            default: break;
            }
        }
        STAG_HOP_SWITCH(bs, (k_hop_guarded<LF, S, BS><<<nblk_m(g.Vh, BS), BS, 0, s>>>(g, 1, U, p, t, sc)));
        return STAG_OK;
    }
    static int launch_mpdot(stag_ctx ctx, MixedSlot& m, const LF& U, int stage, cudaStream_t s, CgScalars* sc)
    {
        const Geom g = ctx->g;
        S t = m.template spinor<S>(m.t), p = m.template spinor<S>(m.p), Ap = m.template spinor<S>(m.Ap);
        const int nb = nblk_m(g.Vh, MHOP_BS);
        const GridSum gs = grid_sum_of(ctx);
        if constexpr (LinkStage<LF>::value) {
            switch (stage) {
            case STAGE_LINKS:
                k_Mp_dot<LF, S, S, MHOP_BS, STAGE_LINKS><<<nb, MHOP_BS, 0, s>>>(g, U, t, p, Ap, sc, ctx->partials,
                                                                             ctx->counters, gs);
                return STAG_OK;
            case STAGE_SPINORS:
                k_Mp_dot<LF, S, S, MHOP_BS, STAGE_SPINORS><<<nb, MHOP_BS, 0, s>>>(g, U, t, p, Ap, sc, ctx->partials,
                                                                               ctx->counters, gs);
                return STAG_OK;
            case STAGE_LINKS | STAGE_SPINORS:
                k_Mp_dot<LF, S, S, MHOP_BS, STAGE_LINKS | STAGE_SPINORS><<<nb, MHOP_BS, 0, s>>>(
                    g, U, t, p, Ap, sc, ctx->partials, ctx->counters, gs);
                return STAG_OK;
            default: break;
            }
        }
        k_Mp_dot<LF, S, S, MHOP_BS><<<nb, MHOP_BS, 0, s>>>(g, U, t, p, Ap, sc, ctx->partials, ctx->counters, gs);
        return STAG_OK;
    }
    static int launch_update(stag_ctx ctx, MixedSlot& m, int cfg, cudaStream_t s, CgScalars* sc, LoopGraph* lg,
                             int use_cond)
    {
        const Geom g = ctx->g;
        S p = m.template spinor<S>(m.p), Ap = m.template spinor<S>(m.Ap), r = m.template spinor<S>(m.r);
        SX x = m.template spinor<SX>(m.xlo);
        STAG_VEC_SWITCH(cfg, (k_mixed_update<S, SX, BS, SPT><<<nblk_m(g.Vh, BS * SPT), BS, 0, s>>>(
                                 g.Vh, x, r, p, Ap, sc, ctx->partials, ctx->counters, grid_sum_of(ctx),
                                 lg ? lg->w : 0, lg ? lg->i : 0, use_cond)));
        return STAG_OK;
    }
    static int launch_p(stag_ctx ctx, MixedSlot& m, int cfg, cudaStream_t s, const CgScalars* sc)
    {
        S r = m.template spinor<S>(m.r), p = m.template spinor<S>(m.p);
        STAG_VEC_SWITCH(cfg, (k_cg_p<S, BS, SPT><<<nblk_m(ctx->g.Vh, BS * SPT), BS, 0, s>>>(ctx->g.Vh, r, p, sc)));
        return STAG_OK;
    }
    // launch shapes of the inner kernels, chosen once per slot (timed on the
    // slot's vectors with a scalar record that never converges)
    static int tune(stag_ctx ctx, MixedSlot& m, const LF& U, int prec, int recon)
    {
        const int tg = U.tg;
        if (m.tuned[tg]) return STAG_OK;
        CgScalars* tsc = ctx->ws->sc + 62;
        k_mixed_time_init<<<1, 1, 0, ctx->stream>>>(tsc);
        STAG_CUDA_TRY(cudaGetLastError());
        CgShape sh;
        // block sizes, and for half 12-real storage the same with the links
        // and / or the neighbour spinors staged in shared memory (24 and
        // 16 KB a block of 128 threads)
        std::vector<int> hc = {128, 64, 256};
        if (LinkStage<LF>::value) {
            for (int st : {STAGE_LINKS, STAGE_SPINORS, STAGE_LINKS | STAGE_SPINORS}) {
                hc.push_back(128 | (st << HOP_STAGE_SHIFT));
                hc.push_back(64 | (st << HOP_STAGE_SHIFT));
            }
        }
        STAG_TRY(tune_choice(ctx, tune_key(ctx, tg ? "mixed_hop_tg" : "mixed_hop", prec, recon, 1), hc, &sh.hop,
                             [&](int c) { return launch_hop(ctx, m, U, c, ctx->stream, tsc); }));
        if (LinkStage<LF>::value) {
            // Mp_dot writes the record (on vectors that are not yet a solve's,
            // pAp may read as a breakdown): it is reset before every launch
            // and after the last
            STAG_TRY(tune_choice(ctx, tune_key(ctx, tg ? "mixed_mpdot_stage_tg" : "mixed_mpdot_stage", prec, recon, 1),
                                 {0, STAGE_LINKS, STAGE_SPINORS, STAGE_LINKS | STAGE_SPINORS}, &sh.mpdot_stage,
                                 [&](int c) {
                                     k_mixed_time_init<<<1, 1, 0, ctx->stream>>>(tsc);
                                     return launch_mpdot(ctx, m, U, c, ctx->stream, tsc);
                                 }));
            k_mixed_time_init<<<1, 1, 0, ctx->stream>>>(tsc);
            STAG_CUDA_TRY(cudaGetLastError());
        }
        const std::vector<int> vc = {vcfg(256, 1), vcfg(128, 1), vcfg(256, 2), vcfg(128, 2)};
        STAG_TRY(tune_choice(ctx, tune_key(ctx, "mixed_update", prec, recon, 1), vc, &sh.upd,
                             [&](int c) { return launch_update(ctx, m, c, ctx->stream, tsc, nullptr, 0); }));
        STAG_TRY(tune_choice(ctx, tune_key(ctx, "mixed_p", prec, recon, 1), vc, &sh.pk,
                             [&](int c) { return launch_p(ctx, m, c, ctx->stream, tsc); }));
        m.shape[tg] = sh;
        m.tuned[tg] = true;
        return STAG_OK;
    }
    static int enqueue_main(stag_ctx ctx, MixedSlot& m, const LF& U, cudaStream_t s, LoopGraph* lg, int use_cond)
    {
        const Geom g = ctx->g;
        S t = m.template spinor<S>(m.t), p = m.template spinor<S>(m.p), Ap = m.template spinor<S>(m.Ap);
        const CgShape& sh = m.shape[U.tg];
        STAG_TRY(launch_hop(ctx, m, U, sh.hop, s, m.sc));
        STAG_TRY(launch_mpdot(ctx, m, U, sh.mpdot_stage, s, m.sc));
        STAG_TRY(launch_update(ctx, m, sh.upd, s, m.sc, lg, use_cond));
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    static int enqueue_reliable(stag_ctx ctx, MixedSlot& m, const LF64T& U64, cudaStream_t s, LoopGraph* lg,
                                int use_cond, int guard)
    {
        const Geom g = ctx->g;
        Workspace* ws = ctx->ws;
        SX x = m.template spinor<SX>(m.xlo);
        S r = m.template spinor<S>(m.r);
        // double-float arithmetic reads x as double-float pairs kept in the
        // workspace's p (unused by this solver), and t in the same storage
        constexpr bool DFX = std::is_same<SD64, SpinorDF>::value;
        typedef typename std::conditional<DFX, float4, double2>::type VT;
        const SD64 xin{(VT*)(DFX ? ws->p : ws->x)}, tv{(VT*)ws->t};
        k_accum_x<SX, MBLAS_BS><<<nblk_m(g.Vh, MBLAS_BS), MBLAS_BS, 0, s>>>(g.Vh, ws->x, x, m.sc, guard,
                                                                           DFX ? (float4*)ws->p : nullptr);
        k_hop<LF64T, SD64, MHOP_BS><<<nblk_m(g.Vh, MHOP_BS), MHOP_BS, 0, s>>>(g, 1, U64, xin, tv, m.sc, guard);
        k_true_resid_f64<LF64T, SD64, MHOP_BS><<<nblk_m(g.Vh, MHOP_BS), MHOP_BS, 0, s>>>(
            g, U64, tv, ws->x, ws->b, ws->r, m.sc, ctx->partials, ctx->counters, guard);
        k_reliable_finish<S, MBLAS_BS><<<nblk_m(g.Vh, MBLAS_BS), MBLAS_BS, 0, s>>>(g.Vh, ws->r, r, m.sc,
                                                                                  lg ? lg->w : 0, use_cond, guard);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    static int enqueue_p(stag_ctx ctx, MixedSlot& m, int tg, cudaStream_t s)
    {
        STAG_TRY(launch_p(ctx, m, m.shape[tg].pk, s, m.sc));
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }

    // tg: the links lk (and the reliable update's) are the temporal-gauge
    // copies; the caller transforms b and x
    static int solve(stag_ctx ctx, MixedSlot& m, const void* lk, int tg, double2* x_out, const double2* b_in,
                     double mass, const stag_solver_params& prm, stag_solver_stats* st)
    {
        const auto t0 = std::chrono::steady_clock::now();
        Workspace* ws = ctx->ws;
        const Geom g = ctx->g;
        const void* lk64 = nullptr;
        const int p64 = std::is_same<typename LF64T::real, DF>::value ? STAG_F64X : STAG_F64;
        STAG_TRY(tg ? ensure_links_tg(ctx, p64, 18, &lk64) : ensure_links(ctx, p64, 18, &lk64));
        const LF U{(const typename LF::store*)lk, g.Vh, tg};
        const LF64T U64{(const typename LF64T::store*)lk64, g.Vh, tg};
        const int maxiter = prm.maxiter > 0 ? prm.maxiter : 100000;
        const double delta = prm.delta > 0 ? prm.delta : DEFAULT_RELIABLE_DELTA;
        STAG_TRY(tune(ctx, m, U, prm.inner_prec, prm.inner_recon));
        // b' = 2^-k b (largest component in [1, 2)): the float / half inner
        // storage and the double-float passes stay in range for any b; x = 2^k x'
        STAG_TRY(normalise_fields(ctx, b_in, ws->b, 1, (size_t)3 * g.Vh, SLOT_SOLVE, ctx->stream));
        k_mixed_start<S, SX, MBLAS_BS><<<nblk_m(g.Vh, MBLAS_BS), MBLAS_BS, 0, ctx->stream>>>(
            g.Vh, ws->b, ws->x, ws->r, m.template spinor<S>(m.r), m.template spinor<S>(m.p),
            m.template spinor<SX>(m.xlo), m.sc, prm.tol, maxiter, mass * mass, delta, ctx->partials, ctx->counters);
        STAG_CUDA_TRY(cudaGetLastError());
        if (prm.use_graph) {
            if (!m.lg[tg].exec || m.graph_arith[tg] != p64) {
                LoopGraph& lg = m.lg[tg];
                STAG_TRY(build_loop_graph(
                    ctx->cap_stream, lg, true,
                    [&](cudaStream_t s) { return enqueue_main(ctx, m, U, s, &lg, 1); },
                    [&](cudaStream_t s) { return enqueue_reliable(ctx, m, U64, s, &lg, 1, 0); },
                    [&](cudaStream_t s) { return enqueue_p(ctx, m, tg, s); }));
                m.graph_arith[tg] = p64;
            }
            STAG_CUDA_TRY(cudaGraphLaunch(m.lg[tg].exec, ctx->stream));
        } else {
            const int every = prm.check_every > 0 ? prm.check_every : 25;
            for (;;) {
                for (int k = 0; k < every; ++k) {
                    STAG_TRY(enqueue_main(ctx, m, U, ctx->stream, nullptr, 0));
                    STAG_TRY(enqueue_reliable(ctx, m, U64, ctx->stream, nullptr, 0, 1));
                    STAG_TRY(enqueue_p(ctx, m, tg, ctx->stream));
                }
                STAG_CUDA_TRY(cudaMemcpyAsync(ws->sc_host, m.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost,
                                              ctx->stream));
                STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
                if (ws->sc_host->done) break;
            }
        }
        CgScalars* hs = ws->sc_host;
        STAG_CUDA_TRY(cudaMemcpyAsync(hs, m.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, ctx->stream));
        STAG_TRY(scale_fields_out(ctx, ws->x, x_out, 1, (size_t)3 * g.Vh, SLOT_SOLVE, 1, ctx->stream));
        STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        int status = STAG_OK;
        if (hs->status == STAG_BREAKDOWN) status = STAG_BREAKDOWN;
        else if (hs->rr0 > 0.0 && !(hs->rr_true <= hs->tol2)) status = STAG_NOT_CONVERGED;
        if (st) {
            st->status = status;
            st->iters = hs->iter;
            st->restarts = 0;
            st->reliable_updates = hs->n_reliable;
            st->true_rel_residual = hs->rr0 > 0 ? sqrt(hs->rr_true / hs->rr0) : 0.0;
            st->iter_rel_residual = hs->rr0 > 0 ? sqrt(hs->rr / hs->rr0) : 0.0;
            st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        }
        return status;
    }
};

int ensure_cg_f64(stag_ctx ctx);

static int ensure_mixed(stag_ctx ctx, int prec, int recon, MixedSlot** out)
{
    STAG_TRY(ensure_cg_f64(ctx));
    Workspace* ws = ctx->ws;
    MixedSlot& m = ws->mixed[prec == STAG_F16 ? 1 : 0][recon == 12 ? 1 : 0];
    if (!m.ready) {
        const size_t lo = lo_spinor_bytes(ctx->g, prec);
        const size_t xb = lo_spinor_bytes(ctx->g, STAG_F32);
        STAG_CUDA_TRY(cudaMalloc(&m.r, lo));
        STAG_CUDA_TRY(cudaMalloc(&m.p, lo));
        STAG_CUDA_TRY(cudaMalloc(&m.Ap, lo));
        STAG_CUDA_TRY(cudaMalloc(&m.t, lo));
        STAG_CUDA_TRY(cudaMalloc(&m.xlo, xb));
        STAG_CUDA_TRY(cudaMalloc(&m.sc, sizeof(CgScalars)));
        m.Vh = ctx->g.Vh;
        m.ready = true;
    }
    *out = &m;
    return STAG_OK;
}

template <class LF64T, class SD64>
static int dispatch_inner(stag_ctx ctx, MixedSlot& m, const void* lk, int tg, double2* x_out, const double2* b_in,
                          double mass, const stag_solver_params& prm, stag_solver_stats* st)
{
    const int prec = prm.inner_prec, recon = prm.inner_recon;
    if (prec == STAG_F32) {
        if (recon == 12)
            return MixedPlan<SpinorF32, SpinorF32, LinkField<float2, 12>, LF64T, SD64>::solve(ctx, m, lk, tg, x_out,
                                                                                             b_in, mass, prm, st);
        return MixedPlan<SpinorF32, SpinorF32, LinkField<float2, 18>, LF64T, SD64>::solve(ctx, m, lk, tg, x_out, b_in,
                                                                                         mass, prm, st);
    }
    if (recon == 12)
        return MixedPlan<SpinorF16, SpinorF32, LinkField<__half2, 12>, LF64T, SD64>::solve(ctx, m, lk, tg, x_out,
                                                                                          b_in, mass, prm, st);
    return MixedPlan<SpinorF16, SpinorF32, LinkField<__half2, 18>, LF64T, SD64>::solve(ctx, m, lk, tg, x_out, b_in,
                                                                                      mass, prm, st);
}

static int mixed_arith(stag_ctx ctx, MixedSlot& m, const void* lk, int tg, double2* x_out, const double2* b_in,
                       double mass, const stag_solver_params& prm, stag_solver_stats* st)
{
    int arith = STAG_F64;
    STAG_TRY(resolve_f64_arith(ctx, prm.f64_arith, &arith));
    if (arith == STAG_F64X)
        return dispatch_inner<LinkFieldDF<18>, SpinorDF>(ctx, m, lk, tg, x_out, b_in, mass, prm, st);
    return dispatch_inner<LinkField<double2, 18>, SpinorF64>(ctx, m, lk, tg, x_out, b_in, mass, prm, st);
}

int cg_solve_mixed(stag_ctx ctx, double2* x_out, const double2* b_in, double mass, const stag_solver_params& prm,
                   stag_solver_stats* st)
{
    const int prec = prm.inner_prec, recon = prm.inner_recon;
    if ((prec != STAG_F32 && prec != STAG_F16) || (recon != 18 && recon != 12)) {
        set_error("mixed solver: inner_prec must be STAG_F32 or STAG_F16 and inner_recon 18 or 12");
        return STAG_EUNSUPPORTED;
    }
    STAG_TRY(check_float_inner_links(ctx));
    MixedSlot* m = nullptr;
    STAG_TRY(ensure_mixed(ctx, prec, recon, &m));
    const void* lk = nullptr;
    if (!prm.temporal_gauge) {
        STAG_TRY(ensure_links(ctx, prec, recon, &lk));
        return mixed_arith(ctx, *m, lk, 0, x_out, b_in, mass, prm, st);
    }
    // temporal gauge: M' x' = g b with every operator pass on U' (the inner
    // iteration and the reliable updates), x = g^dagger x'
    const double2* G = nullptr;
    double2* gb = nullptr;
    STAG_TRY(ensure_links_tg(ctx, prec, recon, &lk));
    STAG_TRY(ensure_tg_gauge(ctx, &G));
    STAG_TRY(ensure_tg_tmp(ctx, 1, &gb));
    STAG_TRY(tg_apply(ctx, G, b_in, gb, 1, 0));
    const int rc = mixed_arith(ctx, *m, lk, 1, x_out, gb, mass, prm, st);
    if (rc < 0) return rc;
    STAG_TRY(tg_apply(ctx, G, x_out, x_out, 1, 1));
    STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return rc;
}

void free_mixed(Workspace* ws)
{
    for (auto& row : ws->mixed)
        for (auto& m : row) {
            m.lg[0].destroy();
            m.lg[1].destroy();
            void* bufs[] = {m.r, m.p, m.Ap, m.t, m.xlo, m.sc};
            for (void* b : bufs)
                if (b) cudaFree(b);
            m = MixedSlot();
        }
}

int check_ctx(stag_ctx ctx);
int check_half_field(const void* p, const char* what);

}  // namespace stag

using namespace stag;

extern "C" int stag_cg_solve_mixed(stag_ctx ctx, double* x_even, const double* b_even, double mass,
                                   const stag_solver_params* params, stag_solver_stats* stats)
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
    return cg_solve_mixed(ctx, (double2*)x_even, (const double2*)b_even, mass, prm, stats);
}
