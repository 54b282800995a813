// multishift.cu -- multi-shift CG: (M + sigma_i) x_i = b for all shifts from a
// single Krylov space, M = m^2 - D_eo D_oe.
//
// Phase 1 (inner precision, one graph launch): CG on the smallest shift s0;
// every other system follows with the shifted-CG coefficients (residuals
// r_i = zeta_i r):
//   zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1} /
//        (a_k b_{k-1} (zeta_{k-1} - zeta_k) + zeta_{k-1} a_{k-1} (1 + (sigma - s0) a_k))
//   a_k^i = a_k zeta_{k+1}/zeta_k,  b_k^i = b_k (zeta_{k+1}/zeta_k)^2
//   x_i += a_k^i p_i,  p_i = zeta_{k+1} r + b_k^i p_i
// One operator application per iteration for all shifts; the x_i and p_i
// updates of every shift happen in one pass over the lattice.  A shift stops
// once zeta_i^2 |r|^2 <= tol^2 |b|^2.
// Phase 2: each shifted solution seeds a batched reliable-update solve of its
// own system (batched.cu), which brings every true residual, recomputed in
// double precision, below tol.
#include <chrono>
#include <new>
#include <vector>

#include "cg_kernels.cuh"
#include "graph.h"
#include "workspace.h"

namespace stag {

constexpr int MS_BS = 128;
constexpr int MS_BLAS = 256;

struct MsShift {
    double sigma;      // shift relative to the base system
    double zeta, zeta_prev, beta_s;
    int active;
    int pad;
};
struct MsState {
    double alpha_prev, beta_prev;
    int nshift, base;
    MsShift s[STAG_MAX_RHS];
};

// r = lo(b), p_i = r, x_i = 0; base scalars from |b|^2.
template <class S, int BS>
__global__ void __launch_bounds__(BS) k_ms_start(int Vh, const double2* b, S r, S P, S X, size_t stride, int nshift,
                                                 CgScalars* sc, MsState* ms, const double* shifts, int base,
                                                 double tol, int maxiter, double m2, double* part, unsigned* cnt)
{
    __shared__ double red[BS / 32];
    __shared__ bool last;
    typedef typename S::real real;
    const int h = blockIdx.x * BS + threadIdx.x;
    double d = 0.0;
    if (h < Vh) {
        Vec3<real> v, z;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 q = b[(size_t)h * 3 + c];
            d = fma(q.x, q.x, d);
            d = fma(q.y, q.y, d);
            v.c[c].re = (real)q.x;
            v.c[c].im = (real)q.y;
            z.c[c].re = z.c[c].im = 0;
        }
        r.store(h, v);
        for (int i = 0; i < nshift; ++i) {
            P.at(i, stride).store(h, v);
            X.at(i, stride).store(h, z);
        }
    }
    const double s = block_sum<BS>(d, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    if (!arrive_last(cnt, &last)) return;
    const double bb = sum_partials<BS>(part, gridDim.x, red);
    if (threadIdx.x == 0) {
        *cnt = 0;
        CgScalars c = {};
        c.rr = c.rr0 = c.rr_true = bb;
        c.tol2 = tol * tol * bb;
        c.maxiter = maxiter;
        c.m2 = m2;
        c.sigma = shifts[base];
        c.done = (bb == 0.0) ? 1 : 0;
        *sc = c;
        ms->alpha_prev = 1.0;
        ms->beta_prev = 0.0;
        ms->nshift = nshift;
        ms->base = base;
        for (int i = 0; i < nshift; ++i) {
            ms->s[i].sigma = shifts[i] - shifts[base];
            ms->s[i].zeta = ms->s[i].zeta_prev = 1.0;
            ms->s[i].beta_s = 0.0;
            ms->s[i].active = bb > 0.0;
        }
    }
}

// Coefficients zeta_{k+1} and a_k^i of every active shift (same arithmetic in
// every block, so all blocks agree bit for bit).
__device__ __forceinline__ void ms_coeffs(const CgScalars* sc, const MsState* ms, double* zn, double* as)
{
    const int i = threadIdx.x;
    if (i < ms->nshift) {
        const MsShift& q = ms->s[i];
        const double a = sc->alpha;
        double z = 1.0;
        if (q.active && i != ms->base) {
            z = q.zeta * q.zeta_prev * ms->alpha_prev /
                (a * ms->beta_prev * (q.zeta_prev - q.zeta) + q.zeta_prev * ms->alpha_prev * (1.0 + q.sigma * a));
        }
        zn[i] = z;
        as[i] = q.active ? a * z / q.zeta : 0.0;
    }
}

// r -= a Ap; x_i += a_i p_i for active shifts; |r|^2; then the scalar recurrences.
template <class S, int BS>
__global__ void __launch_bounds__(BS) k_ms_update(int Vh, S r, S Ap, S P, S X, size_t stride, CgScalars* sc,
                                                  MsState* ms, double* part, unsigned* cnt,
                                                  cudaGraphConditionalHandle wh, int use_cond)
{
    __shared__ double red[BS / 32];
    __shared__ bool last;
    __shared__ double zn[STAG_MAX_RHS], as[STAG_MAX_RHS];
    __shared__ int act[STAG_MAX_RHS];
    if (sc->done) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(wh, 0);
        return;
    }
    typedef typename S::real real;
    const int n = ms->nshift;
    ms_coeffs(sc, ms, zn, as);
    if (threadIdx.x < n) act[threadIdx.x] = ms->s[threadIdx.x].active;
    __syncthreads();
    const real alpha = (real)sc->alpha;
    const int h = blockIdx.x * BS + threadIdx.x;
    real d = real(0);
    if (h < Vh) {
        Vec3<real> rv = r.load_rw(h);
        const Vec3<real> av = Ap.load(h);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rv.c[c].re = fma(-alpha, av.c[c].re, rv.c[c].re);
            rv.c[c].im = fma(-alpha, av.c[c].im, rv.c[c].im);
        }
        r.store(h, rv);
        d = site_dot(rv, rv);
        for (int i = 0; i < n; ++i) {
            if (!act[i]) continue;
            const real ai = (real)as[i];
            const S Xi = X.at(i, stride);
            Vec3<real> xv = Xi.load_rw(h);
            const Vec3<real> pv = P.at(i, stride).load(h);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xv.c[c].re = fma(ai, pv.c[c].re, xv.c[c].re);
                xv.c[c].im = fma(ai, pv.c[c].im, xv.c[c].im);
            }
            Xi.store(h, xv);
        }
    }
    const double bs = block_sum<BS>(d, red);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
    if (!arrive_last(cnt, &last)) return;
    const double rr_new = sum_partials<BS>(part, gridDim.x, red);
    if (threadIdx.x == 0) {
        *cnt = 0;
        const double beta = rr_new / sc->rr;
        for (int i = 0; i < n; ++i) {
            MsShift& q = ms->s[i];
            if (!q.active) continue;
            const double ratio = zn[i] / q.zeta;
            q.beta_s = beta * ratio * ratio;
            q.zeta_prev = q.zeta;
            q.zeta = zn[i];
            if (i != ms->base && q.zeta * q.zeta * rr_new <= sc->tol2) q.active = 0;
        }
        ms->alpha_prev = sc->alpha;
        ms->beta_prev = beta;
        sc->beta = beta;
        sc->rr = rr_new;
        sc->iter += 1;
        if (!isfinite(rr_new)) {
            sc->status = STAG_BREAKDOWN;
            sc->done = 1;
        } else if (rr_new <= sc->tol2 || sc->iter >= sc->maxiter) {
            sc->done = 1;
        }
        if (use_cond) cudaGraphSetConditional(wh, sc->done ? 0 : 1);
    }
}

// p_i = zeta_i r + beta_i p_i for active shifts (zeta_base = 1).
template <class S, int BS>
__global__ void __launch_bounds__(BS) k_ms_p(int Vh, S r, S P, size_t stride, const CgScalars* sc, const MsState* ms)
{
    __shared__ double zs[STAG_MAX_RHS], bsh[STAG_MAX_RHS];
    __shared__ int act[STAG_MAX_RHS];
    if (sc->done) return;
    typedef typename S::real real;
    const int n = ms->nshift;
    if (threadIdx.x < n) {
        zs[threadIdx.x] = ms->s[threadIdx.x].zeta;
        bsh[threadIdx.x] = ms->s[threadIdx.x].beta_s;
        act[threadIdx.x] = ms->s[threadIdx.x].active;
    }
    __syncthreads();
    const int h = blockIdx.x * BS + threadIdx.x;
    if (h >= Vh) return;
    const Vec3<real> rv = r.load(h);
    for (int i = 0; i < n; ++i) {
        if (!act[i]) continue;
        const real z = (real)zs[i], bt = (real)bsh[i];
        const S Pi = P.at(i, stride);
        Vec3<real> pv = Pi.load_rw(h);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pv.c[c].re = fma(bt, pv.c[c].re, z * rv.c[c].re);
            pv.c[c].im = fma(bt, pv.c[c].im, z * rv.c[c].im);
        }
        Pi.store(h, pv);
    }
}

template <class S, class LF>
struct MsPlan {
    static int enqueue_iter(stag_ctx ctx, MsSlot& m, const LF& U, cudaStream_t s, LoopGraph* lg, int use_cond)
    {
        const Geom g = ctx->g;
        const S P = m.template spinor<S>(m.P), X = m.template spinor<S>(m.X);
        const S pb = P.at(m.base, m.stride);
        const S t = m.template spinor<S>(m.t), Ap = m.template spinor<S>(m.Ap), r = m.template spinor<S>(m.r);
        const int gh = (g.Vh + MS_BS - 1) / MS_BS, gb = (g.Vh + MS_BLAS - 1) / MS_BLAS;
        k_hop_guarded<LF, S, MS_BS><<<gh, MS_BS, 0, s>>>(g, 1, U, pb, t, m.sc);
        k_Mp_dot<LF, S, S, MS_BS><<<gh, MS_BS, 0, s>>>(g, U, t, pb, Ap, m.sc, ctx->partials, ctx->counters + 2,
                                                       grid_sum_of(ctx));
        k_ms_update<S, MS_BLAS><<<gb, MS_BLAS, 0, s>>>(g.Vh, r, Ap, P, X, m.stride, m.sc, m.ms, ctx->partials,
                                                       ctx->counters + 2, lg ? lg->w : 0, use_cond);
        k_ms_p<S, MS_BLAS><<<gb, MS_BLAS, 0, s>>>(g.Vh, r, P, m.stride, m.sc, m.ms);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }

    static int run(stag_ctx ctx, MsSlot& m, const void* lk, int tg, const double2* b, double mass,
                   const double* shifts_dev, double tol, int maxiter, const stag_solver_params& prm)
    {
        const Geom g = ctx->g;
        const LF U{(const typename LF::store*)lk, g.Vh, tg};
        const S P = m.template spinor<S>(m.P), X = m.template spinor<S>(m.X), r = m.template spinor<S>(m.r);
        k_ms_start<S, MS_BLAS><<<(g.Vh + MS_BLAS - 1) / MS_BLAS, MS_BLAS, 0, ctx->stream>>>(
            g.Vh, b, r, P, X, m.stride, m.nshift, m.sc, m.ms, shifts_dev, m.base, tol, maxiter, mass * mass,
            ctx->partials, ctx->counters + 2);
        STAG_CUDA_TRY(cudaGetLastError());
        if (prm.use_graph) {
            if (!m.lg.exec || m.graph_n != m.nshift || m.graph_base != m.base || m.graph_tg != tg) {
                LoopGraph& lg = m.lg;
                auto none = [](cudaStream_t) { return STAG_OK; };
                STAG_TRY(build_loop_graph(ctx->cap_stream, lg, false,
                                          [&](cudaStream_t s) { return enqueue_iter(ctx, m, U, s, &lg, 1); }, none,
                                          none));
                m.graph_n = m.nshift;
                m.graph_base = m.base;
                m.graph_tg = tg;
            }
            STAG_CUDA_TRY(cudaGraphLaunch(m.lg.exec, ctx->stream));
        } else {
            const int every = prm.check_every > 0 ? prm.check_every : 25;
            CgScalars hs;
            for (;;) {
                for (int k = 0; k < every; ++k) STAG_TRY(enqueue_iter(ctx, m, U, ctx->stream, nullptr, 0));
                STAG_CUDA_TRY(cudaMemcpyAsync(&hs, m.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, ctx->stream));
                STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
                if (hs.done) break;
            }
        }
        return STAG_OK;
    }
};

void MsSlot::release()
{
    lg.destroy();
    void* bufs[] = {P, X, r, Ap, t, sc, ms, shifts, brep};
    for (void* q : bufs)
        if (q) cudaFree(q);
    *this = MsSlot();
}

int batched_solve(stag_ctx ctx, double2* X, const double2* B, int nrhs, double mass, const double* shifts_host,
                  const double2* X0, const stag_solver_params& prm, stag_solver_stats* stats, int tg);

int multishift_solve(stag_ctx ctx, double2* X, const double2* b, const double* shifts, int nshift, double mass,
                     const stag_solver_params& prm, stag_solver_stats* stats)
{
    const auto t0 = std::chrono::steady_clock::now();
    const int prec = prm.inner_prec == STAG_F64 ? STAG_F64 : STAG_F32;
    const int recon = prm.inner_recon == 18 ? 18 : 12;
    if (prec != STAG_F64) STAG_TRY(check_float_inner_links(ctx));
    if (!ctx->ws) {
        ctx->ws = new (std::nothrow) Workspace();
        if (!ctx->ws) return STAG_ENOMEM;
    }
    MsSlot& m = ctx->ws->ms[prec == STAG_F64 ? 0 : 1];
    const Geom& g = ctx->g;
    if (m.ready && m.cap < nshift) m.release();
    if (!m.ready) {
        m.Vh = g.Vh;
        m.cap = nshift;
        m.stride = lo_spinor_bytes(g, prec);
        STAG_CUDA_TRY(cudaMalloc(&m.P, nshift * m.stride));
        STAG_CUDA_TRY(cudaMalloc(&m.X, nshift * m.stride));
        STAG_CUDA_TRY(cudaMalloc(&m.r, m.stride));
        STAG_CUDA_TRY(cudaMalloc(&m.Ap, m.stride));
        STAG_CUDA_TRY(cudaMalloc(&m.t, m.stride));
        STAG_CUDA_TRY(cudaMalloc(&m.sc, sizeof(CgScalars)));
        STAG_CUDA_TRY(cudaMalloc(&m.ms, sizeof(MsState)));
        STAG_CUDA_TRY(cudaMalloc(&m.shifts, STAG_MAX_RHS * sizeof(double)));
        STAG_CUDA_TRY(cudaMalloc(&m.brep, (size_t)nshift * g.Vh * 3 * sizeof(double2)));
        m.ready = true;
    }
    int base = 0;
    for (int i = 1; i < nshift; ++i)
        if (shifts[i] < shifts[base]) base = i;
    m.nshift = nshift;
    m.base = base;
    STAG_CUDA_TRY(cudaMemcpyAsync(m.shifts, shifts, nshift * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    // temporal gauge: both phases on U' for b' = g b; X = g^dagger X' at the end
    const int tg = prm.temporal_gauge ? 1 : 0;
    const void* lk = nullptr;
    const double2* G = nullptr;
    STAG_TRY(tg ? ensure_links_tg(ctx, prec, recon, &lk) : ensure_links(ctx, prec, recon, &lk));
    if (tg) {
        double2* gb = nullptr;
        STAG_TRY(ensure_tg_gauge(ctx, &G));
        STAG_TRY(ensure_tg_tmp(ctx, 1, &gb));
        STAG_TRY(tg_apply(ctx, G, b, gb, 1, 0));
        b = gb;
    }
    const int maxiter = prm.maxiter > 0 ? prm.maxiter : 100000;
    // b' = 2^-k b (largest component in [1, 2)) in the first replica: the Krylov
    // phase and the refinement solve for b', the solutions are scaled by 2^k
    // at the end
    const size_t fbytes = (size_t)g.Vh * 3 * sizeof(double2);
    STAG_TRY(normalise_fields(ctx, b, m.brep, 1, (size_t)3 * g.Vh, SLOT_OUTER, ctx->stream));
    const double2* bn = m.brep;
    // the Krylov phase stops at the inner precision's reach; refinement does the rest
    const double tol1 = prec == STAG_F64 ? prm.tol : (prm.tol > 1e-6 ? prm.tol : 1e-6);
    if (prec == STAG_F64) {
        if (recon == 18) STAG_TRY((MsPlan<SpinorF64, LinkField<double2, 18>>::run(ctx, m, lk, tg, bn, mass, m.shifts, tol1, maxiter, prm)));
        else STAG_TRY((MsPlan<SpinorF64, LinkField<double2, 12>>::run(ctx, m, lk, tg, bn, mass, m.shifts, tol1, maxiter, prm)));
    } else {
        if (recon == 18) STAG_TRY((MsPlan<SpinorF32, LinkField<float2, 18>>::run(ctx, m, lk, tg, bn, mass, m.shifts, tol1, maxiter, prm)));
        else STAG_TRY((MsPlan<SpinorF32, LinkField<float2, 12>>::run(ctx, m, lk, tg, bn, mass, m.shifts, tol1, maxiter, prm)));
    }
    CgScalars hs;
    STAG_CUDA_TRY(cudaMemcpyAsync(&hs, m.sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, ctx->stream));
    // shifted solutions -> double initial guesses; b' replicated per system
    if (prec == STAG_F64) {
        STAG_CUDA_TRY(cudaMemcpyAsync(X, m.X, nshift * fbytes, cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
        STAG_TRY(convert_lo_to_f64(ctx, prec, m.X, X, nshift, ctx->stream));
    }
    for (int i = 1; i < nshift; ++i)
        STAG_CUDA_TRY(cudaMemcpyAsync((char*)m.brep + i * fbytes, m.brep, fbytes, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
    STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    const int ms_iters = hs.iter;
    if (hs.status == STAG_BREAKDOWN) {
        set_error("multi-shift iteration broke down");
    }
    stag_solver_params p2 = prm;
    p2.inner_prec = prec == STAG_F64 ? STAG_F64 : prm.inner_prec;
    p2.inner_recon = prm.inner_recon;
    p2.maxiter = maxiter > ms_iters ? maxiter - ms_iters : 1;
    const int rc = batched_solve(ctx, X, (const double2*)m.brep, nshift, mass, shifts, X, p2, stats, tg);
    if (rc < 0) return rc;
    STAG_TRY(scale_fields_out(ctx, X, X, nshift, (size_t)3 * g.Vh, SLOT_OUTER, 0, ctx->stream));
    if (tg) STAG_TRY(tg_apply(ctx, G, X, X, nshift, 1));
    STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (stats) {
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int i = 0; i < nshift; ++i) {
            stats[i].restarts = ms_iters;   // iterations of the shared Krylov phase
            stats[i].iters += ms_iters;
            stats[i].seconds = secs;
        }
    }
    return rc;
}

int check_ctx(stag_ctx ctx);
int check_half_field(const void* p, const char* what);

}  // namespace stag

using namespace stag;

extern "C" int stag_cg_solve_multishift(stag_ctx ctx, double* X, const double* b, const double* shifts, int nshift,
                                        double mass, const stag_solver_params* params, stag_solver_stats* stats)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(X, "X"));
    STAG_TRY(check_half_field(b, "b"));
    if (!shifts || nshift < 1 || nshift > STAG_MAX_RHS) {
        set_error("shifts must be a host array of 1..%d values", STAG_MAX_RHS);
        return STAG_EINVAL;
    }
    for (int i = 0; i < nshift; ++i)
        if (!(shifts[i] >= 0.0) || !isfinite(shifts[i])) {
            set_error("shift %d is negative or not finite", i);
            return STAG_EINVAL;
        }
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
    return multishift_solve(ctx, (double2*)X, (const double2*)b, shifts, nshift, mass, prm, stats);
}
