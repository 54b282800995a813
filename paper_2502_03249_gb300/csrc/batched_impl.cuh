// batched_impl.cuh -- batched reliable-update CG: n independent systems
// (M + sigma_k) x_k = b_k, M = m^2 - D_eo D_oe, advanced together so that each
// operator pass loads every link once for NB right-hand sides (NB chosen by
// the autotuner).  Inner storage F64, F32 or F16 (with 18- or 12-real links);
// the solution of each system is accumulated in double precision and its true
// residual recomputed in double precision when its inner residual has dropped
// by delta below the maximum since its last update, or has reached tol.  With
// F64 inner storage and delta = 0 this is plain batched CG with a final true
// residual check.  Systems that have converged are masked out of every pass.
//
// Serves stag_cg_solve_multi (shared shift 0) and the double-precision
// refinement of stag_cg_solve_multishift (one shift per system, the shifted
// solutions as initial guesses).
//
// Graph: while (W) { hop; Mp_dot; update; if (I) { accum_x; hop64; resid64; finish } p }
#pragma once

#include <chrono>
#include <new>
#include <vector>

#include "batched.cuh"
#include "df64.cuh"
#include "cg_kernels.cuh"
#include "graph.h"
#include "tune.h"
#include "workspace.h"

namespace stag {

constexpr int BBS = 128;      // threads (sites) per block of every batched kernel

// Right-hand sides per thread of the double-precision passes (reliable
// updates): the systems reach their updates at different iterations, so a
// pass usually works on one or two of them.  IEEE double (FP64-ALU bound)
// shares each link load among 4; double-float uses 1 per thread, which keeps
// its operator at 96 registers and full occupancy (4 per thread needs 128-152).
template <class LF64> struct Nb64 { static constexpr int value = 4; };
template <> struct Nb64<LinkFieldDF<18>> { static constexpr int value = 1; };

struct BatchScal {
    CgScalars* sc;      // [nrhs]
    int nrhs;
    double* part;       // [nrhs][gx]
    unsigned* cnt;      // one counter over all blocks (or over finished systems)
    int gx;             // blocks along the sites
    unsigned* cnt_sys;  // [nrhs] one counter per system: blocks that wrote its partial
};

// Per-system completion of a reduction: after the block has written its
// partials of the systems in `mine` (bit k: system k0 + k), count it in for
// each of them.  Returns the systems this block finished last (the whole row
// of gx blocks has written their partials), whose final sums it must form;
// those counters are reset.  Each system is finalised by its own last block,
// so the systems' final sums run in parallel.
template <int NB>
__device__ __forceinline__ unsigned arrive_last_sys(const BatchScal& bs, int k0, unsigned mine, unsigned* smem)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned last = 0;
        if (mine) {
            __threadfence();
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (mine & (1u << k)) {
                    if (atomicAdd(bs.cnt_sys + k0 + k, 1u) == (unsigned)bs.gx - 1) {
                        last |= 1u << k;
                        bs.cnt_sys[k0 + k] = 0;
                    }
                }
        }
        *smem = last;
    }
    __syncthreads();
    return *smem;
}

__device__ __forceinline__ bool active(const CgScalars& s) { return !s.done; }
__device__ __forceinline__ bool updating(const CgScalars& s) { return !s.done && s.reliable; }

// Masks of the NB systems starting at k0 that a pass works on.
template <int NB>
__device__ __forceinline__ unsigned mask_active(const BatchScal& b, int k0)
{
    unsigned m = 0;
#pragma unroll
    for (int k = 0; k < NB; ++k)
        if (k0 + k < b.nrhs && active(b.sc[k0 + k])) m |= 1u << k;
    return m;
}
template <int NB>
__device__ __forceinline__ unsigned mask_updating(const BatchScal& b, int k0)
{
    unsigned m = 0;
#pragma unroll
    for (int k = 0; k < NB; ++k)
        if (k0 + k < b.nrhs && updating(b.sc[k0 + k])) m |= 1u << k;
    return m;
}

// ------------------------------------------------------------- start

// x_hi = x0 (or 0), xlo = 0, rr0 = |b|^2 per system; every system marked for a
// residual recomputation.  grid (gx, nrhs).
// b holds the normalised right-hand sides 2^-k_k B_k; x0 (unnormalised
// initial guesses) is brought to the same scale.
template <class SX>
__global__ void __launch_bounds__(BBS) k_b_init(int Vh, const double2* b, const double2* x0, double2* x_hi, SX xlo,
                                                size_t sx_stride, BatchScal bs, double tol, int maxiter, double m2,
                                                const double* shifts, double delta, const int* kexp)
{
    __shared__ double red[BBS / 32];
    __shared__ bool last;
    const int k = blockIdx.y, h = blockIdx.x * BBS + threadIdx.x;
    double d = 0.0;
    if (h < Vh) {
        const size_t o = ((size_t)k * Vh + h) * 3;
        Vec3<typename SX::real> z;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 bv = b[o + c];
            d = fma(bv.x, bv.x, d);
            d = fma(bv.y, bv.y, d);
            if (x0) {
                const double2 v = x0[o + c];
                x_hi[o + c] = make_double2(scalbn(v.x, -kexp[k]), scalbn(v.y, -kexp[k]));
            } else {
                x_hi[o + c] = make_double2(0.0, 0.0);
            }
            z.c[c].re = z.c[c].im = 0;
        }
        xlo.at(k, sx_stride).store(h, z);
    }
    const double s = block_sum<BBS>(d, red);
    if (threadIdx.x == 0) bs.part[(size_t)k * bs.gx + blockIdx.x] = s;
    if (!arrive_last(bs.cnt, &last)) return;
    for (int kk = 0; kk < bs.nrhs; ++kk) {
        const double bb = sum_partials<BBS>(bs.part + (size_t)kk * bs.gx, bs.gx, red);
        if (threadIdx.x == 0) {
            CgScalars c = {};
            c.rr0 = c.rr = c.rmax2 = c.rr_true = bb;
            c.tol2 = tol * tol * bb;
            c.delta2 = delta * delta;
            c.maxiter = maxiter;
            c.m2 = m2;
            c.sigma = shifts ? shifts[kk] : 0.0;
            c.rr_prev = bb;
            c.done = (bb == 0.0) ? 1 : 0;
            c.reliable = 1;
            bs.sc[kk] = c;
        }
    }
    if (threadIdx.x == 0) *bs.cnt = 0;
}

// ------------------------------------------------------- operator passes

// t_k = D_oe p_k for the systems selected by MODE.  MODE 0 (active systems,
// the iteration): grid (gx, nrhs / NB), row y takes systems y NB ... .  MODE 1
// (systems due a reliable update, usually one or two): grid (gx, 1), every
// block loops over the groups of NB systems and skips those with none due, so
// no block is launched for systems that have nothing to do.
template <class LF, class S, int NB, int MODE>
__global__ void __launch_bounds__(BBS, (MultiMinBlocks<LF, NB>::value)) k_b_hop(Geom g, LF U, S in, S out,
                                                                               size_t stride, BatchScal bs)
{
    const int h = blockIdx.x * BBS + threadIdx.x;
    if (h >= g.Vh) return;
    const int kbeg = MODE == 0 ? blockIdx.y * NB : 0, kend = MODE == 0 ? kbeg + NB : bs.nrhs;
    for (int k0 = kbeg; k0 < kend; k0 += NB) {
        const unsigned mask = MODE == 0 ? mask_active<NB>(bs, k0) : mask_updating<NB>(bs, k0);
        if (!mask) continue;
        Vec3<typename LF::real> acc[NB];
        dslash_site_multi<LF, S, NB>(g, 1, h, U, in, stride, k0, mask, acc);
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if (mask & (1u << k)) out.at(k0 + k, stride).store(h, acc[k]);
    }
}

// Ap_k = (m^2 + sigma_k) p_k - D_eo t_k, pAp_k, alpha_k = rr_k / pAp_k.
template <class LF, class S, int NB>
__global__ void __launch_bounds__(BBS, (MultiMinBlocks<LF, NB>::value)) k_b_Mp_dot(Geom g, LF U, S t, S p, S Ap,
                                                                                  size_t stride, BatchScal bs)
{
    __shared__ double red[(BBS / 32) * (NB > 1 ? NB : 1)];
    __shared__ unsigned lastm;
    typedef typename S::real real;
    const int k0 = blockIdx.y * NB;
    const unsigned mask = mask_active<NB>(bs, k0);
    const int h = blockIdx.x * BBS + threadIdx.x;
    double d[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) d[k] = 0.0;
    if (mask && h < g.Vh) {
        Vec3<real> acc[NB];
        dslash_site_multi<LF, S, NB>(g, 0, h, U, t, stride, k0, mask, acc);
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            if (!(mask & (1u << k))) continue;
            const real m2s = (real)(bs.sc[k0 + k].m2 + bs.sc[k0 + k].sigma);
            const Vec3<real> pv = p.at(k0 + k, stride).load(h);
            Vec3<real> a;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a.c[c].re = fma(m2s, pv.c[c].re, -acc[k].c[c].re);
                a.c[c].im = fma(m2s, pv.c[c].im, -acc[k].c[c].im);
            }
            Ap.at(k0 + k, stride).store(h, a);
            d[k] = site_dot(pv, a);
        }
    }
    {
        const double s = block_sum_n<BBS, NB>(d, mask, red);
        if (threadIdx.x < NB && (mask & (1u << threadIdx.x)))
            bs.part[(size_t)(k0 + threadIdx.x) * bs.gx + blockIdx.x] = s;
    }
    const unsigned fin = arrive_last_sys<NB>(bs, k0, mask, &lastm);
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        if (!(fin & (1u << k))) continue;
        const int kk = k0 + k;
        const double pAp = sum_partials<BBS>(bs.part + (size_t)kk * bs.gx, bs.gx, red);
        if (threadIdx.x == 0) {
            CgScalars& c = bs.sc[kk];
            c.pAp = pAp;
            if (!(pAp > 0.0) || !isfinite(pAp)) {
                c.status = STAG_BREAKDOWN;
                c.done = 1;
                c.reliable = 0;
            } else {
                c.alpha = c.rr / pAp;
            }
        }
    }
}

// x_k += alpha_k p_k, r_k -= alpha_k Ap_k, rr_k; flag reliable updates.  grid (gx, nrhs).
template <class S, class SX>
__global__ void __launch_bounds__(BBS) k_b_update(int Vh, SX x, size_t sx_stride, S r, S p, S Ap, size_t stride,
                                                  BatchScal bs, cudaGraphConditionalHandle wh,
                                                  cudaGraphConditionalHandle ih, int use_cond)
{
    __shared__ double red[BBS / 32];
    __shared__ unsigned lastm;
    typedef typename S::real real;
    const int k = blockIdx.y, h = blockIdx.x * BBS + threadIdx.x;
    const bool on = active(bs.sc[k]);
    double d = 0.0;
    if (on && h < Vh) {
        const real alpha = (real)bs.sc[k].alpha;
        const SX xk = x.at(k, sx_stride);
        const S rk = r.at(k, stride);
        Vec3<typename SX::real> xv = xk.load_rw(h);
        Vec3<real> rv = rk.load_rw(h);
        const Vec3<real> pv = p.at(k, stride).load(h), av = Ap.at(k, stride).load(h);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xv.c[c].re = fma(alpha, pv.c[c].re, xv.c[c].re);
            xv.c[c].im = fma(alpha, pv.c[c].im, xv.c[c].im);
            rv.c[c].re = fma(-alpha, av.c[c].re, rv.c[c].re);
            rv.c[c].im = fma(-alpha, av.c[c].im, rv.c[c].im);
        }
        xk.store(h, xv);
        rk.store(h, rv);
        d = site_dot(rv, rv);
    }
    if (on) {
        const double s = block_sum<BBS>(d, red);
        if (threadIdx.x == 0) bs.part[(size_t)k * bs.gx + blockIdx.x] = s;
    }
    // Which systems are active does not change during this kernel; with none
    // active, block (0, 0) ends the graph loop.
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        int n_on = 0;
        for (int kk = 0; kk < bs.nrhs; ++kk) n_on += active(bs.sc[kk]);
        if (n_on == 0 && use_cond) {
            cudaGraphSetConditional(ih, 0);
            cudaGraphSetConditional(wh, 0);
        }
    }
    // system k finished by its last block ...
    if (!arrive_last_sys<1>(bs, k, on ? 1u : 0u, &lastm)) return;
    const double rr_new = sum_partials<BBS>(bs.part + (size_t)k * bs.gx, bs.gx, red);
    if (threadIdx.x != 0) return;
    CgScalars& c = bs.sc[k];
    c.rr_prev = c.rr;
    c.beta = rr_new / c.rr;
    c.rr = rr_new;
    c.iter += 1;
    if (rr_new > c.rmax2) c.rmax2 = rr_new;
    c.reliable = !isfinite(rr_new) || rr_new < c.delta2 * c.rmax2 || rr_new <= c.tol2 || c.iter >= c.maxiter;
    // ... and the last system to finish sets the loop's conditions
    int n_on = 0;
    for (int kk = 0; kk < bs.nrhs; ++kk) n_on += active(bs.sc[kk]);
    __threadfence();
    if (atomicAdd(bs.cnt, 1u) != (unsigned)n_on - 1) return;
    *bs.cnt = 0;
    __threadfence();
    // other systems' flags were written by other blocks in this kernel: read past L1
    const volatile CgScalars* vs = bs.sc;
    int any_rel = 0;
    for (int kk = 0; kk < bs.nrhs; ++kk) any_rel |= !vs[kk].done && vs[kk].reliable;
    if (use_cond) {
        cudaGraphSetConditional(ih, any_rel ? 1 : 0);
        cudaGraphSetConditional(wh, 1);
    }
}

// x_hi_k += xlo_k, xlo_k = 0 for systems due a reliable update.  grid (gx, 1):
// each block loops over the systems and skips those not due.
template <class SX>
__global__ void __launch_bounds__(BBS) k_b_accum_x(int Vh, double2* x_hi, SX xlo, size_t sx_stride, BatchScal bs)
{
    const int h = blockIdx.x * BBS + threadIdx.x;
    if (h >= Vh) return;
    for (int k = 0; k < bs.nrhs; ++k) {
        if (!updating(bs.sc[k])) continue;
        const SX xk = xlo.at(k, sx_stride);
        const Vec3<typename SX::real> v = xk.load_rw(h);
        Vec3<typename SX::real> z;
        const size_t o = ((size_t)k * Vh + h) * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double2 xv = x_hi[o + c];
            xv.x += (double)v.c[c].re;
            xv.y += (double)v.c[c].im;
            x_hi[o + c] = xv;
            z.c[c].re = z.c[c].im = 0;
        }
        xk.store(h, z);
    }
}

// One group of NB systems of k_b_resid64 (below).
template <class LF, class SD, int NB>
__device__ __forceinline__ void resid64_group(const Geom& g, const LF& U, const double2* t, const double2* x_hi,
                                              const double2* b, double2* r_hi, const BatchScal& bs, int k0,
                                              double* red, unsigned* lastm_p)
{
    unsigned& lastm = *lastm_p;
    const unsigned mask = mask_updating<NB>(bs, k0);
    if (!mask) return;   // uniform over the block
    const int h = blockIdx.x * BBS + threadIdx.x;
    const size_t stride = (size_t)g.Vh * 3 * sizeof(double2);
    double d[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) d[k] = 0.0;
    if (mask && h < g.Vh) {
        Vec3<typename LF::real> acc[NB];
        dslash_site_multi<LF, SD, NB>(g, 0, h, U, SD{(double2*)t}, stride, k0, mask, acc);
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            if (!(mask & (1u << k))) continue;
            const double m2s = bs.sc[k0 + k].m2 + bs.sc[k0 + k].sigma;
            const size_t o = ((size_t)(k0 + k) * g.Vh + h) * 3;
            const Vec3<double> Dt = vconv<double>(acc[k]);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double2 xv = x_hi[o + c], bv = b[o + c];
                const double re = bv.x - fma(m2s, xv.x, -Dt.c[c].re);
                const double im = bv.y - fma(m2s, xv.y, -Dt.c[c].im);
                r_hi[o + c] = make_double2(re, im);
                d[k] = fma(re, re, d[k]);
                d[k] = fma(im, im, d[k]);
            }
        }
    }
    {
        const double s = block_sum_n<BBS, NB>(d, mask, red);
        if (threadIdx.x < NB && (mask & (1u << threadIdx.x)))
            bs.part[(size_t)(k0 + threadIdx.x) * bs.gx + blockIdx.x] = s;
    }
    const unsigned fin = arrive_last_sys<NB>(bs, k0, mask, &lastm);
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        if (!(fin & (1u << k))) continue;
        const double rr = sum_partials<BBS>(bs.part + (size_t)(k0 + k) * bs.gx, bs.gx, red);
        if (threadIdx.x == 0) bs.sc[k0 + k].rr_true = rr;
    }
}

// r_hi_k = b_k - (m^2 + sigma_k) x_hi_k + D_eo t_k, rr_true_k (double) for updating systems.
// The operator pass runs in LF's arithmetic (IEEE double, or double-float on
// the same double vectors through SD), the epilogue in double.  grid (gx, 1):
// each block loops over the groups of NB systems and skips those with none
// due; every system due gets one partial from every block and is finished by
// its own last block, as in the iteration's reductions.
template <class LF, class SD, int NB>
__global__ void __launch_bounds__(BBS, (MultiMinBlocks<LF, NB>::value)) k_b_resid64(Geom g, LF U, const double2* t,
                                                                                        const double2* x_hi,
                                                                                        const double2* b, double2* r_hi,
                                                                                        BatchScal bs)
{
    __shared__ double red[(BBS / 32) * (NB > 1 ? NB : 1)];
    __shared__ unsigned lastm;
    for (int k0 = 0; k0 < bs.nrhs; k0 += NB)
        resid64_group<LF, SD, NB>(g, U, t, x_hi, b, r_hi, bs, k0, red, &lastm);
}

// r_k = lo(r_hi_k) (and p_k = r_k at the start); then, in the last block,
// restart each updated system's recurrence from its true residual and decide
// convergence.  grid (gx, 1): each block loops over the systems due.
template <class S>
__global__ void __launch_bounds__(BBS) k_b_finish(int Vh, const double2* r_hi, S r, S p, size_t stride, BatchScal bs,
                                                  int start, cudaGraphConditionalHandle wh, int use_cond)
{
    __shared__ bool last;
    typedef typename S::real real;
    const int h = blockIdx.x * BBS + threadIdx.x;
    for (int k = 0; k < bs.nrhs && h < Vh; ++k) {
        if (!updating(bs.sc[k])) continue;
        Vec3<real> v;
        const size_t o = ((size_t)k * Vh + h) * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 q = r_hi[o + c];
            v.c[c].re = (real)q.x;
            v.c[c].im = (real)q.y;
        }
        r.at(k, stride).store(h, v);
        if (start) p.at(k, stride).store(h, v);
    }
    if (!arrive_last(bs.cnt, &last)) return;
    if (threadIdx.x == 0) {
        int any_on = 0;
        for (int kk = 0; kk < bs.nrhs; ++kk) {
            CgScalars& c = bs.sc[kk];
            if (updating(c)) {
                const double rt = c.rr_true;
                if (!start) c.n_reliable += 1;
                if (!isfinite(rt)) {
                    c.status = STAG_BREAKDOWN;
                    c.done = 1;
                } else if (rt <= c.tol2) {
                    c.done = 1;
                } else if (c.iter >= c.maxiter) {
                    c.status = STAG_NOT_CONVERGED;
                    c.done = 1;
                }
                c.beta = start ? 0.0 : rt / c.rr_prev;
                c.rr = rt;
                c.rmax2 = rt;
            }
            c.reliable = 0;
            any_on |= !c.done;
        }
        *bs.cnt = 0;
        if (use_cond) cudaGraphSetConditional(wh, any_on ? 1 : 0);
    }
}

// p_k = r_k + beta_k p_k.  grid (gx, nrhs).
template <class S>
__global__ void __launch_bounds__(BBS) k_b_p(int Vh, S r, S p, size_t stride, BatchScal bs)
{
    typedef typename S::real real;
    const int k = blockIdx.y, h = blockIdx.x * BBS + threadIdx.x;
    if (!active(bs.sc[k]) || h >= Vh) return;
    const real beta = (real)bs.sc[k].beta;
    const S pk = p.at(k, stride);
    const Vec3<real> rv = r.at(k, stride).load(h);
    Vec3<real> pv = pk.load_rw(h);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        pv.c[c].re = fma(beta, pv.c[c].re, rv.c[c].re);
        pv.c[c].im = fma(beta, pv.c[c].im, rv.c[c].im);
    }
    pk.store(h, pv);
}

// ------------------------------------------------------------- driver

typedef LinkField<double2, 18> LF64B;

// LF64 / SD64: link field and spinor view of the double-precision passes
// (reliable updates): IEEE double (LinkField<double2,18>, SpinorF64) or
// double-float on the same double vectors (LinkFieldDF<18>, SpinorF64asDF).
template <class S, class SX, class LF, int NB, class LF64, class SD64>
struct BatchPlan {
    static constexpr int NB64 = Nb64<LF64>::value;
    static S spin(const BatchSlot& m, void* buf) { return m.template spinor<S>(buf); }
    static SX spinx(const BatchSlot& m, void* buf) { return m.template spinor<SX>(buf); }

    static int enqueue_start(stag_ctx ctx, BatchSlot& m, const LF64& U64, cudaStream_t s, const double2* x0,
                             double tol, int maxiter, double mass, const double* shifts_dev, double delta)
    {
        const Geom g = ctx->g;
        const BatchScal bs{m.sc, m.nrhs, m.part, ctx->counters + 1, m.gx, m.cnt_sys};
        const dim3 gb(m.gx, m.nrhs), g1(m.gx, 1);
        k_b_init<SX><<<gb, BBS, 0, s>>>(g.Vh, m.b, x0, m.x_hi, spinx(m, m.xlo), m.sx_stride, bs, tol, maxiter,
                                        mass * mass, shifts_dev, delta, ctx->scale_k + SLOT_SOLVE);
        k_b_hop<LF64, SD64, NB64, 1><<<g1, BBS, 0, s>>>(g, U64, SD64{m.x_hi}, SD64{m.t64}, m.f64_stride, bs);
        k_b_resid64<LF64, SD64, NB64><<<g1, BBS, 0, s>>>(g, U64, m.t64, m.x_hi, m.b, m.r_hi, bs);
        k_b_finish<S><<<g1, BBS, 0, s>>>(g.Vh, m.r_hi, spin(m, m.r), spin(m, m.p), m.s_stride, bs, 1, 0, 0);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    static int enqueue_main(stag_ctx ctx, BatchSlot& m, const LF& U, cudaStream_t s, LoopGraph* lg, int use_cond)
    {
        const Geom g = ctx->g;
        const BatchScal bs{m.sc, m.nrhs, m.part, ctx->counters + 1, m.gx, m.cnt_sys};
        const dim3 gb(m.gx, m.nrhs), gn(m.gx, (m.nrhs + NB - 1) / NB);
        k_b_hop<LF, S, NB, 0><<<gn, BBS, 0, s>>>(g, U, spin(m, m.p), spin(m, m.t), m.s_stride, bs);
        k_b_Mp_dot<LF, S, NB><<<gn, BBS, 0, s>>>(g, U, spin(m, m.t), spin(m, m.p), spin(m, m.Ap), m.s_stride, bs);
        k_b_update<S, SX><<<gb, BBS, 0, s>>>(g.Vh, spinx(m, m.xlo), m.sx_stride, spin(m, m.r), spin(m, m.p),
                                             spin(m, m.Ap), m.s_stride, bs, lg ? lg->w : 0, lg ? lg->i : 0, use_cond);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    static int enqueue_reliable(stag_ctx ctx, BatchSlot& m, const LF64& U64, cudaStream_t s, LoopGraph* lg,
                                int use_cond)
    {
        const Geom g = ctx->g;
        const BatchScal bs{m.sc, m.nrhs, m.part, ctx->counters + 1, m.gx, m.cnt_sys};
        // one grid row: the blocks loop over the (usually one or two) systems due
        const dim3 g1(m.gx, 1);
        k_b_accum_x<SX><<<g1, BBS, 0, s>>>(g.Vh, m.x_hi, spinx(m, m.xlo), m.sx_stride, bs);
        k_b_hop<LF64, SD64, NB64, 1><<<g1, BBS, 0, s>>>(g, U64, SD64{m.x_hi}, SD64{m.t64}, m.f64_stride, bs);
        k_b_resid64<LF64, SD64, NB64><<<g1, BBS, 0, s>>>(g, U64, m.t64, m.x_hi, m.b, m.r_hi, bs);
        k_b_finish<S><<<g1, BBS, 0, s>>>(g.Vh, m.r_hi, spin(m, m.r), spin(m, m.p), m.s_stride, bs, 0,
                                         lg ? lg->w : 0, use_cond);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    static int enqueue_p(stag_ctx ctx, BatchSlot& m, cudaStream_t s)
    {
        const BatchScal bs{m.sc, m.nrhs, m.part, ctx->counters + 1, m.gx, m.cnt_sys};
        k_b_p<S><<<dim3(m.gx, m.nrhs), BBS, 0, s>>>(ctx->g.Vh, spin(m, m.r), spin(m, m.p), m.s_stride, bs);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }

    static int run(stag_ctx ctx, BatchSlot& m, const void* lk, const double2* x0, double mass,
                   const double* shifts_dev, const stag_solver_params& prm, double delta, int arith)
    {
        const void* lk64 = nullptr;
        STAG_TRY(ensure_links(ctx, arith, 18, &lk64));
        const LF U{(const typename LF::store*)lk, ctx->g.Vh};
        const LF64 U64{(const typename LF64::store*)lk64, ctx->g.Vh};
        const int maxiter = prm.maxiter > 0 ? prm.maxiter : 100000;
        STAG_TRY(enqueue_start(ctx, m, U64, ctx->stream, x0, prm.tol, maxiter, mass, shifts_dev, delta));
        if (prm.use_graph) {
            if (!m.lg.exec || m.graph_nb != NB || m.graph_arith != arith) {
                LoopGraph& lg = m.lg;
                STAG_TRY(build_loop_graph(
                    ctx->cap_stream, lg, true, [&](cudaStream_t s) { return enqueue_main(ctx, m, U, s, &lg, 1); },
                    [&](cudaStream_t s) { return enqueue_reliable(ctx, m, U64, s, &lg, 1); },
                    [&](cudaStream_t s) { return enqueue_p(ctx, m, s); }));
                m.graph_nb = NB;
                m.graph_arith = arith;
            }
            STAG_CUDA_TRY(cudaGraphLaunch(m.lg.exec, ctx->stream));
        } else {
            const int every = prm.check_every > 0 ? prm.check_every : 25;
            std::vector<CgScalars> hs(m.nrhs);
            for (;;) {
                for (int k = 0; k < every; ++k) {
                    STAG_TRY(enqueue_main(ctx, m, U, ctx->stream, nullptr, 0));
                    STAG_TRY(enqueue_reliable(ctx, m, U64, ctx->stream, nullptr, 0));
                    STAG_TRY(enqueue_p(ctx, m, ctx->stream));
                }
                STAG_CUDA_TRY(cudaMemcpyAsync(hs.data(), m.sc, sizeof(CgScalars) * m.nrhs, cudaMemcpyDeviceToHost,
                                              ctx->stream));
                STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
                bool any = false;
                for (auto& c : hs) any |= !c.done;
                if (!any) break;
            }
        }
        return STAG_OK;
    }
};

template <class S, class SX, class LF, class LF64, class SD64>
static int run_with_nb_arith(stag_ctx ctx, BatchSlot& m, const void* lk, const double2* x0, double mass,
                             const double* shifts_dev, const stag_solver_params& prm, double delta, int nb, int arith)
{
    switch (nb) {
    case 1: return BatchPlan<S, SX, LF, 1, LF64, SD64>::run(ctx, m, lk, x0, mass, shifts_dev, prm, delta, arith);
    case 2: return BatchPlan<S, SX, LF, 2, LF64, SD64>::run(ctx, m, lk, x0, mass, shifts_dev, prm, delta, arith);
    case 4: return BatchPlan<S, SX, LF, 4, LF64, SD64>::run(ctx, m, lk, x0, mass, shifts_dev, prm, delta, arith);
    case 8: return BatchPlan<S, SX, LF, 8, LF64, SD64>::run(ctx, m, lk, x0, mass, shifts_dev, prm, delta, arith);
    case 16: return BatchPlan<S, SX, LF, 16, LF64, SD64>::run(ctx, m, lk, x0, mass, shifts_dev, prm, delta, arith);
    default: set_error("unsupported rhs block %d", nb); return STAG_EINVAL;
    }
}

// The double-precision passes follow prm.f64_arith (IEEE double or double-float).
template <class S, class SX, class LF>
static int run_with_nb(stag_ctx ctx, BatchSlot& m, const void* lk, const double2* x0, double mass,
                       const double* shifts_dev, const stag_solver_params& prm, double delta, int nb)
{
    if (prm.f64_arith == STAG_F64X)
        return run_with_nb_arith<S, SX, LF, LinkFieldDF<18>, SpinorF64asDF>(ctx, m, lk, x0, mass, shifts_dev, prm,
                                                                           delta, nb, STAG_F64X);
    if (prm.f64_arith != STAG_F64) {
        set_error("f64_arith must be STAG_F64 or STAG_F64X");
        return STAG_EINVAL;
    }
    return run_with_nb_arith<S, SX, LF, LF64B, SpinorF64>(ctx, m, lk, x0, mass, shifts_dev, prm, delta, nb, STAG_F64);
}

// The plans for one inner storage each, compiled in their own translation
// units (batched_f64.cu, batched_f32.cu, batched_f16.cu): every rhs block and
// double-pass arithmetic is a set of kernels.
int batched_run_f64(stag_ctx ctx, BatchSlot& m, int recon, const void* lk, const double2* x0, double mass,
                    const double* shifts_dev, const stag_solver_params& prm, double delta, int nb);
int batched_run_f32(stag_ctx ctx, BatchSlot& m, int recon, const void* lk, const double2* x0, double mass,
                    const double* shifts_dev, const stag_solver_params& prm, double delta, int nb);
int batched_run_f16(stag_ctx ctx, BatchSlot& m, int recon, const void* lk, const double2* x0, double mass,
                    const double* shifts_dev, const stag_solver_params& prm, double delta, int nb);

}  // namespace stag
