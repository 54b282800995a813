// cg_kernels.cuh -- the kernels of one conjugate-gradient iteration on
// M = m^2 - D_eo D_oe (+ sigma), for any spinor storage S and link field LF.
//
// One iteration is four launches:
//   hop     t  = D_oe p                                   (odd sites)
//   Mp_dot  Ap = (m^2 + sigma) p - D_eo t, pAp = Re<p,Ap>,  alpha = rr / pAp
//   update  x += alpha p, r -= alpha Ap, rr' = |r|^2,      beta = rr'/rr
//   p       p  = r + beta p
// Scalars live in a CgScalars record in device memory; each reduction ends in
// the last block to arrive, which sums the per-block partials in a fixed order
// (deterministic) and updates the record.  Once the record says done, every
// kernel of the iteration returns at once, and the update kernel clears the
// condition of the enclosing CUDA-graph loop.
#pragma once

#include "ctx.h"
#include "df64.cuh"
#include "dslash.cuh"

namespace stag {

// Site contribution to a real inner product in the storage's arithmetic
// (float sites: six terms in float; the block sums of float values run in
// float-float and end in double, df64.cuh).
template <typename T>
__device__ __forceinline__ T site_dot(const Vec3<T>& a, const Vec3<T>& b)
{
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s = fma(a.c[c].re, b.c[c].re, s);
        s = fma(a.c[c].im, b.c[c].im, s);
    }
    return s;
}

// Minimum resident blocks of an operator kernel of BS threads: the 128-thread
// bound of the link field (OpMinBlocksS) kept at the same registers per thread.
template <class LF, class S, int BS> struct OpMinBlocksBS {
    static constexpr int v = OpMinBlocksS<LF, S>::value * 128 / BS;
    static constexpr int value = v > 0 ? v : 1;
};

// MODE: links and/or neighbour spinors staged in shared memory
// (dslash_site_staged, STAGE_LINKS | STAGE_SPINORS), the same result bit for bit.
template <class LF, class S, int BS, int MODE = 0>
__global__ void __launch_bounds__(BS, (OpMinBlocksBS<LF, S, BS>::value)) k_hop_guarded(Geom g, int p, LF U, S in, S out, const CgScalars* sc)
{
    if (sc->done) return;
    const int h = blockIdx.x * BS + threadIdx.x;
    if (h >= g.Vh) return;
    if constexpr (MODE != 0) {
        __shared__ uint4 st[StageWords<LF, S, BS, MODE>::value];
        out.store(h, dslash_site_staged<BS, MODE>(g, p, h, U, in, st));
    } else {
        out.store(h, dslash_site(g, p, h, U, in));
    }
}

// SD is the storage view the operator reads t through (S itself, or a
// double-float view of double storage); the epilogue runs in S's arithmetic.
template <class LF, class SD, class S, int BS, int MODE = 0>
__global__ void __launch_bounds__(BS, (OpMinBlocksS<LF, SD>::value)) k_Mp_dot(Geom g, LF U, SD t, S p, S Ap, CgScalars* sc,
                                               double* part, unsigned* cnt, GridSum gs)
{
    __shared__ double red[BS / 32];
    __shared__ uint4 st[StageWords<LF, SD, BS, MODE>::value];
    if (sc->done) return;
    typedef typename S::real real;
    const real m2s = (real)(sc->m2 + sc->sigma);
    const int h = blockIdx.x * BS + threadIdx.x;
    real d = real(0);
    if (h < g.Vh) {
        const Vec3<real> Dt = vconv<real>(dslash_site_sel<BS, MODE>(g, 0, h, U, t, st));
        const Vec3<real> pv = p.load(h);
        Vec3<real> a;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a.c[c].re = fma(m2s, pv.c[c].re, -Dt.c[c].re);
            a.c[c].im = fma(m2s, pv.c[c].im, -Dt.c[c].im);
        }
        Ap.store(h, a);
        d = site_dot(pv, a);
    }
    const double bs = block_sum<BS>(d, red);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
    double pAp;
    if (!grid_sum_finish<BS>(part, gridDim.x, blockIdx.x, 1, gs, cnt, red, &pAp)) return;
    if (threadIdx.x == 0) {
        sc->pAp = pAp;
        if (!(pAp > 0.0) || !isfinite(pAp)) {
            sc->status = STAG_BREAKDOWN;
            sc->done = 1;
        } else {
            sc->alpha = sc->rr / pAp;
        }
    }
}

// x += alpha p, r -= alpha Ap, rr' = |r|^2 over SPT sites per thread (the
// partials in 128-site chunks, common.cuh: every launch shape gives the same
// bits); the last block sets beta, the convergence flag and the graph loop's
// condition.
template <class S, int BS, int SPT>
__global__ void __launch_bounds__(BS) k_cg_update(int Vh, S x, S r, S p, S Ap, CgScalars* sc, double* part,
                                                  unsigned* cnt, GridSum gs, cudaGraphConditionalHandle cond,
                                                  int use_cond)
{
    __shared__ double red[BS / 32 * SPT];
    if (sc->done) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
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
            Vec3<real> xv = x.load_rw(h), rv = r.load_rw(h);
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
        sc->beta = rr_new / sc->rr;
        sc->rr = rr_new;
        sc->iter += 1;
        if (!isfinite(rr_new)) {
            sc->status = STAG_BREAKDOWN;
            sc->done = 1;
        } else if (rr_new <= sc->tol2 || sc->iter >= sc->maxiter) {
            sc->done = 1;
        }
        if (use_cond) cudaGraphSetConditional(cond, sc->done ? 0 : 1);
    }
}

// p = r + beta p over SPT sites per thread
template <class S, int BS, int SPT>
__global__ void __launch_bounds__(BS) k_cg_p(int Vh, S r, S p, const CgScalars* sc)
{
    if (sc->done) return;
    typedef typename S::real real;
    const real beta = (real)sc->beta;
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int h = (blockIdx.x * SPT + j) * BS + threadIdx.x;
        if (h >= Vh) return;
        const Vec3<real> rv = r.load(h);
        Vec3<real> pv = p.load_rw(h);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pv.c[c].re = fma(beta, pv.c[c].re, rv.c[c].re);
            pv.c[c].im = fma(beta, pv.c[c].im, rv.c[c].im);
        }
        p.store(h, pv);
    }
}

// Candidate launch shapes of the vector kernels (vcfg codes), the first the default.
inline const int* vec_cfgs(int* n)
{
    static const int c[] = {vcfg(256, 1), vcfg(128, 1), vcfg(256, 2), vcfg(128, 2)};
    *n = 4;
    return c;
}

template <class LF, class SD, class S, int BS>
__global__ void __launch_bounds__(BS) k_xpay_hop(Geom g, LF U, SD t, S x, S out, double a)
{
    // out = a x - D_eo t  on even sites
    typedef typename S::real real;
    const int h = blockIdx.x * BS + threadIdx.x;
    if (h >= g.Vh) return;
    const Vec3<real> Dt = vconv<real>(dslash_site(g, 0, h, U, t));
    const Vec3<real> xv = x.load(h);
    Vec3<real> o;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        o.c[c].re = fma((real)a, xv.c[c].re, -Dt.c[c].re);
        o.c[c].im = fma((real)a, xv.c[c].im, -Dt.c[c].im);
    }
    out.store(h, o);
}

// out = D_{p,1-p} in; with guard set, only when a reliable update is due.
template <class LF, class S, int BS>
__global__ void __launch_bounds__(BS, (OpMinBlocksS<LF, S>::value)) k_hop(Geom g, int p, LF U, S in, S out, const CgScalars* sc, int guard)
{
    if (guard && !sc->reliable) return;
    const int h = blockIdx.x * BS + threadIdx.x;
    if (h >= g.Vh) return;
    out.store(h, dslash_site(g, p, h, U, in));
}

// r = b - (m^2 + sigma) x + D_eo t  (t = D_oe x), rr_true = |r|^2, double precision.
// With guard set, only when a reliable update is due.
template <class LF, class SD, int BS>
__global__ void __launch_bounds__(BS) k_true_resid_f64(Geom g, LF U, SD t, const double2* x,
                                                       const double2* b, double2* r, CgScalars* sc, double* part,
                                                       unsigned* cnt, int guard)
{
    __shared__ double red[BS / 32];
    __shared__ bool last;
    if (guard && !sc->reliable) return;
    const int h = blockIdx.x * BS + threadIdx.x;
    double d = 0.0;
    const double m2s = sc->m2 + sc->sigma;
    if (h < g.Vh) {
        const Vec3<double> Dt = vconv<double>(dslash_site(g, 0, h, U, t));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 xv = x[(size_t)h * 3 + c], bv = b[(size_t)h * 3 + c];
            const double re = bv.x - fma(m2s, xv.x, -Dt.c[c].re);
            const double im = bv.y - fma(m2s, xv.y, -Dt.c[c].im);
            r[(size_t)h * 3 + c] = make_double2(re, im);
            d = fma(re, re, d);
            d = fma(im, im, d);
        }
    }
    const double bs = block_sum<BS>(d, red);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
    if (!arrive_last(cnt, &last)) return;
    const double rr = sum_partials<BS>(part, gridDim.x, red);
    if (threadIdx.x == 0) {
        *cnt = 0;
        sc->rr_true = rr;
    }
}

}  // namespace stag
