// cg_df.cuh -- the conjugate-gradient iteration on M = m^2 - D_eo D_oe (+ sigma)
// with the Krylov vectors x, r, p, Ap and t = D_oe p held as double-floats
// (SpinorDF): the steps of cg_kernels.cuh,
//   hop     t  = D_oe p
//   Mp_dot  Ap = (m^2 + sigma) p - D_eo t,  pAp = Re<p,Ap>,  alpha = rr / pAp
//   update  x += alpha p, r -= alpha Ap,    rr' = |r|^2,     beta = rr'/rr
//   p       p  = r + beta p
// in four launches, or in three when the solver's vectors fit in L2: then the
// direction update p = r + beta p of one iteration is applied where the next
// iteration first reads p (the hop reads r and p at its neighbours through
// SpinorDFDir, Mp_dot forms and stores p at its own site; bit for bit the
// values of the separate pass).  On larger lattices the second neighbour
// gather costs more than the pass it saves.  Every per-site operation
// runs in double-float arithmetic on the FP32 pipe (GB300 executes FP64 at
// 1/64 of the FP32 rate).  The scalars alpha, beta and the reductions'
// results stay double in the CgScalars record; beta = 0 after a (re)start,
// where p already holds r.
#pragma once

#include "cg_kernels.cuh"
#include "df64.cuh"

namespace stag {

__device__ __forceinline__ void df_site_dot(DF& d, const Vec3<DF>& a, const Vec3<DF>& b)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        df_mac(d, a.c[c].re, b.c[c].re);
        df_mac(d, a.c[c].im, b.c[c].im);
    }
}

// Fresh start: x = 0, r = p = b (split into double-floats), rr = rr0 = |b|^2.
template <int BS>
__global__ void __launch_bounds__(BS) k_dfcg_start(int Vh, const double2* b, SpinorDF x, SpinorDF r, SpinorDF p,
                                                   CgScalars* sc, double tol, int maxiter, double m2, double sigma,
                                                   double* part, unsigned* cnt)
{
    __shared__ double red[BS / 32];
    __shared__ bool last;
    const int h = blockIdx.x * BS + threadIdx.x;
    DF d(0);
    if (h < Vh) {
        const Vec3<DF> v = SpinorF64asDF{(double2*)b}.load(h);
        Vec3<DF> z;
#pragma unroll
        for (int c = 0; c < 3; ++c) z.c[c].re = z.c[c].im = DF(0);
        x.store(h, z);
        r.store(h, v);
        p.store(h, v);
        df_site_dot(d, v, v);
    }
    const double bs = block_sum_df<BS>(d, red);
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

// The search direction as the first operator pass of an iteration reads it:
// r + beta p, formed at load time from the stored r and p with the
// previous iteration's beta (bit for bit the value Mp_dot then stores).
struct SpinorDFDir {
    typedef DF real;
    SpinorDF r, p;
    DF beta;
    __device__ __forceinline__ Vec3<DF> load(int h) const
    {
        const Vec3<DF> rv = r.load(h), pv = p.load(h);
        Vec3<DF> o;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.c[c].re = df_fma(beta, pv.c[c].re, rv.c[c].re);
            o.c[c].im = df_fma(beta, pv.c[c].im, rv.c[c].im);
        }
        return o;
    }
};

// t = D_oe (r + beta p) on odd sites (p itself is updated by Mp_dot).
template <class LF, int BS>
__global__ void __launch_bounds__(BS, (OpMinBlocksBS<LF, SpinorDF, BS>::value)) k_dfcg_hop(Geom g, LF U, SpinorDF r,
                                                                                       SpinorDF p, SpinorDF t,
                                                                                       const CgScalars* sc)
{
    if (sc->done) return;
    const int h = blockIdx.x * BS + threadIdx.x;
    if (h >= g.Vh) return;
    const SpinorDFDir in{r, p, split_double(sc->beta)};
    t.store(h, dslash_site(g, 1, h, U, in));
}

// DIR: p = r + beta p (stored) first.  Ap = (m^2 + sigma) p - D_eo t and the
// block partials of Re<p, Ap>; the last block sets alpha (or flags a breakdown).
template <class LF, int BS, bool DIR>
__global__ void __launch_bounds__(BS, (OpMinBlocksS<LF, SpinorDF>::value)) k_dfcg_Mp_dot(Geom g, LF U, SpinorDF t, SpinorDF r,
                                                                          SpinorDF p, SpinorDF Ap, CgScalars* sc,
                                                                          double* part, unsigned* cnt, GridSum gs)
{
    __shared__ double red[BS / 32];
    if (sc->done) return;
    const DF m2s = split_double(sc->m2 + sc->sigma);
    const int h = blockIdx.x * BS + threadIdx.x;
    DF d(0);
    if (h < g.Vh) {
        const Vec3<DF> Dt = dslash_site(g, 0, h, U, t);
        Vec3<DF> pv;
        if (DIR) {
            pv = SpinorDFDir{r, p, split_double(sc->beta)}.load(h);
            p.store(h, pv);
        } else {
            pv = p.load(h);
        }
        Vec3<DF> a;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a.c[c].re = df_fma(m2s, pv.c[c].re, df_neg(Dt.c[c].re));
            a.c[c].im = df_fma(m2s, pv.c[c].im, df_neg(Dt.c[c].im));
        }
        Ap.store(h, a);
        df_site_dot(d, pv, a);
    }
    const double bs = block_sum_df<BS>(d, red);
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

// chunk_partials (common.cuh) for double-float site values: each warp sums its
// 32 sites in double-float by a butterfly, converts to double, and the chunk
// adds its four warp sums in ascending order.
template <int BS, int SPT>
__device__ __forceinline__ void chunk_partials_df(const DF* v, double* part, int nchunks, double* smem)
{
    constexpr int NW = BS / 32, NCH = BS * SPT / RCHUNK;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        DF x = v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const DF y(__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o));
            x = df_add(x, y);
        }
        if (lane == 0) smem[j * NW + w] = df_to_double(x);
    }
    __syncthreads();
    if (threadIdx.x < NCH) {
        const int c = threadIdx.x, ch = blockIdx.x * NCH + c;
        const double x = ((smem[4 * c] + smem[4 * c + 1]) + smem[4 * c + 2]) + smem[4 * c + 3];
        if (ch < nchunks) part[ch] = x;
    }
    __syncthreads();
}

// x += alpha p, r -= alpha Ap, rr' = |r|^2 over SPT sites per thread (partials
// in 128-site chunks: every launch shape gives the same bits); the last block
// sets beta, the convergence flag and the graph loop's condition.
template <int BS, int SPT>
__global__ void __launch_bounds__(BS) k_dfcg_update(int Vh, SpinorDF x, SpinorDF r, SpinorDF p, SpinorDF Ap,
                                                    CgScalars* sc, double* part, unsigned* cnt, GridSum gs,
                                                    cudaGraphConditionalHandle cond, int use_cond)
{
    __shared__ double red[BS / 32 * SPT];
    if (sc->done) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
        return;
    }
    const DF alpha = split_double(sc->alpha), nalpha = df_neg(alpha);
    DF d[SPT];
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int h = (blockIdx.x * SPT + j) * BS + threadIdx.x;
        d[j] = DF(0);
        if (h < Vh) {
            Vec3<DF> xv = x.load_rw(h), rv = r.load_rw(h);
            const Vec3<DF> pv = p.load(h), av = Ap.load(h);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xv.c[c].re = df_fma(alpha, pv.c[c].re, xv.c[c].re);
                xv.c[c].im = df_fma(alpha, pv.c[c].im, xv.c[c].im);
                rv.c[c].re = df_fma(nalpha, av.c[c].re, rv.c[c].re);
                rv.c[c].im = df_fma(nalpha, av.c[c].im, rv.c[c].im);
            }
            x.store(h, xv);
            r.store(h, rv);
            df_site_dot(d[j], rv, rv);
        }
    }
    const int nch = (Vh + RCHUNK - 1) / RCHUNK;
    chunk_partials_df<BS, SPT>(d, part, nch, red);
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

// p = r + beta p as a pass of its own (the four-launch iteration), SPT sites per thread
template <int BS, int SPT>
__global__ void __launch_bounds__(BS) k_dfcg_p(int Vh, SpinorDF r, SpinorDF p, const CgScalars* sc)
{
    if (sc->done) return;
    const DF beta = split_double(sc->beta);
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int h = (blockIdx.x * SPT + j) * BS + threadIdx.x;
        if (h >= Vh) return;
        const Vec3<DF> rv = r.load(h);
        Vec3<DF> pv = p.load_rw(h);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pv.c[c].re = df_fma(beta, pv.c[c].re, rv.c[c].re);
            pv.c[c].im = df_fma(beta, pv.c[c].im, rv.c[c].im);
        }
        p.store(h, pv);
    }
}

// r = b - ((m^2 + sigma) x - D_eo t)  (t = D_oe x), rr_true = |r|^2.  The
// operator pass runs in double-float; the epilogue (once per solve pass, not
// per iteration) in IEEE double on x converted exactly as the solver returns
// it, so that rr_true is the residual of the returned solution to double
// rounding.  r is stored back as double-floats for a restart.
template <class LF, int BS>
__global__ void __launch_bounds__(BS, (OpMinBlocksS<LF, SpinorDF>::value)) k_dfcg_true_resid(Geom g, LF U, SpinorDF t, SpinorDF x,
                                                                              const double2* b, SpinorDF r,
                                                                              CgScalars* sc, double* part,
                                                                              unsigned* cnt)
{
    __shared__ double red[BS / 32];
    __shared__ bool last;
    const double m2s = sc->m2 + sc->sigma;
    const int h = blockIdx.x * BS + threadIdx.x;
    double d = 0.0;
    if (h < g.Vh) {
        const Vec3<double> Dt = vconv<double>(dslash_site(g, 0, h, U, t));
        const Vec3<DF> xv = x.load(h);
        Vec3<DF> rv;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 bv = b[(size_t)h * 3 + c];
            const double re = bv.x - fma(m2s, df_to_double(xv.c[c].re), -Dt.c[c].re);
            const double im = bv.y - fma(m2s, df_to_double(xv.c[c].im), -Dt.c[c].im);
            rv.c[c].re = split_double(re);
            rv.c[c].im = split_double(im);
            d = fma(re, re, d);
            d = fma(im, im, d);
        }
        r.store(h, rv);
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
