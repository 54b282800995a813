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
#include <type_traits>
#include <vector>

#include "batched.cuh"
#include "df64.cuh"
#include "multi_tile.cuh"
#include "cg_kernels.cuh"
#include "graph.h"
#include "tune.h"
#include "workspace.h"

namespace stag {

constexpr int BBS = 128;      // threads (sites) per block of every batched kernel

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

// mask_active of the n <= 32 systems kb ... kb + n - 1 with one load per
// lane and a ballot (every warp of a block forms the same mask; all lanes of
// the warp must call it).
__device__ __forceinline__ unsigned mask_active_ballot(const BatchScal& b, int kb, int n)
{
    const int lane = threadIdx.x & 31;
    const bool a = lane < n && kb + lane < b.nrhs && active(b.sc[kb + lane]);
    return __ballot_sync(0xffffffffu, a);
}

// ------------------------------------------------------------- start

// x_hi = x0 (or 0), xlo = 0, rr0 = |b|^2 per system; every system marked for a
// residual recomputation.  grid (gx, nrhs).
// b holds the normalised right-hand sides 2^-k_k B_k; x0 (unnormalised
// initial guesses) is brought to the same scale.
// x_df (double-float arithmetic only, else NULL) keeps x_hi split into
// double-float pairs, the storage the reliable updates' operator reads.
template <class SX>
__global__ void __launch_bounds__(BBS) k_b_init(int Vh, const double2* b, const double2* x0, double2* x_hi, SX xlo,
                                                size_t sx_stride, BatchScal bs, double tol, int maxiter, double m2,
                                                const double* shifts, double delta, const int* kexp, float4* x_df)
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
            double2 xv = make_double2(0.0, 0.0);
            if (x0) {
                const double2 v = x0[o + c];
                xv = make_double2(scalbn(v.x, -kexp[k]), scalbn(v.y, -kexp[k]));
            }
            x_hi[o + c] = xv;
            if (x_df) {
                const DF re = split_double(xv.x), im = split_double(xv.y);
                x_df[o + c] = make_float4(re.hi, re.lo, im.hi, im.lo);
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
    real d[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) d[k] = real(0);
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

// ----------------------------------------- tile kernels (multi_tile.cuh)

// t_k = D_oe p_k for the active systems, links staged per tile and shared by
// the block's G NBT systems.  grid (tiles, ceil(nrhs / (G NBT))).
template <class LF, class S, int G, int NBT>
__global__ void __launch_bounds__(32 * TileSW<G>::value * G, TileMinBlocks<32 * TileSW<G>::value * G, NBT>::value)
    k_tile_b_hop(Geom g, LF U, S in, S out, size_t stride, BatchScal bs)
{
    __shared__ uint4 sm[TileSmem<LF, G>::value / 16];
    constexpr int SW = TileSW<G>::value, TS = 32 * SW;
    const int kb = blockIdx.y * G * NBT;
    const unsigned bmask = mask_active_ballot(bs, kb, G * NBT);
    if (!bmask) return;   // uniform over the block
    const int h = blockIdx.x * TS + threadIdx.x % TS;
    const int k0 = kb + (threadIdx.x / TS) * NBT;
    const unsigned mask = (bmask >> ((threadIdx.x / TS) * NBT)) & ((1u << NBT) - 1u);
    SiteNbrs s;
    site_nbrs(g, 1, h < g.Vh ? h : g.Vh - 1, s);
    Vec3<typename LF::real> acc[NBT];
    tile_site_multi<LF, S, G, NBT>(g, 1, h, s, U, in, stride, k0, mask, sm, acc);
    if (h >= g.Vh) return;
#pragma unroll
    for (int k = 0; k < NBT; ++k)
        if (mask & (1u << k)) out.at(k0 + k, stride).store(h, acc[k]);
}

// Ap_k = (m^2 + sigma_k) p_k - D_eo t_k and the partial sums of <p_k, Ap_k>,
// as k_b_Mp_dot with the tile operator.  The block's partial of system k is
// the sum over its SW site warps of the warp sums (fixed order), stored at
// part[k * tiles + tile]; k_b_alpha forms the totals (no arrival counting
// here: with 16 systems per block and thousands of tiles, the per-block
// atomics and the serial final sums of the last arrivers cost more than the
// operator).  grid (tiles, ceil(nrhs / (G NBT))).
template <class LF, class S, int G, int NBT>
__global__ void __launch_bounds__(32 * TileSW<G>::value * G, TileMinBlocks<32 * TileSW<G>::value * G, NBT>::value)
    k_tile_b_Mp_dot(Geom g, LF U, S t, S p, S Ap, size_t stride, BatchScal bs)
{
    constexpr int SW = TileSW<G>::value, TS = 32 * SW, NT = TS * G, NW = NT / 32;
    __shared__ uint4 sm[TileSmem<LF, G>::value / 16];
    __shared__ double wsum[NW * NBT];
    typedef typename S::real real;
    const int kb = blockIdx.y * G * NBT;
    const unsigned bmask = mask_active_ballot(bs, kb, G * NBT);
    if (!bmask) return;   // uniform over the block
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = blockIdx.x * TS + threadIdx.x % TS;
    const int k0 = kb + (threadIdx.x / TS) * NBT;
    const unsigned mask = (bmask >> ((threadIdx.x / TS) * NBT)) & ((1u << NBT) - 1u);
    SiteNbrs s;
    site_nbrs(g, 0, h < g.Vh ? h : g.Vh - 1, s);
    Vec3<real> acc[NBT];
    tile_site_multi<LF, S, G, NBT>(g, 0, h, s, U, t, stride, k0, mask, sm, acc);
    real d[NBT];
#pragma unroll
    for (int k = 0; k < NBT; ++k) d[k] = real(0);
    if (h < g.Vh) {
#pragma unroll
        for (int k = 0; k < NBT; ++k) {
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
    if constexpr (std::is_same<real, float>::value && (NBT & (NBT - 1)) == 0) {
        const double x = warp_sum_n<NBT>(d);
        const int k = lane / (32 / NBT);
        if (lane == warp_sum_n_lane<NBT>(k)) wsum[w * NBT + k] = x;
    } else {
#pragma unroll
        for (int k = 0; k < NBT; ++k) {
            const double x = warp_sum(d[k]);
            if (lane == 0) wsum[w * NBT + k] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x < G * NBT && (bmask & (1u << threadIdx.x))) {
        const int gi = threadIdx.x / NBT, k = threadIdx.x % NBT;
        double x = 0.0;
#pragma unroll
        for (int sw = 0; sw < SW; ++sw) x += wsum[(gi * SW + sw) * NBT + k];
        bs.part[(size_t)(kb + threadIdx.x) * bs.gx + blockIdx.x] = x;
    }
}

// pAp_k = the sum of system k's bs.gx partials (fixed order), alpha_k =
// rr_k / pAp_k, or a breakdown.  One block per system (grid nrhs).
template <int BS>
__global__ void __launch_bounds__(BS) k_b_alpha(BatchScal bs)
{
    __shared__ double red[BS / 32];
    const int k = blockIdx.x;
    if (!active(bs.sc[k])) return;
    const double pAp = sum_partials<BS>(bs.part + (size_t)k * bs.gx, bs.gx, red);
    if (threadIdx.x == 0) {
        CgScalars& c = bs.sc[k];
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

// ------------------------------------- reliable updates with link tiles
//
// The double-precision passes of a reliable update, for every system due,
// with the links of a tile of 32 sites staged once for up to 16 systems
// (multi_tile.cuh, G = 16 groups of one system): the systems' updates are
// gathered into the same iterations (k_b_update), so that one pass over the
// links serves all of them.  grid (tiles, ceil(nrhs / 16)).
constexpr int RG = 16;

// t64_k = D_oe x_hi_k for the systems due.
template <class LF, class SD>
__global__ void __launch_bounds__(32 * RG, 2) k_tile_b_hop64(Geom g, LF U, SD in, SD out, size_t stride,
                                                             BatchScal bs)
{
    __shared__ uint4 sm[TileSmem<LF, RG>::value / 16];
    const int kb = blockIdx.y * RG;
    if (!mask_updating<RG>(bs, kb)) return;   // uniform over the block
    const int h = blockIdx.x * 32 + threadIdx.x % 32;
    const int k0 = kb + threadIdx.x / 32;
    const unsigned mask = mask_updating<1>(bs, k0);
    SiteNbrs s;
    site_nbrs(g, 1, h < g.Vh ? h : g.Vh - 1, s);
    Vec3<typename LF::real> acc[1];
    tile_site_multi<LF, SD, RG, 1>(g, 1, h, s, U, in, stride, k0, mask, sm, acc);
    if (h < g.Vh && mask) out.at(k0, stride).store(h, acc[0]);
}

// r_hi_k = b_k - ((m^2 + sigma_k) x_hi_k - D_eo t64_k) in double and the
// tile's partial of |r_hi_k|^2 at part[k * tiles + tile]; k_b_rrtrue sums them.
template <class LF, class SD>
__global__ void __launch_bounds__(32 * RG, 2) k_tile_b_resid64(Geom g, LF U, SD t, const double2* x_hi,
                                                               const double2* b, double2* r_hi, BatchScal bs)
{
    __shared__ uint4 sm[TileSmem<LF, RG>::value / 16];
    const int kb = blockIdx.y * RG;
    if (!mask_updating<RG>(bs, kb)) return;   // uniform over the block
    const int lane = threadIdx.x % 32;
    const int h = blockIdx.x * 32 + lane;
    const int k0 = kb + threadIdx.x / 32;
    const unsigned mask = mask_updating<1>(bs, k0);
    const size_t stride = (size_t)g.Vh * 3 * sizeof(double2);
    SiteNbrs s;
    site_nbrs(g, 0, h < g.Vh ? h : g.Vh - 1, s);
    Vec3<typename LF::real> acc[1];
    tile_site_multi<LF, SD, RG, 1>(g, 0, h, s, U, t, stride, k0, mask, sm, acc);
    double d = 0.0;
    if (h < g.Vh && mask) {
        const double m2s = bs.sc[k0].m2 + bs.sc[k0].sigma;
        const size_t o = ((size_t)k0 * g.Vh + h) * 3;
        const Vec3<double> Dt = vconv<double>(acc[0]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 xv = x_hi[o + c], bv = b[o + c];
            const double re = bv.x - fma(m2s, xv.x, -Dt.c[c].re);
            const double im = bv.y - fma(m2s, xv.y, -Dt.c[c].im);
            r_hi[o + c] = make_double2(re, im);
            d = fma(re, re, d);
            d = fma(im, im, d);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0 && mask) bs.part[(size_t)k0 * bs.gx + blockIdx.x] = d;
}

// rr_true_k = the sum of system k's bs.gx partials (fixed order), systems due.
template <int BS>
__global__ void __launch_bounds__(BS) k_b_rrtrue(BatchScal bs)
{
    __shared__ double red[BS / 32];
    const int k = blockIdx.x;
    if (!updating(bs.sc[k])) return;
    const double rr = sum_partials<BS>(bs.part + (size_t)k * bs.gx, bs.gx, red);
    if (threadIdx.x == 0) bs.sc[k].rr_true = rr;
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
    real d = real(0);
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
    volatile CgScalars* vs = bs.sc;
    int any_rel = 0;
    for (int kk = 0; kk < bs.nrhs; ++kk) any_rel |= !vs[kk].done && vs[kk].reliable;
    // When one system is due, every active system takes its reliable update
    // in the same pass: the double-precision passes share each link load
    // among all systems due (k_tile_b_hop64 / k_tile_b_resid64), so that a few
    // gathered passes replace one pass every iteration or two for whichever
    // system happens to be due.  (An update replaces the iterated residual by
    // the true one and keeps the direction; doing it earlier than needed
    // costs no accuracy.)
    if (any_rel)
        for (int kk = 0; kk < bs.nrhs; ++kk)
            if (!vs[kk].done) vs[kk].reliable = 1;
    if (use_cond) {
        cudaGraphSetConditional(ih, any_rel ? 1 : 0);
        cudaGraphSetConditional(wh, 1);
    }
}

// x_hi_k += xlo_k, xlo_k = 0 for systems due a reliable update.  grid (gx, 1):
// each block loops over the systems and skips those not due.
template <class SX>
__global__ void __launch_bounds__(BBS) k_b_accum_x(int Vh, double2* x_hi, SX xlo, size_t sx_stride, BatchScal bs,
                                                   float4* x_df)
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
            if (x_df) {
                const DF re = split_double(xv.x), im = split_double(xv.y);
                x_df[o + c] = make_float4(re.hi, re.lo, im.hi, im.lo);
            }
            z.c[c].re = z.c[c].im = 0;
        }
        xk.store(h, z);
    }
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
// double-float (LinkFieldDF<18>, SpinorDF on double-float copies of the vectors).
// CFG: the multi-vector configuration of the iteration's operator passes
// (multi_tile.cuh): G = 1 register-blocked with NBT right-hand sides per
// thread, G > 1 link tiles shared by G NBT right-hand sides.
template <class S, class SX, class LF, int CFG, class LF64, class SD64>
struct BatchPlan {
    static constexpr int G = mcfg_G(CFG), NBT = mcfg_NBT(CFG);
    static S spin(const BatchSlot& m, void* buf) { return m.template spinor<S>(buf); }
    static SX spinx(const BatchSlot& m, void* buf) { return m.template spinor<SX>(buf); }

    // the reliable update's double-precision operator passes (link tiles
    // shared by up to 16 systems due) and the true residual norms
    // SD64: the operator's vector storage, double (IEEE) or double-float pairs
    // (x_df, a split copy of x_hi kept by k_b_init / k_b_accum_x, so that no
    // neighbour load splits doubles)
    static constexpr bool DFX = std::is_same<SD64, SpinorDF>::value;
    static SD64 view64(void* p) { return SD64{(typename std::conditional<DFX, float4, double2>::type*)p}; }
    static float4* xdf(const BatchSlot& m) { return DFX ? (float4*)m.x_df : nullptr; }
    static int enqueue_hop_resid64(stag_ctx ctx, BatchSlot& m, const LF64& U64, cudaStream_t s)
    {
        const Geom g = ctx->g;
        const int tiles = (g.Vh + 31) / 32;
        const BatchScal bst{m.sc, m.nrhs, m.part, ctx->counters + 1, tiles, m.cnt_sys};
        const dim3 gt(tiles, (m.nrhs + RG - 1) / RG);
        k_tile_b_hop64<LF64, SD64><<<gt, 32 * RG, 0, s>>>(g, U64, view64(DFX ? m.x_df : m.x_hi), view64(m.t64),
                                                          m.f64_stride, bst);
        k_tile_b_resid64<LF64, SD64><<<gt, 32 * RG, 0, s>>>(g, U64, view64(m.t64), m.x_hi, m.b, m.r_hi, bst);
        k_b_rrtrue<256><<<m.nrhs, 256, 0, s>>>(bst);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    static int enqueue_start(stag_ctx ctx, BatchSlot& m, const LF64& U64, cudaStream_t s, const double2* x0,
                             double tol, int maxiter, double mass, const double* shifts_dev, double delta)
    {
        const Geom g = ctx->g;
        const BatchScal bs{m.sc, m.nrhs, m.part, ctx->counters + 1, m.gx, m.cnt_sys};
        const dim3 gb(m.gx, m.nrhs), g1(m.gx, 1);
        k_b_init<SX><<<gb, BBS, 0, s>>>(g.Vh, m.b, x0, m.x_hi, spinx(m, m.xlo), m.sx_stride, bs, tol, maxiter,
                                        mass * mass, shifts_dev, delta, ctx->scale_k + SLOT_SOLVE, xdf(m));
        STAG_TRY(enqueue_hop_resid64(ctx, m, U64, s));
        k_b_finish<S><<<g1, BBS, 0, s>>>(g.Vh, m.r_hi, spin(m, m.r), spin(m, m.p), m.s_stride, bs, 1, 0, 0);
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    static int enqueue_main(stag_ctx ctx, BatchSlot& m, const LF& U, cudaStream_t s, LoopGraph* lg, int use_cond)
    {
        const Geom g = ctx->g;
        const BatchScal bs{m.sc, m.nrhs, m.part, ctx->counters + 1, m.gx, m.cnt_sys};
        const dim3 gb(m.gx, m.nrhs);
        if constexpr (G == 1) {
            const dim3 gn(m.gx, (m.nrhs + NBT - 1) / NBT);
            k_b_hop<LF, S, NBT, 0><<<gn, BBS, 0, s>>>(g, U, spin(m, m.p), spin(m, m.t), m.s_stride, bs);
            k_b_Mp_dot<LF, S, NBT><<<gn, BBS, 0, s>>>(g, U, spin(m, m.t), spin(m, m.p), spin(m, m.Ap), m.s_stride,
                                                      bs);
        } else {
            constexpr int TS = 32 * TileSW<G>::value;
            const int tiles = (g.Vh + TS - 1) / TS;
            const BatchScal bst{m.sc, m.nrhs, m.part, ctx->counters + 1, tiles, m.cnt_sys};
            const dim3 gt(tiles, (m.nrhs + G * NBT - 1) / (G * NBT));
            k_tile_b_hop<LF, S, G, NBT><<<gt, TS * G, 0, s>>>(g, U, spin(m, m.p), spin(m, m.t), m.s_stride, bst);
            k_tile_b_Mp_dot<LF, S, G, NBT><<<gt, TS * G, 0, s>>>(g, U, spin(m, m.t), spin(m, m.p), spin(m, m.Ap),
                                                                 m.s_stride, bst);
            k_b_alpha<256><<<m.nrhs, 256, 0, s>>>(bst);
        }
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
        k_b_accum_x<SX><<<g1, BBS, 0, s>>>(g.Vh, m.x_hi, spinx(m, m.xlo), m.sx_stride, bs, xdf(m));
        STAG_TRY(enqueue_hop_resid64(ctx, m, U64, s));
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
        STAG_TRY(m.tg ? ensure_links_tg(ctx, arith, 18, &lk64) : ensure_links(ctx, arith, 18, &lk64));
        const LF U{(const typename LF::store*)lk, ctx->g.Vh, m.tg};
        const LF64 U64{(const typename LF64::store*)lk64, ctx->g.Vh, m.tg};
        const int maxiter = prm.maxiter > 0 ? prm.maxiter : 100000;
        STAG_TRY(enqueue_start(ctx, m, U64, ctx->stream, x0, prm.tol, maxiter, mass, shifts_dev, delta));
        if (prm.use_graph) {
            if (!m.lg.exec || m.graph_nb != CFG || m.graph_arith != arith || m.graph_tg != m.tg) {
                LoopGraph& lg = m.lg;
                STAG_TRY(build_loop_graph(
                    ctx->cap_stream, lg, true, [&](cudaStream_t s) { return enqueue_main(ctx, m, U, s, &lg, 1); },
                    [&](cudaStream_t s) { return enqueue_reliable(ctx, m, U64, s, &lg, 1); },
                    [&](cudaStream_t s) { return enqueue_p(ctx, m, s); }));
                m.graph_nb = CFG;
                m.graph_arith = arith;
                m.graph_tg = m.tg;
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
                             const double* shifts_dev, const stag_solver_params& prm, double delta, int cfg, int arith)
{
#define STAG_BATCH_CFG(Gv, Nv)                                                                              \
    case mcfg(Gv, Nv):                                                                                      \
        return BatchPlan<S, SX, LF, mcfg(Gv, Nv), LF64, SD64>::run(ctx, m, lk, x0, mass, shifts_dev, prm, delta, \
                                                                   arith)
    switch (cfg) {
        STAG_BATCH_CFG(1, 1);
        STAG_BATCH_CFG(1, 2);
        STAG_BATCH_CFG(1, 4);
        STAG_BATCH_CFG(1, 8);
        STAG_BATCH_CFG(1, 16);
    default: break;
    }
    if constexpr (TileOK<LF>::value) {
        switch (cfg) {
            STAG_BATCH_CFG(2, 1);
            STAG_BATCH_CFG(2, 2);
            STAG_BATCH_CFG(4, 1);
            STAG_BATCH_CFG(2, 4);
            STAG_BATCH_CFG(4, 2);
            STAG_BATCH_CFG(8, 1);
            STAG_BATCH_CFG(2, 8);
            STAG_BATCH_CFG(4, 4);
            STAG_BATCH_CFG(8, 2);
            STAG_BATCH_CFG(16, 1);
        default: break;
        }
    }
#undef STAG_BATCH_CFG
    set_error("unsupported multi-vector configuration (%d groups x %d)", mcfg_G(cfg), mcfg_NBT(cfg));
    return STAG_EINVAL;
}

// The double-precision passes follow prm.f64_arith (IEEE double or double-float).
template <class S, class SX, class LF>
static int run_with_nb(stag_ctx ctx, BatchSlot& m, const void* lk, const double2* x0, double mass,
                       const double* shifts_dev, const stag_solver_params& prm, double delta, int nb)
{
    if (prm.f64_arith == STAG_F64X)
        return run_with_nb_arith<S, SX, LF, LinkFieldDF<18>, SpinorDF>(ctx, m, lk, x0, mass, shifts_dev, prm,
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
