// tgauge.cuh -- the double-float operator on links in temporal gauge.
//
// The paper stores 6 links per site by fixing the temporal gauge: with
// g(x, t = 0) = 1 and g(x, t + 1) = g(x, t) U_t(x, t), the transformed links
// U'_mu(x) = g(x) U_mu(x) g(x + mu)^dagger have U'_t = 1 except on the last
// time slice, where U'_t(x, Lt - 1) = g(x, Lt - 1) U_t(x, Lt - 1) (the
// Polyakov line; g = 1 again at t = 0).  Gauge covariance gives
// D[U'] = g D[U] g^dagger, so M x = b is solved as M' x' = g b, x = g^dagger x'.
//
// Storage (double-float float4 per complex element): the three spatial
// directions in the usual planes [((par*3 + mu)*9 + k)*V/2 + h], then the
// temporal links of the last slice, [(par*9 + k)*Vs/2 + hs], hs the index
// within the slice (h = hs + t Vs/2 with Vs = Lx Ly Lz).  A time hop through an
// identity link adds the neighbour spinor without a link load or product.
#pragma once

#include "df64.cuh"

namespace stag {

struct LinkFieldTG {
    typedef DF real;
    typedef float4 store;
    const float4* base;
    int Vh, Vsh, Lt;
    __device__ __forceinline__ Mat3<DF> load9(const float4* q, size_t stride) const
    {
        Mat3<DF> U;
        const unsigned long long pol = l2_evict_first_policy();
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float4 f = ld_stream(q + (size_t)k * stride, pol);
            U.m[k].re = DF(f.x, f.y);
            U.m[k].im = DF(f.z, f.w);
        }
        return U;
    }
    // spatial direction mu < 3 at half site h of parity par
    __device__ __forceinline__ Mat3<DF> load(int par, int mu, int h) const
    {
        return load9(base + ((size_t)(par * 3 + mu) * 9) * Vh + h, Vh);
    }
    // temporal link of the last slice, slice index hs, parity par
    __device__ __forceinline__ Mat3<DF> load_t(int par, int hs) const
    {
        return load9(base + (size_t)54 * Vh + ((size_t)par * 9) * Vsh + hs, Vsh);
    }
};

template <> struct OpMinBlocksS<LinkFieldTG, SpinorDF> { static constexpr int value = 7; };

// acc += v (an exact sum into the hop accumulator, like df_mac with y = 1)
__device__ __forceinline__ void df_acc(DF& acc, const DF& v)
{
    float s, e;
    two_sum(acc.hi, v.hi, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, v.lo));
}

// D_{p,1-p} at half site h on temporal-gauge links (the overload of
// dslash_site for LinkFieldTG; the same eta and boundary signs).
template <class SIn>
__device__ __forceinline__ Vec3<DF> dslash_site(const Geom& g, int p, int h, const LinkFieldTG& U, const SIn& in)
{
    SiteNbrs s;
    site_nbrs(g, p, h, s);
    Vec3<DF> acc;
#pragma unroll
    for (int a = 0; a < 3; ++a) acc.c[a].re = acc.c[a].im = DF(0);
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        mv_acc(acc, U.load(p, mu, h), vflip(in.load(s.fwd[mu]), s.sf[mu]));
        mdv_acc(acc, U.load(1 - p, mu, s.bwd[mu]), vflip(in.load(s.bwd[mu]), s.sb[mu]));
    }
    const int t = h / U.Vsh;
    const Vec3<DF> vf = vflip(in.load(s.fwd[3]), s.sf[3]);
    if (t == U.Lt - 1) {
        mv_acc(acc, U.load_t(p, h - t * U.Vsh), vf);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            df_acc(acc.c[a].re, vf.c[a].re);
            df_acc(acc.c[a].im, vf.c[a].im);
        }
    }
    // the backward time link sits at x - t, on the last slice when t == 0
    const Vec3<DF> vb = vflip(in.load(s.bwd[3]), s.sb[3]);
    if (t == 0) {
        mdv_acc(acc, U.load_t(1 - p, s.bwd[3] - (U.Lt - 1) * U.Vsh), vb);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            df_acc(acc.c[a].re, vb.c[a].re);
            df_acc(acc.c[a].im, vb.c[a].im);
        }
    }
    return acc;
}

}  // namespace stag
