// dslash.cuh -- the per-site staggered hop sum of Sec. 4.2, Eq. (staggered),
// restricted to one output parity, for any link / spinor storage.
#pragma once

#include "common.cuh"

namespace stag {

// D_{p,1-p} psi at output half site h of parity p:
//   sum_mu [ eta_mu(x) U_{x,mu} psi_{x+mu} - eta_mu(x-mu) U^dagger_{x-mu,mu} psi_{x-mu} ]
// Forward links live at x (parity p), backward links at x-mu (parity 1-p).
// Eight hops, 570 flop per site in the paper's count (Sec. 4.3).
template <class LF, class SIn>
__device__ __forceinline__ Vec3<typename LF::real> dslash_site(const Geom& g, int p, int h,
                                                               const LF& U, const SIn& in)
{
    typedef typename LF::real real;
    SiteNbrs s;
    site_nbrs(g, p, h, s);
    Vec3<real> acc;
#pragma unroll
    for (int a = 0; a < 3; ++a) acc.c[a].re = acc.c[a].im = real(0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        // temporal-gauge links (U.tg): the time hops through identity links
        // are plain sums (warp-uniform wherever Vs/2 is a multiple of 32: a
        // warp's sites then share one time slice)
        if (mu == 3 && unit_fwd_time(U, s)) {
            hop_add(acc, load_flipped(in, s.fwd[mu], s.sf[mu]));
        } else {
            const Mat3<real> Uf = U.load(p, mu, h);
            const Vec3<real> vf = load_flipped(in, s.fwd[mu], s.sf[mu]);
            mv_acc(acc, Uf, vf);
        }
        if (mu == 3 && unit_bwd_time(U, s)) {
            hop_add(acc, load_flipped(in, s.bwd[mu], s.sb[mu]));
        } else {
            const Mat3<real> Ub = U.load(1 - p, mu, s.bwd[mu]);
            const Vec3<real> vb = load_flipped(in, s.bwd[mu], s.sb[mu]);
            mdv_acc(acc, Ub, vb);
        }
    }
    return acc;
}

// dslash_site with the site's links (MODE bit STAGE_LINKS, LinkStage) and/or
// its 8 neighbour spinors (bit STAGE_SPINORS, SpinorStage) copied to shared
// memory first: every copy of the site is issued before the first product,
// one copy group per direction, and direction mu waits only for its own
// group.  st holds StageWords<LF, SIn, BS, MODE>::value words for a block of
// BS threads.  The hop matrices, spinors and arithmetic are those of
// dslash_site, so the result is the same bit for bit; what changes is how
// many bytes each thread has in flight (192 bytes of half 12-real links and
// 128 bytes of half spinors, without holding registers for them).
constexpr int STAGE_LINKS = 1, STAGE_SPINORS = 2;

template <int N>
__device__ __forceinline__ void cp_async_wait_dir(int mu)
{
    if (mu == 0) cp_async_wait<N - 1>();
    else if (mu == 1) cp_async_wait<(N > 2 ? N - 2 : 0)>();
    else if (mu == 2) cp_async_wait<(N > 3 ? N - 3 : 0)>();
    else cp_async_wait<0>();
}

// Shared-memory words of a kernel of BS threads staging by MODE (one unused
// word when MODE is 0): the links first, then the spinor slots, 8 per thread
// ([hop][thread] 16-byte words, then [hop][thread] 8-byte words for float).
template <class LF, int BS, bool ON> struct LinkStageWords { static constexpr int value = 0; };
template <class LF, int BS> struct LinkStageWords<LF, BS, true> { static constexpr int value = LinkStage<LF>::words(BS); };
template <class LF, class SIn, int BS, int MODE> struct StageWords {
    static constexpr int LINKS = LinkStageWords<LF, BS, (MODE & STAGE_LINKS) != 0>::value;
    static constexpr int SPIN = (MODE & STAGE_SPINORS) ? 8 * BS * (std::is_same<SIn, SpinorF32>::value ? 3 : 2) / 2 : 0;
    static constexpr int value = LINKS + SPIN > 0 ? LINKS + SPIN : 1;
};
template <class LF, class SIn, int BS, int MODE> struct StageOK {
    static constexpr bool value = MODE == 0 || (((MODE & STAGE_LINKS) == 0 || LinkStage<LF>::value) &&
                                                ((MODE & STAGE_SPINORS) == 0 || SpinorStage<SIn>::value));
};

template <int BS, int MODE, class LF, class SIn>
__device__ __forceinline__ Vec3<typename LF::real> dslash_site_staged(const Geom& g, int p, int h, const LF& U,
                                                                      const SIn& in, uint4* st)
{
    static_assert(MODE != 0 && StageOK<LF, SIn, BS, MODE>::value, "no shared-memory staging for these fields");
    typedef typename LF::real real;
    constexpr bool SL = (MODE & STAGE_LINKS) != 0, SP = (MODE & STAGE_SPINORS) != 0;
    constexpr int LW = StageWords<LF, SIn, BS, MODE>::LINKS;
    // spinor slot of hop k: 16-byte word at sa[k BS + i], 8-byte word at sb[k BS + i]
    uint4* sa = st + LW;
    uint2* sb2 = reinterpret_cast<uint2*>(sa + 8 * BS);
    const int tid = threadIdx.x;
    SiteNbrs s;
    site_nbrs(g, p, h, s);
    const unsigned long long pol = l2_evict_first_policy();
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        if constexpr (SL) {
            if (!(mu == 3 && unit_fwd_time(U, s))) LinkStage<LF>::issue(U, p, mu, h, st, BS, 2 * mu, pol);
            if (!(mu == 3 && unit_bwd_time(U, s))) LinkStage<LF>::issue(U, 1 - p, mu, s.bwd[mu], st, BS, 2 * mu + 1, pol);
        }
        if constexpr (SP) {
            SpinorStage<SIn>::issue(in, s.fwd[mu], sa + (2 * mu) * BS + tid, sb2 + (2 * mu) * BS + tid);
            SpinorStage<SIn>::issue(in, s.bwd[mu], sa + (2 * mu + 1) * BS + tid, sb2 + (2 * mu + 1) * BS + tid);
        }
        cp_async_commit();
    }
    auto spinor = [&](int k, int nb, uint32_t sbit) {
        if constexpr (SP) return SpinorStage<SIn>::get_flipped(in, sa + k * BS + tid, sb2 + k * BS + tid, sbit);
        else return load_flipped(in, nb, sbit);
    };
    auto link = [&](int k, int par, int mu, int hh) {
        if constexpr (SL) return LinkStage<LF>::get(st, BS, k);
        else return U.load(par, mu, hh);
    };
    Vec3<real> acc;
#pragma unroll
    for (int a = 0; a < 3; ++a) acc.c[a].re = acc.c[a].im = real(0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        cp_async_wait_dir<4>(mu);
        if (mu == 3 && unit_fwd_time(U, s)) {
            hop_add(acc, spinor(2 * mu, s.fwd[mu], s.sf[mu]));
        } else {
            const Mat3<real> Uf = link(2 * mu, p, mu, h);
            const Vec3<real> vf = spinor(2 * mu, s.fwd[mu], s.sf[mu]);
            mv_acc(acc, Uf, vf);
        }
        if (mu == 3 && unit_bwd_time(U, s)) {
            hop_add(acc, spinor(2 * mu + 1, s.bwd[mu], s.sb[mu]));
        } else {
            const Mat3<real> Ub = link(2 * mu + 1, 1 - p, mu, s.bwd[mu]);
            const Vec3<real> vb = spinor(2 * mu + 1, s.bwd[mu], s.sb[mu]);
            mdv_acc(acc, Ub, vb);
        }
    }
    return acc;
}

// The operator at site h through dslash_site_staged when MODE is set (the
// caller's kernel declares the staging words), through dslash_site otherwise.
template <int BS, int MODE, class LF, class SIn>
__device__ __forceinline__ Vec3<typename LF::real> dslash_site_sel(const Geom& g, int p, int h, const LF& U,
                                                                   const SIn& in, uint4* st)
{
    if constexpr (MODE != 0) return dslash_site_staged<BS, MODE>(g, p, h, U, in, st);
    else return dslash_site(g, p, h, U, in);
}

// Minimum resident blocks (of 128 threads) requested from the compiler for an
// operator kernel on link field LF: 1 (no bound) by default; double-float
// links cap registers at 96 (5 blocks), float links at 72 (7) and half links
// at 64 (8), which raises occupancy without spilling (measured 4 %, 5 % and
// 7 % faster at 48^3 x 12).
template <class LF> struct OpMinBlocks { static constexpr int value = 1; };
template <int R> struct OpMinBlocks<LinkField<__half2, R>> { static constexpr int value = 8; };
// float links: 72 registers (48^3 x 12 F32/12: 42.5 against 44.7 us at 128)
template <int R> struct OpMinBlocks<LinkField<float2, R>> { static constexpr int value = 7; };
// the same for a link field and the spinor storage the operator reads
template <class LF, class S> struct OpMinBlocksS { static constexpr int value = OpMinBlocks<LF>::value; };

// Conversion of an operator result to the epilogue's arithmetic type (the
// identity here; double-float results convert to double in df64.cuh).
template <class R, class X> struct VConv;
template <class R> struct VConv<R, R> {
    static __device__ __forceinline__ Vec3<R> f(const Vec3<R>& v) { return v; }
};
template <class R, class X>
__device__ __forceinline__ Vec3<R> vconv(const Vec3<X>& v) { return VConv<R, X>::f(v); }

}  // namespace stag
