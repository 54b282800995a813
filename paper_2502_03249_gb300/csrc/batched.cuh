// batched.cuh -- the staggered operator applied to NB right-hand sides per
// thread: every link is loaded once per site and used for all NB vectors
// (the paper's multi-vector Dslash, Sec. 4.3, NMULTI), plus the per-system
// masks the batched solvers use.
#pragma once

#include "dslash.cuh"

namespace stag {

// Minimum resident blocks of 128 threads for a batched operator kernel: the
// single-RHS bound of the link field for NB = 1; on float arithmetic 7 for up
// to 4 right-hand sides per block (72 registers) and 6 for 8 (80 registers,
// a few dozen bytes of spill), which the latency-bound multi-vector passes
// need more than registers (32^3 x 16, 16 RHS: 105.1 -> 99.7 ms, the
// autotuner now choosing blocks of 4; at 4 and 5 blocks per SM the kernels
// took 96-127 registers); else 4 (at most 128 registers; unbounded, the
// compiler takes up to 222 for NB = 8 and runs 2 blocks per SM).
template <class LF, int NB> struct MultiMinBlocks {
    static constexpr int value = NB == 1 ? OpMinBlocks<LF>::value
                                         : (sizeof(typename LF::real) != 4 ? 4 : (NB <= 4 ? 7 : (NB <= 8 ? 6 : 4)));
};

// acc[k] = (D_{p,1-p} in_{k0+k})_h for the k with bit k of mask set.
// in.at(j, stride) is field j of the multi field.
template <class LF, class S, int NB>
__device__ __forceinline__ void dslash_site_multi(const Geom& g, int p, int h, const LF& U, const S& in,
                                                  size_t stride, int k0, unsigned mask,
                                                  Vec3<typename LF::real>* acc)
{
    typedef typename LF::real real;
    SiteNbrs s;
    site_nbrs(g, p, h, s);
#pragma unroll
    for (int k = 0; k < NB; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[k].c[a].re = acc[k].c[a].im = real(0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        // identity time links of temporal-gauge fields (U.tg): plain sums
        if (mu == 3 && unit_fwd_time(U, s)) {
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (mask & (1u << k)) hop_add(acc[k], load_flipped(in.at(k0 + k, stride), s.fwd[mu], s.sf[mu]));
        } else {
            const Mat3<real> Uf = U.load(p, mu, h);
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (mask & (1u << k)) mv_acc(acc[k], Uf, load_flipped(in.at(k0 + k, stride), s.fwd[mu], s.sf[mu]));
        }
        if (mu == 3 && unit_bwd_time(U, s)) {
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (mask & (1u << k)) hop_add(acc[k], load_flipped(in.at(k0 + k, stride), s.bwd[mu], s.sb[mu]));
        } else {
            const Mat3<real> Ub = U.load(1 - p, mu, s.bwd[mu]);
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (mask & (1u << k)) mdv_acc(acc[k], Ub, load_flipped(in.at(k0 + k, stride), s.bwd[mu], s.sb[mu]));
        }
    }
}

}  // namespace stag
