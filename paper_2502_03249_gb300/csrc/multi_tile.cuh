// multi_tile.cuh -- the multi-vector operator (Sec. 4.3, NMULTI) with the
// links of a tile of sites staged once in shared memory for a block of
// right-hand sides.
//
// A block of G x SW warps covers TS = 32 SW consecutive half sites of the
// output parity and G NBT right-hand sides: warp w computes the NBT systems
// k0 + (w / SW) NBT ... of site (w % SW) 32 + lane.  Two phases:
//
//  1. every thread loads its site's hop matrices -- the 8 links, row 2 rebuilt
//     for 12-real storage, the hop's sign (eta_mu, the time-boundary sign, the
//     minus of the backward term) folded in, and the adjoint taken for the
//     backward hops -- for the hops h0, h0 + G, ... (h0 = its warp's group), so
//     the block reads each link exactly once, and stores them in shared memory;
//  2. after one barrier every thread applies the 8 hop matrices to its NBT
//     spinors.  Each link load and rebuild is shared by G NBT right-hand sides
//     while a thread keeps only NBT accumulators, so blocks of 16 right-hand
//     sides run without the register spills of 16 accumulators per thread.
//
// The hops are summed in the order of dslash_site (forward then backward, mu =
// 0..3) with the same FMAs (the signs and the conjugation are exact), so the
// result equals the single-vector operator bit for bit.
//
// Configurations are named by cfg = (G << 8) | NBT; G = 1 is the
// register-blocked kernel without staging (batched.cuh), which the tile
// kernels leave to that code.
#pragma once

#include <vector>

#include "batched.cuh"
#include "df64.cuh"

namespace stag {

constexpr int mcfg(int G, int NBT) { return (G << 8) | NBT; }
constexpr int mcfg_G(int c) { return c >> 8; }
constexpr int mcfg_NBT(int c) { return c & 0xff; }
constexpr int mcfg_block(int c) { return (c >> 8) * (c & 0xff); }

// Tile kernels are built for links in float arithmetic (float and half
// storage); double links use the register-blocked kernels (G = 1).
template <class LF> struct TileOK { static constexpr bool value = sizeof(typename LF::real) == 4; };

// Candidate configurations of a multi-vector pass over nrhs right-hand sides:
// the register-blocked blocks 1..16 and, for float arithmetic, the tile
// splits of blocks 2..16; blocks above the smallest power of two >= nrhs are
// left out (they would only mask lanes).
template <class LF>
inline std::vector<int> multi_cfg_candidates(int nrhs)
{
    int cap = 1;
    while (cap < nrhs) cap *= 2;
    std::vector<int> c;
    for (int nb : {1, 2, 4, 8, 16})
        if (nb <= cap) c.push_back(mcfg(1, nb));
    if (TileOK<LF>::value) {
        for (int cfg : {mcfg(2, 1), mcfg(2, 2), mcfg(4, 1), mcfg(2, 4), mcfg(4, 2), mcfg(8, 1), mcfg(2, 8), mcfg(4, 4),
                        mcfg(8, 2), mcfg(16, 1)})
            if (mcfg_block(cfg) <= cap) c.push_back(cfg);
    }
    return c;
}

// Site warps per group: blocks of at least 128 threads.
template <int G> struct TileSW { static constexpr int value = G >= 4 ? 1 : (G == 2 ? 2 : 4); };

// Minimum resident blocks per SM requested for a tile kernel of NT threads
// with NBT right-hand sides per thread: 1024 threads per SM (64 registers)
// for up to two accumulators, 768 (85 registers) for four, which the four
// accumulators, the four neighbour spinors in flight and the hop matrix need.
template <int NT, int NBT> struct TileMinBlocks {
    static constexpr int threads = NBT >= 8 ? 512 : NBT >= 4 ? 768 : 1024;
    static constexpr int value = NT >= threads ? 1 : threads / NT;
};

// Hop matrices in shared memory, 16-byte chunks: float links as four float4
// (elements 0..7) and one float2 (element 8) padded to 16 bytes; double links
// as nine double2.  Layout [hop][chunk][site] of uint4: a warp reading one
// chunk of 32 consecutive sites reads 512 contiguous bytes.
template <typename T> struct HopStore;
template <> struct HopStore<float> {
    static constexpr int NV = 5;
    static __device__ __forceinline__ void put(uint4* sm, int TS, int hop, int sl, const Mat3<float>& H)
    {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            reinterpret_cast<float4*>(sm)[(hop * NV + c) * TS + sl] =
                make_float4(H.m[2 * c].re, H.m[2 * c].im, H.m[2 * c + 1].re, H.m[2 * c + 1].im);
        reinterpret_cast<float4*>(sm)[(hop * NV + 4) * TS + sl] = make_float4(H.m[8].re, H.m[8].im, 0.f, 0.f);
    }
    static __device__ __forceinline__ Mat3<float> get(const uint4* sm, int TS, int hop, int sl)
    {
        Mat3<float> H;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float4 q = reinterpret_cast<const float4*>(sm)[(hop * NV + c) * TS + sl];
            H.m[2 * c] = {q.x, q.y};
            H.m[2 * c + 1] = {q.z, q.w};
        }
        const float4 q = reinterpret_cast<const float4*>(sm)[(hop * NV + 4) * TS + sl];
        H.m[8] = {q.x, q.y};
        return H;
    }
};
template <> struct HopStore<double> {
    static constexpr int NV = 9;
    static __device__ __forceinline__ void put(uint4* sm, int TS, int hop, int sl, const Mat3<double>& H)
    {
#pragma unroll
        for (int c = 0; c < 9; ++c)
            reinterpret_cast<double2*>(sm)[(hop * NV + c) * TS + sl] = make_double2(H.m[c].re, H.m[c].im);
    }
    static __device__ __forceinline__ Mat3<double> get(const uint4* sm, int TS, int hop, int sl)
    {
        Mat3<double> H;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const double2 q = reinterpret_cast<const double2*>(sm)[(hop * NV + c) * TS + sl];
            H.m[c] = {q.x, q.y};
        }
        return H;
    }
};

// double-float links (the reliable updates' operator): nine float4 (re_hi,
// re_lo, im_hi, im_lo)
template <> struct HopStore<DF> {
    static constexpr int NV = 9;
    static __device__ __forceinline__ void put(uint4* sm, int TS, int hop, int sl, const Mat3<DF>& H)
    {
#pragma unroll
        for (int c = 0; c < 9; ++c)
            reinterpret_cast<float4*>(sm)[(hop * NV + c) * TS + sl] =
                make_float4(H.m[c].re.hi, H.m[c].re.lo, H.m[c].im.hi, H.m[c].im.lo);
    }
    static __device__ __forceinline__ Mat3<DF> get(const uint4* sm, int TS, int hop, int sl)
    {
        Mat3<DF> H;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const float4 q = reinterpret_cast<const float4*>(sm)[(hop * NV + c) * TS + sl];
            H.m[c].re = DF(q.x, q.y);
            H.m[c].im = DF(q.z, q.w);
        }
        return H;
    }
};

// The hop matrix of hop = 2 mu + back at output site h (neighbours s):
// forward  s_f U_{x,mu},  backward  s_b U^dagger_{x-mu,mu}  (s the sign bits).
template <class LF>
__device__ __forceinline__ Mat3<typename LF::real> hop_matrix(const LF& U, int p, int h, const SiteNbrs& s, int hop)
{
    typedef typename LF::real real;
    const int mu = hop >> 1;
    Mat3<real> H;
    if (!(hop & 1)) {
        const Mat3<real> L = U.load(p, mu, h);
        const uint32_t sb = s.sf[mu];
#pragma unroll
        for (int e = 0; e < 9; ++e) H.m[e] = {flip(L.m[e].re, sb), flip(L.m[e].im, sb)};
    } else {
        const Mat3<real> L = U.load(1 - p, mu, s.bwd[mu]);
        const uint32_t sb = s.sb[mu];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                H.m[a * 3 + b] = {flip(L.m[b * 3 + a].re, sb), flip(L.m[b * 3 + a].im, sb ^ 0x80000000u)};
    }
    return H;
}

// Phase 2 for one thread: acc[k] += the 8 hops applied to field f[k] at the
// neighbours of s, for the k of mask (ALL: every k, no tests), the hop
// matrices read from the tile in shared memory.
template <class LF, class S, int NBT, bool ALL>
__device__ __forceinline__ void tile_apply_hops(const SiteNbrs& s, const LF& U, const S* f, unsigned mask,
                                                const uint4* sm, int TS, int sl, Vec3<typename LF::real>* acc)
{
    typedef typename LF::real real;
#pragma unroll
    for (int hop = 0; hop < 8; ++hop) {
        const int nb = (hop & 1) ? s.bwd[hop >> 1] : s.fwd[hop >> 1];
        // the neighbour spinors in batches of up to four loads in flight
        constexpr int NL = NBT < 4 ? NBT : 4;
        if (unit_hop(U, s, hop)) {
            // identity time link of a temporal-gauge field: the signed spinor
            // is added (what the product with the hop matrix +-1 gives)
            const uint32_t sb = (hop & 1) ? s.sb[3] : s.sf[3];
#pragma unroll
            for (int kb = 0; kb < NBT; kb += NL) {
                Vec3<real> v[NL];
#pragma unroll
                for (int k = 0; k < NL; ++k)
                    if (ALL || (mask & (1u << (kb + k)))) v[k] = load_flipped(f[kb + k], nb, sb);
#pragma unroll
                for (int k = 0; k < NL; ++k)
                    if (ALL || (mask & (1u << (kb + k)))) hop_add(acc[kb + k], v[k]);
            }
            continue;
        }
        const Mat3<real> H = HopStore<real>::get(sm, TS, hop, sl);
#pragma unroll
        for (int kb = 0; kb < NBT; kb += NL) {
            Vec3<real> v[NL];
#pragma unroll
            for (int k = 0; k < NL; ++k)
                if (ALL || (mask & (1u << (kb + k)))) v[k] = f[kb + k].load(nb);
#pragma unroll
            for (int k = 0; k < NL; ++k)
                if (ALL || (mask & (1u << (kb + k)))) mv_acc(acc[kb + k], H, v[k]);
        }
    }
}

// Phase 1 and 2 for one thread: stage the tile's hop matrices, then
// acc[k] = (D_{p,1-p} in_{k0+k})_h for the k of mask.  All threads of the
// block call this (it contains a barrier); h >= Vh and mask = 0 only skip work.
template <class LF, class S, int G, int NBT>
__device__ __forceinline__ void tile_site_multi(const Geom& g, int p, int h, const SiteNbrs& s, const LF& U,
                                                const S& in, size_t stride, int k0, unsigned mask, uint4* sm,
                                                Vec3<typename LF::real>* acc)
{
    typedef typename LF::real real;
    constexpr int SW = TileSW<G>::value, TS = 32 * SW;
    const int sl = threadIdx.x % TS, grp = threadIdx.x / TS;
    const bool on = h < g.Vh;
    // this thread stages hops grp, grp + G, ...: unrolled so that the
    // neighbour arrays are indexed statically (registers, not local memory)
#pragma unroll
    for (int hop = 0; hop < 8; ++hop)
        if (on && hop % G == grp && !unit_hop(U, s, hop))
            HopStore<real>::put(sm, TS, hop, sl, hop_matrix(U, p, h, s, hop));
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NBT; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[k].c[a].re = acc[k].c[a].im = real(0);
    if (!on || !mask) return;
    // the thread's NBT fields, and the hop loop without per-system tests
    // when all of them are active (the usual case)
    S f[NBT];
#pragma unroll
    for (int k = 0; k < NBT; ++k) f[k] = in.at(k0 + k, stride);
    if (mask == (1u << NBT) - 1u) {
        tile_apply_hops<LF, S, NBT, true>(s, U, f, mask, sm, TS, sl, acc);
        return;
    }
    tile_apply_hops<LF, S, NBT, false>(s, U, f, mask, sm, TS, sl, acc);
}

// Shared memory of a tile kernel (bytes).
template <class LF, int G> struct TileSmem {
    static constexpr int value = 8 * HopStore<typename LF::real>::NV * 32 * TileSW<G>::value * 16;
};

// out_k = D_{p,1-p} in_k for k < nrhs, one block per tile of sites and G NBT
// right-hand sides (grid (tiles, ceil(nrhs / (G NBT)))).
template <class LF, class S, int G, int NBT>
__global__ void __launch_bounds__(32 * TileSW<G>::value * G, TileMinBlocks<32 * TileSW<G>::value * G, NBT>::value)
    k_tile_dslash(Geom g, int p, LF U, S in, S out, size_t stride, int nrhs)
{
    __shared__ uint4 sm[TileSmem<LF, G>::value / 16];
    constexpr int SW = TileSW<G>::value, TS = 32 * SW;
    const int w = threadIdx.x >> 5;
    const int h = blockIdx.x * TS + threadIdx.x % TS;
    const int k0 = blockIdx.y * G * NBT + (w / SW) * NBT;
    unsigned mask = 0;
#pragma unroll
    for (int k = 0; k < NBT; ++k)
        if (k0 + k < nrhs) mask |= 1u << k;
    SiteNbrs s;
    site_nbrs(g, p, h < g.Vh ? h : g.Vh - 1, s);
    Vec3<typename LF::real> acc[NBT];
    tile_site_multi<LF, S, G, NBT>(g, p, h, s, U, in, stride, k0, mask, sm, acc);
    if (h >= g.Vh) return;
#pragma unroll
    for (int k = 0; k < NBT; ++k)
        if (mask & (1u << k)) out.at(k0 + k, stride).store(h, acc[k]);
}

}  // namespace stag
