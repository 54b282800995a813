// common.cuh -- device-side building blocks shared by the libstag kernels:
// lattice geometry of one parity, complex 3-vectors and 3x3 matrices, the
// internal storage layouts of links and spinors, and block reductions.
#pragma once

#include <type_traits>
#include <utility>

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace stag {

// ---------------------------------------------------------------- geometry
//
// A half field of parity p holds the V/2 sites with (x+y+z+t) mod 2 == p,
// indexed h = i/2 with i = x + Lx*(y + Ly*(z + Lz*t)).  Writing h = xh + Lxh*r
// (Lxh = Lx/2, r the row index of (y,z,t)), the site's x is 2*xh + ((p+y+z+t)&1).
// Division of a non-negative int by an invariant positive divisor with one
// multiply-high, two adds and two shifts instead of the integer division
// routine: Granlund and Montgomery's unsigned method ("Division by invariant
// integers using multiplication", 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n) gives
// floor(n / d) = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) for every
// 0 <= n < 2^32.
struct FastDiv {
    uint32_t m;
    uint32_t s1, s2;
};

__host__ __device__ inline FastDiv make_fastdiv(int d)
{
    uint32_t l = 0;
    while ((1ull << l) < (unsigned long long)d) ++l;
    FastDiv f;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - (unsigned long long)d)) / (unsigned long long)d + 1ull);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}

__device__ __forceinline__ int fast_div(int n, const FastDiv& f)
{
    const uint32_t un = (uint32_t)n, t = __umulhi(f.m, un);
    return (int)((t + ((un - t) >> f.s1)) >> f.s2);
}

struct Geom {
    int L[4];     // Lx, Ly, Lz, Lt
    int Lxh;      // Lx / 2
    int Vh;       // V / 2
    FastDiv dxh, dy, dz;   // division by Lxh, Ly, Lz
};

// Geometry of an Lx x Ly x Lz x Lt lattice (extents even and >= 2).
__host__ inline Geom make_geom(const int dims[4])
{
    Geom g;
    for (int mu = 0; mu < 4; ++mu) g.L[mu] = dims[mu];
    g.Lxh = dims[0] / 2;
    g.Vh = (int)((long long)dims[0] * dims[1] * dims[2] * dims[3] / 2);
    g.dxh = make_fastdiv(g.Lxh);
    g.dy = make_fastdiv(dims[1]);
    g.dz = make_fastdiv(dims[2]);
    return g;
}

struct SiteNbrs {
    int h;             // own half index
    int fwd[4];        // half index of x + mu (other parity)
    int bwd[4];        // half index of x - mu (other parity)
    uint32_t sf[4];    // sign bit (0 or 0x80000000) of eta_mu(x) * boundary, forward hop
    uint32_t sb[4];    // sign bit of -eta_mu(x-mu) * boundary, backward hop
};

// Neighbours and hop signs of output site h of parity p.  eta_mu(x-mu) equals
// eta_mu(x) because eta_mu does not depend on x_mu (even extents keep this
// true across the periodic wrap).  The backward term of Eq. (staggered) carries
// an explicit minus, folded into sb.
__device__ __forceinline__ void site_nbrs(const Geom& g, int p, int h, SiteNbrs& s)
{
    const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
    const int r = fast_div(h, g.dxh);
    const int xh = h - r * g.Lxh;
    const int zt = fast_div(r, g.dy);
    const int y = r - zt * Ly;
    const int t = fast_div(zt, g.dz);
    const int z = zt - t * Lz;
    const int x = 2 * xh + ((p + y + z + t) & 1);
    s.h = h;
    const int rowh = g.Lxh * r;
    s.fwd[0] = ((x + 1 == Lx) ? 0 : x + 1) / 2 + rowh;
    s.bwd[0] = ((x == 0) ? Lx - 1 : x - 1) / 2 + rowh;
    const int sy = g.Lxh, sz = g.Lxh * Ly, st = g.Lxh * Ly * Lz;
    s.fwd[1] = h + ((y + 1 == Ly) ? -(Ly - 1) * sy : sy);
    s.bwd[1] = h + ((y == 0) ? (Ly - 1) * sy : -sy);
    s.fwd[2] = h + ((z + 1 == Lz) ? -(Lz - 1) * sz : sz);
    s.bwd[2] = h + ((z == 0) ? (Lz - 1) * sz : -sz);
    s.fwd[3] = h + ((t + 1 == Lt) ? -(Lt - 1) * st : st);
    s.bwd[3] = h + ((t == 0) ? (Lt - 1) * st : -st);
    const uint32_t SB = 0x80000000u;
    const uint32_t e1 = (x & 1) ? SB : 0u;
    const uint32_t e2 = ((x + y) & 1) ? SB : 0u;
    const uint32_t e3 = ((x + y + z) & 1) ? SB : 0u;
    const uint32_t bf3 = (t == Lt - 1) ? SB : 0u;   // forward hop crosses the time boundary
    const uint32_t bb3 = (t == 0) ? SB : 0u;        // backward hop crosses it
    s.sf[0] = 0u;
    s.sf[1] = e1;
    s.sf[2] = e2;
    s.sf[3] = e3 ^ bf3;
    s.sb[0] = SB;
    s.sb[1] = e1 ^ SB;
    s.sb[2] = e2 ^ SB;
    s.sb[3] = e3 ^ bb3 ^ SB;
}

// Forward neighbour (half index) and the sign bit of the forward hop (eta_mu
// times the time-boundary sign) of half site h of parity p in direction mu,
// the same values as site_nbrs for a runtime mu (no local array).
__device__ __forceinline__ void fwd_nbr(const Geom& g, int p, int h, int mu, int& fw, uint32_t& sf)
{
    const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
    const int r = fast_div(h, g.dxh);
    const int xh = h - r * g.Lxh;
    const int zt = fast_div(r, g.dy);
    const int y = r - zt * Ly;
    const int t = fast_div(zt, g.dz);
    const int z = zt - t * Lz;
    const int x = 2 * xh + ((p + y + z + t) & 1);
    const uint32_t SB = 0x80000000u;
    if (mu == 0) {
        fw = ((x + 1 == Lx) ? 0 : x + 1) / 2 + g.Lxh * r;
        sf = 0u;
        return;
    }
    const int c = (mu == 1) ? y : (mu == 2) ? z : t;
    const int Lc = (mu == 1) ? Ly : (mu == 2) ? Lz : Lt;
    const int st = (mu == 1) ? g.Lxh : (mu == 2) ? g.Lxh * Ly : g.Lxh * Ly * Lz;
    fw = h + ((c + 1 == Lc) ? -(Lc - 1) * st : st);
    const int ep = (mu == 1) ? x : (mu == 2) ? x + y : x + y + z;
    sf = ((ep & 1) ? SB : 0u) ^ ((mu == 3 && t == Lt - 1) ? SB : 0u);
}

// ------------------------------------------------------- complex arithmetic

template <typename T> struct Cplx { T re, im; };

template <typename T> struct Vec3 { Cplx<T> c[3]; };
template <typename T> struct Mat3 { Cplx<T> m[9]; };   // row major

__device__ __forceinline__ double flip(double v, uint32_t sbit)
{
    // v with its sign bit xor-ed with sbit (an exact negation when sbit is set)
    long long b = __double_as_longlong(v);
    b ^= ((long long)sbit) << 32;
    return __longlong_as_double(b);
}
__device__ __forceinline__ float flip(float v, uint32_t sbit)
{
    return __uint_as_float(__float_as_uint(v) ^ sbit);
}

template <typename T>
__device__ __forceinline__ Vec3<T> vflip(const Vec3<T>& v, uint32_t s)
{
    Vec3<T> o;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o.c[a].re = flip(v.c[a].re, s);
        o.c[a].im = flip(v.c[a].im, s);
    }
    return o;
}

// acc += U v
template <typename T>
__device__ __forceinline__ void mv_acc(Vec3<T>& acc, const Mat3<T>& U, const Vec3<T>& v)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T re = acc.c[a].re, im = acc.c[a].im;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const Cplx<T> u = U.m[a * 3 + b];
            re = fma(u.re, v.c[b].re, re);
            re = fma(-u.im, v.c[b].im, re);
            im = fma(u.re, v.c[b].im, im);
            im = fma(u.im, v.c[b].re, im);
        }
        acc.c[a].re = re;
        acc.c[a].im = im;
    }
}

// acc += U^dagger v
template <typename T>
__device__ __forceinline__ void mdv_acc(Vec3<T>& acc, const Mat3<T>& U, const Vec3<T>& v)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T re = acc.c[a].re, im = acc.c[a].im;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const Cplx<T> u = U.m[b * 3 + a];
            re = fma(u.re, v.c[b].re, re);
            re = fma(u.im, v.c[b].im, re);
            im = fma(u.re, v.c[b].im, im);
            im = fma(-u.im, v.c[b].re, im);
        }
        acc.c[a].re = re;
        acc.c[a].im = im;
    }
}

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Third row of an SU(3) matrix from its first two: conj(row0 x row1) (Sec. 4.3).
// Every product and sum is spelled out (explicit FMA and rounded operations),
// so that all kernels that reconstruct a link round it identically: the
// compiler may not contract the expression differently per instantiation.
template <typename T>
__device__ __forceinline__ void reconstruct_row2(Mat3<T>& U)
{
    const Cplx<T>* a = &U.m[0];
    const Cplx<T>* b = &U.m[3];
    // c_k = conj(a_i b_j - a_j b_i) for (k,i,j) cyclic: each part one
    // product and three FMAs (the conjugate's sign folded into the operands)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = (k + 1) % 3, j = (k + 2) % 3;
        // re = a_i.re b_j.re - a_i.im b_j.im - a_j.re b_i.re + a_j.im b_i.im
        T re = mul_rn(a[j].im, b[i].im);
        re = fma(-a[j].re, b[i].re, re);
        re = fma(-a[i].im, b[j].im, re);
        re = fma(a[i].re, b[j].re, re);
        // -im = a_j.re b_i.im + a_j.im b_i.re - a_i.re b_j.im - a_i.im b_j.re
        T im = mul_rn(a[j].re, b[i].im);
        im = fma(a[j].im, b[i].re, im);
        im = fma(-a[i].re, b[j].im, im);
        im = fma(-a[i].im, b[j].re, im);
        U.m[6 + k].re = re;
        U.m[6 + k].im = im;
    }
}

// ------------------------------------------------------------ link storage
//
// Links are stored per parity, direction and matrix element, structure of
// arrays over half sites, so that a warp reading element k of 32 consecutive
// sites touches one contiguous run:
//     base[((par*4 + mu)*NE + k)*Vh + h],   NE = 9 (18-real) or 6 (12-real)
// with element type double2 (F64), float2 (F32) or __half2 (F16).

template <typename S> struct StoreTraits;
template <> struct StoreTraits<double2> { typedef double real; };
template <> struct StoreTraits<float2> { typedef float real; };
template <> struct StoreTraits<__half2> { typedef float real; };

__device__ __forceinline__ Cplx<double> to_cplx(double2 v) { return {v.x, v.y}; }
__device__ __forceinline__ Cplx<float> to_cplx(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ Cplx<float> to_cplx(__half2 v)
{
    float2 f = __half22float2(v);
    return {f.x, f.y};
}

template <typename S>
__device__ __forceinline__ S ldg_nc(const S* p) { return __ldg(p); }
template <>
__device__ __forceinline__ __half2 ldg_nc<__half2>(const __half2* p)
{
    unsigned int u = __ldg(reinterpret_cast<const unsigned int*>(p));
    return *reinterpret_cast<__half2*>(&u);
}

// Streaming loads for data read once per kernel (the links: each half
// operator reads every link once): L2 evict-first policy (the line is the
// first to go when its set needs room) and no L1 allocation.  A half operator
// streams the whole gauge field (151 MB of double-float links at 32^3 x 8,
// more than the 129 MB L2); loaded this way the links no longer push the
// solvers' vectors out of L2 between the kernels of an iteration (measured:
// double-float CG iteration 76.5 -> 70.5 us at 32^3 x 8, 323 -> 310 us at
// 48^3 x 12).
__device__ __forceinline__ unsigned long long l2_evict_first_policy()
{
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ float4 ld_stream(const float4* p, unsigned long long pol)
{
    float4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint4 ld_stream(const uint4* p, unsigned long long pol)
{
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint2 ld_stream(const uint2* p, unsigned long long pol)
{
    uint2 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
        : "=r"(v.x), "=r"(v.y)
        : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ unsigned int ld_stream(const unsigned int* p, unsigned long long pol)
{
    unsigned int v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double2 ld_stream(const double2* p, unsigned long long pol)
{
    double2 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
        : "=d"(v.x), "=d"(v.y)
        : "l"(p), "l"(pol));
    return v;
}
// Asynchronous copies from global to shared memory (cp.async): the data do
// not pass through registers, so a thread can have all of its site's links
// in flight at once.  A thread's copies complete in the groups it commits
// and are visible to that thread once it has waited for them (wait_group N:
// at most the N most recent groups still pending); the links take the same
// L2 evict-first policy as the streaming loads.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, unsigned long long pol)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, unsigned long long pol)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;" ::"r"(sa), "l"(gmem), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, unsigned long long pol)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2;" ::"r"(sa), "l"(gmem), "l"(pol)
                 : "memory");
}
// spinor copies: default L2 policy (the vectors stay L2-resident), L1 allocated
// (neighbouring sites of a block share lines)
__device__ __forceinline__ void cp_async16_ca(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8_ca(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename S, int RECON>
struct LinkField {
    typedef typename StoreTraits<S>::real real;
    typedef S store;
    static constexpr int NE = (RECON == 12) ? 6 : 9;
    const S* base;
    int Vh;
    int tg = 0;   // 1: temporal-gauge links, identity time links skipped (see below)
    __device__ __forceinline__ Mat3<real> load(int par, int mu, int h) const
    {
        Mat3<real> U;
        const S* p = base + ((size_t)(par * 4 + mu) * NE) * Vh + h;
        const unsigned long long pol = l2_evict_first_policy();
#pragma unroll
        for (int k = 0; k < NE; ++k) U.m[k] = to_cplx(ld_stream(p + (size_t)k * Vh, pol));
        if (RECON == 12) reconstruct_row2(U);
        return U;
    }
};

// Float and half links are stored in 16-byte chunks so that a thread loads a
// whole link with two to five vector loads.  For each (parity, direction) the
// NE elements of a link (8 bytes each for float, 4 for half) are cut into NC
// full 16-byte chunks plus a remainder of RB bytes; chunk j of all sites is a
// plane [Vh] of uint4, the remainder a plane [Vh] of RB-byte words:
//     block(par, mu) = base + (par*4 + mu) * NE*EB*Vh bytes
//     chunk j at block + j*16*Vh + 16*h,  remainder at block + NC*16*Vh + RB*h
template <int EB, int NE> struct LinkChunks {
    static constexpr int BYTES = EB * NE;
    static constexpr int NC = BYTES / 16;
    static constexpr int RB = BYTES % 16;     // 0, 4 or 8
    static constexpr int WORDS = BYTES / 4;
    // all 32-bit words of the link at (block, h)
    static __device__ __forceinline__ void load(const char* block, int Vh, int h, uint32_t* w)
    {
        const unsigned long long pol = l2_evict_first_policy();
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const uint4 q = ld_stream(reinterpret_cast<const uint4*>(block + (size_t)j * 16 * Vh) + h, pol);
            w[4 * j] = q.x;
            w[4 * j + 1] = q.y;
            w[4 * j + 2] = q.z;
            w[4 * j + 3] = q.w;
        }
        const char* rem = block + (size_t)NC * 16 * Vh;
        if constexpr (RB == 8) {
            const uint2 q = ld_stream(reinterpret_cast<const uint2*>(rem) + h, pol);
            w[4 * NC] = q.x;
            w[4 * NC + 1] = q.y;
        } else if constexpr (RB == 4) {
            w[4 * NC] = ld_stream(reinterpret_cast<const unsigned int*>(rem) + h, pol);
        }
    }
    // Staging in shared memory (LinkStage below): chunk j of the link goes to
    // sq[j * stride], the remainder to sr[0] (a word of RB bytes).
    static __device__ __forceinline__ void stage(const char* block, int Vh, int h, uint4* sq, void* sr, int stride,
                                                 unsigned long long pol)
    {
#pragma unroll
        for (int j = 0; j < NC; ++j)
            cp_async16(sq + (size_t)j * stride, reinterpret_cast<const uint4*>(block + (size_t)j * 16 * Vh) + h, pol);
        const char* rem = block + (size_t)NC * 16 * Vh;
        if constexpr (RB == 8) cp_async8(sr, reinterpret_cast<const uint2*>(rem) + h, pol);
        else if constexpr (RB == 4) cp_async4(sr, reinterpret_cast<const unsigned int*>(rem) + h, pol);
    }
    static __device__ __forceinline__ void unstage(const uint4* sq, const void* sr, int stride, uint32_t* w)
    {
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const uint4 q = sq[(size_t)j * stride];
            w[4 * j] = q.x;
            w[4 * j + 1] = q.y;
            w[4 * j + 2] = q.z;
            w[4 * j + 3] = q.w;
        }
        if constexpr (RB == 8) {
            const uint2 q = *reinterpret_cast<const uint2*>(sr);
            w[4 * NC] = q.x;
            w[4 * NC + 1] = q.y;
        } else if constexpr (RB == 4) {
            w[4 * NC] = *reinterpret_cast<const unsigned int*>(sr);
        }
    }
    static __device__ __forceinline__ void store(char* block, int Vh, int h, const uint32_t* w)
    {
#pragma unroll
        for (int j = 0; j < NC; ++j)
            reinterpret_cast<uint4*>(block + (size_t)j * 16 * Vh)[h] =
                make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
        char* rem = block + (size_t)NC * 16 * Vh;
        if constexpr (RB == 8) reinterpret_cast<uint2*>(rem)[h] = make_uint2(w[4 * NC], w[4 * NC + 1]);
        else if constexpr (RB == 4) reinterpret_cast<unsigned int*>(rem)[h] = w[4 * NC];
    }
};

template <int RECON>
struct LinkField<float2, RECON> {
    typedef float real;
    typedef float2 store;
    static constexpr int NE = (RECON == 12) ? 6 : 9;
    typedef LinkChunks<8, NE> C;
    const float2* base;
    int Vh;
    int tg = 0;
    __device__ __forceinline__ Mat3<float> load(int par, int mu, int h) const
    {
        uint32_t w[C::WORDS];
        C::load(reinterpret_cast<const char*>(base) + (size_t)(par * 4 + mu) * C::BYTES * Vh, Vh, h, w);
        Mat3<float> U;
#pragma unroll
        for (int k = 0; k < NE; ++k) U.m[k] = {__uint_as_float(w[2 * k]), __uint_as_float(w[2 * k + 1])};
        if (RECON == 12) reconstruct_row2(U);
        return U;
    }
};

template <int RECON>
struct LinkField<__half2, RECON> {
    typedef float real;
    typedef __half2 store;
    static constexpr int NE = (RECON == 12) ? 6 : 9;
    typedef LinkChunks<4, NE> C;
    const __half2* base;
    int Vh;
    int tg = 0;
    __device__ __forceinline__ const char* block(int par, int mu) const
    {
        return reinterpret_cast<const char*>(base) + (size_t)(par * 4 + mu) * C::BYTES * Vh;
    }
    static __device__ __forceinline__ Mat3<float> decode(const uint32_t* w)
    {
        Mat3<float> U;
#pragma unroll
        for (int k = 0; k < NE; ++k) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
            U.m[k] = {f.x, f.y};
        }
        if (RECON == 12) reconstruct_row2(U);
        return U;
    }
    __device__ __forceinline__ Mat3<float> load(int par, int mu, int h) const
    {
        uint32_t w[C::WORDS];
        C::load(block(par, mu), Vh, h, w);
        return decode(w);
    }
};

// Shared-memory staging of the 8 links of one output site per thread
// (dslash_site_staged): for a block of BS threads, chunk j of hop k (0..7) of
// thread i at q[(k NC + j) BS + i], its remainder word at r[k BS + i] with r
// after the 8 NC BS chunks; a warp reading one slot reads contiguous words.
// Built for half 12-real links (24 bytes per link, 192 bytes per thread).
template <class LF> struct LinkStage { static constexpr bool value = false; };
template <> struct LinkStage<LinkField<__half2, 12>> {
    static constexpr bool value = true;
    typedef LinkField<__half2, 12>::C C;
    // uint4 words of shared memory for a block of BS threads
    __host__ __device__ static constexpr int words(int BS) { return 8 * C::NC * BS + (C::RB ? (8 * BS * C::RB + 15) / 16 : 0); }
    static __device__ __forceinline__ uint4* chunks(uint4* st, int BS, int k) { return st + (size_t)k * C::NC * BS + threadIdx.x; }
    static __device__ __forceinline__ void* rem(uint4* st, int BS, int k)
    {
        return reinterpret_cast<char*>(st + 8 * C::NC * BS) + ((size_t)k * BS + threadIdx.x) * C::RB;
    }
    static __device__ __forceinline__ void issue(const LinkField<__half2, 12>& U, int par, int mu, int h, uint4* st,
                                                 int BS, int k, unsigned long long pol)
    {
        C::stage(U.block(par, mu), U.Vh, h, chunks(st, BS, k), rem(st, BS, k), BS, pol);
    }
    static __device__ __forceinline__ Mat3<float> get(uint4* st, int BS, int k)
    {
        uint32_t w[C::WORDS];
        C::unstage(chunks(st, BS, k), rem(st, BS, k), BS, w);
        return LinkField<__half2, 12>::decode(w);
    }
};

// ---------------------------------------------------------- spinor storage
//
// F64: the canonical layout, complex128 [h][3] (double2 per colour).
// F32: structure of arrays, float2 [c][Vh] per colour.
// F16: structure of arrays, __half2 [c][Vh] codes plus a float norm [Vh]; the
//      value is code * norm, the norm being the largest magnitude of the six
//      real components of the site.
// A multi field is n such fields back to back (stride = one field).

struct SpinorF64 {
    typedef double real;
    double2* p;
    // field k of a multi field whose fields are stride bytes apart
    __host__ __device__ __forceinline__ SpinorF64 at(int k, size_t stride) const
    {
        return SpinorF64{(double2*)((char*)p + (size_t)k * stride)};
    }
    __device__ __forceinline__ Vec3<double> load(int h) const
    {
        Vec3<double> v;
        const double2* q = p + (size_t)h * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) v.c[c] = to_cplx(__ldg(q + c));
        return v;
    }
    __device__ __forceinline__ Vec3<double> load_rw(int h) const
    {
        Vec3<double> v;
        const double2* q = p + (size_t)h * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) v.c[c] = to_cplx(q[c]);
        return v;
    }
    __device__ __forceinline__ void store(int h, const Vec3<double>& v) const
    {
        double2* q = p + (size_t)h * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) q[c] = make_double2(v.c[c].re, v.c[c].im);
    }
};

// F32: two planes per field, colours 0 and 1 as a float4 [Vh], colour 2 as a
// float2 [Vh] right after it (24 bytes per site, two vector loads).
struct SpinorF32 {
    typedef float real;
    float2* p;   // start of the field (the float4 plane)
    int Vh;
    __host__ __device__ __forceinline__ SpinorF32 at(int k, size_t stride) const
    {
        return SpinorF32{(float2*)((char*)p + (size_t)k * stride), Vh};
    }
    __device__ __forceinline__ const float4* pa() const { return reinterpret_cast<const float4*>(p); }
    __device__ __forceinline__ const float2* pb() const { return reinterpret_cast<const float2*>(pa() + Vh); }
    __device__ __forceinline__ Vec3<float> unpack(float4 a, float2 b) const
    {
        Vec3<float> v;
        v.c[0] = {a.x, a.y};
        v.c[1] = {a.z, a.w};
        v.c[2] = {b.x, b.y};
        return v;
    }
    __device__ __forceinline__ Vec3<float> load(int h) const { return unpack(__ldg(pa() + h), __ldg(pb() + h)); }
    __device__ __forceinline__ Vec3<float> load_rw(int h) const { return unpack(pa()[h], pb()[h]); }
    __device__ __forceinline__ void store(int h, const Vec3<float>& v) const
    {
        reinterpret_cast<float4*>(p)[h] = make_float4(v.c[0].re, v.c[0].im, v.c[1].re, v.c[1].im);
        const_cast<float2*>(pb())[h] = make_float2(v.c[2].re, v.c[2].im);
    }
};

// F16: one 16-byte record per site: three __half2 codes and the float norm;
// the value is code * norm, the norm being the largest magnitude of the six
// real components of the site.
struct SpinorF16 {
    typedef float real;
    uint4* p;
    int Vh;
    __host__ __device__ __forceinline__ SpinorF16 at(int k, size_t stride) const
    {
        return SpinorF16{(uint4*)((char*)p + (size_t)k * stride), Vh};
    }
    __device__ __forceinline__ Vec3<float> unpack(uint4 q) const
    {
        const float n = __uint_as_float(q.w);
        const unsigned int w[3] = {q.x, q.y, q.z};
        Vec3<float> v;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[c]));
            v.c[c].re = f.x * n;
            v.c[c].im = f.y * n;
        }
        return v;
    }
    __device__ __forceinline__ Vec3<float> load(int h) const { return unpack(__ldg(p + h)); }
    __device__ __forceinline__ Vec3<float> load_rw(int h) const { return unpack(p[h]); }
    // The site's value times the sign of sign bit sbit: the sign goes onto the
    // norm (one operation instead of six; code * (-n) = -(code * n) exactly).
    __device__ __forceinline__ Vec3<float> load_signed(int h, uint32_t sbit) const
    {
        uint4 q = __ldg(p + h);
        q.w ^= sbit;
        return unpack(q);
    }
    // Encode: norm = max |component| (float), code = RN_half(component / norm)
    // with an IEEE float division; a zero site stores zeros.
    __device__ __forceinline__ void store(int h, const Vec3<float>& v) const
    {
        float n = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) n = fmaxf(n, fmaxf(fabsf(v.c[c].re), fabsf(v.c[c].im)));
        unsigned int w[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float re = 0.f, im = 0.f;
            if (n > 0.f) {
                re = __fdiv_rn(v.c[c].re, n);
                im = __fdiv_rn(v.c[c].im, n);
            }
            const __half2 q = __floats2half2_rn(re, im);
            w[c] = *reinterpret_cast<const unsigned int*>(&q);
        }
        p[h] = make_uint4(w[0], w[1], w[2], __float_as_uint(n));
    }
};

// Neighbour spinors copied to shared memory ahead of their use (cp.async):
// a slot is one 16-byte word (a) plus, for float storage, one 8-byte word (b);
// get returns what the storage's load returns, get_flipped what load_flipped
// returns, from the same bytes.
template <class S> struct SpinorStage { static constexpr bool value = false; };
template <> struct SpinorStage<SpinorF32> {
    static constexpr bool value = true;
    static __device__ __forceinline__ void issue(const SpinorF32& in, int h, uint4* a, uint2* b)
    {
        cp_async16_ca(a, in.pa() + h);
        cp_async8_ca(b, in.pb() + h);
    }
    static __device__ __forceinline__ Vec3<float> get(const SpinorF32& in, const uint4* a, const uint2* b)
    {
        const uint4 q = *a;
        const uint2 r = *b;
        return in.unpack(make_float4(__uint_as_float(q.x), __uint_as_float(q.y), __uint_as_float(q.z),
                                     __uint_as_float(q.w)),
                         make_float2(__uint_as_float(r.x), __uint_as_float(r.y)));
    }
    static __device__ __forceinline__ Vec3<float> get_flipped(const SpinorF32& in, const uint4* a, const uint2* b,
                                                              uint32_t sbit)
    {
        return vflip(get(in, a, b), sbit);
    }
};
template <> struct SpinorStage<SpinorF16> {
    static constexpr bool value = true;
    static __device__ __forceinline__ void issue(const SpinorF16& in, int h, uint4* a, uint2*)
    {
        cp_async16_ca(a, in.p + h);
    }
    static __device__ __forceinline__ Vec3<float> get(const SpinorF16& in, const uint4* a, const uint2*)
    {
        return in.unpack(*a);
    }
    static __device__ __forceinline__ Vec3<float> get_flipped(const SpinorF16& in, const uint4* a, const uint2*,
                                                              uint32_t sbit)
    {
        uint4 q = *a;
        q.w ^= sbit;
        return in.unpack(q);
    }
};

// A neighbour's spinor times the hop's sign (sign bit sbit): the value with
// its components' signs flipped, or, for storage that can do it with fewer
// operations (a per-site norm), the same value formed at load.
template <class S>
__device__ __forceinline__ Vec3<typename S::real> load_flipped(const S& in, int h, uint32_t sbit)
{
    return vflip(in.load(h), sbit);
}
__device__ __forceinline__ Vec3<float> load_flipped(const SpinorF16& in, int h, uint32_t sbit)
{
    return in.load_signed(h, sbit);
}

// ------------------------------------------------------ temporal gauge
//
// The paper reads 6 links per site by fixing the temporal gauge (Sec. 4.3):
// with g(x, t = 0) = 1 and g(x, t + 1) = g(x, t) U_t(x, t), the links
// U'_mu(x) = g(x) U_mu(x) g(x + mu)^dagger have U'_t = 1 except on the last
// time slice, where U'_t(x, Lt - 1) = g(x, Lt - 1) U_t(x, Lt - 1).  Gauge
// covariance gives D[U'] = g D[U] g^dagger, so M x = b is solved as
// M' x' = g b, x = g^dagger x' (tgauge.cu builds g and U').
//
// U' is stored in the usual layout of its storage, the time planes holding
// U'_t exactly (the identity off the last slice), so every kernel computes
// D[U'] correctly from it.  A link field with tg = 1 tells the operator
// kernels to skip the identity time links: a time hop off the last slice
// adds the neighbour's spinor with no link load and no product.  The flag is
// a kernel argument, not a template parameter, so every kernel serves both.

// Link fields without the flag (used by code paths that never see
// temporal-gauge links) are always read in full.
template <class LF, class = void> struct HasTG : std::false_type {};
template <class LF> struct HasTG<LF, std::void_t<decltype(std::declval<LF>().tg)>> : std::true_type {};

// The time hops of output site s.h through identity links (tg = 1 only):
// forward unless the site is on the last slice (x + t wraps: s.fwd[3] < h),
// backward unless it is on slice 0 (x - t wraps: s.bwd[3] > h).
template <class LF>
__device__ __forceinline__ bool unit_fwd_time(const LF& U, const SiteNbrs& s)
{
    if constexpr (HasTG<LF>::value) return U.tg && s.fwd[3] > s.h;
    else return false;
}
template <class LF>
__device__ __forceinline__ bool unit_bwd_time(const LF& U, const SiteNbrs& s)
{
    if constexpr (HasTG<LF>::value) return U.tg && s.bwd[3] < s.h;
    else return false;
}
// hop number 2 mu + back (0..7) through an identity link
template <class LF>
__device__ __forceinline__ bool unit_hop(const LF& U, const SiteNbrs& s, int hop)
{
    return hop == 6 ? unit_fwd_time(U, s) : (hop == 7 ? unit_bwd_time(U, s) : false);
}

// acc += v (a hop through an identity link), one rounding per component:
// the sum the product with the identity matrix forms (mv_acc), and never
// contracted with a multiplication inside v's load (the half spinors' norm)
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
template <typename T>
__device__ __forceinline__ void hop_add(Vec3<T>& acc, const Vec3<T>& v)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc.c[a].re = add_rn(acc.c[a].re, v.c[a].re);
        acc.c[a].im = add_rn(acc.c[a].im, v.c[a].im);
    }
}

// ------------------------------------------------------------ reductions

template <int BS>
__device__ __forceinline__ double block_sum(double v, double* smem)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) smem[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (l < BS / 32) ? smem[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;   // valid in thread 0 (warp 0)
}

// Each block stores its partial sum; the last block to arrive (counted with an
// atomic after a fence) sees every partial.  Nobody waits, so the pattern is
// safe for any grid size and shape (all blocks of a 1-, 2- or 3-D grid are
// counted).  Returns true in all threads of the last block.
__device__ __forceinline__ bool arrive_last(unsigned int* counter, bool* smem_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int nblocks = gridDim.x * gridDim.y * gridDim.z;
        unsigned int prev = atomicAdd(counter, 1u);
        *smem_flag = (prev == nblocks - 1);
    }
    __syncthreads();
    return *smem_flag;
}

// Block sums of NB per-thread values at once (the bits of mask select them;
// mask is uniform over the block): each warp reduces through shuffles, one
// barrier, then thread k adds the warps' results for value k in warp order.
// Valid in thread k < NB for value k.  smem: BS / 32 * NB doubles.
template <int BS, int NB>
__device__ __forceinline__ double block_sum_n(const double* v, unsigned mask, double* smem)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        if (!(mask & (1u << k))) continue;
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (l == 0) smem[w * NB + k] = x;
    }
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < NB && (mask & (1u << threadIdx.x))) {
#pragma unroll
        for (int ww = 0; ww < BS / 32; ++ww) s += smem[ww * NB + threadIdx.x];
    }
    __syncthreads();
    return s;
}

// Deterministic sum of n partials by one block (fixed order for fixed n):
// thread j adds part[j], part[j + BS], ... in that order.  The loads are
// issued eight at a time so that they are in flight together (the last block
// of a reduction otherwise waits one L2 round trip per partial).
template <int BS>
__device__ __forceinline__ double sum_partials(const double* part, int n, double* smem)
{
    double s = 0.0;
    for (int k0 = threadIdx.x; k0 < n; k0 += 8 * BS) {
        double v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (k0 + j * BS < n) ? __ldcg(part + k0 + j * BS) : 0.0;
#pragma unroll
        for (int j = 0; j < 8; ++j) s += v[j];
    }
    return block_sum<BS>(s, smem);
}

// ------------------------------------- reductions in fixed 128-site chunks
//
// The vector kernels the autotuner may launch with different block sizes and
// sites per thread reduce in a shape that does not depend on either: every
// partial covers one chunk of 128 consecutive sites (four warps of 32); a warp
// reduces its 32 sites by a butterfly, the chunk adds its four warp sums in
// ascending order, and the final sum runs over the chunk partials with 128
// lanes in a fixed pattern.  All launch shapes therefore give the same bits.
constexpr int RCHUNK = 128;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// A block of BS threads with SPT sites per thread (thread t of the block holds
// sites base + j BS + t, base = blockIdx.x BS SPT): v[j] are the threads'
// per-site values.  Writes the block's BS SPT / 128 chunk partials to
// part[blockIdx.x * BS * SPT / 128 + c] (chunks past nchunks are skipped).
// smem: BS / 32 * SPT doubles.  All threads must call it.
template <int BS, int SPT>
__device__ __forceinline__ void chunk_partials(const double* v, double* part, int nchunks, double* smem)
{
    static_assert((BS * SPT) % RCHUNK == 0 && BS % 32 == 0, "chunks of 128 sites");
    constexpr int NW = BS / 32, NCH = BS * SPT / RCHUNK;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const double s = warp_sum(v[j]);
        if (lane == 0) smem[j * NW + w] = s;   // index = (site offset in the block) / 32
    }
    __syncthreads();
    if (threadIdx.x < NCH) {
        const int c = threadIdx.x, ch = blockIdx.x * NCH + c;
        const double x = ((smem[4 * c] + smem[4 * c + 1]) + smem[4 * c + 2]) + smem[4 * c + 3];
        if (ch < nchunks) part[ch] = x;
    }
    __syncthreads();
}

// Sum of n chunk partials in a fixed order by the first 128 threads of the
// block (BS >= 128; every thread must call it): lane l adds part[l],
// part[l + 128], ... in order, then the four warps' butterfly sums are added
// in ascending order.  Valid in thread 0.  smem: 4 doubles.
template <int BS>
__device__ __forceinline__ double sum_chunks(const double* part, int n, double* smem)
{
    static_assert(BS >= 128, "128 lanes");
    double s = 0.0;
    if (threadIdx.x < 128) {
        for (int k0 = threadIdx.x; k0 < n; k0 += 8 * 128) {
            double v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = (k0 + j * 128 < n) ? __ldcg(part + k0 + j * 128) : 0.0;
#pragma unroll
            for (int j = 0; j < 8; ++j) s += v[j];
        }
        s = warp_sum(s);
        if ((threadIdx.x & 31) == 0) smem[threadIdx.x >> 5] = s;
    }
    __syncthreads();
    const double r = ((smem[0] + smem[1]) + smem[2]) + smem[3];
    __syncthreads();
    return r;
}

// Two-level finish of a grid-wide sum over n unit partials part[0 .. n)
// (128-site chunks or one per block), in a fixed order, without a long serial
// tail.  Units form groups of RGROUP: the block that completes a group (an
// atomic count of the units written) sums the group's partials with one
// warp's butterfly into gpart[group] and resets the group's counter; the
// block that completes the last group sums the group partials in the fixed
// 128-lane pattern of sum_chunks.  Which block does a step does not change
// the bits.  Replaces "the last block to arrive sums all n partials", whose
// serial sum kept one SM busy for several microseconds after the others had
// finished (48^3 x 12: 5184 partials).
constexpr int RGROUP = 32;
struct GridSum {
    double* gpart;    // one partial per group
    unsigned* gcnt;   // units arrived per group: zero between uses (reset by each group's finisher)
};

// Called by all threads of every block after the block wrote its units
// part[u0 .. u0 + nu) (nu >= 1, all in one group: RGROUP is a multiple of
// the units per block).  True in the one block that finishes the sum, with
// the total in *total for every thread of that block; *cnt counts finished
// groups and is reset there.
template <int BS>
__device__ __forceinline__ bool grid_sum_finish(const double* part, int n, int u0, int nu, GridSum gs,
                                                unsigned* cnt, double* red, double* total)
{
    static_assert(BS >= 128, "the final sum uses 128 lanes");
    __shared__ int gs_flag;
    const int grp = u0 / RGROUP, ngroups = (n + RGROUP - 1) / RGROUP;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned gsz = (unsigned)min(RGROUP, n - grp * RGROUP);
        const unsigned prev = atomicAdd(gs.gcnt + grp, (unsigned)nu);
        gs_flag = (prev + (unsigned)nu == gsz) ? 1 : 0;
    }
    __syncthreads();
    if (!gs_flag) return false;
    if (threadIdx.x < 32) {
        const int j = grp * RGROUP + (int)threadIdx.x;
        const double v = warp_sum(j < n ? __ldcg(part + j) : 0.0);
        if (threadIdx.x == 0) {
            gs.gpart[grp] = v;
            gs.gcnt[grp] = 0;
            __threadfence();
            const unsigned prev = atomicAdd(cnt, 1u);
            gs_flag = (prev == (unsigned)ngroups - 1) ? 1 : 0;
        }
    }
    __syncthreads();
    if (!gs_flag) return false;
    *total = sum_chunks<BS>(gs.gpart, ngroups, red);
    if (threadIdx.x == 0) *cnt = 0;
    return true;
}

// Launch shape of a vector kernel: block size and sites per thread, coded
// (BS << 4) | SPT for the autotuner.
constexpr int vcfg(int BS, int SPT) { return (BS << 4) | SPT; }
constexpr int vcfg_BS(int c) { return c >> 4; }
constexpr int vcfg_SPT(int c) { return c & 15; }

}  // namespace stag
