// df64.cuh -- double-float ("f32x2") arithmetic for the double-precision
// operator on GB300.
//
// GB300 runs FP64 at 1/64 of the FP32 rate (about 1.2 TFLOP/s), which makes a
// double-precision Dslash ALU-bound at ~40 % of its HBM roofline.  Here each
// double is carried as an unevaluated sum hi + lo of two floats (48-bit
// significand) and the hop sums run on the FP32 pipe:
//
//  * product of two double-floats x*y: hi part p = RN(xh*yh) and its exact
//    error RN(xh*yh - p) by one FMA, plus the cross terms xh*yl + xl*yh
//    (the xl*yl term is below 2^-48 relative and dropped);
//  * accumulation: the hi parts are summed with Knuth's error-free TwoSum, the
//    rounding errors and low parts are collected in a float companion, so a
//    whole hop sum keeps ~2^-44 relative to the sum of magnitudes.
//
// Every operation uses the _rn intrinsics so the compiler cannot contract or
// reassociate the error-free transformations.  Inputs are doubles: the links
// are split once at upload (hi = RN(x), lo = RN(x - hi) in double), the
// spinors are split on load with integer operations only (no FP64 instruction
// in the hot loop); results are formed as double(hi) + double(lo).  The
// integer split keeps the full 48 bits for |x| >= 2^-74 (smaller magnitudes
// keep 24 bits; zero and subnormal doubles become zero).
#pragma once

#include "dslash.cuh"

namespace stag {

struct DF {
    float hi, lo;
    __device__ __forceinline__ DF() {}
    __device__ __forceinline__ DF(int v) : hi((float)v), lo(0.f) {}
    __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ DF flip(DF v, uint32_t sbit)
{
    return DF(__uint_as_float(__float_as_uint(v.hi) ^ sbit), __uint_as_float(__float_as_uint(v.lo) ^ sbit));
}

// acc += s * x * y, s = +1 or -1 given as a sign bit applied to x.
__device__ __forceinline__ void df_mac(DF& acc, const DF& x, const DF& y)
{
    const float ph = __fmul_rn(x.hi, y.hi);
    float pl = __fmaf_rn(x.hi, y.hi, -ph);
    pl = __fmaf_rn(x.hi, y.lo, pl);
    pl = __fmaf_rn(x.lo, y.hi, pl);
    // TwoSum(acc.hi, ph)
    const float s = __fadd_rn(acc.hi, ph);
    const float bb = __fsub_rn(s, acc.hi);
    const float e = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(ph, bb));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pl));
}

__device__ __forceinline__ DF df_neg(const DF& x) { return DF(-x.hi, -x.lo); }

// acc += U v
template <>
__device__ __forceinline__ void mv_acc<DF>(Vec3<DF>& acc, const Mat3<DF>& U, const Vec3<DF>& v)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const Cplx<DF> u = U.m[a * 3 + b];
            df_mac(acc.c[a].re, u.re, v.c[b].re);
            df_mac(acc.c[a].re, df_neg(u.im), v.c[b].im);
            df_mac(acc.c[a].im, u.re, v.c[b].im);
            df_mac(acc.c[a].im, u.im, v.c[b].re);
        }
    }
}

// acc += U^dagger v
template <>
__device__ __forceinline__ void mdv_acc<DF>(Vec3<DF>& acc, const Mat3<DF>& U, const Vec3<DF>& v)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const Cplx<DF> u = U.m[b * 3 + a];
            df_mac(acc.c[a].re, u.re, v.c[b].re);
            df_mac(acc.c[a].re, u.im, v.c[b].im);
            df_mac(acc.c[a].im, u.re, v.c[b].im);
            df_mac(acc.c[a].im, df_neg(u.im), v.c[b].re);
        }
    }
}

// Split a double into hi + lo floats with integer operations only:
// hi = x truncated to 24 significant bits, lo = the remaining 29 bits rounded
// to 24 bits (exact for |x| in the float range with |x| >= 2^-74).
__device__ __forceinline__ DF split_double(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
    const unsigned sign = h32 & 0x80000000u;
    const int e = (int)((h32 >> 20) & 0x7FFu);
    const int ef = e - 896;   // float biased exponent of x (1023 - 127 = 896)
    if (ef < 1 || ef > 254) {
        // zero, subnormal, or outside the float range: no split
        return DF(__double2float_rn(x), 0.f);
    }
    const float hi = __uint_as_float(sign | ((unsigned)ef << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29));
    const unsigned m29 = l32 & 0x1FFFFFFFu;   // value m29 * 2^(e - 1075)
    const int es = e - 948;                   // float biased exponent of 2^(e - 1075)
    float lo = 0.f;
    if (es >= 1) lo = __fmul_rn(__uint2float_rn(m29), __uint_as_float((unsigned)es << 23));
    return DF(hi, __uint_as_float(__float_as_uint(lo) | sign));
}

__device__ __forceinline__ double df_to_double(const DF& v) { return (double)v.hi + (double)v.lo; }

// split_double(2^-k x) with the scaling done on the exponent field (integer
// operations only): exact, like the split itself, for 2^-k |x| in
// [2^-74, 2^128).
__device__ __forceinline__ DF split_double_scaled(double x, int k)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FFu);
    if (e == 0) return DF(0.f, 0.f);   // zero or subnormal: far below any normalised field's scale
    const int es = e - k;
    if (es < 1 || es > 2046) return split_double(scalbn(x, -k));   // outside the double range: the slow path
    return split_double(__longlong_as_double((long long)((b & ~(0x7FFull << 52)) | ((unsigned long long)es << 52))));
}

// 2^k f as a double from the float's fields (integer operations only), for a
// normal float f and a result inside the normal double range (0 for a zero
// or subnormal f, whose contribution is below the rounding of the sum it
// enters).
__device__ __forceinline__ double f2d_scaled(float f, int k)
{
    const uint32_t u = __float_as_uint(f);
    const int e = (int)((u >> 23) & 0xFFu);
    if (e == 0) return 0.0;
    const int ed = e + 896 + k;   // 1023 - 127 = 896
    if (ed < 1 || ed > 2046) return scalbn((double)f, k);
    return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                            ((unsigned long long)ed << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// 2^k (hi + lo) in double: one FP64 addition
__device__ __forceinline__ double df_to_double_scaled(const DF& v, int k)
{
    return f2d_scaled(v.hi, k) + f2d_scaled(v.lo, k);
}

// Canonical double spinor ([h][3] complex128) read and written as double-floats.
struct SpinorF64asDF {
    typedef DF real;
    double2* p;
    __host__ __device__ __forceinline__ SpinorF64asDF at(int k, size_t stride) const
    {
        return SpinorF64asDF{(double2*)((char*)p + (size_t)k * stride)};
    }
    __device__ __forceinline__ Vec3<DF> load(int h) const
    {
        Vec3<DF> v;
        const double2* q = p + (size_t)h * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 d = __ldg(q + c);
            v.c[c].re = split_double(d.x);
            v.c[c].im = split_double(d.y);
        }
        return v;
    }
    __device__ __forceinline__ void store(int h, const Vec3<DF>& v) const
    {
        double2* q = p + (size_t)h * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) q[c] = make_double2(df_to_double(v.c[c].re), df_to_double(v.c[c].im));
    }
};

// ---------------------------------------------------- double-float vectors
//
// The double-float solver keeps its Krylov vectors as double-floats, so that
// no FP64 instruction (conversion or arithmetic) runs per site inside the
// iteration: the BLAS below and the operator's loads and stores use the FP32
// pipe only.  Stored values are normalised (|lo| <= ulp(hi) / 2).

// Knuth's error-free sum: s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (s, e) -> normalised double-float (Dekker's fast two-sum, |e| small against s)
__device__ __forceinline__ DF df_norm(float s, float e)
{
    const float h = __fadd_rn(s, e);
    return DF(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ DF df_add(const DF& a, const DF& b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return df_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

// a x + y: the product's high part and its exact FMA error plus the cross
// terms, summed into y with an error-free sum of the high parts.
__device__ __forceinline__ DF df_fma(const DF& a, const DF& x, const DF& y)
{
    const float ph = __fmul_rn(a.hi, x.hi);
    float pl = __fmaf_rn(a.hi, x.hi, -ph);
    pl = __fmaf_rn(a.hi, x.lo, pl);
    pl = __fmaf_rn(a.lo, x.hi, pl);
    float s, e;
    two_sum(y.hi, ph, s, e);
    return df_norm(s, __fadd_rn(e, __fadd_rn(y.lo, pl)));
}

// Double-float vector storage: per site three float4 (re_hi, re_lo, im_hi,
// im_lo) in the canonical site order, 48 bytes like a double spinor.
struct SpinorDF {
    typedef DF real;
    float4* p;
    __host__ __device__ __forceinline__ SpinorDF at(int k, size_t stride) const
    {
        return SpinorDF{(float4*)((char*)p + (size_t)k * stride)};
    }
    __device__ __forceinline__ Vec3<DF> load(int h) const
    {
        Vec3<DF> v;
        const float4* q = p + (size_t)h * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 f = __ldg(q + c);
            v.c[c].re = DF(f.x, f.y);
            v.c[c].im = DF(f.z, f.w);
        }
        return v;
    }
    // for vectors this kernel also writes
    __device__ __forceinline__ Vec3<DF> load_rw(int h) const
    {
        Vec3<DF> v;
        const float4* q = p + (size_t)h * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 f = q[c];
            v.c[c].re = DF(f.x, f.y);
            v.c[c].im = DF(f.z, f.w);
        }
        return v;
    }
    __device__ __forceinline__ void store(int h, const Vec3<DF>& v) const
    {
        float4* q = p + (size_t)h * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const DF re = df_norm(v.c[c].re.hi, v.c[c].re.lo), im = df_norm(v.c[c].im.hi, v.c[c].im.lo);
            q[c] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
    }
};

// Block sum of one double-float per thread: warps reduce in double-float
// through shuffles (every lane ends with the same bits, so the order is
// fixed), warp results are combined in double.  Valid in thread 0.
template <int BS>
__device__ __forceinline__ double block_sum_df(DF v, double* smem)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DF w(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
        v = df_add(v, w);
    }
    const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) smem[wi] = df_to_double(v);
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (l < BS / 32) ? smem[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;
}

// Links split at upload: per complex element a float4 (re_hi, re_lo, im_hi,
// im_lo), same structure-of-arrays layout and byte count as the double copy.
template <int RECON>
struct LinkFieldDF {
    typedef DF real;
    typedef float4 store;
    static_assert(RECON == 18, "double-float links are stored with 18 reals");
    const float4* base;
    int Vh;
    int tg = 0;   // temporal-gauge links (common.cuh)
    __device__ __forceinline__ Mat3<DF> load(int par, int mu, int h) const
    {
        Mat3<DF> U;
        const float4* q = base + ((size_t)(par * 4 + mu) * 9) * Vh + h;
        const unsigned long long pol = l2_evict_first_policy();
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float4 f = ld_stream(q + (size_t)k * Vh, pol);
            U.m[k].re = DF(f.x, f.y);
            U.m[k].im = DF(f.z, f.w);
        }
        return U;
    }
};

// ------------------------------------------- sums of float site values
//
// The reductions of the float kernels (the mixed and batched solvers' inner
// iterations) add float site values across the warp in float-float
// arithmetic (Knuth's TwoSum, FP32 pipe) and convert the warp sum to double
// once: no FP64 addition per lane, which on GB300 (FP64 at 1/64 of the FP32
// rate) cost a sizable part of those kernels.  Same fixed butterfly shape as
// the double sums, so the results do not depend on the launch shape.

// Warp sum of one float per lane, in double (every lane gets the same bits).
__device__ __forceinline__ double warp_sum(float v)
{
    DF x(v, 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DF y(__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o));
        x = df_add(x, y);
    }
    return df_to_double_scaled(x, 0);
}

// Warp sums of N float values per lane (N a power of two, at most 32), each
// equal bit for bit to warp_sum of that value, for about the cost of one:
// the first log2 N levels of the butterfly are transposed -- at the level of
// offset o a lane keeps the half of its values that its lane bit o selects
// and adds the partner's copies of them -- so every level pairs the same
// lanes as warp_sum and df_add is commutative bit for bit (its TwoSum error
// is exact in either order).  Value k ends in the lanes k (32 / N) ...
// (k + 1) (32 / N) - 1; warp_sum_n_lane(k) names the first of them.
template <int N>
__device__ __forceinline__ double warp_sum_n(const float* v)
{
    static_assert(N >= 1 && N <= 32 && (N & (N - 1)) == 0, "N a power of two <= 32");
    const int lane = threadIdx.x & 31;
    DF x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = DF(v[i], 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int m = (N * o) / 16;   // values a lane holds before this level
        if (m > 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < m / 2; ++i) {
                const DF keep = up ? x[i + m / 2] : x[i];
                const DF send = up ? x[i] : x[i + m / 2];
                const DF recv(__shfl_xor_sync(0xffffffffu, send.hi, o), __shfl_xor_sync(0xffffffffu, send.lo, o));
                x[i] = df_add(keep, recv);
            }
        } else {
            const DF y(__shfl_xor_sync(0xffffffffu, x[0].hi, o), __shfl_xor_sync(0xffffffffu, x[0].lo, o));
            x[0] = df_add(x[0], y);
        }
    }
    return df_to_double_scaled(x[0], 0);
}
template <int N>
__device__ __forceinline__ int warp_sum_n_lane(int k) { return k * (32 / N); }

// block_sum (common.cuh) of float values
template <int BS>
__device__ __forceinline__ double block_sum(float v, double* smem)
{
    const double x = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) smem[w] = x;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (l < BS / 32) ? smem[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;
}

// block_sum_n (common.cuh) of float values
template <int BS, int NB>
__device__ __forceinline__ double block_sum_n(const float* v, unsigned mask, double* smem)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if constexpr ((NB & (NB - 1)) == 0) {
        // values outside mask are zero: summed, not stored
        const double x = warp_sum_n<NB>(v);
        const int k = l / (32 / NB);
        if (l == warp_sum_n_lane<NB>(k) && (mask & (1u << k))) smem[w * NB + k] = x;
    } else {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            if (!(mask & (1u << k))) continue;
            const double x = warp_sum(v[k]);
            if (l == 0) smem[w * NB + k] = x;
        }
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

// chunk_partials (common.cuh) of float values
template <int BS, int SPT>
__device__ __forceinline__ void chunk_partials(const float* v, double* part, int nchunks, double* smem)
{
    static_assert((BS * SPT) % RCHUNK == 0 && BS % 32 == 0, "chunks of 128 sites");
    constexpr int NW = BS / 32, NCH = BS * SPT / RCHUNK;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr ((SPT & (SPT - 1)) == 0) {
        const double s = warp_sum_n<SPT>(v);
        const int j = lane / (32 / SPT);
        if (lane == warp_sum_n_lane<SPT>(j)) smem[j * NW + w] = s;
    } else {
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            const double s = warp_sum(v[j]);
            if (lane == 0) smem[j * NW + w] = s;
        }
    }
    __syncthreads();
    if (threadIdx.x < NCH) {
        const int c = threadIdx.x, ch = blockIdx.x * NCH + c;
        const double x = ((smem[4 * c] + smem[4 * c + 1]) + smem[4 * c + 2]) + smem[4 * c + 3];
        if (ch < nchunks) part[ch] = x;
    }
    __syncthreads();
}

// acc += v, exactly summed into the accumulator (the identity hops of
// temporal-gauge links: the sum df_mac forms for the product 1 * v)
__device__ __forceinline__ void df_acc(DF& acc, const DF& v)
{
    float s, e;
    two_sum(acc.hi, v.hi, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, v.lo));
}
template <>
__device__ __forceinline__ void hop_add<DF>(Vec3<DF>& acc, const Vec3<DF>& v)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        df_acc(acc.c[a].re, v.c[a].re);
        df_acc(acc.c[a].im, v.c[a].im);
    }
}

template <int R> struct OpMinBlocks<LinkFieldDF<R>> { static constexpr int value = 5; };
// on double-float vectors (no conversions) the operator fits 72 registers:
// 7 blocks per SM, 32^3 x 8 in 1.2 waves (measured 30.4 against 32.3 us;
// 48^3 x 12 unchanged)
template <int R> struct OpMinBlocksS<LinkFieldDF<R>, SpinorDF> { static constexpr int value = 7; };

// Double-float operator results enter double-precision epilogues as double.
template <> struct VConv<double, DF> {
    static __device__ __forceinline__ Vec3<double> f(const Vec3<DF>& v)
    {
        Vec3<double> o;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o.c[c].re = df_to_double(v.c[c].re);
            o.c[c].im = df_to_double(v.c[c].im);
        }
        return o;
    }
};
}  // namespace stag
