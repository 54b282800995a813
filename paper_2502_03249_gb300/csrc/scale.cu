// scale.cu -- exact power-of-two normalisation of the fields the double
// precision solvers and the double-float operator take in.
//
// Double-float arithmetic (df64.cuh) carries a double as two floats, so it
// keeps 48 significant bits only inside the float exponent range (magnitudes
// from 2^-74 to 2^127), and the inner iterations of the mixed solvers store
// floats or halves.  A right-hand side b is therefore solved as
//   M x' = b',  b' = 2^-k b,  x = 2^k x',
// with k = floor(log2 max|b component|), so that b' has its largest component
// in [1, 2).  Multiplying by a power of two is exact (components more than
// 2^1022 below the largest may lose bits; they are below the double rounding
// of the largest anyway), M is linear, and the relative residual |b - Mx|/|b|
// is unchanged, so the solvers behave the same on b and on any 2^j b.  The
// double-float operator entry points scale their input the same way and the
// output back.
//
// Each field's exponent is found on the device (no host round trip): the
// largest magnitude by an atomic maximum over the bit patterns of the
// absolute values (non-negative doubles order like their bit patterns as
// unsigned integers), then k = ilogb(max) (0 for a zero field).
#include "ctx.h"
#include "df64.cuh"

namespace stag {

constexpr int SC_BS = 256;
constexpr int SC_ITEMS = 4;   // double2 elements per thread of the max pass

// bits[f] = max over field f of the bit pattern of |component|.  grid (gx, nfield)
__global__ void __launch_bounds__(SC_BS) k_field_maxabs(const double2* __restrict__ v, size_t field_elems,
                                                       unsigned long long* bits)
{
    const int f = blockIdx.y;
    const double2* q = v + (size_t)f * field_elems;
    unsigned long long m = 0;
    const size_t i0 = ((size_t)blockIdx.x * SC_BS) * SC_ITEMS + threadIdx.x;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        const size_t i = i0 + (size_t)j * SC_BS;
        if (i < field_elems) {
            const double2 d = q[i];
            const unsigned long long a = (unsigned long long)__double_as_longlong(fabs(d.x));
            const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(d.y));
            m = max(m, max(a, b));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ unsigned long long wm[SC_BS / 32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
#pragma unroll
        for (int w = 0; w < SC_BS / 32; ++w) b = max(b, wm[w]);
        // a NaN's pattern is above every finite one: the exponent pass treats it as 0
        if (b) atomicMax(bits + f, b);
    }
}

// kexp[f] = ilogb(largest magnitude of field f), 0 for a zero or non-finite field.
__global__ void k_field_exponent(const unsigned long long* bits, int nfield, int* kexp)
{
    const int f = threadIdx.x;
    if (f >= nfield) return;
    const double m = __longlong_as_double((long long)bits[f]);
    kexp[f] = (m > 0.0 && isfinite(m)) ? ilogb(m) : 0;
}

// out_f = 2^(sign * kexp[f * kstride]) in_f (in place allowed).  grid (gx, nfield)
__global__ void __launch_bounds__(SC_BS) k_field_scale(const double2* in, double2* out, size_t field_elems,
                                                      const int* kexp, int kstride, int sign)
{
    const int f = blockIdx.y;
    const size_t i = (size_t)blockIdx.x * SC_BS + threadIdx.x;
    if (i >= field_elems) return;
    const int k = sign * kexp[f * kstride];
    const size_t o = (size_t)f * field_elems + i;
    const double2 d = in[o];
    out[o] = make_double2(scalbn(d.x, k), scalbn(d.y, k));
}

// canonical doubles scaled by 2^-kexp[f] -> double-float pairs (SpinorDF storage)
__global__ void __launch_bounds__(SC_BS) k_field_split_scaled(const double2* __restrict__ in, float4* __restrict__ out,
                                                             size_t field_elems, const int* kexp, int extra)
{
    const int f = blockIdx.y;
    const size_t i = (size_t)blockIdx.x * SC_BS + threadIdx.x;
    if (i >= field_elems) return;
    const int k = -(kexp[f] + extra);
    const size_t o = (size_t)f * field_elems + i;
    const double2 d = in[o];
    const DF re = split_double(scalbn(d.x, k)), im = split_double(scalbn(d.y, k));
    out[o] = make_float4(re.hi, re.lo, im.hi, im.lo);
}

// double-float pairs -> canonical doubles scaled by 2^(kexp[f * kstride] + extra)
__global__ void __launch_bounds__(SC_BS) k_field_join_scaled(const float4* __restrict__ in, double2* __restrict__ out,
                                                            size_t field_elems, const int* kexp, int kstride,
                                                            int extra)
{
    const int f = blockIdx.y;
    const size_t i = (size_t)blockIdx.x * SC_BS + threadIdx.x;
    if (i >= field_elems) return;
    const int k = kexp[f * kstride] + extra;
    const size_t o = (size_t)f * field_elems + i;
    const float4 q = in[o];
    out[o] = make_double2(scalbn(df_to_double(DF(q.x, q.y)), k), scalbn(df_to_double(DF(q.z, q.w)), k));
}

static inline unsigned gx_of(size_t n, int per) { return (unsigned)((n + per - 1) / per); }

int ensure_scale_scratch(stag_ctx ctx)
{
    if (!ctx->scale_bits) STAG_CUDA_TRY(cudaMalloc(&ctx->scale_bits, sizeof(unsigned long long) * SCALE_SLOTS));
    if (!ctx->scale_k) STAG_CUDA_TRY(cudaMalloc(&ctx->scale_k, sizeof(int) * SCALE_SLOTS));
    return STAG_OK;
}

// Exponents of nfield fields of field_elems double2 each into ctx->scale_k[slot ...].
int field_exponents(stag_ctx ctx, const double2* v, int nfield, size_t field_elems, int slot, cudaStream_t s)
{
    if (nfield < 1 || slot < 0 || slot + nfield > SCALE_SLOTS) {
        set_error("field_exponents: %d fields at slot %d", nfield, slot);
        return STAG_EINVAL;
    }
    STAG_TRY(ensure_scale_scratch(ctx));
    STAG_CUDA_TRY(cudaMemsetAsync(ctx->scale_bits + slot, 0, sizeof(unsigned long long) * nfield, s));
    k_field_maxabs<<<dim3(gx_of(field_elems, SC_BS * SC_ITEMS), nfield), SC_BS, 0, s>>>(v, field_elems,
                                                                                      ctx->scale_bits + slot);
    k_field_exponent<<<1, 64, 0, s>>>(ctx->scale_bits + slot, nfield, ctx->scale_k + slot);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

// out = 2^-k in per field (k from slot; kstride 0: every field uses scale_k[slot]).
int scale_fields_in(stag_ctx ctx, const double2* in, double2* out, int nfield, size_t field_elems, int slot,
                    int kstride, cudaStream_t s)
{
    k_field_scale<<<dim3(gx_of(field_elems, SC_BS), nfield), SC_BS, 0, s>>>(in, out, field_elems,
                                                                           ctx->scale_k + slot, kstride, -1);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

int scale_fields_out(stag_ctx ctx, const double2* in, double2* out, int nfield, size_t field_elems, int slot,
                     int kstride, cudaStream_t s)
{
    k_field_scale<<<dim3(gx_of(field_elems, SC_BS), nfield), SC_BS, 0, s>>>(in, out, field_elems,
                                                                           ctx->scale_k + slot, kstride, 1);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

// Normalise nfield fields: exponents into slot, out = 2^-k in.
int normalise_fields(stag_ctx ctx, const double2* in, double2* out, int nfield, size_t field_elems, int slot,
                     cudaStream_t s)
{
    STAG_TRY(field_exponents(ctx, in, nfield, field_elems, slot, s));
    return scale_fields_in(ctx, in, out, nfield, field_elems, slot, 1, s);
}

// Canonical doubles -> double-float storage of 2^-(k + extra) in, k per field (slot).
int split_fields_scaled(stag_ctx ctx, const double2* in, float4* out, int nfield, size_t field_elems, int slot,
                        int extra, cudaStream_t s)
{
    k_field_split_scaled<<<dim3(gx_of(field_elems, SC_BS), nfield), SC_BS, 0, s>>>(in, out, field_elems,
                                                                                  ctx->scale_k + slot, extra);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

// Double-float storage -> canonical doubles 2^(k + extra) in.
int join_fields_scaled(stag_ctx ctx, const float4* in, double2* out, int nfield, size_t field_elems, int slot,
                       int kstride, int extra, cudaStream_t s)
{
    k_field_join_scaled<<<dim3(gx_of(field_elems, SC_BS), nfield), SC_BS, 0, s>>>(in, out, field_elems,
                                                                                 ctx->scale_k + slot, kstride, extra);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

// Exponent of the largest link element (host value; one stream synchronisation),
// computed once per upload and cached.
int link_max_exponent(stag_ctx ctx, int* out)
{
    if (ctx->link_exp_known) {
        *out = ctx->link_exp;
        return STAG_OK;
    }
    STAG_TRY(ensure_scale_scratch(ctx));
    const size_t n = (size_t)ctx->V * 4 * 9;
    STAG_TRY(field_exponents(ctx, (const double2*)ctx->links[0], 1, n, SCALE_SLOTS - 1, ctx->stream));
    int k = 0;
    STAG_CUDA_TRY(cudaMemcpyAsync(&k, ctx->scale_k + SCALE_SLOTS - 1, sizeof(int), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    ctx->link_exp = k;
    ctx->link_exp_known = true;
    *out = k;
    return STAG_OK;
}

// The float / half inner iterations keep M's products inside the float range
// only for links of moderate magnitude; solvers refuse other links.
int check_float_inner_links(stag_ctx ctx)
{
    int e = 0;
    STAG_TRY(link_max_exponent(ctx, &e));
    if (e > FLOAT_INNER_LINK_EXP || e < -FLOAT_INNER_LINK_EXP) {
        set_error("float / half inner iterations need links whose largest element lies within 2^-%d .. 2^%d "
                  "(here 2^%d); use inner_prec STAG_F64",
                  FLOAT_INNER_LINK_EXP, FLOAT_INNER_LINK_EXP + 1, e);
        return STAG_EUNSUPPORTED;
    }
    return STAG_OK;
}

}  // namespace stag
