// pack.cu -- conversions between the canonical host-facing layouts and the
// internal device layouts: the gauge field upload, its 12-real / float / half
// copies (Sec. 4.3 link compression) and reduced-precision spinor codes.
#include "ctx.h"
#include "df64.cuh"

namespace stag {

// canonical U[i][mu][a][b] (complex128) -> internal F64/18:
//   out[((par*4 + mu)*9 + k)*Vh + i/2],  par = parity of site i
__global__ void k_pack_gauge(Geom g, const double2* __restrict__ U, double2* __restrict__ out)
{
    const long long V = 2LL * g.Vh;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (site, mu)
    if (idx >= 4 * V) return;
    const long long i = idx >> 2;
    const int mu = (int)(idx & 3);
    const int x = (int)(i % g.L[0]);
    long long r = i / g.L[0];
    const int y = (int)(r % g.L[1]);
    r /= g.L[1];
    const int z = (int)(r % g.L[2]);
    const int t = (int)(r / g.L[2]);
    const int par = (x + y + z + t) & 1;
    const long long h = i >> 1;
    const double2* src = U + idx * 9;
    double2* dst = out + ((size_t)(par * 4 + mu) * 9) * g.Vh + h;
#pragma unroll
    for (int k = 0; k < 9; ++k) dst[(size_t)k * g.Vh] = src[k];
}

// internal F64/18 -> F64/12: elements 0..5 (rows 0 and 1) kept, same layout.
__global__ void k_derive_links_f64_12(int Vh, const double2* __restrict__ in, double2* __restrict__ out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (par, mu, h)
    if (idx >= 8LL * Vh) return;
    const long long pm = idx / Vh, h = idx - pm * Vh;
#pragma unroll
    for (int k = 0; k < 6; ++k) out[(pm * 6 + k) * Vh + h] = in[(pm * 9 + k) * Vh + h];
}

// internal F64/18 -> float (EB = 8) or half (EB = 4) links in 16-byte chunks,
// elements 0..NE-1 (NE = 6 keeps rows 0 and 1).  Conversions round to nearest
// (double -> float, then float -> half).
template <int EB, int NE>
__global__ void k_derive_links_vec(int Vh, const double2* __restrict__ in, char* __restrict__ out)
{
    typedef LinkChunks<EB, NE> C;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (par, mu, h)
    if (idx >= 8LL * Vh) return;
    const long long pm = idx / Vh, h = idx - pm * Vh;
    uint32_t w[C::WORDS];
#pragma unroll
    for (int k = 0; k < NE; ++k) {
        const double2 v = in[(pm * 9 + k) * Vh + h];
        const float re = (float)v.x, im = (float)v.y;
        if constexpr (EB == 8) {
            w[2 * k] = __float_as_uint(re);
            w[2 * k + 1] = __float_as_uint(im);
        } else {
            const __half2 q = __floats2half2_rn(re, im);
            w[k] = *reinterpret_cast<const uint32_t*>(&q);
        }
    }
    C::store(out + (size_t)pm * C::BYTES * Vh, Vh, (int)h, w);
}

// internal F64/18 -> double-float split (hi = RN(x), lo = RN(x - hi)) per real
// of x = 2^-e U (e = 0 unless the links lie outside the double-float range).
__global__ void k_split_links(int Vh, const double2* __restrict__ in, float4* __restrict__ out, int e)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (par, mu, h)
    if (idx >= 8LL * Vh) return;
    const long long pm = idx / Vh, h = idx - pm * Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 v = in[(pm * 9 + k) * Vh + h];
        if (e) v = make_double2(scalbn(v.x, -e), scalbn(v.y, -e));
        const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
        out[(pm * 9 + k) * Vh + h] = make_float4(rh, __double2float_rn(v.x - (double)rh), ih,
                                                 __double2float_rn(v.y - (double)ih));
    }
}

int upload_gauge(stag_ctx ctx, const double* U, int on_device)
{
    const size_t n = (size_t)ctx->V * 4 * 9;
    const double2* src = (const double2*)U;
    double2* staging = nullptr;
    if (!on_device) {
        STAG_CUDA_TRY(cudaMallocAsync(&staging, n * sizeof(double2), ctx->stream));
        STAG_CUDA_TRY(cudaMemcpyAsync(staging, U, n * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
        src = staging;
    }
    // Derived copies are kept at their addresses and re-derived in place on
    // their next use: CUDA graphs captured by the solvers hold these pointers.
    for (int s = 1; s < 8; ++s) ctx->link_stale[s] = ctx->links[s] != nullptr;
    for (int s = 0; s < 8; ++s) ctx->tg_link_stale[s] = ctx->tg_links[s] != nullptr;
    ctx->tg_stale = true;
    ctx->link_exp_known = false;
    if (!ctx->links[0]) {
        STAG_CUDA_TRY(cudaMalloc(&ctx->links[0], n * sizeof(double2)));
        ctx->link_bytes[0] = n * sizeof(double2);
    }
    const long long work = 4 * ctx->V;
    const int BS = 256;
    k_pack_gauge<<<(unsigned)((work + BS - 1) / BS), BS, 0, ctx->stream>>>(ctx->g, src, (double2*)ctx->links[0]);
    STAG_CUDA_TRY(cudaGetLastError());
    if (staging) STAG_CUDA_TRY(cudaFreeAsync(staging, ctx->stream));
    if (!on_device) STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));   // host buffer may be reused
    ctx->have_gauge = true;
    return STAG_OK;
}

int derive_link_copy(stag_ctx ctx, const double2* src, int prec, int recon, int e, void** dst, size_t* bytes_out)
{
    const int NE = recon == 12 ? 6 : 9;
    const size_t esz = (prec == STAG_F64 || prec == STAG_F64X) ? 16 : (prec == STAG_F32 ? 8 : 4);
    const size_t bytes = (size_t)8 * ctx->g.Vh * NE * esz;
    void* p = *dst;
    if (!p) STAG_CUDA_TRY(cudaMalloc(&p, bytes));
    *dst = p;
    *bytes_out = bytes;
    const long long work = 8LL * ctx->g.Vh;
    const int BS = 256;
    const unsigned grid = (unsigned)((work + BS - 1) / BS);
    const int Vh = ctx->g.Vh;
    if (prec == STAG_F64X) k_split_links<<<grid, BS, 0, ctx->stream>>>(Vh, src, (float4*)p, e);
    else if (prec == STAG_F64) k_derive_links_f64_12<<<grid, BS, 0, ctx->stream>>>(Vh, src, (double2*)p);
    else if (prec == STAG_F32 && NE == 9) k_derive_links_vec<8, 9><<<grid, BS, 0, ctx->stream>>>(Vh, src, (char*)p);
    else if (prec == STAG_F32) k_derive_links_vec<8, 6><<<grid, BS, 0, ctx->stream>>>(Vh, src, (char*)p);
    else if (NE == 9) k_derive_links_vec<4, 9><<<grid, BS, 0, ctx->stream>>>(Vh, src, (char*)p);
    else k_derive_links_vec<4, 6><<<grid, BS, 0, ctx->stream>>>(Vh, src, (char*)p);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

int ensure_links(stag_ctx ctx, int prec, int recon, const void** out)
{
    if (!ctx->have_gauge) {
        set_error("no gauge field uploaded");
        return STAG_ENOGAUGE;
    }
    if (prec < STAG_F64 || prec > STAG_F64X || (recon != 18 && recon != 12) || (prec == STAG_F64X && recon != 18)) {
        set_error("unsupported links: prec %d recon %d", prec, recon);
        return STAG_EUNSUPPORTED;
    }
    const int slot = link_slot(prec, recon);
    if (!ctx->links[slot] || ctx->link_stale[slot]) {
        int e = 0;
        if (prec == STAG_F64X) {
            // links whose largest element leaves the double-float range are
            // stored as 2^-e U (operator results scaled back by 2^e)
            STAG_TRY(link_max_exponent(ctx, &e));
            ctx->df_link_exp = (e > DF_LINK_SAFE_EXP || e < -DF_LINK_SAFE_EXP) ? e : 0;
            e = ctx->df_link_exp;
        }
        STAG_TRY(derive_link_copy(ctx, (const double2*)ctx->links[0], prec, recon, e, &ctx->links[slot],
                                  &ctx->link_bytes[slot]));
        ctx->link_stale[slot] = false;
    }
    *out = ctx->links[slot];
    return STAG_OK;
}

int resolve_f64_arith(stag_ctx ctx, int requested, int* out)
{
    if (requested != STAG_F64 && requested != STAG_F64X) {
        set_error("f64_arith must be STAG_F64 or STAG_F64X");
        return STAG_EINVAL;
    }
    if (requested == STAG_F64X) {
        const void* lk = nullptr;
        STAG_TRY(ensure_links(ctx, STAG_F64X, 18, &lk));
        if (ctx->df_link_exp != 0) requested = STAG_F64;
    }
    *out = requested;
    return STAG_OK;
}

// ----------------------------------------------------------- spinor codes

size_t lo_spinor_bytes(const Geom& g, int prec)
{
    // STAG_F64: canonical complex128; STAG_F64X: double-float pairs, same size
    if (prec == STAG_F32) return (size_t)g.Vh * 3 * sizeof(float2);
    if (prec == STAG_F16) return (size_t)g.Vh * 16;   // three __half2 codes + float norm per site
    return (size_t)g.Vh * 3 * sizeof(double2);
}

template <class SOut>
__global__ void k_to_lo(int Vh, int nvec, const double2* __restrict__ in, SOut out, size_t out_stride_bytes)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nvec * Vh) return;
    const int v = (int)(idx / Vh), h = (int)(idx - (long long)v * Vh);
    Vec3<float> f;
    const double2* q = in + ((size_t)v * Vh + h) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        f.c[c].re = (float)q[c].x;
        f.c[c].im = (float)q[c].y;
    }
    out.at(v, out_stride_bytes).store(h, f);
}

template <class SIn>
__global__ void k_from_lo(int Vh, int nvec, SIn in, size_t in_stride_bytes, double2* __restrict__ out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nvec * Vh) return;
    const int v = (int)(idx / Vh), h = (int)(idx - (long long)v * Vh);
    const Vec3<float> f = in.at(v, in_stride_bytes).load_rw(h);
    double2* q = out + ((size_t)v * Vh + h) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) q[c] = make_double2((double)f.c[c].re, (double)f.c[c].im);
}

// canonical complex128 <-> double-float storage (the double-float solver's vectors)
__global__ void k_split_spinor(size_t n, const double2* __restrict__ in, float4* __restrict__ out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 d = in[i];
    const DF re = split_double(d.x), im = split_double(d.y);
    out[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
}

__global__ void k_df_to_double(size_t n, const float4* __restrict__ x, double2* __restrict__ out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 f = x[i];
    out[i] = make_double2(df_to_double(DF(f.x, f.y)), df_to_double(DF(f.z, f.w)));
}

int convert_f64_to_lo(stag_ctx ctx, int prec, const double2* in, void* out, int nvec, cudaStream_t s)
{
    const int Vh = ctx->g.Vh;
    const long long work = (long long)nvec * Vh;
    const int BS = 256;
    const unsigned grid = (unsigned)((work + BS - 1) / BS);
    const size_t stride = lo_spinor_bytes(ctx->g, prec);
    if (prec == STAG_F64X) {
        const size_t n = (size_t)nvec * Vh * 3;
        k_split_spinor<<<(unsigned)((n + BS - 1) / BS), BS, 0, s>>>(n, in, (float4*)out);
    } else if (prec == STAG_F32) {
        k_to_lo<SpinorF32><<<grid, BS, 0, s>>>(Vh, nvec, in, SpinorF32{(float2*)out, Vh}, stride);
    } else if (prec == STAG_F16) {
        k_to_lo<SpinorF16><<<grid, BS, 0, s>>>(Vh, nvec, in, SpinorF16{(uint4*)out, Vh}, stride);
    } else {
        set_error("convert_f64_to_lo: bad precision %d", prec);
        return STAG_EUNSUPPORTED;
    }
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

int convert_lo_to_f64(stag_ctx ctx, int prec, const void* in, double2* out, int nvec, cudaStream_t s)
{
    const int Vh = ctx->g.Vh;
    const long long work = (long long)nvec * Vh;
    const int BS = 256;
    const unsigned grid = (unsigned)((work + BS - 1) / BS);
    const size_t stride = lo_spinor_bytes(ctx->g, prec);
    if (prec == STAG_F64X) {
        const size_t n = (size_t)nvec * Vh * 3;
        k_df_to_double<<<(unsigned)((n + BS - 1) / BS), BS, 0, s>>>(n, (const float4*)in, out);
    } else if (prec == STAG_F32) {
        k_from_lo<SpinorF32><<<grid, BS, 0, s>>>(Vh, nvec, SpinorF32{(float2*)in, Vh}, stride, out);
    } else if (prec == STAG_F16) {
        k_from_lo<SpinorF16><<<grid, BS, 0, s>>>(Vh, nvec, SpinorF16{(uint4*)in, Vh}, stride, out);
    } else {
        set_error("convert_lo_to_f64: bad precision %d", prec);
        return STAG_EUNSUPPORTED;
    }
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

}  // namespace stag
