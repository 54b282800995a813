// dslash.cu -- the half-lattice staggered operator D_eo / D_oe (Sec. 4.2,
// Eq. (staggered)) for every supported storage, one output site per thread.
#include "ctx.h"
#include "df64.cuh"
#include "dslash.cuh"

namespace stag {

template <class LF, class SIn, class SOut, int BS>
__global__ void __launch_bounds__(BS, (OpMinBlocksS<LF, SIn>::value)) k_dslash(Geom g, int p, LF U, SIn in, SOut out)
{
    const int h = blockIdx.x * BS + threadIdx.x;
    if (h >= g.Vh) return;
    out.store(h, dslash_site(g, p, h, U, in));
}

template <class LF, class SIn, class SOut>
static int run_dslash(stag_ctx ctx, const LF& U, const SIn& in, const SOut& out, int p,
                      cudaStream_t s)
{
    constexpr int BS = 128;
    const int grid = (ctx->g.Vh + BS - 1) / BS;
    k_dslash<LF, SIn, SOut, BS><<<grid, BS, 0, s>>>(ctx->g, p, U, in, out);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

int launch_dslash(stag_ctx ctx, int prec, int recon, int par_out, void* out, const void* in,
                  cudaStream_t s)
{
    const void* lk = nullptr;
    STAG_TRY(ensure_links(ctx, prec, recon, &lk));
    const int Vh = ctx->g.Vh;
    if (prec == STAG_F64) {
        SpinorF64 si{(double2*)in}, so{(double2*)out};
        if (recon == 18) return run_dslash(ctx, LinkField<double2, 18>{(const double2*)lk, Vh}, si, so, par_out, s);
        return run_dslash(ctx, LinkField<double2, 12>{(const double2*)lk, Vh}, si, so, par_out, s);
    }
    if (prec == STAG_F64X) {
        SpinorF64asDF si{(double2*)in}, so{(double2*)out};
        return run_dslash(ctx, LinkFieldDF<18>{(const float4*)lk, Vh}, si, so, par_out, s);
    }
    if (prec == STAG_F32) {
        SpinorF32 si{(float2*)in, Vh}, so{(float2*)out, Vh};
        if (recon == 18) return run_dslash(ctx, LinkField<float2, 18>{(const float2*)lk, Vh}, si, so, par_out, s);
        return run_dslash(ctx, LinkField<float2, 12>{(const float2*)lk, Vh}, si, so, par_out, s);
    }
    if (prec == STAG_F16) {
        SpinorF16 si{(uint4*)in, Vh}, so{(uint4*)out, Vh};
        if (recon == 18) return run_dslash(ctx, LinkField<__half2, 18>{(const __half2*)lk, Vh}, si, so, par_out, s);
        return run_dslash(ctx, LinkField<__half2, 12>{(const __half2*)lk, Vh}, si, so, par_out, s);
    }
    set_error("unsupported precision %d", prec);
    return STAG_EUNSUPPORTED;
}

// The operator on a precision's internal storage: as launch_dslash, except
// that STAG_F64X reads and writes double-float vectors (the storage of the
// double-float solver) instead of converting canonical doubles on the fly.
int launch_dslash_internal(stag_ctx ctx, int prec, int recon, int par_out, void* out, const void* in,
                           cudaStream_t s)
{
    if (prec != STAG_F64X) return launch_dslash(ctx, prec, recon, par_out, out, in, s);
    const void* lk = nullptr;
    STAG_TRY(ensure_links(ctx, prec, recon, &lk));
    return run_dslash(ctx, LinkFieldDF<18>{(const float4*)lk, ctx->g.Vh}, SpinorDF{(float4*)in},
                      SpinorDF{(float4*)out}, par_out, s);
}

}  // namespace stag
