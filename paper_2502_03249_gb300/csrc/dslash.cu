// dslash.cu -- the half-lattice staggered operator D_eo / D_oe (Sec. 4.2,
// Eq. (staggered)) for every supported storage, one output site per thread.
#include "ctx.h"
#include "df64.cuh"
#include "dslash.cuh"
#include "tune.h"

namespace stag {

template <class LF, class SIn, class SOut, int BS, int MODE>
__global__ void __launch_bounds__(BS, (OpMinBlocksS<LF, SIn>::value)) k_dslash(Geom g, int p, LF U, SIn in, SOut out)
{
    const int h = blockIdx.x * BS + threadIdx.x;
    if (h >= g.Vh) return;
    if constexpr (MODE != 0) {
        __shared__ uint4 st[StageWords<LF, SIn, BS, MODE>::value];
        out.store(h, dslash_site_staged<BS, MODE>(g, p, h, U, in, st));
    } else {
        out.store(h, dslash_site(g, p, h, U, in));
    }
}

// Half 12-real links and half spinors can be staged in shared memory
// (dslash_site_staged, stage = STAGE_* bits) where the context's decision says
// so: the autotuner's choice, timed by stag_dslash_repeat (an operator entry
// point outside stream capture), and the unstaged kernel until a decision
// exists.
template <class LF, class SIn, class SOut>
static int run_dslash(stag_ctx ctx, const LF& U, const SIn& in, const SOut& out, int p,
                      cudaStream_t s, int stage = 0)
{
    constexpr int BS = 128;
    const int grid = (ctx->g.Vh + BS - 1) / BS;
    if constexpr (LinkStage<LF>::value && SpinorStage<SIn>::value) {
        switch (stage) {
        case STAGE_LINKS: k_dslash<LF, SIn, SOut, BS, STAGE_LINKS><<<grid, BS, 0, s>>>(ctx->g, p, U, in, out); break;
        case STAGE_SPINORS: k_dslash<LF, SIn, SOut, BS, STAGE_SPINORS><<<grid, BS, 0, s>>>(ctx->g, p, U, in, out); break;
        case STAGE_LINKS | STAGE_SPINORS:
            k_dslash<LF, SIn, SOut, BS, STAGE_LINKS | STAGE_SPINORS><<<grid, BS, 0, s>>>(ctx->g, p, U, in, out);
            break;
        default: k_dslash<LF, SIn, SOut, BS, 0><<<grid, BS, 0, s>>>(ctx->g, p, U, in, out); break;
        }
    } else {
        k_dslash<LF, SIn, SOut, BS, 0><<<grid, BS, 0, s>>>(ctx->g, p, U, in, out);
    }
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

int launch_dslash(stag_ctx ctx, int prec, int recon, int par_out, void* out, const void* in,
                  cudaStream_t s, int links)
{
    if (prec == STAG_F64X)
        return dslash_f64x_canonical(ctx, par_out, (double2*)out, (const double2*)in, 1, links, 1, nullptr, s);
    const void* lk = nullptr;
    int tg = 0;
    STAG_TRY(op_links_for(ctx, links, prec, recon, &lk, &tg));
    const int Vh = ctx->g.Vh;
    if (prec == STAG_F64) {
        SpinorF64 si{(double2*)in}, so{(double2*)out};
        if (recon == 18) return run_dslash(ctx, LinkField<double2, 18>{(const double2*)lk, Vh, tg}, si, so, par_out, s);
        return run_dslash(ctx, LinkField<double2, 12>{(const double2*)lk, Vh, tg}, si, so, par_out, s);
    }
    if (prec == STAG_F32) {
        SpinorF32 si{(float2*)in, Vh}, so{(float2*)out, Vh};
        if (recon == 18) return run_dslash(ctx, LinkField<float2, 18>{(const float2*)lk, Vh, tg}, si, so, par_out, s);
        return run_dslash(ctx, LinkField<float2, 12>{(const float2*)lk, Vh, tg}, si, so, par_out, s);
    }
    if (prec == STAG_F16) {
        SpinorF16 si{(uint4*)in, Vh}, so{(uint4*)out, Vh};
        if (recon == 18) return run_dslash(ctx, LinkField<__half2, 18>{(const __half2*)lk, Vh, tg}, si, so, par_out, s);
        return run_dslash(ctx, LinkField<__half2, 12>{(const __half2*)lk, Vh, tg}, si, so, par_out, s,
                          ctx->half_stage[tg] > 0 ? ctx->half_stage[tg] : 0);
    }
    set_error("unsupported precision %d", prec);
    return STAG_EUNSUPPORTED;
}

int tune_half_stage(stag_ctx ctx, int links, void* out, const void* in)
{
    const void* lk = nullptr;
    int tg = 0;
    STAG_TRY(op_links_for(ctx, links, STAG_F16, 12, &lk, &tg));
    if (ctx->half_stage[tg] >= 0) return STAG_OK;
    const int Vh = ctx->g.Vh;
    const LinkField<__half2, 12> U{(const __half2*)lk, Vh, tg};
    const SpinorF16 si{(uint4*)in, Vh}, so{(uint4*)out, Vh};
    int choice = 0;
    STAG_TRY(tune_choice(ctx, tune_key(ctx, tg ? "dslash_stage_tg" : "dslash_stage", STAG_F16, 12, 1),
                         {0, STAGE_LINKS, STAGE_SPINORS, STAGE_LINKS | STAGE_SPINORS}, &choice,
                         [&](int c) { return run_dslash(ctx, U, si, so, 0, ctx->stream, c); }));
    ctx->half_stage[tg] = choice;
    return STAG_OK;
}

// Scratch of the double-float operator on canonical fields: nfield input and
// nfield output fields of double-float pairs (48 bytes per site each).
int dfx_fields(stag_ctx ctx, int nfield, float4** in, float4** out)
{
    const size_t per = lo_spinor_bytes(ctx->g, STAG_F64X);
    const size_t bytes = 2 * per * (size_t)nfield;
    if (ctx->dfx_tmp_bytes < bytes) {
        if (ctx->dfx_tmp) cudaFree(ctx->dfx_tmp);
        ctx->dfx_tmp = nullptr;
        ctx->dfx_tmp_bytes = 0;
        STAG_CUDA_TRY(cudaMalloc(&ctx->dfx_tmp, bytes));
        ctx->dfx_tmp_bytes = bytes;
    }
    *in = (float4*)ctx->dfx_tmp;
    *out = (float4*)((char*)ctx->dfx_tmp + per * (size_t)nfield);
    return STAG_OK;
}

// out_k = D_{par_out, 1-par_out} in_k (k < nfield) on canonical complex128
// fields in double-float arithmetic, accurate over the whole double range:
// each field is scaled by an exact power of two into double-float storage,
// the operator runs on that storage (the multi-vector kernel with rhs_block nb
// for nfield > 1), and the result is scaled back by the field's exponent and
// the links' (scale.cu).  The largest component is put at 2^60, high in the
// float range (outputs stay below 2^61 * 48 * 2^41 < 2^127), so that
// components down to 2^-134 of it keep their full 48 bits as well.
constexpr int DFX_TOP = 60;
int dslash_f64x_canonical(stag_ctx ctx, int par_out, double2* out, const double2* in, int nfield, int links,
                          int nb, int* nb_used, cudaStream_t s)
{
    const void* lk = nullptr;
    int tg = 0;
    STAG_TRY(op_links_for(ctx, links, STAG_F64X, 18, &lk, &tg));
    float4 *ti = nullptr, *to = nullptr;
    STAG_TRY(dfx_fields(ctx, nfield, &ti, &to));
    const size_t elems = (size_t)3 * ctx->g.Vh;
    STAG_TRY(field_exponents(ctx, in, nfield, elems, SLOT_OPER, s));
    STAG_TRY(split_fields_scaled(ctx, in, ti, nfield, elems, SLOT_OPER, -DFX_TOP, s));
    if (nfield == 1) {
        STAG_TRY(run_dslash(ctx, LinkFieldDF<18>{(const float4*)lk, ctx->g.Vh, tg}, SpinorDF{ti}, SpinorDF{to},
                            par_out, s));
        if (nb_used) *nb_used = 1;
    } else {
        STAG_TRY(multi_dslash_internal(ctx, STAG_F64X, 18, par_out, to, ti, nfield, nb, nb_used, links));
    }
    return join_fields_scaled(ctx, to, out, nfield, elems, SLOT_OPER, 1, ctx->df_link_exp - DFX_TOP, s);
}

// The operator on a precision's internal storage: as launch_dslash, except
// that STAG_F64X reads and writes double-float vectors (the storage of the
// double-float solver) instead of converting canonical doubles on the fly.
int launch_dslash_internal(stag_ctx ctx, int prec, int recon, int par_out, void* out, const void* in,
                           cudaStream_t s, int links)
{
    if (prec != STAG_F64X) return launch_dslash(ctx, prec, recon, par_out, out, in, s, links);
    const void* lk = nullptr;
    int tg = 0;
    STAG_TRY(op_links_for(ctx, links, prec, recon, &lk, &tg));
    return run_dslash(ctx, LinkFieldDF<18>{(const float4*)lk, ctx->g.Vh, tg}, SpinorDF{(float4*)in},
                      SpinorDF{(float4*)out}, par_out, s);
}

}  // namespace stag
