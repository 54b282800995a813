// multi.cu -- the multi-vector operator (Sec. 4.3, NMULTI): each link loaded
// once per site for a block of right-hand sides, the block chosen by the
// autotuner; used by the batched solvers, stag_dslash_multi and the
// measurement entry points.
#include "batched_impl.cuh"

namespace stag {

// Multi operator pass for the autotuner and the public multi Dslash.
template <class LF, class S, int NB>
__global__ void __launch_bounds__(BBS, (MultiMinBlocks<LF, NB>::value)) k_multi_dslash(Geom g, int p, LF U, S in,
                                                                                      S out, size_t stride, int nrhs)
{
    const int k0 = blockIdx.y * NB;
    unsigned mask = 0;
#pragma unroll
    for (int k = 0; k < NB; ++k)
        if (k0 + k < nrhs) mask |= 1u << k;
    const int h = blockIdx.x * BBS + threadIdx.x;
    if (h >= g.Vh) return;
    Vec3<typename LF::real> acc[NB];
    dslash_site_multi<LF, S, NB>(g, p, h, U, in, stride, k0, mask, acc);
#pragma unroll
    for (int k = 0; k < NB; ++k)
        if (mask & (1u << k)) out.at(k0 + k, stride).store(h, acc[k]);
}

template <class LF, class S>
int launch_multi_dslash_nb(stag_ctx ctx, int nb, const LF& U, const S& in, const S& out, size_t stride, int nrhs,
                           int p, cudaStream_t s)
{
    const int gx = (ctx->g.Vh + BBS - 1) / BBS;
    const dim3 grid(gx, (nrhs + nb - 1) / nb);
    switch (nb) {
    case 1: k_multi_dslash<LF, S, 1><<<grid, BBS, 0, s>>>(ctx->g, p, U, in, out, stride, nrhs); break;
    case 2: k_multi_dslash<LF, S, 2><<<grid, BBS, 0, s>>>(ctx->g, p, U, in, out, stride, nrhs); break;
    case 4: k_multi_dslash<LF, S, 4><<<grid, BBS, 0, s>>>(ctx->g, p, U, in, out, stride, nrhs); break;
    case 8: k_multi_dslash<LF, S, 8><<<grid, BBS, 0, s>>>(ctx->g, p, U, in, out, stride, nrhs); break;
    case 16: k_multi_dslash<LF, S, 16><<<grid, BBS, 0, s>>>(ctx->g, p, U, in, out, stride, nrhs); break;
    default: set_error("unsupported rhs block %d", nb); return STAG_EINVAL;
    }
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

template <class LF, class S, int G, int NBT>
static int launch_tile(stag_ctx ctx, const LF& U, const S& in, const S& out, size_t stride, int nrhs, int p,
                       cudaStream_t s)
{
    constexpr int TS = 32 * TileSW<G>::value;
    const dim3 grid((ctx->g.Vh + TS - 1) / TS, (nrhs + G * NBT - 1) / (G * NBT));
    k_tile_dslash<LF, S, G, NBT><<<grid, TS * G, 0, s>>>(ctx->g, p, U, in, out, stride, nrhs);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

// One multi-vector operator pass in configuration cfg (multi_tile.cuh):
// G = 1 the register-blocked kernel with NBT right-hand sides per thread,
// G > 1 the tile kernel (float arithmetic only).
template <class LF, class S>
int launch_multi_cfg(stag_ctx ctx, int cfg, const LF& U, const S& in, const S& out, size_t stride, int nrhs, int p,
                     cudaStream_t s)
{
    if (mcfg_G(cfg) == 1) return launch_multi_dslash_nb(ctx, mcfg_NBT(cfg), U, in, out, stride, nrhs, p, s);
    if constexpr (TileOK<LF>::value) {
        switch (cfg) {
        case mcfg(2, 1): return launch_tile<LF, S, 2, 1>(ctx, U, in, out, stride, nrhs, p, s);
        case mcfg(2, 2): return launch_tile<LF, S, 2, 2>(ctx, U, in, out, stride, nrhs, p, s);
        case mcfg(4, 1): return launch_tile<LF, S, 4, 1>(ctx, U, in, out, stride, nrhs, p, s);
        case mcfg(2, 4): return launch_tile<LF, S, 2, 4>(ctx, U, in, out, stride, nrhs, p, s);
        case mcfg(4, 2): return launch_tile<LF, S, 4, 2>(ctx, U, in, out, stride, nrhs, p, s);
        case mcfg(8, 1): return launch_tile<LF, S, 8, 1>(ctx, U, in, out, stride, nrhs, p, s);
        case mcfg(2, 8): return launch_tile<LF, S, 2, 8>(ctx, U, in, out, stride, nrhs, p, s);
        case mcfg(4, 4): return launch_tile<LF, S, 4, 4>(ctx, U, in, out, stride, nrhs, p, s);
        case mcfg(8, 2): return launch_tile<LF, S, 8, 2>(ctx, U, in, out, stride, nrhs, p, s);
        case mcfg(16, 1): return launch_tile<LF, S, 16, 1>(ctx, U, in, out, stride, nrhs, p, s);
        default: break;
        }
    }
    set_error("unsupported multi-vector configuration (%d groups x %d)", mcfg_G(cfg), mcfg_NBT(cfg));
    return STAG_EINVAL;
}

// The configuration of an explicitly requested rhs block (0: autotuned).
template <class LF>
int multi_cfg_of_block(int block)
{
    if (!TileOK<LF>::value || block <= 1) return mcfg(1, block < 1 ? 1 : block);
    return block == 2 ? mcfg(2, 1) : block == 4 ? mcfg(4, 1) : block == 8 ? mcfg(4, 2) : mcfg(4, 4);
}

// Apply the multi Dslash on internal-storage multi fields; nb = 0 asks the
// autotuner (timed on these buffers, cached per context and shape) for the
// configuration; *nb_used receives the right-hand sides sharing a link load.
template <class LF, class S>
static int multi_dslash_tuned(stag_ctx ctx, const char* tag, int tag_prec, int tag_recon, const LF& U, const S& in,
                              const S& out, size_t stride, int nrhs, int p, int nb, int* nb_used,
                              int* cfg_used = nullptr)
{
    int cfg = nb >= 256 ? nb : multi_cfg_of_block<LF>(nb);   // >= 256: an explicit configuration code
    if (nb >= 256) {
        bool ok = false;
        for (int c : multi_cfg_candidates<LF>(16)) ok |= c == cfg;
        if (!ok) {
            set_error("multi-vector configuration %d x %d is not offered for this storage", mcfg_G(cfg), mcfg_NBT(cfg));
            return STAG_EINVAL;
        }
    }
    if (nb == 0) {
        // the default when timing is off: the whole batch per link load (at
        // most 16; 4 for the register-blocked double kernels)
        int cap = 1;
        while (cap < nrhs && cap < 16) cap *= 2;
        cfg = multi_cfg_of_block<LF>(TileOK<LF>::value ? cap : (cap < 4 ? cap : 4));
        const std::string key = tune_key(ctx, tag, tag_prec, tag_recon, nrhs);
        STAG_TRY(tune_choice(ctx, key, multi_cfg_candidates<LF>(nrhs), &cfg, [&](int c) {
            return launch_multi_cfg(ctx, c, U, in, out, stride, nrhs, p, ctx->stream);
        }));
    }
    if (nb_used) *nb_used = mcfg_block(cfg);
    if (cfg_used) *cfg_used = cfg;
    return launch_multi_cfg(ctx, cfg, U, in, out, stride, nrhs, p, ctx->stream);
}

int multi_cfg_for(int prec, int block)
{
    if (block >= 256) return block;   // an explicit configuration code
    return (prec == STAG_F32 || prec == STAG_F16) ? multi_cfg_of_block<LinkField<float2, 12>>(block)
                                                  : multi_cfg_of_block<LinkField<double2, 18>>(block);
}

int multi_dslash(stag_ctx ctx, int prec, int recon, int par_out, void* out, const void* in, int nrhs, int nb,
                 int* nb_used, int* cfg_used, int links)
{
    const void* lk = nullptr;
    int tg = 0;
    STAG_TRY(op_links_for(ctx, links, prec, recon, &lk, &tg));
    const int Vh = ctx->g.Vh;
    // the autotuner's key names the link field (6 or 8 link reads per site)
    const char* tag = links == STAG_LINKS_UPLOADED ? "multi_dslash"
                      : links == STAG_LINKS_TEMPORAL ? "multi_dslash_tg" : "multi_dslash_tgfull";
    const size_t stride = lo_spinor_bytes(ctx->g, prec);
    if (prec == STAG_F64) {
        SpinorF64 si{(double2*)in}, so{(double2*)out};
        if (recon == 18)
            return multi_dslash_tuned(ctx, tag, prec, recon, LinkField<double2, 18>{(const double2*)lk, Vh, tg}, si, so, stride, nrhs,
                                      par_out, nb, nb_used, cfg_used);
        return multi_dslash_tuned(ctx, tag, prec, recon, LinkField<double2, 12>{(const double2*)lk, Vh, tg}, si, so, stride, nrhs,
                                  par_out, nb, nb_used, cfg_used);
    }
    if (prec == STAG_F64X) {
        // canonical fields in double-float arithmetic go through the
        // normalising dslash_f64x_canonical, internal ones through
        // multi_dslash_internal
        set_error("multi_dslash: double-float fields are not canonical storage here");
        return STAG_EINVAL;
    }
    if (prec == STAG_F32) {
        SpinorF32 si{(float2*)in, Vh}, so{(float2*)out, Vh};
        if (recon == 18)
            return multi_dslash_tuned(ctx, tag, prec, recon, LinkField<float2, 18>{(const float2*)lk, Vh, tg}, si, so, stride, nrhs,
                                      par_out, nb, nb_used, cfg_used);
        return multi_dslash_tuned(ctx, tag, prec, recon, LinkField<float2, 12>{(const float2*)lk, Vh, tg}, si, so, stride, nrhs,
                                  par_out, nb, nb_used, cfg_used);
    }
    SpinorF16 si{(uint4*)in, Vh}, so{(uint4*)out, Vh};
    if (recon == 18)
        return multi_dslash_tuned(ctx, tag, prec, recon, LinkField<__half2, 18>{(const __half2*)lk, Vh, tg}, si, so, stride, nrhs,
                                  par_out, nb, nb_used, cfg_used);
    return multi_dslash_tuned(ctx, tag, prec, recon, LinkField<__half2, 12>{(const __half2*)lk, Vh, tg}, si, so, stride, nrhs, par_out,
                              nb, nb_used, cfg_used);
}

// The multi operator on a precision's internal storage (as multi_dslash,
// except that STAG_F64X reads and writes double-float vectors).
int multi_dslash_internal(stag_ctx ctx, int prec, int recon, int par_out, void* out, const void* in, int nrhs,
                          int nb, int* nb_used, int links)
{
    if (prec != STAG_F64X) return multi_dslash(ctx, prec, recon, par_out, out, in, nrhs, nb, nb_used, nullptr, links);
    const void* lk = nullptr;
    int tg = 0;
    STAG_TRY(op_links_for(ctx, links, prec, recon, &lk, &tg));
    const char* tag = links == STAG_LINKS_UPLOADED ? "multi_dslash_df"
                      : links == STAG_LINKS_TEMPORAL ? "multi_dslash_df_tg" : "multi_dslash_df_tgfull";
    return multi_dslash_tuned(ctx, tag, prec, recon, LinkFieldDF<18>{(const float4*)lk, ctx->g.Vh, tg},
                              SpinorDF{(float4*)in}, SpinorDF{(float4*)out}, lo_spinor_bytes(ctx->g, prec), nrhs,
                              par_out, nb, nb_used);
}

int check_ctx(stag_ctx ctx);
int check_half_field(const void* p, const char* what);

}  // namespace stag

using namespace stag;

extern "C" {

int stag_dslash_multi(stag_ctx ctx, double* out, const double* in, int nrhs, int out_parity, int prec, int recon,
                      int rhs_block)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(out, "out"));
    STAG_TRY(check_half_field(in, "in"));
    if (out == in) {
        set_error("out and in must not alias");
        return STAG_EINVAL;
    }
    if (nrhs < 1 || nrhs > STAG_MAX_RHS || (out_parity != 0 && out_parity != 1)) {
        set_error("nrhs must be in [1, %d] and out_parity 0 or 1", STAG_MAX_RHS);
        return STAG_EINVAL;
    }
    if (rhs_block != 0 && rhs_block != 1 && rhs_block != 2 && rhs_block != 4 && rhs_block != 8 && rhs_block != 16 &&
        rhs_block < 256) {
        set_error("rhs_block must be 0 (autotune), 1, 2, 4, 8, 16 or a configuration code (G << 8) | NBT");
        return STAG_EINVAL;
    }
    if (prec < STAG_F64 || prec > STAG_F64X || (recon != 18 && recon != 12) || (prec == STAG_F64X && recon != 18)) {
        set_error("unsupported prec %d / recon %d", prec, recon);
        return STAG_EUNSUPPORTED;
    }
    if (!ctx->have_gauge) {
        set_error("no gauge field uploaded");
        return STAG_ENOGAUGE;
    }
    if (prec == STAG_F64)
        return multi_dslash(ctx, prec, recon, out_parity, out, in, nrhs, rhs_block, nullptr, nullptr, ctx->op_links);
    if (prec == STAG_F64X)
        return dslash_f64x_canonical(ctx, out_parity, (double2*)out, (const double2*)in, nrhs, ctx->op_links,
                                     rhs_block ? rhs_block : 0, nullptr, ctx->stream);
    const size_t lo = lo_spinor_bytes(ctx->g, prec) * nrhs;
    STAG_TRY(ensure_lo_tmp_public(ctx, lo));
    STAG_TRY(convert_f64_to_lo(ctx, prec, (const double2*)in, ctx->tmp_lo_in, nrhs, ctx->stream));
    STAG_TRY(multi_dslash(ctx, prec, recon, out_parity, ctx->tmp_lo_out, ctx->tmp_lo_in, nrhs, rhs_block, nullptr,
                          nullptr, ctx->op_links));
    return convert_lo_to_f64(ctx, prec, ctx->tmp_lo_out, (double2*)out, nrhs, ctx->stream);
}

}  // extern "C"
