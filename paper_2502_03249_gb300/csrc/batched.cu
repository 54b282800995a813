// batched.cu -- the batched solver's driver: workspace slots, the rhs-block
// choice, the dispatch to the plans of each inner storage (batched_f64.cu,
// batched_f32.cu, batched_f16.cu; the kernels and plans are in
// batched_impl.cuh), the statistics, and stag_cg_solve_multi.
#include "batched_impl.cuh"

namespace stag {

// ------------------------------------------------------------- slots

int ensure_cg_f64(stag_ctx ctx);

static int ensure_batch(stag_ctx ctx, int prec, int recon, int nrhs, BatchSlot** out)
{
    if (!ctx->ws) {
        ctx->ws = new (std::nothrow) Workspace();
        if (!ctx->ws) return STAG_ENOMEM;
    }
    BatchSlot& m = ctx->ws->batch[prec][recon == 12 ? 1 : 0];
    if (m.ready && m.cap < nrhs) m.release();
    if (!m.ready) {
        const Geom& g = ctx->g;
        m.Vh = g.Vh;
        m.cap = nrhs;
        m.s_stride = lo_spinor_bytes(g, prec);
        m.sx_stride = lo_spinor_bytes(g, prec == STAG_F64 ? STAG_F64 : STAG_F32);
        m.f64_stride = (size_t)g.Vh * 3 * sizeof(double2);
        m.prec = prec;
        m.gx = (g.Vh + BBS - 1) / BBS;
        const size_t n = (size_t)nrhs;
        STAG_CUDA_TRY(cudaMalloc(&m.r, n * m.s_stride));
        STAG_CUDA_TRY(cudaMalloc(&m.p, n * m.s_stride));
        STAG_CUDA_TRY(cudaMalloc(&m.Ap, n * m.s_stride));
        STAG_CUDA_TRY(cudaMalloc(&m.t, n * m.s_stride));
        STAG_CUDA_TRY(cudaMalloc(&m.xlo, n * m.sx_stride));
        STAG_CUDA_TRY(cudaMalloc(&m.x_hi, n * m.f64_stride));
        STAG_CUDA_TRY(cudaMalloc(&m.r_hi, n * m.f64_stride));
        STAG_CUDA_TRY(cudaMalloc(&m.b, n * m.f64_stride));
        STAG_CUDA_TRY(cudaMalloc(&m.t64, n * m.f64_stride));
        STAG_CUDA_TRY(cudaMalloc(&m.x_df, n * m.f64_stride));
        STAG_CUDA_TRY(cudaMalloc(&m.sc, n * sizeof(CgScalars)));
        // partials: one per block of BBS sites, or per tile of 32 (tile kernels)
        STAG_CUDA_TRY(cudaMalloc(&m.part, n * (size_t)((g.Vh + 31) / 32) * sizeof(double)));
        STAG_CUDA_TRY(cudaMalloc(&m.shifts, n * sizeof(double)));
        STAG_CUDA_TRY(cudaMalloc(&m.cnt_sys, n * sizeof(unsigned)));
        STAG_CUDA_TRY(cudaMemset(m.cnt_sys, 0, n * sizeof(unsigned)));
        m.ready = true;
    }
    if (m.nrhs != nrhs) m.lg.destroy();   // the graph bakes the batch size into its grids
    m.nrhs = nrhs;
    *out = &m;
    return STAG_OK;
}

// X (device, [nrhs][Vh][3] complex128) = solutions of (M + shifts_k) X_k = B_k.
// shifts_host: NULL (all zero) or nrhs host values; X0: NULL or initial guesses.
// tg = 1: every operator pass on the temporal-gauge links U' (M' = g M g^dagger);
// B, X0 and X are then the transformed fields (the caller applies g and g^dagger).
int batched_solve(stag_ctx ctx, double2* X, const double2* B, int nrhs, double mass, const double* shifts_host,
                  const double2* X0, const stag_solver_params& prm, stag_solver_stats* stats, int tg)
{
    const auto t0 = std::chrono::steady_clock::now();
    const int prec = prm.inner_prec, recon = prm.inner_recon;
    if (prec < STAG_F64 || prec > STAG_F16 || (recon != 18 && recon != 12)) {
        set_error("batched solver: unsupported inner precision %d / compression %d", prec, recon);
        return STAG_EUNSUPPORTED;
    }
    if (prec != STAG_F64) STAG_TRY(check_float_inner_links(ctx));
    BatchSlot* mp = nullptr;
    STAG_TRY(ensure_batch(ctx, prec, recon, nrhs, &mp));
    BatchSlot& m = *mp;
    const void* lk = nullptr;
    STAG_TRY(tg ? ensure_links_tg(ctx, prec, recon, &lk) : ensure_links(ctx, prec, recon, &lk));
    m.tg = tg;
    const double delta = prec == STAG_F64 ? 0.0 : (prm.delta > 0 ? prm.delta : DEFAULT_RELIABLE_DELTA);
    const size_t vbytes = (size_t)nrhs * m.f64_stride;
    stag_solver_params prm2 = prm;
    STAG_TRY(resolve_f64_arith(ctx, prm.f64_arith, &prm2.f64_arith));
    // B_k' = 2^-k_k B_k, each with its largest component in [1, 2); X_k = 2^k_k X_k'
    STAG_TRY(normalise_fields(ctx, B, m.b, nrhs, (size_t)3 * ctx->g.Vh, SLOT_SOLVE, ctx->stream));
    const double* shifts_dev = nullptr;
    if (shifts_host) {
        STAG_CUDA_TRY(cudaMemcpyAsync(m.shifts, shifts_host, nrhs * sizeof(double), cudaMemcpyHostToDevice,
                                      ctx->stream));
        shifts_dev = m.shifts;
    }
    // right-hand sides per operator pass: given, or tuned on the inner operator
    int nb = prm.rhs_block;
    if (nb != 0 && nb != 1 && nb != 2 && nb != 4 && nb != 8 && nb != 16 && nb < 256) {
        set_error("rhs_block must be 0 (autotune), 1, 2, 4, 8, 16 or a configuration code (G << 8) | NBT");
        return STAG_EINVAL;
    }
    // the configuration (multi_tile.cuh) of a given block, or the autotuner's
    // choice for the inner operator on these buffers
    int cfg = multi_cfg_for(prec, nb);
    if (nb == 0) STAG_TRY(multi_dslash(ctx, prec, recon, 1, m.t, m.p, nrhs, 0, &nb, &cfg, tg));
    int rc;
    if (prec == STAG_F64) rc = batched_run_f64(ctx, m, recon, lk, X0, mass, shifts_dev, prm2, delta, cfg);
    else if (prec == STAG_F32) rc = batched_run_f32(ctx, m, recon, lk, X0, mass, shifts_dev, prm2, delta, cfg);
    else rc = batched_run_f16(ctx, m, recon, lk, X0, mass, shifts_dev, prm2, delta, cfg);
    STAG_TRY(rc);
    std::vector<CgScalars> hs(nrhs);
    STAG_CUDA_TRY(cudaMemcpyAsync(hs.data(), m.sc, sizeof(CgScalars) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
    STAG_TRY(scale_fields_out(ctx, m.x_hi, X, nrhs, (size_t)3 * ctx->g.Vh, SLOT_SOLVE, 1, ctx->stream));
    STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    int status = STAG_OK;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < nrhs; ++k) {
        const CgScalars& c = hs[k];
        int sk = STAG_OK;
        if (c.rr0 == 0.0) {
            STAG_CUDA_TRY(cudaMemsetAsync(X + (size_t)k * 3 * ctx->g.Vh, 0, m.f64_stride, ctx->stream));
        } else if (c.status == STAG_BREAKDOWN) {
            sk = STAG_BREAKDOWN;
        } else if (!(c.rr_true <= c.tol2)) {
            sk = STAG_NOT_CONVERGED;
        }
        if (sk > status) status = sk;
        if (stats) {
            stats[k].status = sk;
            stats[k].iters = c.iter;
            stats[k].restarts = 0;
            stats[k].reliable_updates = c.n_reliable;
            stats[k].true_rel_residual = c.rr0 > 0 ? sqrt(c.rr_true / c.rr0) : 0.0;
            stats[k].iter_rel_residual = c.rr0 > 0 ? sqrt(c.rr / c.rr0) : 0.0;
            stats[k].seconds = secs;
        }
    }
    STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    ctx->last_rhs_block = mcfg_block(cfg);
    ctx->last_multi_cfg = cfg;
    return status;
}

void BatchSlot::release()
{
    lg.destroy();
    void* bufs[] = {r, p, Ap, t, xlo, x_hi, r_hi, b, t64, x_df, sc, part, shifts, cnt_sys};
    for (void* q : bufs)
        if (q) cudaFree(q);
    *this = BatchSlot();
}

void free_batches(Workspace* ws)
{
    for (auto& row : ws->batch)
        for (auto& m : row) m.release();
}

int check_ctx(stag_ctx ctx);
int check_half_field(const void* p, const char* what);

}  // namespace stag

using namespace stag;

extern "C" {

int stag_cg_solve_multi(stag_ctx ctx, double* X, const double* B, int nrhs, double mass,
                        const stag_solver_params* params, stag_solver_stats* stats)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(X, "X"));
    STAG_TRY(check_half_field(B, "B"));
    if (nrhs < 1 || nrhs > STAG_MAX_RHS) {
        set_error("nrhs must be in [1, %d]", STAG_MAX_RHS);
        return STAG_EINVAL;
    }
    stag_solver_params prm;
    stag_solver_params_default(&prm);
    if (params) prm = *params;
    if (!(prm.tol > 0.0)) {
        set_error("tol must be positive");
        return STAG_EINVAL;
    }
    if (!ctx->have_gauge) {
        set_error("no gauge field uploaded");
        return STAG_ENOGAUGE;
    }
    if (!prm.temporal_gauge)
        return batched_solve(ctx, (double2*)X, (const double2*)B, nrhs, mass, nullptr, nullptr, prm, stats, 0);
    // temporal gauge: M' X' = g B on U', X = g^dagger X'
    const double2* G = nullptr;
    double2* gb = nullptr;
    STAG_TRY(ensure_tg_gauge(ctx, &G));
    STAG_TRY(ensure_tg_tmp(ctx, nrhs, &gb));
    STAG_TRY(tg_apply(ctx, G, (const double2*)B, gb, nrhs, 0));
    const int rc = batched_solve(ctx, (double2*)X, gb, nrhs, mass, nullptr, nullptr, prm, stats, 1);
    if (rc < 0) return rc;
    STAG_TRY(tg_apply(ctx, G, (const double2*)X, (double2*)X, nrhs, 1));
    STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return rc;
}

int stag_last_rhs_block(stag_ctx ctx)
{
    if (!ctx) return STAG_EINVAL;
    return ctx->last_rhs_block;
}

}  // extern "C"
