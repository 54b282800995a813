// api.cu -- C ABI entry points of libstag: contexts, gauge upload and the
// operator applications.  Every function validates its arguments before it
// enqueues any work, so a negative return leaves the outputs untouched.
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "ctx.h"

namespace stag {

static thread_local char g_last_error[512] = "";

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

void free_workspace(stag_ctx ctx);   // cg.cu
void free_tune_cache(stag_ctx ctx);  // tune.cu

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Device buffers must be 16-byte aligned device (or managed) memory.
static int check_dev_ptr(const void* p, const char* what)
{
    if (!p) {
        set_error("%s is NULL", what);
        return STAG_EINVAL;
    }
    if (!aligned16(p)) {
        set_error("%s is not 16-byte aligned", what);
        return STAG_EINVAL;
    }
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        set_error("%s is not a CUDA pointer", what);
        return STAG_EINVAL;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
        set_error("%s is not device memory", what);
        return STAG_EINVAL;
    }
    return STAG_OK;
}

int check_ctx(stag_ctx ctx)
{
    if (!ctx) {
        set_error("context is NULL");
        return STAG_EINVAL;
    }
    STAG_CUDA_TRY(cudaSetDevice(ctx->device));
    return STAG_OK;
}

int check_half_field(const void* p, const char* what) { return check_dev_ptr(p, what); }

static int ensure_lo_tmp(stag_ctx ctx, size_t bytes)
{
    ctx->prepared_prec = -1;   // every user of the scratch fields overwrites a prepared field
    if (ctx->tmp_lo_bytes >= bytes) return STAG_OK;
    if (ctx->tmp_lo_in) cudaFree(ctx->tmp_lo_in);
    if (ctx->tmp_lo_out) cudaFree(ctx->tmp_lo_out);
    ctx->tmp_lo_in = ctx->tmp_lo_out = nullptr;
    ctx->tmp_lo_bytes = 0;
    STAG_CUDA_TRY(cudaMalloc(&ctx->tmp_lo_in, bytes));
    STAG_CUDA_TRY(cudaMalloc(&ctx->tmp_lo_out, bytes));
    ctx->tmp_lo_bytes = bytes;
    return STAG_OK;
}

int ensure_lo_tmp_public(stag_ctx ctx, size_t bytes) { return ensure_lo_tmp(ctx, bytes); }

// out (parity par_out) = D in, boundary fields complex128.
static int dslash_entry(stag_ctx ctx, double* out, const double* in, int prec, int recon, int par_out)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(out, "out"));
    STAG_TRY(check_half_field(in, "in"));
    if (out == in) {
        set_error("out and in must not alias");
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
    if (prec == STAG_F64 || prec == STAG_F64X)
        return launch_dslash(ctx, prec, recon, par_out, out, in, ctx->stream, ctx->op_links);
    STAG_TRY(ensure_lo_tmp(ctx, lo_spinor_bytes(ctx->g, prec)));
    STAG_TRY(convert_f64_to_lo(ctx, prec, (const double2*)in, ctx->tmp_lo_in, 1, ctx->stream));
    STAG_TRY(launch_dslash(ctx, prec, recon, par_out, ctx->tmp_lo_out, ctx->tmp_lo_in, ctx->stream, ctx->op_links));
    return convert_lo_to_f64(ctx, prec, ctx->tmp_lo_out, (double2*)out, 1, ctx->stream);
}

int apply_M_f64(stag_ctx ctx, double2* out, const double2* in, double mass, double2* tmp_odd,
                cudaStream_t s);   // cg.cu

}  // namespace stag

using namespace stag;

extern "C" {

int stag_abi_version(void) { return STAG_ABI_VERSION; }

const char* stag_last_error(void) { return g_last_error; }

const char* stag_strerror(int code)
{
    switch (code) {
    case STAG_OK: return "success";
    case STAG_NOT_CONVERGED: return "solver did not converge within maxiter";
    case STAG_BREAKDOWN: return "solver breakdown: <p, M p> not positive or not finite";
    case STAG_EINVAL: return "invalid argument";
    case STAG_EGEOM: return "invalid lattice extents (each must be even and >= 2)";
    case STAG_ENOMEM: return "out of memory";
    case STAG_ECUDA: return "CUDA error";
    case STAG_ENOGAUGE: return "no gauge field uploaded";
    case STAG_EUNSUPPORTED: return "unsupported precision or compression";
    default: return "unknown status";
    }
}

int stag_create(stag_ctx* out, const int dims[4], void* stream)
{
    if (!out || !dims) {
        set_error("stag_create: NULL argument");
        return STAG_EINVAL;
    }
    *out = nullptr;
    long long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2 || dims[mu] % 2) {
            set_error("extent %d of direction %d is not even and >= 2", dims[mu], mu);
            return STAG_EGEOM;
        }
        V *= dims[mu];
    }
    if (V >= (1LL << 31)) {
        set_error("volume %lld too large (limit 2^31)", V);
        return STAG_EGEOM;
    }
    stag_ctx ctx = new (std::nothrow) stag_ctx_s();
    if (!ctx) return STAG_ENOMEM;
    memset((void*)ctx, 0, sizeof(*ctx));
    ctx->g = make_geom(dims);
    ctx->V = V;
    ctx->stream = (cudaStream_t)stream;
    ctx->prepared_prec = -1;
    ctx->half_stage[0] = ctx->half_stage[1] = -1;
    int rc = STAG_OK;
    do {
        if (cudaGetDevice(&ctx->device) != cudaSuccess) { rc = STAG_ECUDA; break; }
        if (cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
            rc = STAG_ECUDA;
            break;
        }
        if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) { rc = STAG_ECUDA; break; }
        ctx->max_blocks = (ctx->g.Vh + 31) / 32 + 1024;
        if (cudaMalloc(&ctx->partials, sizeof(double) * (size_t)ctx->max_blocks * 2) != cudaSuccess) { rc = STAG_ENOMEM; break; }
        if (cudaMalloc(&ctx->counters, sizeof(unsigned) * 64) != cudaSuccess) { rc = STAG_ENOMEM; break; }
        if (cudaMemset(ctx->counters, 0, sizeof(unsigned) * 64) != cudaSuccess) { rc = STAG_ECUDA; break; }
        const size_t ng = (size_t)ctx->max_blocks / RGROUP + 2;
        if (cudaMalloc(&ctx->gsum_part, sizeof(double) * ng) != cudaSuccess) { rc = STAG_ENOMEM; break; }
        if (cudaMalloc(&ctx->gsum_cnt, sizeof(unsigned) * ng) != cudaSuccess) { rc = STAG_ENOMEM; break; }
        if (cudaMemset(ctx->gsum_cnt, 0, sizeof(unsigned) * ng) != cudaSuccess) { rc = STAG_ECUDA; break; }
        if (cudaMalloc(&ctx->tmp_odd, sizeof(double2) * 3 * (size_t)ctx->g.Vh) != cudaSuccess) { rc = STAG_ENOMEM; break; }
    } while (0);
    if (rc != STAG_OK) {
        set_error("stag_create: %s", cudaGetErrorString(cudaGetLastError()));
        stag_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return STAG_OK;
}

int stag_destroy(stag_ctx ctx)
{
    if (!ctx) return STAG_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream || ctx->cap_stream) cudaStreamSynchronize(ctx->stream);
    free_workspace(ctx);
    free_tune_cache(ctx);
    for (int s = 0; s < 8; ++s)
        if (ctx->links[s]) cudaFree(ctx->links[s]);
    if (ctx->partials) cudaFree(ctx->partials);
    if (ctx->counters) cudaFree(ctx->counters);
    if (ctx->gsum_part) cudaFree(ctx->gsum_part);
    if (ctx->gsum_cnt) cudaFree(ctx->gsum_cnt);
    if (ctx->tg_g) cudaFree(ctx->tg_g);
    if (ctx->tg_defect) cudaFree(ctx->tg_defect);
    for (int s = 0; s < 8; ++s)
        if (ctx->tg_links[s]) cudaFree(ctx->tg_links[s]);
    if (ctx->tg_tmp) cudaFree(ctx->tg_tmp);
    if (ctx->tmp_odd) cudaFree(ctx->tmp_odd);
    if (ctx->tmp_lo_in) cudaFree(ctx->tmp_lo_in);
    if (ctx->tmp_lo_out) cudaFree(ctx->tmp_lo_out);
    if (ctx->full_tmp) cudaFree(ctx->full_tmp);
    if (ctx->scale_bits) cudaFree(ctx->scale_bits);
    if (ctx->scale_k) cudaFree(ctx->scale_k);
    if (ctx->dfx_tmp) cudaFree(ctx->dfx_tmp);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
    return STAG_OK;
}

int stag_set_stream(stag_ctx ctx, void* stream)
{
    STAG_TRY(check_ctx(ctx));
    ctx->stream = (cudaStream_t)stream;
    return STAG_OK;
}

int stag_set_operator_links(stag_ctx ctx, int links)
{
    STAG_TRY(check_ctx(ctx));
    if (links != STAG_LINKS_UPLOADED && links != STAG_LINKS_TEMPORAL && links != STAG_LINKS_TEMPORAL_FULL) {
        set_error("links must be STAG_LINKS_UPLOADED, STAG_LINKS_TEMPORAL or STAG_LINKS_TEMPORAL_FULL");
        return STAG_EINVAL;
    }
    ctx->op_links = links;
    return STAG_OK;
}

int stag_get_dims(stag_ctx ctx, int dims[4], long long* volume)
{
    if (!ctx) {
        set_error("context is NULL");
        return STAG_EINVAL;
    }
    if (dims)
        for (int mu = 0; mu < 4; ++mu) dims[mu] = ctx->g.L[mu];
    if (volume) *volume = ctx->V;
    return STAG_OK;
}

int stag_upload_gauge(stag_ctx ctx, const double* U, int on_device)
{
    STAG_TRY(check_ctx(ctx));
    if (!U) {
        set_error("U is NULL");
        return STAG_EINVAL;
    }
    if (on_device) STAG_TRY(check_dev_ptr(U, "U"));
    return upload_gauge(ctx, U, on_device);
}

int stag_dslash_eo(stag_ctx ctx, double* out_even, const double* in_odd, int prec, int recon)
{
    return dslash_entry(ctx, out_even, in_odd, prec, recon, 0);
}

int stag_dslash_oe(stag_ctx ctx, double* out_odd, const double* in_even, int prec, int recon)
{
    return dslash_entry(ctx, out_odd, in_even, prec, recon, 1);
}

int stag_dslash_prepare_multi(stag_ctx ctx, const double* in, int nrhs, int prec)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(in, "in"));
    if (prec < STAG_F64 || prec > STAG_F64X) {
        set_error("unsupported prec %d", prec);
        return STAG_EUNSUPPORTED;
    }
    if (nrhs < 1 || nrhs > STAG_MAX_RHS) {
        set_error("nrhs must be in [1, %d]", STAG_MAX_RHS);
        return STAG_EINVAL;
    }
    const size_t bytes = lo_spinor_bytes(ctx->g, prec);
    STAG_TRY(ensure_lo_tmp(ctx, bytes * nrhs));
    if (prec == STAG_F64)
        STAG_CUDA_TRY(cudaMemcpyAsync(ctx->tmp_lo_in, in, bytes * nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
    else
        STAG_TRY(convert_f64_to_lo(ctx, prec, (const double2*)in, ctx->tmp_lo_in, nrhs, ctx->stream));
    ctx->prepared_prec = prec;
    ctx->prepared_nrhs = nrhs;
    ctx->repeat_done = 0;
    return STAG_OK;
}

int stag_dslash_prepare(stag_ctx ctx, const double* in, int prec)
{
    return stag_dslash_prepare_multi(ctx, in, 1, prec);
}

int stag_dslash_repeat_multi(stag_ctx ctx, int prec, int recon, int rhs_block, int nrep)
{
    STAG_TRY(check_ctx(ctx));
    if (ctx->prepared_prec != prec || !ctx->tmp_lo_in) {
        set_error("call stag_dslash_prepare_multi with this precision first");
        return STAG_EINVAL;
    }
    if (nrep < 1 || recon != 18 && recon != 12 || (prec == STAG_F64X && recon != 18)) {
        set_error("nrep must be >= 1 and recon 18 or 12");
        return STAG_EINVAL;
    }
    if (rhs_block != 0 && rhs_block != 1 && rhs_block != 2 && rhs_block != 4 && rhs_block != 8 && rhs_block != 16 &&
        rhs_block < 256) {
        set_error("rhs_block must be 0 (autotune), 1, 2, 4, 8, 16 or a configuration code (G << 8) | NBT");
        return STAG_EINVAL;
    }
    if (!ctx->have_gauge) {
        set_error("no gauge field uploaded");
        return STAG_ENOGAUGE;
    }
    int nb = rhs_block;
    for (int k = 0; k < nrep; ++k)
        STAG_TRY(multi_dslash_internal(ctx, prec, recon, 0, ctx->tmp_lo_out, ctx->tmp_lo_in, ctx->prepared_nrhs,
                                       rhs_block, &nb, ctx->op_links));
    ctx->last_rhs_block = nb;
    ctx->repeat_done = 1;
    return STAG_OK;
}

int stag_dslash_result(stag_ctx ctx, double* out)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(out, "out"));
    if (!ctx->repeat_done || ctx->prepared_prec < 0) {
        set_error("no stag_dslash_repeat since the last stag_dslash_prepare");
        return STAG_EINVAL;
    }
    const int prec = ctx->prepared_prec, n = ctx->prepared_nrhs;
    if (prec == STAG_F64)
        STAG_CUDA_TRY(cudaMemcpyAsync(out, ctx->tmp_lo_out, lo_spinor_bytes(ctx->g, prec) * n,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    else
        STAG_TRY(convert_lo_to_f64(ctx, prec, ctx->tmp_lo_out, (double2*)out, n, ctx->stream));
    return STAG_OK;
}

int stag_dslash_repeat(stag_ctx ctx, int prec, int recon, int nrep)
{
    STAG_TRY(check_ctx(ctx));
    if (ctx->prepared_prec != prec || !ctx->tmp_lo_in || ctx->prepared_nrhs != 1) {
        set_error("call stag_dslash_prepare with this precision first");
        return STAG_EINVAL;
    }
    if (nrep < 1 || recon != 18 && recon != 12 || (prec == STAG_F64X && recon != 18)) {
        set_error("nrep must be >= 1 and recon 18 or 12");
        return STAG_EINVAL;
    }
    if (!ctx->have_gauge) {
        set_error("no gauge field uploaded");
        return STAG_ENOGAUGE;
    }
    if (prec == STAG_F16 && recon == 12)
        STAG_TRY(tune_half_stage(ctx, ctx->op_links, ctx->tmp_lo_out, ctx->tmp_lo_in));
    for (int k = 0; k < nrep; ++k)
        STAG_TRY(launch_dslash_internal(ctx, prec, recon, 0, ctx->tmp_lo_out, ctx->tmp_lo_in, ctx->stream,
                                        ctx->op_links));
    ctx->repeat_done = 1;
    return STAG_OK;
}

int stag_apply_M(stag_ctx ctx, double* out_even, const double* in_even, double mass)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(out_even, "out_even"));
    STAG_TRY(check_half_field(in_even, "in_even"));
    if (out_even == in_even) {
        set_error("out and in must not alias");
        return STAG_EINVAL;
    }
    if (!ctx->have_gauge) {
        set_error("no gauge field uploaded");
        return STAG_ENOGAUGE;
    }
    return apply_M_f64(ctx, (double2*)out_even, (const double2*)in_even, mass, ctx->tmp_odd, ctx->stream);
}

}  // extern "C"
