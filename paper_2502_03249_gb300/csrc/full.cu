// full.cu -- the full-lattice system (m + D) psi = b through the even-odd
// Schur complement (D of Sec. 4.2, Eq. (staggered); M the even-odd normal
// matrix the solvers invert):
//   even rows:  m psi_e + D_eo psi_o = b_e,   odd rows:  D_oe psi_e + m psi_o = b_o
//   => M psi_e = m b_e - D_eo b_o,  psi_o = (b_o - D_oe psi_e) / m.
#include "cg_kernels.cuh"
#include "df64.cuh"
#include "workspace.h"

namespace stag {

constexpr int FULL_BS = 128;

// canonical full field [V][3] <-> two half fields of [V/2][3] (site i -> i/2 of its parity)
__global__ void k_split_full(Geom g, const double2* __restrict__ full, double2* __restrict__ ev,
                             double2* __restrict__ od)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2LL * g.Vh) return;
    const int x = (int)(i % g.L[0]);
    long long r = i / g.L[0];
    const int y = (int)(r % g.L[1]);
    r /= g.L[1];
    const int z = (int)(r % g.L[2]);
    const int t = (int)(r / g.L[2]);
    double2* dst = ((x + y + z + t) & 1) ? od : ev;
#pragma unroll
    for (int c = 0; c < 3; ++c) dst[(size_t)(i >> 1) * 3 + c] = full[(size_t)i * 3 + c];
}

__global__ void k_join_full(Geom g, const double2* __restrict__ ev, const double2* __restrict__ od,
                            double2* __restrict__ full)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2LL * g.Vh) return;
    const int x = (int)(i % g.L[0]);
    long long r = i / g.L[0];
    const int y = (int)(r % g.L[1]);
    r /= g.L[1];
    const int z = (int)(r % g.L[2]);
    const int t = (int)(r / g.L[2]);
    const double2* src = ((x + y + z + t) & 1) ? od : ev;
#pragma unroll
    for (int c = 0; c < 3; ++c) full[(size_t)i * 3 + c] = src[(size_t)(i >> 1) * 3 + c];
}

// out = a x + c D_{p,1-p} t  (double vectors, operator in LF/SD arithmetic)
template <class LF, class SD>
__global__ void __launch_bounds__(FULL_BS) k_axpby_hop(Geom g, int p, LF U, SD t, const double2* x, double2* out,
                                                       double a, double c)
{
    const int h = blockIdx.x * FULL_BS + threadIdx.x;
    if (h >= g.Vh) return;
    const Vec3<double> Dt = vconv<double>(dslash_site(g, p, h, U, t));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double2 xv = x[(size_t)h * 3 + k];
        out[(size_t)h * 3 + k] = make_double2(fma(a, xv.x, c * Dt.c[k].re), fma(a, xv.y, c * Dt.c[k].im));
    }
}

template <class LF, class SD>
static int axpby_hop(stag_ctx ctx, const LF& U, int p, const double2* t, const double2* x, double2* out, double a,
                     double c)
{
    const int grid = (ctx->g.Vh + FULL_BS - 1) / FULL_BS;
    k_axpby_hop<LF, SD><<<grid, FULL_BS, 0, ctx->stream>>>(ctx->g, p, U, SD{(double2*)t}, x, out, a, c);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

int cg_solve_f64(stag_ctx ctx, double2* x_out, const double2* b_in, double mass, double sigma,
                 const stag_solver_params& prm, stag_solver_stats* st);
int cg_solve_mixed(stag_ctx ctx, double2* x_out, const double2* b_in, double mass, const stag_solver_params& prm,
                   stag_solver_stats* st);
int check_ctx(stag_ctx ctx);
int check_half_field(const void* p, const char* what);

// Buffers: four half fields (b_e, b_o, rhs_e, psi_e) carved from one allocation kept in the context.
static int full_buffers(stag_ctx ctx, double2** bufs)
{
    const size_t n = (size_t)3 * ctx->g.Vh;
    if (!ctx->full_tmp) STAG_CUDA_TRY(cudaMalloc(&ctx->full_tmp, 4 * n * sizeof(double2)));
    for (int k = 0; k < 4; ++k) bufs[k] = (double2*)ctx->full_tmp + k * n;
    return STAG_OK;
}

// out = a x + c y (double vectors)
__global__ void k_axpby(long long n, const double2* x, const double2* y, double2* out, double a, double c)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 xv = x[i], yv = y[i];
    out[i] = make_double2(fma(a, xv.x, c * yv.x), fma(a, xv.y, c * yv.y));
}

static int axpby(stag_ctx ctx, const double2* x, const double2* y, double2* out, double a, double c)
{
    const long long n = 3LL * ctx->g.Vh;
    k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, x, y, out, a, c);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

// The Schur steps with the double-float operator on canonical fields (which
// normalises its input, so any scale of b is served): the operator result
// goes to the output buffer first, then the axpby.
static int schur_pre_df(stag_ctx ctx, double2* const* B, double mass)
{
    STAG_TRY(dslash_f64x_canonical(ctx, 0, B[2], B[1], 1, STAG_LINKS_UPLOADED, 1, nullptr, ctx->stream));   // D_eo b_o
    return axpby(ctx, B[0], B[2], B[2], mass, -1.0);                                   // m b_e - D_eo b_o
}

static int schur_post_df(stag_ctx ctx, double2* const* B, double2* psi_o, double mass)
{
    STAG_TRY(dslash_f64x_canonical(ctx, 1, psi_o, B[3], 1, STAG_LINKS_UPLOADED, 1, nullptr, ctx->stream));   // D_oe psi_e
    return axpby(ctx, B[1], psi_o, psi_o, 1.0 / mass, -1.0 / mass);                      // (b_o - D_oe psi_e)/m
}

template <class LF, class SD>
static int schur_pre(stag_ctx ctx, const LF& U, double2* const* B, double mass)
{
    return axpby_hop<LF, SD>(ctx, U, 0, B[1], B[0], B[2], mass, -1.0);   // rhs_e = m b_e - D_eo b_o
}

template <class LF, class SD>
static int schur_post(stag_ctx ctx, const LF& U, double2* const* B, double2* psi_o, double mass)
{
    return axpby_hop<LF, SD>(ctx, U, 1, B[3], B[1], psi_o, 1.0 / mass, -1.0 / mass);   // (b_o - D_oe psi_e)/m
}

}  // namespace stag

using namespace stag;

extern "C" int stag_solve_full(stag_ctx ctx, double* psi, const double* b, double mass,
                               const stag_solver_params* params, stag_solver_stats* stats)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(psi, "psi"));
    STAG_TRY(check_half_field(b, "b"));
    if ((const double*)psi == b) {
        set_error("psi and b must not alias");
        return STAG_EINVAL;
    }
    if (!(mass > 0.0) || !isfinite(mass)) {
        set_error("the full-lattice solve needs a mass > 0 (m + D is singular or ill-posed otherwise)");
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
    double2* B[4];
    STAG_TRY(full_buffers(ctx, B));
    const Geom g = ctx->g;
    const unsigned grid = (unsigned)((2LL * g.Vh + 255) / 256);
    k_split_full<<<grid, 256, 0, ctx->stream>>>(g, (const double2*)b, B[0], B[1]);
    STAG_CUDA_TRY(cudaGetLastError());
    int arith = STAG_F64;
    STAG_TRY(resolve_f64_arith(ctx, prm.f64_arith, &arith));
    const bool dfx = arith == STAG_F64X;
    const void* lk = nullptr;
    STAG_TRY(ensure_links(ctx, STAG_F64, 18, &lk));
    if (dfx) STAG_TRY(schur_pre_df(ctx, B, mass));
    else STAG_TRY((schur_pre<LinkField<double2, 18>, SpinorF64>(ctx, LinkField<double2, 18>{(const double2*)lk, g.Vh}, B, mass)));
    const int rc = prm.inner_prec == STAG_F64 ? cg_solve_f64(ctx, B[3], B[2], mass, 0.0, prm, stats)
                                              : cg_solve_mixed(ctx, B[3], B[2], mass, prm, stats);
    if (rc < 0) return rc;
    // psi_o goes to the odd-parity scratch slot of B[0] (b_e is no longer needed)
    double2* psi_o = B[0];
    if (dfx) STAG_TRY(schur_post_df(ctx, B, psi_o, mass));
    else STAG_TRY((schur_post<LinkField<double2, 18>, SpinorF64>(ctx, LinkField<double2, 18>{(const double2*)lk, g.Vh}, B, psi_o, mass)));
    k_join_full<<<grid, 256, 0, ctx->stream>>>(g, B[3], psi_o, (double2*)psi);
    STAG_CUDA_TRY(cudaGetLastError());
    STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return rc;
}
