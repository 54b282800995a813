// tgauge.cu -- the temporal-gauge transform (Sec. 4.3; the layout and the
// operator's use of it are described in common.cuh): the gauge matrices g,
// the transformed links U' = g U g^dagger in every storage, and g / g^dagger
// applied to even-site vectors.  Computed in IEEE double from the internal
// F64/18 links once per gauge upload, on first use; the reduced-precision
// and double-float copies are derived from the double U' like the untransformed
// copies are from U.
#include <string.h>

#include "ctx.h"

namespace stag {

__device__ __forceinline__ Cplx<double> cmul(Cplx<double> a, Cplx<double> b)
{
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ Cplx<double> cmulc(Cplx<double> a, Cplx<double> b)   // a conj(b)
{
    return {fma(a.re, b.re, a.im * b.im), fma(a.im, b.re, -a.re * b.im)};
}

__device__ __forceinline__ Mat3<double> load_link64(const double2* L, int Vh, int par, int mu, int h)
{
    Mat3<double> U;
    const double2* q = L + ((size_t)(par * 4 + mu) * 9) * Vh + h;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double2 v = q[(size_t)k * Vh];
        U.m[k] = {v.x, v.y};
    }
    return U;
}

// C = A B
__device__ __forceinline__ Mat3<double> mm(const Mat3<double>& A, const Mat3<double>& B)
{
    Mat3<double> C;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            Cplx<double> s = {0.0, 0.0};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const Cplx<double> p = cmul(A.m[a * 3 + c], B.m[c * 3 + b]);
                s.re += p.re;
                s.im += p.im;
            }
            C.m[a * 3 + b] = s;
        }
    return C;
}

// C = A B^dagger
__device__ __forceinline__ Mat3<double> mmd(const Mat3<double>& A, const Mat3<double>& B)
{
    Mat3<double> C;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            Cplx<double> s = {0.0, 0.0};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const Cplx<double> p = cmulc(A.m[a * 3 + c], B.m[b * 3 + c]);
                s.re += p.re;
                s.im += p.im;
            }
            C.m[a * 3 + b] = s;
        }
    return C;
}

// g per site, one thread per spatial site walking up in time:
// g(t = 0) = 1, g(t + 1) = g(t) U_t(t).  G: [par][V/2][9] complex128.
__global__ void k_tg_gauge(Geom g, const double2* __restrict__ L, double2* __restrict__ G)
{
    const long long Vs = (long long)g.L[0] * g.L[1] * g.L[2];
    const long long is = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (is >= Vs) return;
    const int x = (int)(is % g.L[0]);
    const int yz = (int)(is / g.L[0]);
    const int y = yz % g.L[1], z = yz / g.L[1];
    Mat3<double> cur;
#pragma unroll
    for (int k = 0; k < 9; ++k) cur.m[k] = {(k % 4 == 0) ? 1.0 : 0.0, 0.0};
    for (int t = 0; t < g.L[3]; ++t) {
        const long long i = is + Vs * t;
        const int par = (x + y + z + t) & 1;
        const int h = (int)(i >> 1);
        double2* dst = G + ((size_t)par * g.Vh + h) * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) dst[k] = make_double2(cur.m[k].re, cur.m[k].im);
        if (t + 1 < g.L[3]) cur = mm(cur, load_link64(L, g.Vh, par, 3, h));
    }
}

__device__ __forceinline__ Mat3<double> load_g(const double2* G, int Vh, int par, int h)
{
    Mat3<double> M;
    const double2* q = G + ((size_t)par * Vh + h) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) M.m[k] = {q[k].x, q[k].y};
    return M;
}

__device__ __forceinline__ void store_link64(double2* q, size_t stride, const Mat3<double>& U)
{
#pragma unroll
    for (int k = 0; k < 9; ++k) q[(size_t)k * stride] = make_double2(U.m[k].re, U.m[k].im);
}

// U'_mu(x) = g(x) U_mu(x) g(x + mu)^dagger for the spatial directions;
// U'_t(x) = g(x) U_t(x) on the last time slice (g = 1 at t = 0) and exactly
// the identity elsewhere.  F64/18 layout [((par*4 + mu)*9 + k)*V/2 + h]; one
// thread per (par, h).
__global__ void k_tg_links(Geom g, const double2* __restrict__ L, const double2* __restrict__ G,
                           double2* __restrict__ out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2LL * g.Vh) return;
    const int par = (int)(idx / g.Vh), h = (int)(idx - (long long)par * g.Vh);
    SiteNbrs s;
    site_nbrs(g, par, h, s);
    const Mat3<double> gx = load_g(G, g.Vh, par, h);
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        const Mat3<double> U = load_link64(L, g.Vh, par, mu, h);
        const Mat3<double> Up = mmd(mm(gx, U), load_g(G, g.Vh, 1 - par, s.fwd[mu]));
        store_link64(out + ((size_t)(par * 4 + mu) * 9) * g.Vh + h, g.Vh, Up);
    }
    const int Vsh = g.Vh / g.L[3];
    const int t = h / Vsh;
    Mat3<double> Ut;
    if (t == g.L[3] - 1) {
        Ut = mm(gx, load_link64(L, g.Vh, par, 3, h));
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) Ut.m[k] = {(k % 4 == 0) ? 1.0 : 0.0, 0.0};
    }
    store_link64(out + ((size_t)(par * 4 + 3) * 9) * g.Vh + h, g.Vh, Ut);
}

// out = g v (dagger = 0) or g^dagger v (dagger = 1) on even sites, for
// nfield fields of V/2 sites back to back; in place allowed.
__global__ void k_tg_apply(int Vh, int nfield, const double2* __restrict__ G, const double2* in, double2* out,
                           int dagger)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nfield * Vh) return;
    const int h = (int)(idx % Vh);
    const Mat3<double> M = load_g(G, Vh, 0, h);
    Cplx<double> v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double2 q = in[(size_t)idx * 3 + c];
        v[c] = {q.x, q.y};
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Cplx<double> s = {0.0, 0.0};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // (g v)_a = g_ac v_c ; (g^dagger v)_a = conj(g_ca) v_c
            const Cplx<double> p = dagger ? cmulc(v[c], M.m[c * 3 + a]) : cmul(M.m[a * 3 + c], v[c]);
            s.re += p.re;
            s.im += p.im;
        }
        out[(size_t)idx * 3 + a] = make_double2(s.re, s.im);
    }
}

// The largest |(U U^dagger - 1)_ij| over all links (its bits, maximised over
// the warp by shuffles and then atomically: non-negative doubles order like
// their bit patterns); one thread per link (par, mu, h).
__global__ void k_tg_unitarity(int Vh, const double2* __restrict__ L, unsigned long long* out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0;
    if (idx < 8LL * Vh) {
        const int pm = (int)(idx / Vh), h = (int)(idx - (long long)pm * Vh);
        const Mat3<double> U = load_link64(L, Vh, pm >> 2, pm & 3, h);
        const Mat3<double> W = mmd(U, U);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const double re = W.m[k].re - ((k % 4 == 0) ? 1.0 : 0.0);
            d = fmax(d, fmax(fabs(re), fabs(W.m[k].im)));
        }
        if (!(d <= 1e300)) d = 1e300;   // NaN or infinity: as far from unitary as it gets
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
    if ((threadIdx.x & 31) == 0 && d > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(d));
}

// The temporal-gauge transform is a gauge transformation only for unitary
// links (g U g^dagger with U'_t = 1 needs U_t U_t^dagger = 1): links further
// than this from unitary are refused rather than solved wrongly.
constexpr double TG_UNITARITY_TOL = 1e-12;

// The gauge matrices g for the current gauge field, computed on first use
// after an upload (kept at their address), after checking that the links
// are unitary.
int ensure_tg_gauge(stag_ctx ctx, const double2** G)
{
    if (!ctx->have_gauge) {
        set_error("no gauge field uploaded");
        return STAG_ENOGAUGE;
    }
    const Geom g = ctx->g;
    if (!ctx->tg_g || ctx->tg_stale) {
        if (!ctx->tg_defect) STAG_CUDA_TRY(cudaMalloc(&ctx->tg_defect, sizeof(unsigned long long)));
        STAG_CUDA_TRY(cudaMemsetAsync(ctx->tg_defect, 0, sizeof(unsigned long long), ctx->stream));
        const long long nl = 8LL * g.Vh;
        k_tg_unitarity<<<(unsigned)((nl + 255) / 256), 256, 0, ctx->stream>>>(g.Vh, (const double2*)ctx->links[0],
                                                                            ctx->tg_defect);
        STAG_CUDA_TRY(cudaGetLastError());
        unsigned long long bits = 0;
        STAG_CUDA_TRY(cudaMemcpyAsync(&bits, ctx->tg_defect, sizeof(bits), cudaMemcpyDeviceToHost, ctx->stream));
        STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        double defect;
        memcpy(&defect, &bits, sizeof(defect));
        if (!(defect <= TG_UNITARITY_TOL)) {
            set_error("temporal gauge needs unitary links: max |U U^dagger - 1| = %.3g (limit %.0e)", defect,
                      TG_UNITARITY_TOL);
            return STAG_EUNSUPPORTED;
        }
        if (!ctx->tg_g) STAG_CUDA_TRY(cudaMalloc(&ctx->tg_g, (size_t)2 * g.Vh * 9 * sizeof(double2)));
        const long long Vs = (long long)g.L[0] * g.L[1] * g.L[2];
        k_tg_gauge<<<(unsigned)((Vs + 127) / 128), 128, 0, ctx->stream>>>(g, (const double2*)ctx->links[0],
                                                                        ctx->tg_g);
        STAG_CUDA_TRY(cudaGetLastError());
        ctx->tg_stale = false;
        // every transformed copy was made from the previous g
        for (int s = 0; s < 8; ++s) ctx->tg_link_stale[s] = ctx->tg_links[s] != nullptr;
    }
    *G = ctx->tg_g;
    return STAG_OK;
}

// U' in the storage (prec, recon): the F64/18 copy (slot 0) from g and U, the
// others derived from it (allocated on first use, re-derived in place after an
// upload: graphs hold these addresses).
int ensure_links_tg(stag_ctx ctx, int prec, int recon, const void** out)
{
    const double2* G = nullptr;
    STAG_TRY(ensure_tg_gauge(ctx, &G));
    const Geom g = ctx->g;
    if (!ctx->tg_links[0] || ctx->tg_link_stale[0]) {
        const size_t bytes = (size_t)8 * g.Vh * 9 * sizeof(double2);
        if (!ctx->tg_links[0]) STAG_CUDA_TRY(cudaMalloc(&ctx->tg_links[0], bytes));
        ctx->tg_link_bytes[0] = bytes;
        const long long n = 2LL * g.Vh;
        k_tg_links<<<(unsigned)((n + 127) / 128), 128, 0, ctx->stream>>>(g, (const double2*)ctx->links[0], G,
                                                                       (double2*)ctx->tg_links[0]);
        STAG_CUDA_TRY(cudaGetLastError());
        ctx->tg_link_stale[0] = false;
        for (int s = 1; s < 8; ++s) ctx->tg_link_stale[s] = ctx->tg_links[s] != nullptr;
    }
    const int slot = link_slot(prec, recon);
    if (slot != 0 && (!ctx->tg_links[slot] || ctx->tg_link_stale[slot])) {
        int e = 0;
        if (prec == STAG_F64X) {
            // the scaling rule of the untransformed double-float copy (|U'| and
            // |U| are bounded alike for the unitary links this path needs)
            STAG_TRY(link_max_exponent(ctx, &e));
            ctx->df_link_exp = (e > DF_LINK_SAFE_EXP || e < -DF_LINK_SAFE_EXP) ? e : 0;
            e = ctx->df_link_exp;
        }
        STAG_TRY(derive_link_copy(ctx, (const double2*)ctx->tg_links[0], prec, recon, e, &ctx->tg_links[slot],
                                  &ctx->tg_link_bytes[slot]));
        ctx->tg_link_stale[slot] = false;
    }
    *out = ctx->tg_links[slot];
    return STAG_OK;
}

// Room for g b of nfield even-site fields (grown on demand; not held by graphs).
int ensure_tg_tmp(stag_ctx ctx, int nfield, double2** out)
{
    if (nfield > ctx->tg_tmp_fields) {
        if (ctx->tg_tmp) {
            STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
            cudaFree(ctx->tg_tmp);
            ctx->tg_tmp = nullptr;
            ctx->tg_tmp_fields = 0;
        }
        STAG_CUDA_TRY(cudaMalloc(&ctx->tg_tmp, (size_t)nfield * 3 * ctx->g.Vh * sizeof(double2)));
        ctx->tg_tmp_fields = nfield;
    }
    *out = ctx->tg_tmp;
    return STAG_OK;
}

int tg_apply(stag_ctx ctx, const double2* G, const double2* in, double2* out, int nfield, int dagger)
{
    const long long n = (long long)nfield * ctx->g.Vh;
    if (n == 0) return STAG_OK;
    k_tg_apply<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(ctx->g.Vh, nfield, G, in, out, dagger);
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

}  // namespace stag
