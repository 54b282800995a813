// force.cu -- the pseudo-fermion action S = phi^dagger M^{-1} phi and its
// derivative with respect to the links (the HMC fermion force; the paper names
// HMC as the setting of the inversion, Sec. 1, and gauge-field derivatives as a
// backend capability, Sec. 3; the force itself is not in the paper).
//
// With X = M^{-1} phi (even sites) and Y = D_oe X (odd sites), varying a link
// changes S by dS = X^dagger dD_eo Y - Y^dagger dD_oe X (D_eo^dagger = -D_oe).
// For the link U_{x,mu}, eta = eta_mu(x) times the boundary sign of the hop:
//   x even: G = 2 eta X_x Y_{x+mu}^dagger,   x odd: G = -2 eta Y_x X_{x+mu}^dagger,
// G the Euclidean gradient (dS = Re sum conj(G_ab) dU_ab, the PyTorch
// convention dS/dRe U + i dS/dIm U).  Under U -> exp(i eps T) U,
// dS/deps = tr(i T P) with P = TA(U G^dagger) = (W - W^dagger)/2 - tr(W - W^dagger)/6.
// G = s u v^dagger is an outer product, so W = U G^dagger = s (U v) u^dagger
// costs one matrix-vector product per link.
#include <chrono>
#include <cmath>
#include <new>

#include "cg_kernels.cuh"
#include "df64.cuh"
#include "workspace.h"

namespace stag {

constexpr int F_BS = 128;

// One thread per (site, mu), in the canonical order i*4 + mu, so each thread
// writes its link's 144 contiguous bytes of P and G.
template <class LF>
__global__ void __launch_bounds__(F_BS) k_force(Geom g, LF U, const double2* X, const double2* Y, double2* P,
                                                double2* G, double scale, int accumulate)
{
    const long long idx = (long long)blockIdx.x * F_BS + threadIdx.x;
    if (idx >= 8LL * g.Vh) return;
    const int i = (int)(idx >> 2);   // lexicographic site (V < 2^31)
    const int mu = (int)(idx & 3);
    // coordinates and parity of site i from its half index (Lx even)
    const int h = i >> 1;
    const int rr = fast_div(h, g.dxh);
    const int x = 2 * (h - rr * g.Lxh) + (i & 1);
    const int zt = fast_div(rr, g.dy);
    const int y = rr - zt * g.L[1];
    const int t = fast_div(zt, g.dz);
    const int z = zt - t * g.L[2];
    const int par = (x + y + z + t) & 1;
    int hf;
    uint32_t sfb;
    fwd_nbr(g, par, h, mu, hf, sfb);
    // eta_mu(x) times the forward boundary sign, as a double
    const double eta = (sfb ? -1.0 : 1.0);
    // u, v and s of G = s u v^dagger
    const double2* up = par == 0 ? X + (size_t)h * 3 : Y + (size_t)h * 3;
    const double2* vp = par == 0 ? Y + (size_t)hf * 3 : X + (size_t)hf * 3;
    const double sg = (par == 0 ? 2.0 : -2.0) * eta * scale;
    // u carries the factor s: G = u v^dagger, W = U G^dagger = (U v) u^dagger.
    // GB300 runs FP64 at 1/64 of the FP32 rate and this kernel is bound by it,
    // so the arithmetic is arranged to the minimum: scale factors folded into
    // the vectors once, and only the upper triangle and the diagonal of the
    // antihermitian P formed (P_ba = -conj(P_ab)).
    Cplx<double> u[3], v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double2 q = __ldg(up + a), w = __ldg(vp + a);
        u[a] = {sg * q.x, sg * q.y};
        v[a] = {w.x, w.y};
    }
    double2* Gp = G ? G + (size_t)idx * 9 : nullptr;
    if (Gp) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                // u_a conj(v_b)
                double2 o = make_double2(fma(u[a].re, v[b].re, u[a].im * v[b].im),
                                         fma(u[a].im, v[b].re, -(u[a].re * v[b].im)));
                if (accumulate) {
                    const double2 q = Gp[a * 3 + b];
                    o.x += q.x;
                    o.y += q.y;
                }
                Gp[a * 3 + b] = o;
            }
    }
    if (P) {
        const Mat3<double> Um = U.load(par, mu, h);
        Cplx<double> w[3];   // (U v) / 2
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                re = fma(Um.m[a * 3 + c].re, v[c].re, re);
                re = fma(-Um.m[a * 3 + c].im, v[c].im, re);
                im = fma(Um.m[a * 3 + c].re, v[c].im, im);
                im = fma(Um.m[a * 3 + c].im, v[c].re, im);
            }
            w[a] = {0.5 * re, 0.5 * im};
        }
        // P = (W - W^dagger)/2 - tr(W - W^dagger)/6 with W_ab = 2 w_a conj(u_b):
        //   P_ab = w_a conj(u_b) - u_a conj(w_b),
        //   P_aa = 2i Im(w_a conj(u_a)) - (2i/3) sum_c Im(w_c conj(u_c))
        double d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = 2.0 * fma(w[a].im, u[a].re, -(w[a].re * u[a].im));
        const double trim = (d[0] + d[1] + d[2]) * (1.0 / 3.0);
        // off-diagonal (a, b) = (0, 1), (0, 2), (1, 2)
        auto offd = [&](int a, int b) {
            return Cplx<double>{fma(w[a].re, u[b].re, w[a].im * u[b].im) - fma(u[a].re, w[b].re, u[a].im * w[b].im),
                                fma(w[a].im, u[b].re, -(w[a].re * u[b].im)) -
                                    fma(u[a].im, w[b].re, -(u[a].re * w[b].im))};
        };
        const Cplx<double> p01 = offd(0, 1), p02 = offd(0, 2), p12 = offd(1, 2);
        const Cplx<double> Pm[9] = {{0.0, d[0] - trim}, p01, p02,
                                    {-p01.re, p01.im}, {0.0, d[1] - trim}, p12,
                                    {-p02.re, p02.im}, {-p12.re, p12.im}, {0.0, d[2] - trim}};
        double2* Pp = P + (size_t)idx * 9;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 o = make_double2(Pm[k].re, Pm[k].im);
            if (accumulate) {
                const double2 q = Pp[k];
                o.x += q.x;
                o.y += q.y;
            }
            Pp[k] = o;
        }
    }
}

// The same force with the projected P formed in double-float arithmetic (the
// FP32 pipe: GB300 runs FP64 at 1/64 of the FP32 rate).  u and v enter
// normalised, u' = 2^-ku sg u and v' = 2^-kv v (ku, kv the exponents of the
// largest components of the fields they come from, so that every product stays
// inside the float range), W' = U v' u'^dagger and P' = TA(W') in double-float,
// and P = 2^(ku + kv) P' in double with an exact scaling.  G = sg u v^dagger,
// when asked for, is formed in IEEE double as in k_force (18 products of
// doubles cost less than converting 18 double-float results).  kexp[0] and
// kexp[1]: the exponents of X and Y.
//
// The thread's site comes from its half index h = i / 2 by the multiply-high
// divisions of the geometry (x = 2 (h mod Lx/2) + (i mod 2), Lx even), and
// |sg| = 2 |scale| = sgn 2^ks is split once on the host (sgn in [1, 2), ks its
// exponent); the sign of sg (the parity, eta and boundary, and scale's) is a
// sign bit applied exactly to u and to the G products.
__global__ void __launch_bounds__(F_BS) k_force_df(Geom g, LinkFieldDF<18> U, const double2* X, const double2* Y,
                                                   double2* P, double2* G, double sg_abs, double sgn, int ks,
                                                   uint32_t sbit_scale, int accumulate, const int* kexp)
{
    const long long idx = (long long)blockIdx.x * F_BS + threadIdx.x;
    if (idx >= 8LL * g.Vh) return;
    const int i = (int)(idx >> 2);   // lexicographic site (V < 2^31)
    const int mu = (int)(idx & 3);
    const int h = i >> 1;
    const int rr = fast_div(h, g.dxh);
    const int x = 2 * (h - rr * g.Lxh) + (i & 1);
    const int zt = fast_div(rr, g.dy);
    const int y = rr - zt * g.L[1];
    const int t = fast_div(zt, g.dz);
    const int z = zt - t * g.L[2];
    const int par = (x + y + z + t) & 1;
    int hf;
    uint32_t sfb;
    fwd_nbr(g, par, h, mu, hf, sfb);
    const uint32_t sbit = (par ? 0x80000000u : 0u) ^ sfb ^ sbit_scale;   // sign of sg
    const double sg = flip(sg_abs, sbit);
    const double2* up = par == 0 ? X + (size_t)h * 3 : Y + (size_t)h * 3;
    const double2* vp = par == 0 ? Y + (size_t)hf * 3 : X + (size_t)hf * 3;
    const int ku = kexp[par], kv = kexp[1 - par];
    double2 uq[3], vq[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        uq[a] = __ldg(up + a);
        vq[a] = __ldg(vp + a);
    }
    if (G) {
        double2* Gp = G + (size_t)idx * 9;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double ure = sg * uq[a].x, uim = sg * uq[a].y;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                double2 o = make_double2(fma(ure, vq[b].x, uim * vq[b].y), fma(uim, vq[b].x, -(ure * vq[b].y)));
                if (accumulate) {
                    const double2 q = Gp[a * 3 + b];
                    o.x += q.x;
                    o.y += q.y;
                }
                Gp[a * 3 + b] = o;
            }
        }
    }
    if (!P) return;
    const DF sgd = split_double(sgn);   // |sg| = sgd 2^ks, sgd in [1, 2)
    Cplx<DF> u[3], v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const DF ur = split_double_scaled(uq[a].x, ku), ui = split_double_scaled(uq[a].y, ku);
        u[a] = {DF(0), DF(0)};
        df_mac(u[a].re, sgd, ur);
        df_mac(u[a].im, sgd, ui);
        // the sign of sg: an exact negation of the products
        u[a] = {flip(u[a].re, sbit), flip(u[a].im, sbit)};
        v[a] = {split_double_scaled(vq[a].x, kv), split_double_scaled(vq[a].y, kv)};
    }
    const Mat3<DF> Um = U.load(par, mu, h);
    Cplx<DF> w[3];   // U v'
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        DF re(0), im(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            df_mac(re, Um.m[a * 3 + c].re, v[c].re);
            df_mac(re, df_neg(Um.m[a * 3 + c].im), v[c].im);
            df_mac(im, Um.m[a * 3 + c].re, v[c].im);
            df_mac(im, Um.m[a * 3 + c].im, v[c].re);
        }
        w[a] = {re, im};
    }
    // with W = 2 w u^dagger / 2 = w u^dagger (the 2 of P = (W - W^dagger)/2 cancels):
    //   P_ab = (w_a conj(u_b) - u_a conj(w_b)) / 2 ... written with w halved below
    // diagonal: P_aa = i (Im(w_a conj(u_a)) - (1/3) sum_c Im(w_c conj(u_c))) times 2 / 2
    DF d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        DF q(0);
        df_mac(q, w[a].im, u[a].re);
        df_mac(q, df_neg(w[a].re), u[a].im);
        d[a] = q;
    }
    const DF tr = df_add(df_add(d[0], d[1]), d[2]);
    const DF third = split_double(1.0 / 3.0);
    DF trim(0);
    df_mac(trim, tr, third);
    auto offd = [&](int a, int b) {
        DF re(0), im(0);
        df_mac(re, w[a].re, u[b].re);
        df_mac(re, w[a].im, u[b].im);
        df_mac(re, df_neg(u[a].re), w[b].re);
        df_mac(re, df_neg(u[a].im), w[b].im);
        df_mac(im, w[a].im, u[b].re);
        df_mac(im, df_neg(w[a].re), u[b].im);
        df_mac(im, df_neg(u[a].im), w[b].re);
        df_mac(im, u[a].re, w[b].im);
        return Cplx<DF>{re, im};
    };
    const Cplx<DF> p01 = offd(0, 1), p02 = offd(0, 2), p12 = offd(1, 2);
    // P_ab = (w_a conj(u_b) - u_a conj(w_b)) / 2, P_aa = i (d_a - trim): the
    // halving and 2^(ku + kv + ks) are one exact scaling of the double result
    const int k = ku + kv + ks - 1;
    auto out = [&](const DF& v_) { return df_to_double_scaled(v_, k); };
    const double d0 = df_to_double_scaled(df_add(d[0], df_neg(trim)), k + 1),
                 d1 = df_to_double_scaled(df_add(d[1], df_neg(trim)), k + 1),
                 d2 = df_to_double_scaled(df_add(d[2], df_neg(trim)), k + 1);
    const double r01 = out(p01.re), i01 = out(p01.im), r02 = out(p02.re), i02 = out(p02.im), r12 = out(p12.re),
                 i12 = out(p12.im);
    const double2 Pm[9] = {make_double2(0.0, d0),    make_double2(r01, i01),   make_double2(r02, i02),
                           make_double2(-r01, i01),  make_double2(0.0, d1),    make_double2(r12, i12),
                           make_double2(-r02, i02),  make_double2(-r12, i12),  make_double2(0.0, d2)};
    double2* Pp = P + (size_t)idx * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        double2 o = Pm[e];
        if (accumulate) {
            const double2 q = Pp[e];
            o.x += q.x;
            o.y += q.y;
        }
        Pp[e] = o;
    }
}

// P alone from X and Y already in double-float storage at one scale: X' =
// 2^-kx X (largest component in [1, 2)) and Y' = D_oe X' from the
// double-float operator, so neither field is joined to double, normalised
// again or split per link.  The arithmetic is that of k_force_df with
// ku = kv = kx (kexp[0]).
__global__ void __launch_bounds__(F_BS) k_force_dfin(Geom g, LinkFieldDF<18> U, const float4* Xd, const float4* Yd,
                                                     double2* P, double sgn, int ks, uint32_t sbit_scale,
                                                     int accumulate, const int* kexp)
{
    const long long idx = (long long)blockIdx.x * F_BS + threadIdx.x;
    if (idx >= 8LL * g.Vh) return;
    const int i = (int)(idx >> 2);   // lexicographic site (V < 2^31)
    const int mu = (int)(idx & 3);
    const int h = i >> 1;
    const int rr = fast_div(h, g.dxh);
    const int x = 2 * (h - rr * g.Lxh) + (i & 1);
    const int zt = fast_div(rr, g.dy);
    const int y = rr - zt * g.L[1];
    const int t = fast_div(zt, g.dz);
    const int z = zt - t * g.L[2];
    const int par = (x + y + z + t) & 1;
    int hf;
    uint32_t sfb;
    fwd_nbr(g, par, h, mu, hf, sfb);
    const uint32_t sbit = (par ? 0x80000000u : 0u) ^ sfb ^ sbit_scale;   // sign of sg
    const float4* up = par == 0 ? Xd + (size_t)h * 3 : Yd + (size_t)h * 3;
    const float4* vp = par == 0 ? Yd + (size_t)hf * 3 : Xd + (size_t)hf * 3;
    const DF sgd = split_double(sgn);   // |sg| = sgd 2^ks
    Cplx<DF> u[3], v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float4 q = __ldg(up + a), w = __ldg(vp + a);
        u[a] = {DF(0), DF(0)};
        df_mac(u[a].re, sgd, DF(q.x, q.y));
        df_mac(u[a].im, sgd, DF(q.z, q.w));
        u[a] = {flip(u[a].re, sbit), flip(u[a].im, sbit)};
        v[a] = {DF(w.x, w.y), DF(w.z, w.w)};
    }
    const Mat3<DF> Um = U.load(par, mu, h);
    Cplx<DF> wv[3];   // U v'
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        DF re(0), im(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            df_mac(re, Um.m[a * 3 + c].re, v[c].re);
            df_mac(re, df_neg(Um.m[a * 3 + c].im), v[c].im);
            df_mac(im, Um.m[a * 3 + c].re, v[c].im);
            df_mac(im, Um.m[a * 3 + c].im, v[c].re);
        }
        wv[a] = {re, im};
    }
    DF d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        DF q(0);
        df_mac(q, wv[a].im, u[a].re);
        df_mac(q, df_neg(wv[a].re), u[a].im);
        d[a] = q;
    }
    const DF tr = df_add(df_add(d[0], d[1]), d[2]);
    const DF third = split_double(1.0 / 3.0);
    DF trim(0);
    df_mac(trim, tr, third);
    auto offd = [&](int a, int b) {
        DF re(0), im(0);
        df_mac(re, wv[a].re, u[b].re);
        df_mac(re, wv[a].im, u[b].im);
        df_mac(re, df_neg(u[a].re), wv[b].re);
        df_mac(re, df_neg(u[a].im), wv[b].im);
        df_mac(im, wv[a].im, u[b].re);
        df_mac(im, df_neg(wv[a].re), u[b].im);
        df_mac(im, df_neg(u[a].im), wv[b].re);
        df_mac(im, u[a].re, wv[b].im);
        return Cplx<DF>{re, im};
    };
    const Cplx<DF> p01 = offd(0, 1), p02 = offd(0, 2), p12 = offd(1, 2);
    const int k = 2 * kexp[0] + ks - 1;
    auto out = [&](const DF& v_) { return df_to_double_scaled(v_, k); };
    const double d0 = df_to_double_scaled(df_add(d[0], df_neg(trim)), k + 1),
                 d1 = df_to_double_scaled(df_add(d[1], df_neg(trim)), k + 1),
                 d2 = df_to_double_scaled(df_add(d[2], df_neg(trim)), k + 1);
    const double r01 = out(p01.re), i01 = out(p01.im), r02 = out(p02.re), i02 = out(p02.im), r12 = out(p12.re),
                 i12 = out(p12.im);
    const double2 Pm[9] = {make_double2(0.0, d0),    make_double2(r01, i01),   make_double2(r02, i02),
                           make_double2(-r01, i01),  make_double2(0.0, d1),    make_double2(r12, i12),
                           make_double2(-r02, i02),  make_double2(-r12, i12),  make_double2(0.0, d2)};
    double2* Pp = P + (size_t)idx * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        double2 o = Pm[e];
        if (accumulate) {
            const double2 q = Pp[e];
            o.x += q.x;
            o.y += q.y;
        }
        Pp[e] = o;
    }
}

// out = c X (the gradient 2 dS X of S with respect to phi), canonical half field.
__global__ void k_scale_copy(long long n, const double2* X, double2* out, double c)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        const double2 v = X[k];
        out[k] = make_double2(c * v.x, c * v.y);
    }
}

// Re <a, b> over a half field, deterministic two-stage sum into *out (device).
template <int BS>
__global__ void __launch_bounds__(BS) k_dot_re(int Vh, const double2* a, const double2* b, double* out, double* part,
                                               unsigned* cnt)
{
    __shared__ double red[BS / 32];
    __shared__ bool last;
    const int h = blockIdx.x * BS + threadIdx.x;
    double d = 0.0;
    if (h < Vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 x = a[(size_t)h * 3 + c], y = b[(size_t)h * 3 + c];
            d = fma(x.x, y.x, d);
            d = fma(x.y, y.y, d);
        }
    }
    const double s = block_sum<BS>(d, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    if (!arrive_last(cnt, &last)) return;
    const double tot = sum_partials<BS>(part, gridDim.x, red);
    if (threadIdx.x == 0) {
        *cnt = 0;
        *out = tot;
    }
}

int ensure_cg_f64(stag_ctx ctx);
int cg_solve_f64(stag_ctx ctx, double2* x_out, const double2* b_in, double mass, double sigma,
                 const stag_solver_params& prm, stag_solver_stats* st);
int cg_solve_mixed(stag_ctx ctx, double2* x_out, const double2* b_in, double mass, const stag_solver_params& prm,
                   stag_solver_stats* st);
int check_ctx(stag_ctx ctx);
int check_half_field(const void* p, const char* what);

int force_from_X(stag_ctx ctx, double2* P, double2* G, const double2* X, double2* phi_grad, double scale,
                 int accumulate = 0)
{
    const void* lk = nullptr;
    STAG_TRY(ensure_links(ctx, STAG_F64, 18, &lk));
    const Geom g = ctx->g;
    const LinkField<double2, 18> U{(const double2*)lk, g.Vh};
    const long long n = 8LL * g.Vh;
    const unsigned grid = (unsigned)((n + F_BS - 1) / F_BS);
    const bool df_ok = ctx->df_link_exp == 0 && scale != 0.0 && isfinite(scale);
    // |sg| = 2 |scale| = sgn 2^ks with sgn in [1, 2) (exact scalings)
    const double sg_abs = 2.0 * fabs(scale);
    const int ks = df_ok ? ilogb(sg_abs) : 0;
    const double sgn = df_ok ? ldexp(sg_abs, -ks) : 0.0;
    const uint32_t sbit_scale = signbit(scale) ? 0x80000000u : 0u;
    if (P && !G && df_ok) {
        // P alone: X' = 2^-kx X split once into double-float storage, Y' =
        // D_oe X' by the double-float operator, both read as they are
        const void* lkdf = nullptr;
        STAG_TRY(ensure_links(ctx, STAG_F64X, 18, &lkdf));
        float4 *xd = nullptr, *yd = nullptr;
        STAG_TRY(dfx_fields(ctx, 1, &xd, &yd));
        const size_t elems = (size_t)3 * g.Vh;
        STAG_TRY(field_exponents(ctx, X, 1, elems, SLOT_FORCE, ctx->stream));
        STAG_TRY(split_fields_scaled(ctx, X, xd, 1, elems, SLOT_FORCE, 0, ctx->stream));
        STAG_TRY(launch_dslash_internal(ctx, STAG_F64X, 18, 1, yd, xd, ctx->stream));
        k_force_dfin<<<grid, F_BS, 0, ctx->stream>>>(g, LinkFieldDF<18>{(const float4*)lkdf, g.Vh}, xd, yd, P, sgn,
                                                     ks, sbit_scale, accumulate, ctx->scale_k + SLOT_FORCE);
        if (phi_grad) {
            const long long m = 3LL * g.Vh;
            k_scale_copy<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(m, X, phi_grad, 2.0 * scale);
        }
        STAG_CUDA_TRY(cudaGetLastError());
        return STAG_OK;
    }
    // Y = D_oe X into the context's odd temporary, with the double-float
    // operator (~1e-14 relative; the IEEE-double one is FP64-bound on GB300)
    STAG_TRY(launch_dslash(ctx, STAG_F64X, 18, 1, ctx->tmp_odd, X, ctx->stream));
    if (P && df_ok) {
        // P in double-float arithmetic on the double-float links, X and Y normalised
        const void* lkdf = nullptr;
        STAG_TRY(ensure_links(ctx, STAG_F64X, 18, &lkdf));
        STAG_TRY(field_exponents(ctx, X, 1, (size_t)3 * g.Vh, SLOT_FORCE, ctx->stream));
        STAG_TRY(field_exponents(ctx, ctx->tmp_odd, 1, (size_t)3 * g.Vh, SLOT_FORCE + 1, ctx->stream));
        k_force_df<<<grid, F_BS, 0, ctx->stream>>>(g, LinkFieldDF<18>{(const float4*)lkdf, g.Vh}, X, ctx->tmp_odd, P,
                                                   G, sg_abs, sgn, ks, sbit_scale, accumulate,
                                                   ctx->scale_k + SLOT_FORCE);
    } else {
        k_force<LinkField<double2, 18>><<<grid, F_BS, 0, ctx->stream>>>(g, U, X, ctx->tmp_odd, P, G, scale,
                                                                        accumulate);
    }
    if (phi_grad) {
        const long long m = 3LL * g.Vh;
        k_scale_copy<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(m, X, phi_grad, 2.0 * scale);
    }
    STAG_CUDA_TRY(cudaGetLastError());
    return STAG_OK;
}

}  // namespace stag

using namespace stag;

extern "C" {

int stag_fermion_force(stag_ctx ctx, double* P, double* G, const double* X_even, double* phi_grad, double scale)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(X_even, "X_even"));
    if (!P && !G && !phi_grad) {
        set_error("at least one of P, G, phi_grad must be given");
        return STAG_EINVAL;
    }
    if (P) STAG_TRY(check_half_field(P, "P"));
    if (G) STAG_TRY(check_half_field(G, "G"));
    if (phi_grad) STAG_TRY(check_half_field(phi_grad, "phi_grad"));
    if ((P && (const double*)P == X_even) || (G && (const double*)G == X_even) ||
        (phi_grad && (const double*)phi_grad == X_even)) {
        set_error("outputs must not alias X_even");
        return STAG_EINVAL;
    }
    if (!ctx->have_gauge) {
        set_error("no gauge field uploaded");
        return STAG_ENOGAUGE;
    }
    return force_from_X(ctx, (double2*)P, (double2*)G, (const double2*)X_even, (double2*)phi_grad, scale);
}

int stag_fermion_force_multi(stag_ctx ctx, double* P, double* G, const double* X, const double* coeffs, int n)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(X, "X"));
    if (!P && !G) {
        set_error("at least one of P, G must be given");
        return STAG_EINVAL;
    }
    if (P) STAG_TRY(check_half_field(P, "P"));
    if (G) STAG_TRY(check_half_field(G, "G"));
    if (!coeffs || n < 1 || n > STAG_MAX_RHS) {
        set_error("coeffs must be a host array of 1..%d values", STAG_MAX_RHS);
        return STAG_EINVAL;
    }
    if (!ctx->have_gauge) {
        set_error("no gauge field uploaded");
        return STAG_ENOGAUGE;
    }
    const size_t stride = (size_t)3 * ctx->g.Vh;
    for (int i = 0; i < n; ++i)
        STAG_TRY(force_from_X(ctx, (double2*)P, (double2*)G, (const double2*)X + i * stride, nullptr, coeffs[i],
                              i > 0));
    return STAG_OK;
}

int stag_fermion_action(stag_ctx ctx, const double* phi_even, double mass, const stag_solver_params* params,
                        double* X_even, double* S, stag_solver_stats* stats)
{
    STAG_TRY(check_ctx(ctx));
    STAG_TRY(check_half_field(phi_even, "phi_even"));
    STAG_TRY(check_half_field(X_even, "X_even"));
    if (!S) {
        set_error("S is NULL");
        return STAG_EINVAL;
    }
    if ((const double*)X_even == phi_even) {
        set_error("X_even must not alias phi_even");
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
    int rc = prm.inner_prec == STAG_F64
                 ? cg_solve_f64(ctx, (double2*)X_even, (const double2*)phi_even, mass, 0.0, prm, stats)
                 : cg_solve_mixed(ctx, (double2*)X_even, (const double2*)phi_even, mass, prm, stats);
    if (rc < 0) return rc;
    STAG_TRY(ensure_cg_f64(ctx));
    const int Vh = ctx->g.Vh;
    double* dS = (double*)(ctx->ws->sc + 63);   // a spare device record
    k_dot_re<256><<<(Vh + 255) / 256, 256, 0, ctx->stream>>>(Vh, (const double2*)phi_even, (const double2*)X_even,
                                                             dS, ctx->partials, ctx->counters);
    STAG_CUDA_TRY(cudaGetLastError());
    STAG_CUDA_TRY(cudaMemcpyAsync(S, dS, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    STAG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return rc;
}

}  // extern "C"
