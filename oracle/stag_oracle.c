/*
 * stag_oracle.c -- plain, slow, double-precision CPU oracle for the staggered
 * Dirac operator, the even-odd normal matrix M = m^2 - D_eo D_oe, conjugate
 * gradient and multi-shift CG on M, and the pseudo-fermion force.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark load this file; the CUDA library never does.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * Written for a reader who checks it against the paper by eye: no blocking,
 * no fusion, sums in plain sequential order, one lattice site at a time.
 * Build with -ffp-contract=off so every result is reproducible bit for bit.
 * A second build with -fopenmp (timing only: the CPU baseline) spreads the
 * loops over independent output sites and vector elements across threads;
 * every reduction stays sequential, so both builds give identical bits.
 *
 * Conventions (inputs produced by lattice_inputs):
 *   site index  i = x + Lx*(y + Ly*(z + Lz*t)), mu = 0,1,2,3 = x,y,z,t;
 *   U[((i*4 + mu)*3 + a)*3 + b] = (U_{x,mu})_{ab}, complex double;
 *   full field  phi[i*3 + a];
 *   half field of parity p: psi[(i/2)*3 + a] over the sites with
 *   (x+y+z+t) mod 2 == p (Lx even makes i/2 a bijection per parity).
 *
 * Parity status of each function (what pins it, see tests/test_oracle.py):
 *   orc_eta, orc_dslash_full, orc_dslash_half  pinned (antihermiticity,
 *       even-odd connectivity, gauge covariance, plaquette flux of the
 *       phases, free-field spectrum with antiperiodic time)
 *   orc_apply_M                              pinned (free spectrum, Schur
 *       identity against the dense full operator)
 *   orc_cg                                   pinned (dense linear solve)
 *   orc_multishift_cg                        pinned (dense shifted solves)
 *   orc_force, orc_action                    pinned (central finite
 *       differences of S, gauge covariance of the force)
 *   orc_reconstruct_row2                     pinned (SU(3) matrices)
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* Geometry                                                                   */
/* ------------------------------------------------------------------------- */

/* Extents must be even (so every row holds one site of each parity) and >= 2. */
int orc_check_dims(const int L[4])
{
    for (int mu = 0; mu < 4; ++mu)
        if (L[mu] < 2 || (L[mu] % 2) != 0)
            return -1;
    return 0;
}

long orc_volume(const int L[4])
{
    return (long)L[0] * L[1] * L[2] * L[3];
}

/* Threads the site loops use: 1 in the parity build, the OpenMP team size in
 * the timing build. */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static long lex_index(const int L[4], const int c[4])
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

static void lex_coords(const int L[4], long i, int c[4])
{
    c[0] = (int)(i % L[0]); i /= L[0];
    c[1] = (int)(i % L[1]); i /= L[1];
    c[2] = (int)(i % L[2]); i /= L[2];
    c[3] = (int)i;
}

static int site_parity(const int c[4])
{
    return (c[0] + c[1] + c[2] + c[3]) % 2;
}

/* Kogut-Susskind phase eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) (Sec. 4.2 only
 * says eta = +-1; this is the usual choice with x varying first). */
int orc_eta(const int L[4], const int c[4], int mu)
{
    (void)L;
    int s = 0;
    for (int nu = 0; nu < mu; ++nu)
        s += c[nu];
    return (s % 2 == 0) ? 1 : -1;
}

/* Coordinates of x + dir*mu_hat with periodic wrap.  The returned sign is the
 * boundary factor of the hop: -1 when it crosses the time boundary
 * (antiperiodic in t), +1 otherwise (periodic in space). */
static int shifted(const int L[4], const int c[4], int mu, int dir, int out[4])
{
    int bc = 1;
    for (int nu = 0; nu < 4; ++nu)
        out[nu] = c[nu];
    out[mu] = c[mu] + dir;
    if (out[mu] >= L[mu]) {
        out[mu] -= L[mu];
        if (mu == 3) bc = -1;
    }
    if (out[mu] < 0) {
        out[mu] += L[mu];
        if (mu == 3) bc = -1;
    }
    return bc;
}

static const cplx *link(const cplx *U, long i, int mu)
{
    return U + (i * 4 + mu) * 9;
}

/* ------------------------------------------------------------------------- */
/* The staggered operator, Sec. 4.2 Eq. (staggered):                           */
/*   (D phi)_x = sum_mu [ eta_mu(x) U_{x,mu} phi_{x+mu}                        */
/*                       - eta_mu(x-mu) U^dagger_{x-mu,mu} phi_{x-mu} ]        */
/* with no factor 1/2 and no mass term; the antiperiodic time boundary enters  */
/* as the sign of the hop that crosses it.                                     */
/* ------------------------------------------------------------------------- */

/* (D phi)_x for one site x; phi_at(j) returns the colour vector at lexicographic
 * site j (or NULL for a site where the field is zero). */
typedef const cplx *(*field_at_fn)(const void *ctx, long j);

static void dslash_site(const int L[4], const cplx *U, const int c[4],
                        field_at_fn phi_at, const void *ctx, cplx out[3])
{
    out[0] = out[1] = out[2] = 0.0;
    long i = lex_index(L, c);
    for (int mu = 0; mu < 4; ++mu) {
        int cf[4], cb[4];
        /* forward hop: + eta_mu(x) U_{x,mu} phi_{x+mu} */
        int bcf = shifted(L, c, mu, +1, cf);
        const cplx *phf = phi_at(ctx, lex_index(L, cf));
        if (phf) {
            const cplx *u = link(U, i, mu);
            double s = (double)(orc_eta(L, c, mu) * bcf);
            for (int a = 0; a < 3; ++a) {
                cplx acc = 0.0;
                for (int b = 0; b < 3; ++b)
                    acc += u[a * 3 + b] * phf[b];
                out[a] += s * acc;
            }
        }
        /* backward hop: - eta_mu(x-mu) U^dagger_{x-mu,mu} phi_{x-mu} */
        int bcb = shifted(L, c, mu, -1, cb);
        const cplx *phb = phi_at(ctx, lex_index(L, cb));
        if (phb) {
            const cplx *u = link(U, lex_index(L, cb), mu);
            double s = (double)(orc_eta(L, cb, mu) * bcb);
            for (int a = 0; a < 3; ++a) {
                cplx acc = 0.0;
                for (int b = 0; b < 3; ++b)
                    acc += conj(u[b * 3 + a]) * phb[b];
                out[a] -= s * acc;
            }
        }
    }
}

static const cplx *full_at(const void *ctx, long j)
{
    return (const cplx *)ctx + j * 3;
}

/* out = D in, full lattice, both fields (V,3). */
int orc_dslash_full(const int L[4], const cplx *U, const cplx *in, cplx *out)
{
    if (orc_check_dims(L)) return -1;
    long V = orc_volume(L);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; ++i) {
        int c[4];
        lex_coords(L, i, c);
        dslash_site(L, U, c, full_at, in, out + i * 3);
    }
    return 0;
}

/* A half field seen as a full field that vanishes on the other parity. */
struct half_view {
    const int *L;
    const cplx *psi;
    int parity;
};

static const cplx *half_at(const void *ctx, long j)
{
    const struct half_view *hv = (const struct half_view *)ctx;
    int c[4];
    lex_coords(hv->L, j, c);
    if (site_parity(c) != hv->parity) return NULL;
    return hv->psi + (j / 2) * 3;
}

/* Half operator D_{p,1-p}: out (parity out_parity, (V/2,3)) = D restricted to
 * output sites of parity out_parity acting on a field living on parity
 * 1-out_parity.  out_parity = 0 gives D_eo, 1 gives D_oe. */
int orc_dslash_half(const int L[4], const cplx *U, int out_parity,
                    const cplx *in_half, cplx *out_half)
{
    if (orc_check_dims(L) || (out_parity != 0 && out_parity != 1)) return -1;
    long V = orc_volume(L);
    struct half_view hv = {L, in_half, 1 - out_parity};
#pragma omp parallel for schedule(static)
    for (long i = 0; i < V; ++i) {
        int c[4];
        lex_coords(L, i, c);
        if (site_parity(c) != out_parity) continue;
        dslash_site(L, U, c, half_at, &hv, out_half + (i / 2) * 3);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Even-odd normal matrix M = m^2 - D_eo D_oe on even sites.                   */
/* ------------------------------------------------------------------------- */

int orc_apply_M(const int L[4], const cplx *U, double mass, const cplx *in_e, cplx *out_e)
{
    if (orc_check_dims(L)) return -1;
    long n = orc_volume(L) / 2 * 3;
    cplx *t = malloc(sizeof(cplx) * n);
    if (!t) return -3;
    orc_dslash_half(L, U, 1, in_e, t);       /* t = D_oe in   (odd)  */
    orc_dslash_half(L, U, 0, t, out_e);      /* out = D_eo t  (even) */
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k)
        out_e[k] = mass * mass * in_e[k] - out_e[k];
    free(t);
    return 0;
}

/* (M + sigma) in */
static int apply_M_shifted(const int L[4], const cplx *U, double mass, double sigma,
                           const cplx *in, cplx *out)
{
    int rc = orc_apply_M(L, U, mass, in, out);
    if (rc) return rc;
    long n = orc_volume(L) / 2 * 3;
    for (long k = 0; k < n; ++k)
        out[k] += sigma * in[k];
    return 0;
}

static cplx dot(long n, const cplx *a, const cplx *b)
{
    cplx s = 0.0;
    for (long k = 0; k < n; ++k)
        s += conj(a[k]) * b[k];
    return s;
}

static double norm2(long n, const cplx *a)
{
    double s = 0.0;
    for (long k = 0; k < n; ++k)
        s += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
    return s;
}

/* ------------------------------------------------------------------------- */
/* Conjugate gradient on (M + sigma) x = b (Hestenes-Stiefel), x0 = 0.         */
/* Iterates on the recursive residual until ||r|| <= tol ||b||, then           */
/* recomputes the true residual b - (M+sigma) x; if that is still above tol    */
/* the iteration restarts from the current x with r = p = true residual.       */
/* Returns 0 converged, 1 not converged within maxiter, 2 breakdown,           */
/* negative on bad input.                                                      */
/* ------------------------------------------------------------------------- */

static int cg_shifted(const int L[4], const cplx *U, double mass, double sigma,
                      const cplx *b, cplx *x, double tol, int maxiter,
                      int *iters_out, double *relres_out)
{
    if (orc_check_dims(L)) return -1;
    long n = orc_volume(L) / 2 * 3;
    cplx *r = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n),
         *Ap = malloc(sizeof(cplx) * n);
    if (!r || !p || !Ap) { free(r); free(p); free(Ap); return -3; }

    int status = 1, k = 0;
    double bb = norm2(n, b), rr;
    for (long j = 0; j < n; ++j) x[j] = 0.0;
    if (bb == 0.0) {
        if (iters_out) *iters_out = 0;
        if (relres_out) *relres_out = 0.0;
        free(r); free(p); free(Ap);
        return 0;
    }
    for (long j = 0; j < n; ++j) r[j] = p[j] = b[j];
    rr = bb;
    for (;;) {
        while (k < maxiter && rr > tol * tol * bb) {
            apply_M_shifted(L, U, mass, sigma, p, Ap);
            double pAp = creal(dot(n, p, Ap));
            if (!(pAp > 0.0)) { status = 2; goto done; }
            double alpha = rr / pAp;
            for (long j = 0; j < n; ++j) x[j] += alpha * p[j];
            for (long j = 0; j < n; ++j) r[j] -= alpha * Ap[j];
            double rr_new = norm2(n, r);
            double beta = rr_new / rr;
            rr = rr_new;
            for (long j = 0; j < n; ++j) p[j] = r[j] + beta * p[j];
            ++k;
        }
        /* true residual */
        apply_M_shifted(L, U, mass, sigma, x, Ap);
        for (long j = 0; j < n; ++j) r[j] = b[j] - Ap[j];
        rr = norm2(n, r);
        if (rr <= tol * tol * bb) { status = 0; break; }
        if (k >= maxiter) { status = 1; break; }
        for (long j = 0; j < n; ++j) p[j] = r[j];   /* restart */
    }
done:
    if (iters_out) *iters_out = k;
    if (relres_out) *relres_out = sqrt(rr / bb);
    free(r); free(p); free(Ap);
    return status;
}

int orc_cg(const int L[4], const cplx *U, double mass, const cplx *b, cplx *x,
           double tol, int maxiter, int *iters_out, double *relres_out)
{
    return cg_shifted(L, U, mass, 0.0, b, x, tol, maxiter, iters_out, relres_out);
}

/* ------------------------------------------------------------------------- */
/* Multi-shift CG: (M + sigma_i) x_i = b for all i from one Krylov space.      */
/* The base system is the smallest shift s0; every other system rides on it    */
/* with the shifted-CG coefficients zeta (residuals r_i = zeta_i r):           */
/*   zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1} /                                  */
/*        ( a_k b_{k-1} (zeta_{k-1} - zeta_k) + zeta_{k-1} a_{k-1} (1 + d a_k) ) */
/*   a_k^i = a_k zeta_{k+1}/zeta_k,  b_k^i = b_k (zeta_{k+1}/zeta_k)^2,         */
/*   x_i += a_k^i p_i,  p_i = zeta_{k+1} r_{k+1} + b_k^i p_i,                   */
/* with d = sigma_i - s0, zeta_0 = zeta_{-1} = 1, a_{-1} = 1, b_{-1} = 0.        */
/* A shifted system stops updating once zeta_i^2 ||r||^2 <= tol^2 ||b||^2.      */
/* X is (nshift, V/2, 3); relres[i] is the recomputed true relative residual.  */
/* Returns 0 if every system reached tol, 1 otherwise, 2 on breakdown.         */
/* ------------------------------------------------------------------------- */

int orc_multishift_cg(const int L[4], const cplx *U, double mass, int nshift,
                      const double *shifts, const cplx *b, cplx *X, double tol,
                      int maxiter, int *iters_out, double *relres)
{
    if (orc_check_dims(L) || nshift < 1) return -1;
    long n = orc_volume(L) / 2 * 3;
    int base = 0;
    for (int s = 1; s < nshift; ++s)
        if (shifts[s] < shifts[base]) base = s;
    double s0 = shifts[base];

    cplx *r = malloc(sizeof(cplx) * n), *Ap = malloc(sizeof(cplx) * n),
         *P = malloc(sizeof(cplx) * n * nshift);
    double *zeta = malloc(sizeof(double) * nshift), *zeta_prev = malloc(sizeof(double) * nshift),
           *zeta_next = malloc(sizeof(double) * nshift);
    int *active = malloc(sizeof(int) * nshift);
    if (!r || !Ap || !P || !zeta || !zeta_prev || !zeta_next || !active) {
        free(r); free(Ap); free(P); free(zeta); free(zeta_prev); free(zeta_next); free(active);
        return -3;
    }

    double bb = norm2(n, b), rr = bb;
    for (int s = 0; s < nshift; ++s) {
        for (long j = 0; j < n; ++j) {
            X[s * n + j] = 0.0;
            P[s * n + j] = b[j];
        }
        zeta[s] = zeta_prev[s] = 1.0;
        active[s] = (bb > 0.0);
    }
    for (long j = 0; j < n; ++j) r[j] = b[j];
    double alpha_prev = 1.0, beta_prev = 0.0;
    int k = 0, status = 0;
    cplx *pb = P + base * n;

    while (k < maxiter && bb > 0.0 && rr > tol * tol * bb) {
        apply_M_shifted(L, U, mass, s0, pb, Ap);
        double pAp = creal(dot(n, pb, Ap));
        if (!(pAp > 0.0)) { status = 2; break; }
        double alpha = rr / pAp;
        for (int s = 0; s < nshift; ++s) {
            if (!active[s]) continue;
            if (s == base) {
                zeta_next[s] = 1.0;
            } else {
                double d = shifts[s] - s0;
                zeta_next[s] = zeta[s] * zeta_prev[s] * alpha_prev /
                    (alpha * beta_prev * (zeta_prev[s] - zeta[s]) +
                     zeta_prev[s] * alpha_prev * (1.0 + d * alpha));
            }
            double alpha_s = alpha * zeta_next[s] / zeta[s];
            for (long j = 0; j < n; ++j) X[s * n + j] += alpha_s * P[s * n + j];
        }
        for (long j = 0; j < n; ++j) r[j] -= alpha * Ap[j];
        double rr_new = norm2(n, r);
        double beta = rr_new / rr;
        for (int s = 0; s < nshift; ++s) {
            if (!active[s]) continue;
            double ratio = zeta_next[s] / zeta[s];
            double beta_s = beta * ratio * ratio;
            for (long j = 0; j < n; ++j)
                P[s * n + j] = zeta_next[s] * r[j] + beta_s * P[s * n + j];
            zeta_prev[s] = zeta[s];
            zeta[s] = zeta_next[s];
            if (s != base && zeta[s] * zeta[s] * rr_new <= tol * tol * bb) active[s] = 0;
        }
        alpha_prev = alpha;
        beta_prev = beta;
        rr = rr_new;
        ++k;
    }
    if (status == 0 && rr > tol * tol * bb) status = 1;
    for (int s = 0; s < nshift; ++s) {
        if (bb == 0.0) { relres[s] = 0.0; continue; }
        apply_M_shifted(L, U, mass, shifts[s], X + s * n, Ap);
        for (long j = 0; j < n; ++j) r[j] = b[j] - Ap[j];
        relres[s] = sqrt(norm2(n, r) / bb);
    }
    if (iters_out) *iters_out = k;
    free(r); free(Ap); free(P); free(zeta); free(zeta_prev); free(zeta_next); free(active);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Pseudo-fermion action and force.                                            */
/* S = phi^dagger M^{-1} phi = Re <phi, X>,  X = M^{-1} phi (even sites).      */
/* With Y = D_oe X, varying a link changes S by                                */
/*   dS = X^dagger dD_eo Y - Y^dagger dD_oe X                                  */
/* (using D_eo^dagger = -D_oe).  For the link U_{x,mu}, eta including the      */
/* boundary sign of the hop x -> x+mu:                                         */
/*   x even: dS = 2 eta Re tr(dU Y_{x+mu} X_x^dagger),  G =  2 eta X_x Y_{x+mu}^dagger */
/*   x odd : dS = -2 eta Re tr(dU X_{x+mu} Y_x^dagger), G = -2 eta Y_x X_{x+mu}^dagger */
/* G is the Euclidean gradient, dS = Re sum_ab conj(G_ab) dU_ab (the PyTorch   */
/* convention dS/dRe U + i dS/dIm U).  Under U -> exp(i eps T) U,              */
/* dS/deps = Re tr(i T W) = tr(i T P) with W = U G^dagger and                  */
/* P = TA(W) = (W - W^dagger)/2 - tr(W - W^dagger)/6 * 1.                      */
/* P and G are (V, 4, 3, 3) like U; either may be NULL.                        */
/* ------------------------------------------------------------------------- */

double orc_action(const int L[4], const cplx *phi_e, const cplx *X_e)
{
    long n = orc_volume(L) / 2 * 3;
    return creal(dot(n, phi_e, X_e));
}

int orc_force(const int L[4], const cplx *U, const cplx *X_e, cplx *P, cplx *G)
{
    if (orc_check_dims(L)) return -1;
    long V = orc_volume(L);
    long n = V / 2 * 3;
    cplx *Y = malloc(sizeof(cplx) * n);
    if (!Y) return -3;
    orc_dslash_half(L, U, 1, X_e, Y);        /* Y = D_oe X on odd sites */

    for (long i = 0; i < V; ++i) {
        int c[4];
        lex_coords(L, i, c);
        int par = site_parity(c);
        for (int mu = 0; mu < 4; ++mu) {
            int cf[4];
            int bc = shifted(L, c, mu, +1, cf);
            long j = lex_index(L, cf);
            double eta = (double)(orc_eta(L, c, mu) * bc);
            cplx g[9];
            if (par == 0) {
                const cplx *Xx = X_e + (i / 2) * 3, *Yf = Y + (j / 2) * 3;
                for (int a = 0; a < 3; ++a)
                    for (int bb = 0; bb < 3; ++bb)
                        g[a * 3 + bb] = 2.0 * eta * Xx[a] * conj(Yf[bb]);
            } else {
                const cplx *Yx = Y + (i / 2) * 3, *Xf = X_e + (j / 2) * 3;
                for (int a = 0; a < 3; ++a)
                    for (int bb = 0; bb < 3; ++bb)
                        g[a * 3 + bb] = -2.0 * eta * Yx[a] * conj(Xf[bb]);
            }
            if (G)
                for (int e = 0; e < 9; ++e) G[(i * 4 + mu) * 9 + e] = g[e];
            if (P) {
                const cplx *u = link(U, i, mu);
                cplx w[9];
                /* W = U G^dagger */
                for (int a = 0; a < 3; ++a)
                    for (int bb = 0; bb < 3; ++bb) {
                        cplx s = 0.0;
                        for (int e = 0; e < 3; ++e)
                            s += u[a * 3 + e] * conj(g[bb * 3 + e]);
                        w[a * 3 + bb] = s;
                    }
                cplx tr = 0.0;
                for (int a = 0; a < 3; ++a)
                    tr += w[a * 3 + a] - conj(w[a * 3 + a]);
                cplx *out = P + (i * 4 + mu) * 9;
                for (int a = 0; a < 3; ++a)
                    for (int bb = 0; bb < 3; ++bb) {
                        out[a * 3 + bb] = 0.5 * (w[a * 3 + bb] - conj(w[bb * 3 + a]));
                        if (a == bb) out[a * 3 + bb] -= tr / 6.0;
                    }
            }
        }
    }
    free(Y);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* 12-real link compression (Sec. 4.3): only rows 0 and 1 are kept; for an     */
/* SU(3) matrix row 2 is the complex conjugate of the cross product of rows 0  */
/* and 1.  n matrices (n,3,3) in, their rebuilt third rows (n,3) out.          */
/* ------------------------------------------------------------------------- */

void orc_reconstruct_row2(long n, const cplx *U, cplx *row2)
{
    for (long k = 0; k < n; ++k) {
        const cplx *a = U + k * 9, *b = U + k * 9 + 3;
        row2[k * 3 + 0] = conj(a[1] * b[2] - a[2] * b[1]);
        row2[k * 3 + 1] = conj(a[2] * b[0] - a[0] * b[2]);
        row2[k * 3 + 2] = conj(a[0] * b[1] - a[1] * b[0]);
    }
}
