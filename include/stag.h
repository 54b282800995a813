/*
 * stag.h -- C ABI of libstag, a staggered Dirac operator and even-odd CG
 * library for one NVIDIA GB300 GPU (sm_103a).
 *
 * Operator (Sec. 4.2, Eq. (staggered) of "Portable Lattice QCD implementation
 * based on OpenCL"):
 *
 *   (D phi)_x = sum_{mu=0..3} [ eta_mu(x) U_{x,mu} phi_{x+mu}
 *                              - eta_mu(x-mu) U^dagger_{x-mu,mu} phi_{x-mu} ]
 *
 * with eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z),
 * periodic boundaries in x, y, z and antiperiodic in t (a hop that crosses the
 * time boundary takes a factor -1).  No factor 1/2, no mass term.  The solvers
 * work on the even-odd normal matrix M = m^2 - D_eo D_oe acting on even sites,
 * which is Hermitian positive definite because D_eo^dagger = -D_oe.
 *
 * Canonical layouts (all complex numbers interleaved re, im as doubles):
 *   site index   i = x + Lx*(y + Ly*(z + Lz*t));  mu = 0,1,2,3 = x,y,z,t
 *   gauge field  U[V][4][3][3] complex, U[i][mu][a][b] = (U_{x,mu})_{ab}
 *   half field   psi[V/2][3] complex over the sites of one parity
 *                ((x+y+z+t) mod 2), indexed h = i/2 (Lx even)
 *   multi field  psi[n][V/2][3] complex, n half fields back to back
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" are CUDA device pointers (for instance a torch
 *     tensor's data_ptr()); the caller owns them and they are only borrowed for
 *     the call.  Buffers must be 16-byte aligned and must not overlap unless a
 *     function says so.
 *   - The library owns everything it allocates inside a context (compressed
 *     links, work vectors, CUDA graphs); stag_destroy frees it.
 *   - Work is enqueued on the context's stream and is asynchronous with respect
 *     to the host, except where a function says it blocks.
 *   - A context is not thread safe: one host thread at a time.
 *   - Return value: 0 = success; negative = error, nothing was written to the
 *     outputs; positive = numerical outcome (outputs and stats are written).
 *     stag_strerror() names a code; stag_last_error() gives the message of the
 *     last failure on the calling thread.
 */
#ifndef STAG_H
#define STAG_H

#ifdef __cplusplus
extern "C" {
#endif

#define STAG_ABI_VERSION 3
#define STAG_MAX_RHS 64   /* largest batch of right-hand sides or shifts */

typedef struct stag_ctx_s *stag_ctx;

enum stag_status {
    STAG_OK = 0,
    STAG_NOT_CONVERGED = 1, /* solver reached maxiter; stats hold the residual reached */
    STAG_BREAKDOWN = 2,     /* <p, Mp> <= 0 or not finite: operator not HPD or data not finite */
    STAG_EINVAL = -1,       /* bad argument: NULL or misaligned pointer, bad enum, bad size */
    STAG_EGEOM = -2,        /* lattice extents not even or < 2, or volume too large */
    STAG_ENOMEM = -3,       /* a device or host allocation failed */
    STAG_ECUDA = -4,        /* a CUDA call failed (see stag_last_error) */
    STAG_ENOGAUGE = -5,     /* no gauge field uploaded to this context yet */
    STAG_EUNSUPPORTED = -6  /* combination of precision / compression not provided */
};

/* Storage precision of an operator application. */
enum stag_prec {
    STAG_F64 = 0, /* double links and spinors, double arithmetic */
    STAG_F32 = 1, /* float links and spinors, float arithmetic */
    STAG_F16 = 2, /* half links, half spinors with a float norm per site, float arithmetic */
    STAG_F64X = 3 /* double links and spinors (same bytes as STAG_F64), double-float arithmetic:
                     each double carried as hi + lo floats (48-bit significand) on the FP32 pipe,
                     whose rate on GB300 is 64x the FP64 one; 18-real links only.  Results agree
                     with STAG_F64 to ~1e-14 relative (2-norm) for fields of any double
                     magnitude: inputs are normalised by exact powers of two on the device
                     (largest component in [1, 2)) and results scaled back, and links whose
                     largest element lies outside 2^-40 .. 2^40 are stored scaled the same way. */
};

/* Link compression (Sec. 4.3): 18 reals per link, or 12 (rows 0 and 1; row 2
 * rebuilt as the complex conjugate of row0 x row1, exact for SU(3) links). */
enum stag_recon { STAG_RECON_18 = 18, STAG_RECON_12 = 12 };

/* ---------------------------------------------------------------- context */

/* Create a context for an Lx x Ly x Lz x Lt lattice on the current CUDA
 * device.  dims: host array {Lx, Ly, Lz, Lt}, each even and >= 2, volume
 * < 2^31.  stream: a cudaStream_t (NULL = the legacy default stream) on which
 * every later call of this context is enqueued.  On success *out holds the new
 * context.  Errors: STAG_EINVAL (out or dims NULL), STAG_EGEOM, STAG_ENOMEM,
 * STAG_ECUDA. */
int stag_create(stag_ctx *out, const int dims[4], void *stream);

/* Free every device and host resource of the context (after synchronising its
 * stream).  NULL is accepted and ignored. */
int stag_destroy(stag_ctx ctx);

/* Change the stream later calls are enqueued on. */
int stag_set_stream(stag_ctx ctx, void *stream);

/* Lattice extents and volume of a context (host outputs, any may be NULL). */
int stag_get_dims(stag_ctx ctx, int dims[4], long long *volume);

/* Upload the gauge field U (canonical [V][4][3][3] complex128) into the
 * context's internal layout.  on_device = 1: U is a device pointer; 0: a host
 * pointer (copied through a device staging buffer).  The field is copied, so U
 * may be freed or changed after the call returns (on_device = 0) or after the
 * stream reaches this point (on_device = 1).  Compressed and reduced-precision
 * copies are derived from it on first use.  Links may be any complex 3x3
 * matrices for the 18-real forms; the 12-real forms assume SU(3). */
int stag_upload_gauge(stag_ctx ctx, const double *U, int on_device);

/* ------------------------------------------------------- operator (Eq. staggered) */

/* Link field of the operator entry points (Sec. 4.3, temporal gauge).  The
 * paper reads 6 links per site by fixing the temporal gauge: with the gauge
 * matrices g(x, t = 0) = 1, g(x, t + 1) = g(x, t) U_t(x, t), the transformed
 * links U' = g U g^dagger (U'_mu(x) = g(x) U_mu(x) g(x + mu)^dagger) have
 * U'_t = 1 except on the last time slice.  The library computes g and U' in
 * double from the uploaded field on first use (unitary links: SU(3) or U(3)).
 *   STAG_LINKS_UPLOADED       (default) the operator entry points apply D[U];
 *   STAG_LINKS_TEMPORAL       they apply D[U'] reading 6 links per site: a time
 *                             hop off the last slice adds the neighbour spinor
 *                             with no link load or product;
 *   STAG_LINKS_TEMPORAL_FULL  they apply D[U'] reading all 8 links (the identity
 *                             links as stored): the same values, for checks.
 * Affects stag_dslash_eo/oe, stag_dslash_multi and stag_dslash_repeat(_multi);
 * solvers, stag_apply_M and the force always act on D[U] (the solvers'
 * temporal_gauge parameter uses U' internally).  Errors: STAG_EINVAL; the
 * operator calls on U' return STAG_EUNSUPPORTED when the uploaded links are
 * not unitary (max |U U^dagger - 1| above 1e-12, checked once per upload). */
enum stag_links { STAG_LINKS_UPLOADED = 0, STAG_LINKS_TEMPORAL = 1, STAG_LINKS_TEMPORAL_FULL = 2 };
int stag_set_operator_links(stag_ctx ctx, int links);

/* out_even = D_eo in_odd: the operator restricted to even output sites acting
 * on a field living on odd sites (both canonical half fields, device).
 * prec/recon select the storage the kernel streams (input and output stay
 * complex128 at the boundary; for STAG_F32/STAG_F16 the input is rounded to
 * that storage first).  Asynchronous.  Errors: STAG_EINVAL, STAG_ENOGAUGE,
 * STAG_EUNSUPPORTED, STAG_ECUDA. */
int stag_dslash_eo(stag_ctx ctx, double *out_even, const double *in_odd, int prec, int recon);

/* out_odd = D_oe in_even, as stag_dslash_eo with the parities exchanged. */
int stag_dslash_oe(stag_ctx ctx, double *out_odd, const double *in_even, int prec, int recon);

/* Measurement support: stag_dslash_prepare converts one canonical half field
 * (device) into the internal storage of prec (once): complex128 for STAG_F64,
 * double-float pairs for STAG_F64X (the storage of the double-float solver's
 * vectors), the float / half codes for STAG_F32 / STAG_F16.
 * stag_dslash_repeat then applies D_eo (Sec. 4.2, Eq. (staggered)) to it nrep
 * times into a context-owned output with no conversions, so that a caller's
 * CUDA events on the context's stream around it time the bare operator
 * kernel.  For half 12-real storage the first repeat per link field (as
 * uploaded, temporal gauge) lets the autotuner time the kernel's
 * shared-memory staging variants (same results bit for bit) unless its cache
 * has the decision, so that call is not capturable in a CUDA graph.
 * stag_dslash_result converts that output back into the canonical
 * device half field out (complex128 [V/2][3]).  Asynchronous.  Errors:
 * STAG_EINVAL (repeat before prepare, other precision, result before repeat,
 * bad pointer), STAG_ENOGAUGE, STAG_EUNSUPPORTED. */
int stag_dslash_prepare(stag_ctx ctx, const double *in, int prec);
int stag_dslash_repeat(stag_ctx ctx, int prec, int recon, int nrep);
int stag_dslash_result(stag_ctx ctx, double *out);

/* The same for nrhs fields (device multi field [nrhs][V/2][3] complex128,
 * nrhs in [1, STAG_MAX_RHS]): stag_dslash_repeat_multi applies the
 * multi-vector operator of stag_dslash_multi (Sec. 4.3, NMULTI: each link
 * loaded once per site for rhs_block vectors; 0 = autotuned) nrep times;
 * stag_dslash_result then writes nrhs fields.  For measurement, rhs_block
 * may also name one configuration of the multi-vector kernels,
 * (G << 8) | NBT: G warp groups of a block sharing one shared-memory tile of
 * links, NBT right-hand sides per thread (G = 1: no tile; the codes offered
 * for the storage, else STAG_EINVAL).  Any other operator call of the
 * context that converts fields (F32 / F16 dslash, dslash_multi) discards the
 * prepared fields (STAG_EINVAL on the next repeat or result).  Errors as above. */
int stag_dslash_prepare_multi(stag_ctx ctx, const double *in, int nrhs, int prec);
int stag_dslash_repeat_multi(stag_ctx ctx, int prec, int recon, int rhs_block, int nrep);

/* Measurement support: times nrep back-to-back launches of the fused CG
 * vector update (x += alpha p, r -= alpha Ap, |r|^2 with its grid reduction;
 * the CG step the paper's Table 1 measures) of the double-precision solver
 * (f64_arith STAG_F64: double vectors and FP64 arithmetic; STAG_F64X:
 * double-float vectors) on the context's work vectors, which it first sets to
 * zero, with CUDA events on the context's stream.  Algorithmic traffic: 4
 * vectors read and 2 written, 288 bytes per even site.  Blocks; writes the
 * mean milliseconds per launch to *ms_per_launch (host).  Errors: STAG_EINVAL,
 * STAG_ENOMEM, STAG_ECUDA. */
int stag_cg_update_time(stag_ctx ctx, int f64_arith, int nrep, double *ms_per_launch);

/* Measurement support for the ALU rooflines (Sec. 4.3 compares the operator
 * with the peak of the arithmetic that binds it): the sustained FMA rate of
 * the FP64 (prec STAG_F64) or FP32 (STAG_F32) pipe of the current device, in
 * TFLOP/s (2 flop per FMA), from one launch of independent FMA chains on every
 * SM (iters FMA steps per chain; ~2048 for FP64 and ~32768 for FP32 run a few
 * milliseconds), timed with CUDA events on the legacy default stream.  Blocks;
 * writes *tflops (host).  Errors: STAG_EINVAL, STAG_ECUDA. */
int stag_fma_probe(int prec, int iters, double *tflops);

/* Multi-vector operator (Sec. 4.3, NMULTI): out_k = D_{p,1-p} in_k for
 * k = 0..nrhs-1, with each link loaded once per site for a block of
 * rhs_block vectors (1, 2, 4, 8 or 16; 0 = autotuned, cached per context).
 * in/out: device multi fields [nrhs][V/2][3] complex128; out_parity 0 gives
 * D_eo (in on odd sites), 1 gives D_oe.  prec/recon as stag_dslash_eo.
 * nrhs in [1, STAG_MAX_RHS].  Asynchronous (the first autotuned call times
 * the candidates and waits for them). */
int stag_dslash_multi(stag_ctx ctx, double *out, const double *in, int nrhs, int out_parity, int prec, int recon,
                      int rhs_block);

/* out_even = M in_even = m^2 in_even - D_eo (D_oe in_even), complex128 double
 * precision, 18-real links.  Uses a context-owned odd temporary. */
int stag_apply_M(stag_ctx ctx, double *out_even, const double *in_even, double mass);

/* Allocation-free variant of stag_apply_M, for callers that cannot allocate
 * device memory: hosts that own every device byte through their own pre-sized
 * arena or caching allocator and forbid libraries to call cudaMalloc behind
 * it, and latency-critical loops that cannot absorb the device-wide
 * synchronisation cudaFree implies (and the latency of cudaMalloc).  It
 * needs no context: the gauge field is read straight from the caller's
 * canonical buffer, and the odd-site intermediate D_oe in lives in a static
 * device array of STAG_NOALLOC_MAX_VH x 3 complex doubles (6 MiB) that every
 * GPU loading the library holds until the process exits.  (The paper has no
 * counterpart; this is an interface for such callers.)
 *   dims: host {Lx, Ly, Lz, Lt}, each even and >= 2, with V/2 <=
 *         STAG_NOALLOC_MAX_VH (larger lattices: STAG_EINVAL with a message);
 *   U: device canonical gauge field [V][4][3][3] complex128;
 *   out_even, in_even: device canonical half fields; must not alias;
 *   stream: cudaStream_t the two kernels are enqueued on (asynchronous).
 * Result: out_even = m^2 in_even - D_eo D_oe in_even, the same arithmetic as
 * stag_apply_M.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture begins.  The address is cached for the life
 * of the device's primary context: resetting the device (cudaDeviceReset)
 * between calls is not supported.  U, out_even and in_even must be memory of
 * the current device (STAG_EINVAL otherwise).  All calls share the one array:
 * calls that overlap on the GPU (other streams, other host threads) race on
 * it and must be serialised by the caller.  Nothing in it needs clearing
 * between calls (every element is written before it is read). */
#define STAG_NOALLOC_MAX_VH (1 << 17)
int stag_apply_M_noalloc(const int dims[4], const double *U, double *out_even, const double *in_even, double mass,
                         void *stream);

/* ---------------------------------------------------------------- solvers */

typedef struct {
    double tol;            /* stop when ||b - M x|| <= tol ||b||, recomputed in double */
    int maxiter;           /* total iteration limit (all restarts together); <= 0: 100000 */
    int use_graph;         /* 1: iterate inside one CUDA graph with a device-side loop;
                              0: host-driven loop (one stream sync per check_every iterations) */
    int check_every;       /* host-driven loop only: iterations between convergence reads */
    double delta;          /* mixed precision: reliable update when ||r|| < delta * max ||r||; <= 0: 0.01 */
    int inner_prec;        /* mixed precision: STAG_F32 or STAG_F16 */
    int inner_recon;       /* mixed precision: STAG_RECON_18 or STAG_RECON_12 */
    int rhs_block;         /* batched solves: right-hand sides per operator pass; 0: autotune */
    int f64_arith;         /* arithmetic of the double-precision operator passes (stag_cg_solve,
                              the reliable updates of the mixed solver): STAG_F64 (IEEE double)
                              or STAG_F64X (double-float; taken as STAG_F64 when the links lie
                              outside the double-float range, see STAG_F64X).  Every solver
                              solves for 2^-k b (largest component in [1, 2)) and returns
                              2^k x, exactly, so any double-range b is served alike */
    int temporal_gauge;    /* 1: solve in temporal gauge (Sec. 4.3, see stag_set_operator_links):
                              M' x' = g b on the links U' = g U g^dagger, reading 6 links per
                              site in every operator pass (inner iterations, reliable updates,
                              multi-vector passes), and return x = g^dagger x'.  M' = g M
                              g^dagger: the same spectrum and iteration; g is unitary, so the
                              same residual norm.  Needs unitary links (SU(3) or U(3)).  All
                              solvers: stag_cg_solve (either f64_arith), _mixed, _multi,
                              _multishift, and the action; STAG_EUNSUPPORTED when the links are
                              not unitary (max |U U^dagger - 1| above 1e-12).  0 (default): the
                              links as uploaded. */
} stag_solver_params;

typedef struct {
    int status;               /* same code the call returned */
    int iters;                /* operator applications of the (inner) iteration */
    int restarts;             /* times the iteration restarted from the true residual */
    int reliable_updates;     /* mixed precision: double-precision residual recomputations */
    double true_rel_residual; /* ||b - M x|| / ||b|| recomputed in double at the end */
    double iter_rel_residual; /* the iterated (recursive) residual at the end */
    double seconds;           /* host wall time of the call, including the final sync */
} stag_solver_stats;

/* Fill *p with defaults: tol 1e-10, maxiter 100000, use_graph 1, check_every 25,
 * delta 0.01, inner_prec STAG_F32, inner_recon STAG_RECON_12, rhs_block 0,
 * f64_arith STAG_F64X (double-float operator passes: on GB300 about twice as
 * fast as IEEE double ones, which are FP64-ALU-bound, with results equal to
 * ~1e-14 relative). */
void stag_solver_params_default(stag_solver_params *p);

/* Solve M x = b by conjugate gradient in double precision (Sec. 1 and
 * Sec. 4.2: inversion of the staggered operator by CG, here on the even-odd
 * normal matrix).  x_even, b_even: device canonical half fields.  x starts at
 * zero.  The iterated residual drives the loop; at the end the true residual
 * is recomputed in double and the iteration restarts from it while it is above
 * tol and iterations remain.  Blocks until the solution and *stats (may be
 * NULL) are final.  Returns STAG_OK, STAG_NOT_CONVERGED, STAG_BREAKDOWN or a
 * negative error. */
int stag_cg_solve(stag_ctx ctx, double *x_even, const double *b_even, double mass,
                  const stag_solver_params *params, stag_solver_stats *stats);

/* As stag_cg_solve for the shifted system (M + sigma) x = b, sigma >= 0. */
int stag_cg_solve_shifted(stag_ctx ctx, double *x_even, const double *b_even, double mass, double sigma,
                          const stag_solver_params *params, stag_solver_stats *stats);

/* Mixed-precision CG with reliable updates on M x = b.  The inner iteration
 * stores links and vectors in params->inner_prec (STAG_F32, or STAG_F16 with a
 * float norm per site) with params->inner_recon links, in float arithmetic; the
 * solution is accumulated in double precision and the residual recomputed in
 * double precision (18-real double links) whenever the inner residual has
 * dropped by params->delta below its maximum since the previous recomputation,
 * and when the inner iteration reaches tol.  Converged means the double
 * precision true residual is <= tol.  Arguments, blocking and return codes as
 * stag_cg_solve; stats->reliable_updates counts the recomputations.  (The paper
 * cites mixed-precision GPU solvers in its bibliography but has no such
 * solver itself.) */
int stag_cg_solve_mixed(stag_ctx ctx, double *x_even, const double *b_even, double mass,
                        const stag_solver_params *params, stag_solver_stats *stats);

/* Batched CG: solve M X_k = B_k for nrhs right-hand sides in one CUDA graph
 * launch, every operator pass applying each loaded link to params->rhs_block
 * systems (0 = autotuned).  X, B: device multi fields [nrhs][V/2][3]
 * complex128, nrhs in [1, STAG_MAX_RHS].  params->inner_prec selects the
 * iteration's storage: STAG_F64 (plain double-precision CG), or STAG_F32 /
 * STAG_F16 with params->inner_recon links and double-precision reliable
 * updates as in stag_cg_solve_mixed, per system.  Converged systems drop out
 * of the passes.  stats: NULL or an array of nrhs records.  Blocks until done;
 * returns the worst status over the systems (STAG_OK, STAG_NOT_CONVERGED,
 * STAG_BREAKDOWN) or a negative error.  (The paper applies the operator to
 * several vectors at once, Sec. 4.3; the batched solver around it is not in
 * the paper.) */
int stag_cg_solve_multi(stag_ctx ctx, double *X, const double *B, int nrhs, double mass,
                        const stag_solver_params *params, stag_solver_stats *stats);

/* Multi-shift CG: solve (M + shifts[i]) X_i = b for i = 0..nshift-1 from one
 * Krylov space (one operator application per iteration serves every shift),
 * then bring each X_i to a double-precision true residual <= tol with a
 * batched reliable-update solve seeded by X_i.  shifts: host array of nshift
 * values >= 0 (added to M, any order; the smallest drives the iteration),
 * nshift in [1, STAG_MAX_RHS].  b: device half field [V/2][3]; X: device multi
 * field [nshift][V/2][3].  params->inner_prec STAG_F32 (default) or STAG_F64
 * selects the Krylov phase's storage, params->inner_recon its links; the
 * refinement uses params->inner_prec / inner_recon with reliable updates.
 * stats: NULL or nshift records (iters counts both phases, restarts holds the
 * shared Krylov iterations).  Blocks until done.  (Not in the paper; it is
 * the solver a rational hybrid Monte Carlo force needs.) */
int stag_cg_solve_multishift(stag_ctx ctx, double *X, const double *b, const double *shifts, int nshift,
                             double mass, const stag_solver_params *params, stag_solver_stats *stats);

/* Full-lattice solve of (m + D) psi = b (D of Eq. (staggered), Sec. 4.2)
 * through the even-odd Schur complement: M psi_e = m b_e - D_eo b_o, then
 * psi_o = (b_o - D_oe psi_e) / m.  psi, b: device canonical full fields
 * [V][3] complex128 (lexicographic sites, both parities); mass > 0.  The even
 * solve uses params->inner_prec (STAG_F64: stag_cg_solve, else the mixed
 * solver) and params->tol on M; the full residual is then at most
 * tol (1 + 8/m) relative (|D_eo| <= 8 for unitary links).  stats describe
 * the even solve.  Blocks until done. */
int stag_solve_full(stag_ctx ctx, double *psi, const double *b, double mass, const stag_solver_params *params,
                    stag_solver_stats *stats);

/* ----------------------------------------------------------- HMC force */

/* Pseudo-fermion action S = phi^dagger M^{-1} phi = Re <phi, X>: solves
 * M X = phi (params->inner_prec STAG_F64: stag_cg_solve; STAG_F32/F16:
 * stag_cg_solve_mixed) into X_even and writes S to *S (host).  phi_even,
 * X_even: device canonical half fields (must not alias).  Blocks; returns the
 * solver's status.  (The paper runs CG inside HMC, Sec. 1; the action and its
 * force are the HMC side of that, not in the paper.) */
int stag_fermion_action(stag_ctx ctx, const double *phi_even, double mass, const stag_solver_params *params,
                        double *X_even, double *S, stag_solver_stats *stats);

/* Derivative of S with respect to the links, given X = M^{-1} phi (device
 * canonical half field).  With Y = D_oe X and eta = eta_mu(x) times the
 * boundary sign of the hop x -> x+mu, the Euclidean gradient of link U_{x,mu}
 * is G = 2 eta X_x Y_{x+mu}^dagger (x even) or -2 eta Y_x X_{x+mu}^dagger (x
 * odd), so that dS = Re sum conj(G_ab) dU_ab (the PyTorch convention
 * dS/dRe U + i dS/dIm U); the projected force is P = TA(U G^dagger)
 * = (W - W^dagger)/2 - tr(W - W^dagger)/6 with W = U G^dagger, so that
 * dS/deps = tr(i T P) under U -> exp(i eps T) U.  Outputs (device, canonical
 * [V][4][3][3] complex128, each may be NULL but not all): P, G, and
 * phi_grad = dS/dRe phi + i dS/dIm phi = 2 X ([V/2][3]); all multiplied by
 * scale.  Double-precision arithmetic, 18-real links.  Asynchronous. */
int stag_fermion_force(stag_ctx ctx, double *P, double *G, const double *X_even, double *phi_grad, double scale);

/* Sum of forces sum_i coeffs[i] F(X_i) for n solutions X (device multi field
 * [n][V/2][3]), coeffs a host array of n reals: the force of a rational
 * approximation S = sum_i r_i phi^dagger (M + sigma_i)^{-1} phi with X_i the
 * multi-shift solutions (the shift changes M's diagonal only, so each term
 * has the single-solution form of stag_fermion_force).  P, G as in
 * stag_fermion_force (overwritten).  n in [1, STAG_MAX_RHS].  Asynchronous. */
int stag_fermion_force_multi(stag_ctx ctx, double *P, double *G, const double *X, const double *coeffs, int n);

/* Right-hand sides per operator pass used by the last batched solve or
 * stag_dslash_repeat_multi of this context (the autotuner's choice when
 * rhs_block was 0). */
int stag_last_rhs_block(stag_ctx ctx);

/* ------------------------------------------------------------- autotuner
 *
 * Launch shapes the library chooses by timing (the multi-vector operator's
 * right-hand-side block and tile split of Sec. 4.3's NMULTI, the block sizes
 * and sites per thread of the solvers' operator and vector kernels).  Each
 * decision is keyed by "kernel|LxxLyxLzxLt|p<prec>|r<recon>|n<nrhs>|<gpu>"
 * and timed once: candidates run with CUDA events on the context's stream, L2
 * flushed before every timed launch, the median of three.  Decisions are kept
 * in a process-wide cache backed by a JSON file: environment STAG_TUNE_CACHE
 * (path; empty = no file; default $XDG_CACHE_HOME/stag/tune.json or
 * $HOME/.cache/stag/tune.json) and STAG_TUNE (0 = never time, use defaults;
 * 1 or unset = time what the cache lacks; force = time again what came from
 * the file).  Every candidate of a decision gives the same results bit for
 * bit; only the time differs.  These functions touch no GPU. */

/* Compose a key into out (len bytes); returns its length or STAG_EINVAL. */
int stag_tune_make_key(const char *kernel, const int dims[4], int prec, int recon, int nrhs, const char *gpu,
                       char *out, int len);
/* Replace the in-memory cache by the entries of a cache file (path NULL: the
 * default file); returns the number of entries or STAG_EINVAL. */
int stag_tune_cache_load(const char *path);
/* Write the in-memory cache to a file (path NULL: the default file). */
int stag_tune_cache_save(const char *path);
/* 1 and *choice set if key is cached, else 0. */
int stag_tune_cache_lookup(const char *key, int *choice);
/* Put a decision into the in-memory cache. */
int stag_tune_cache_insert(const char *key, int choice);
/* Empty the in-memory cache (the default file is not read again) and zero
 * the counters. */
void stag_tune_cache_clear(void);
/* Decisions made by timing, and decisions served from the cache, so far. */
int stag_tune_stats(long long *timed, long long *from_cache);

/* ------------------------------------------------------------- utilities */

const char *stag_strerror(int code);
const char *stag_last_error(void);
int stag_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* STAG_H */
