// ctx.h -- host-side internals of libstag: the context object, error
// reporting helpers and the launchers each translation unit exports to the
// others.  Not part of the public ABI (include/stag.h is).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "common.cuh"
#include "stag.h"

namespace stag {

void set_error(const char* fmt, ...);

#define STAG_CUDA_TRY(call)                                                        \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ::stag::set_error("%s failed at %s:%d: %s", #call, __FILE__, __LINE__, \
                              cudaGetErrorString(e_));                             \
            return STAG_ECUDA;                                                     \
        }                                                                          \
    } while (0)

#define STAG_TRY(call)              \
    do {                            \
        int rc_ = (call);           \
        if (rc_ < 0) return rc_;    \
    } while (0)

// Exponent slots of the field normalisation (scale.cu): the solve's own
// right-hand sides, an outer solver's (multi-shift) right-hand side, the
// operator entry points' inputs, and the gauge field.
constexpr int SCALE_SLOTS = 200;
constexpr int SLOT_SOLVE = 0, SLOT_OUTER = 64, SLOT_OPER = 128, SLOT_FORCE = 192, SLOT_LINKS = SCALE_SLOTS - 1;
constexpr int DF_LINK_SAFE_EXP = 40;
// Reliable-update threshold of the mixed, batched and multi-shift solvers
// (||r|| < delta max ||r|| since the last update): 0.01 keeps the float and
// half recurrences accurate (at most one extra iteration at 48^3 x 12,
// m = 0.002) with half the double-precision passes of 0.1 (half inner
// 12.7 -> 11.1 ms, float 15.3 -> 13.6 ms, 16 RHS at 32^3 x 16 73.8 -> 66.0 ms);
// 0.003 added iterations to the half solve.
constexpr double DEFAULT_RELIABLE_DELTA = 0.01;
constexpr int FLOAT_INNER_LINK_EXP = 20;

// Index of a (precision, compression) link copy.
inline int link_slot(int prec, int recon) { return prec * 2 + (recon == 12 ? 1 : 0); }   // 0..7

// Scalars of one CG-type iteration, resident in device memory so the loop
// runs without host round trips.  One record per right-hand side.
struct CgScalars {
    double rr;        // current iterated |r|^2
    double rr0;       // |b|^2
    double pAp;
    double alpha;
    double beta;
    double tol2;      // tol^2 * |b|^2 threshold on |r|^2
    double rr_true;   // last recomputed |b - M x|^2
    double rmax2;     // mixed precision: max |r|^2 since the last reliable update
    double delta2;    // mixed precision: delta^2
    double m2;        // mass^2 of M = m^2 - D_eo D_oe
    double sigma;     // shift added to M (multi-shift base system)
    double rr_prev;   // mixed precision: |r|^2 before the last step (beta after a reliable update)
    int iter;         // M applications so far
    int maxiter;
    int status;       // 0 running/converged, STAG_NOT_CONVERGED, STAG_BREAKDOWN
    int done;         // 1 once the loop must stop
    int reliable;     // mixed precision: a reliable update is due
    int n_reliable;
    int pad[2];
};

struct Workspace;   // solver vectors and graphs (cg.cu)

}  // namespace stag

struct stag_ctx_s {
    stag::Geom g;
    long long V;
    int device;
    int sm_count;
    cudaStream_t stream;
    cudaStream_t cap_stream;   // private stream used only to capture graphs
    bool have_gauge;
    void* links[8];            // link copies, index link_slot(prec, recon)
    size_t link_bytes[8];
    bool link_stale[8];        // derived copy older than the last upload (re-derived in place)
    double2* tg_g;             // temporal gauge: g per site [par][V/2][9] (tgauge.cu)
    void* tg_links[8];         // temporal gauge: the transformed links U' in every storage,
                               // index link_slot(prec, recon); slot 0 (F64/18) is the source
    size_t tg_link_bytes[8];
    bool tg_link_stale[8];
    double2* tg_tmp;           // temporal gauge: g b for a solve (nrhs_cap fields)
    int tg_tmp_fields;
    bool tg_stale;             // tg_g older than the last upload
    unsigned long long* tg_defect;   // max |U U^dagger - 1| of the uploaded links (bits of a double)
    // reduction scratch: partial sums (one double per block) and arrival counters
    double* partials;
    unsigned int* counters;    // 64 counters, each used by one reduction site
    int max_blocks;
    // two-level grid sums (common.cuh GridSum): group partials and group
    // arrival counters (zero between uses), max_blocks / 32 + 2 of each
    double* gsum_part;
    unsigned int* gsum_cnt;
    // temporaries of the operator entry points
    double2* tmp_odd;          // V/2 x 3 complex
    void* tmp_lo_in;           // reduced-precision conversions of an API input/output
    void* tmp_lo_out;
    size_t tmp_lo_bytes;
    stag::Workspace* ws;
    void* full_tmp;            // four half fields for the full-lattice solve
    int prepared_prec;         // storage of tmp_lo_in after stag_dslash_prepare (-1: none)
    int prepared_nrhs;         // fields prepared
    int repeat_done;           // tmp_lo_out holds a stag_dslash_repeat result of those fields
    void* tune;                // autotuner cache (tune.cu)
    int last_rhs_block;        // right-hand sides per pass chosen by the last batched solve
    int last_multi_cfg;        // and its configuration (G << 8 | NBT, multi_tile.cuh)
    // power-of-two normalisation of fields (scale.cu): largest-magnitude bits
    // and exponents per field, SCALE_SLOTS of each
    unsigned long long* scale_bits;
    int* scale_k;
    // double-float links hold 2^-df_link_exp U: 0 for links whose largest
    // element lies within 2^-40 .. 2^40, else that element's exponent (and the
    // double-precision solvers then use IEEE double arithmetic)
    int df_link_exp;
    int link_exp;              // exponent of the largest link element (valid if link_exp_known)
    bool link_exp_known;       // cleared by every upload
    void* dfx_tmp;             // double-float operator on canonical fields: input and output storage
    size_t dfx_tmp_bytes;
    int op_links;              // link field of the operator entry points (stag_set_operator_links)
    int half_stage[2];         // half 12-real operator entry points, links as uploaded / temporal gauge:
                               // STAGE_* bits of what is staged in shared memory, -1 not decided (unstaged)
};

namespace stag {

// pack.cu
int upload_gauge(stag_ctx ctx, const double* U, int on_device);
int ensure_links(stag_ctx ctx, int prec, int recon, const void** out);
int convert_f64_to_lo(stag_ctx ctx, int prec, const double2* in, void* out, int nvec, cudaStream_t s);
int convert_lo_to_f64(stag_ctx ctx, int prec, const void* in, double2* out, int nvec, cudaStream_t s);
size_t lo_spinor_bytes(const Geom& g, int prec);

int ensure_lo_tmp_public(stag_ctx ctx, size_t bytes);
// links: which link field the operator applies (op_links_for below).
int multi_dslash(stag_ctx ctx, int prec, int recon, int par_out, void* out, const void* in, int nrhs, int nb,
                 int* nb_used, int* cfg_used = nullptr, int links = 0);
// multi-vector configuration (multi_tile.cuh) used for an explicit rhs block
int multi_cfg_for(int prec, int block);

// dslash.cu: out = D_{par_out, 1-par_out} in, storage chosen by prec/recon.
// in/out are in the internal storage of prec (F64: canonical AoS).
// links: the link field applied (STAG_LINKS_*, op_links_for below); the
// operator entry points pass ctx->op_links, internal callers the uploaded field.
int launch_dslash(stag_ctx ctx, int prec, int recon, int par_out, void* out, const void* in,
                  cudaStream_t s, int links = STAG_LINKS_UPLOADED);
int launch_dslash_internal(stag_ctx ctx, int prec, int recon, int par_out, void* out, const void* in,
                           cudaStream_t s, int links = STAG_LINKS_UPLOADED);
int multi_dslash_internal(stag_ctx ctx, int prec, int recon, int par_out, void* out, const void* in, int nrhs,
                          int nb, int* nb_used, int links = STAG_LINKS_UPLOADED);
int dslash_f64x_canonical(stag_ctx ctx, int par_out, double2* out, const double2* in, int nfield, int links,
                          int nb, int* nb_used, cudaStream_t s);
// the context's double-float scratch fields: nfield inputs and nfield outputs
// of SpinorDF storage (48 bytes per site each), kept until the next call that
// uses them (the double-float operator entry points, the force)
int dfx_fields(stag_ctx ctx, int nfield, float4** in, float4** out);
// dslash.cu: the staging decision of the half 12-real operator for a link
// field (ctx->half_stage), timed once on in/out (outputs overwritten).  Only
// outside stream capture.
int tune_half_stage(stag_ctx ctx, int links, void* out, const void* in);
// tgauge.cu: the temporal-gauge matrices g and the links U' = g U g^dagger
// (dslash.cuh, TGLinks) in the storage of (prec, recon), built on first use
// after an upload; g b and g^dagger x for nfield even-site fields.
int ensure_tg_gauge(stag_ctx ctx, const double2** G);
int ensure_links_tg(stag_ctx ctx, int prec, int recon, const void** out);
int ensure_tg_tmp(stag_ctx ctx, int nfield, double2** out);
// pack.cu: (re)derive the copy (prec, recon) of the internal F64/18 field src
// into *dst (allocated on first use, then kept at its address).  e: exponent
// the double-float copy is scaled by (2^-e U).
int derive_link_copy(stag_ctx ctx, const double2* src, int prec, int recon, int e, void** dst, size_t* bytes);

// scale.cu
int ensure_scale_scratch(stag_ctx ctx);
int field_exponents(stag_ctx ctx, const double2* v, int nfield, size_t field_elems, int slot, cudaStream_t s);
int scale_fields_in(stag_ctx ctx, const double2* in, double2* out, int nfield, size_t field_elems, int slot,
                    int kstride, cudaStream_t s);
int scale_fields_out(stag_ctx ctx, const double2* in, double2* out, int nfield, size_t field_elems, int slot,
                     int kstride, cudaStream_t s);
int normalise_fields(stag_ctx ctx, const double2* in, double2* out, int nfield, size_t field_elems, int slot,
                     cudaStream_t s);
int split_fields_scaled(stag_ctx ctx, const double2* in, float4* out, int nfield, size_t field_elems, int slot,
                        int extra, cudaStream_t s);
int join_fields_scaled(stag_ctx ctx, const float4* in, double2* out, int nfield, size_t field_elems, int slot,
                       int kstride, int extra, cudaStream_t s);
int link_max_exponent(stag_ctx ctx, int* out);
int check_float_inner_links(stag_ctx ctx);
// The arithmetic a double-precision pass really uses: STAG_F64X unless the
// double-float links are scaled (links outside the double-float range).
int resolve_f64_arith(stag_ctx ctx, int requested, int* out);
int tg_apply(stag_ctx ctx, const double2* G, const double2* in, double2* out, int nfield, int dagger);
inline GridSum grid_sum_of(stag_ctx ctx) { return GridSum{ctx->gsum_part, ctx->gsum_cnt}; }

// The link copy (prec, recon) of a link-field choice: STAG_LINKS_UPLOADED the
// uploaded field, STAG_LINKS_TEMPORAL(_FULL) its temporal-gauge transform;
// *tg = 1 where the identity time links are to be skipped.
inline int op_links_for(stag_ctx ctx, int links, int prec, int recon, const void** out, int* tg)
{
    *tg = links == STAG_LINKS_TEMPORAL ? 1 : 0;
    if (links == STAG_LINKS_UPLOADED) return ensure_links(ctx, prec, recon, out);
    return ensure_links_tg(ctx, prec, recon, out);
}

}  // namespace stag
