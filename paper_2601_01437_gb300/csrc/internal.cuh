// Internal declarations shared by the library's CUDA translation units.
// Nothing here is part of the C ABI (include/irlnqs.h is).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>

#include "irlnqs.h"

#define LM_MAXM 64      // spin orbitals
#define LM_MAXH 256     // hidden units
#define LM_MAXKRYLOV 64 // Krylov dimension
#define LM_HIST_MAX 1024 // IRL cycles recorded per solve (lm_irl_history)
// Captured IRL cycles kept per pencil (keyed by first step, Krylov dimension and
// everything the captured launches take by value), least recently used replaced.
#define LM_CYCLE_GRAPHS 8
#define LM_CYCLE_KEY 12
struct CycleGraph {
    int key[LM_CYCLE_KEY];
    cudaGraphExec_t exec;
    int kernels;    // kernel nodes (launch counter per replay)
    long long used; // last use, for replacement
};
void lm_cycle_graphs_release(lm_pencil *p);

// Bound on polls of one mbarrier phase before a kernel gives up (each
// try_wait may itself suspend for a short, hardware-defined time).
#define LM_SPIN_LIMIT (1u << 22)

// Device error flags (lm_ctx::d_flags): bit set by kernels, read by the host.
enum {
    FLAG_ROW_OUTSIDE_SECTOR = 1,
    FLAG_TIMEOUT = 2,
    FLAG_BAD_ARG = 4,
};

// ---------------------------------------------------------------------------
// Small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// mbarrier + 1-D bulk copy (TMA engine) wrappers, CTA scope.
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Bulk global->shared copy; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait on one phase of an mbarrier: false once LM_SPIN_LIMIT polls or
// limit_ns of wall time (two seconds unless a test asks for less) have passed
// without the phase completing.
#define LM_WAIT_LIMIT_NS 2000000000ull
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns = LM_WAIT_LIMIT_NS) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < LM_SPIN_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// ---------------------------------------------------------------------------
// Handles
// ---------------------------------------------------------------------------
#define LM_PROF_EVENTS 2048
#define LM_PROF_CLASSES 5

struct lm_ctx {
    int device;
    int sms;
    int smem_optin;
    double hbm_bytes_per_ms;  // streaming rate assumed by grid tuning (0: unknown)
    int *d_flags;        // device error flags
    char err[512];
    // counters
    int64_t launches;
    int profile;
    int prof_mask;  // kernel classes bracketed by events while profile is set (bit = class)
    cudaEvent_t ev[LM_PROF_CLASSES][LM_PROF_EVENTS][2];  // [class][pair][start/end]
    int ev_ready;
    int64_t ev_used[LM_PROF_CLASSES];
    int64_t ev_count[LM_PROF_CLASSES];
    int64_t pencil_rows;
};

enum { PROF_BUILD = 0, PROF_PENCIL = 1, PROF_LANCZOS = 2, PROF_PREP = 3, PROF_TRI = 4 };

inline void lm_note_launch(lm_ctx *ctx, int n = 1) { ctx->launches += n; }

// The largest dynamic shared memory a launch of func may request on this device:
// the opt-in limit less the kernel's static shared memory.
inline int lm_max_dyn_smem(const void *func, int smem_optin) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, func) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return smem_optin - (int)fa.sharedSizeBytes;
}
// Event pair around one launch of a profiled kernel class (no-op unless profiling).
inline void lm_prof_begin(lm_ctx *ctx, int cls, cudaStream_t s) {
    if (!ctx->profile || !ctx->ev_ready || !((ctx->prof_mask >> cls) & 1)) return;
    if (ctx->ev_used[cls] < LM_PROF_EVENTS) cudaEventRecord(ctx->ev[cls][ctx->ev_used[cls]][0], s);
}
inline void lm_prof_end(lm_ctx *ctx, int cls, cudaStream_t s) {
    ctx->ev_count[cls]++;
    if (!ctx->profile || !ctx->ev_ready || !((ctx->prof_mask >> cls) & 1)) return;
    if (ctx->ev_used[cls] < LM_PROF_EVENTS) {
        cudaEventRecord(ctx->ev[cls][ctx->ev_used[cls]][1], s);
        ctx->ev_used[cls]++;
    }
}

// Device-side IRL state (one per pencil), all FP64.
struct IrlState {
    double alpha[LM_MAXKRYLOV + 1];
    double beta[LM_MAXKRYLOV + 1];
    double ritz[LM_MAXKRYLOV];
    double u[LM_MAXKRYLOV];                   // lowest eigenvector of T (final)
    double Q[LM_MAXKRYLOV * LM_MAXKRYLOV];    // restart rotations, column-major
    double h1[LM_MAXKRYLOV + 1];              // reduced CGS dots (pass 1)
    double h2[LM_MAXKRYLOV + 1];              // reduced CGS dots (pass 2)
    double lam, res, tnorm, tol_eff, bnorm;
    double rq, rq_s, res_explicit, c0, yty, lam_ritz;
    int jend, broke, conv, err;
    int flags;  // this pencil's device error flags (FLAG_*), cleared at each IRL start
};

// Pinned host scratch of a pencil: the IRL state read-back, and the energy and
// flags of the last build.
struct PencilHost {
    IrlState st;
    double E;
    int flags;
    // staging of small vectors between device and host: shard statistics,
    // vectors handed to a caller's reduction (irl_step_sharded)
    double xfer[2 * 2048 + 64];
};

struct lm_pencil {
    lm_ctx *ctx;
    int n, na, nb, nh, M, M1, P1, ldp;
    int64_t n_rows;
    int enumerated;     // rows = the whole sector
    int given_weights;  // weights from the caller
    int prec;           // low-precision copy kind (LM_FP64 = none)
    int sym;            // resolved default symmetrisation
    int gfree;          // the E_loc estimator's pencil: O_c, E_loc and weights, no G'_c
    float2 *rt, *psim;  // sector rows: tanh z_j and psi mantissa per row (k_row_tables)
    double *rt64;       // sector rows: tanh z_j per row in FP64
    int *psie;          // sector rows: psi exponent per row
    int cycle_graphs;   // 1: IRL cycles on this pencil replay captured CUDA graphs
    struct CycleGraph *cg;  // [LM_CYCLE_GRAPHS] captured cycles (irl.cu), or null
    double e_core;
    // device buffers (FP64 unless noted)
    uint64_t *rows;
    double *wt, *lnpsi, *eloc;
    float2 *wlo;        // normalised weights as double-float
    double *wel;        // w (E_loc - E): the weights of the E_loc-estimator product
    float2 *wello;      // ... as double-float
    double *O, *G;      // N_s x ldp, centred in place
    void *Olo, *Glo;    // low-precision copies (float or bf16) or null
    double *h, *eri, *theta, *tabs;
    float2 *tdf;        // double-float tables for the df64 build
    int arith;          // lm_arith of the last build
    double *stats;      // [0] sum w, [1] E, [2] max lnpsi, [8..8+ldp) mean O
    double *part;       // reduction partials
    int64_t part_len;
    int order_rev;      // the product being enqueued walks each CTA's rows backwards
    int g_pencil;       // CTAs of a product on the stored factors (tunable); an FP64
                        // product of a low-precision pencil always runs on every SM
    // IRL workspace
    double *V;          // ldp x (LM_MAXKRYLOV + 1), column-major
    double *wvec, *yvec, *hy, *sy, *tvec, *dots;
    IrlState *st;       // device
    IrlState *st_host;  // pinned mirror (inside hs)
    PencilHost *hs;     // pinned host scratch
    // Pinned staging of caller host arrays: a copy from or to pageable host
    // memory synchronises its stream (to) or the host (from), which would
    // serialise concurrent instances. Inputs are copied here on the host and
    // sent asynchronously; host outputs land here and are copied out when the
    // job completes. Layout: LM_STAGE_* offsets below.
    unsigned char *hstage;
    size_t st_in_rows, st_in_w, st_out;  // byte offsets of rows, weights, IRL region
    int *d_flags;       // &st->flags: error flags of this pencil's kernels
    unsigned *bar;      // grid-barrier words of the cooperative Lanczos kernel
    double E_host;
    // per IRL cycle of the last irl_step on this pencil (host side): the lowest
    // Ritz value of T_m, the residual estimate beta_m |u_m|, and whether the
    // cycle ran on the low-precision factors
    int n_hist;
    double hist_lam[LM_HIST_MAX], hist_res[LM_HIST_MAX];
    int hist_lowp[LM_HIST_MAX];
    // row shards (lm_shard_*): 1 after lm_shard_build, 2 after lm_shard_sums,
    // 0 once centred (the pencil is usable); shv holds a shard's local product
    // for the caller's reduction (2 ldp doubles, allocated on first use)
    int shard_state;
    double *shv;
    // tensor-core block product (block.cu): tensor maps and scratch, created on
    // first use
    struct BlockState *blk;
    // block Lanczos workspace (blocklz.cu), allocated on first use
    double *blz;
    size_t blz_len;
    // streamed pencil (lm_build_streamed): rows per chunk (0: O and G resident),
    // the chunks' raw statistics [n_chunks][8 + ldp]
    int64_t chunk;
    double *cstats;
};

// ---------------------------------------------------------------------------
// Host helpers (abi.cu)
// ---------------------------------------------------------------------------
int lm_fail(lm_ctx *ctx, int code, const char *fmt, ...);
int lm_cuda_check(lm_ctx *ctx, cudaError_t e, const char *what);
bool lm_is_device_ptr(const void *p);
int lm_read_flags(lm_ctx *ctx, cudaStream_t s, int *flags);
// lm_build_OG in two halves: enqueue the build (and the read-back of E and the
// flags into pinned memory) on `stream`; after that work has completed,
// lm_build_finish checks the flags and publishes E.
// rows_only = 1 stops after the row build (K2-K6), for row shards.
// chunk_rows > 0 makes a streamed pencil: O and G buffers of chunk_rows rows,
// statistics gathered chunk by chunk, products rebuilding the chunks.
int lm_build_enqueue(lm_ctx *ctx, const lm_system *sys, const double *theta,
                     const uint64_t *rows, const double *weights, int64_t n_rows,
                     lm_precision prec, void *stream, lm_pencil **inout, int rows_only = 0,
                     int64_t chunk_rows = 0, int gfree = 0);
int lm_build_finish(lm_pencil *p);
size_t lm_pencil_footprint(lm_ctx *ctx, int n, int nh, int64_t n_rows, int prec);
// Staging regions: h at 0, eri after it, theta after that (ldp doubles), rows
// at st_in_rows, weights at st_in_w; the IRL region at st_out holds four ldp
// vectors: theta_inout, c, dtheta, v0.
enum { LM_STAGE_TIO = 0, LM_STAGE_C = 1, LM_STAGE_DTH = 2, LM_STAGE_V0 = 3 };
double *lm_stage_irl(lm_pencil *p, int which);
// Copy n bytes of a caller array (device, pinned or pageable host) to device
// memory on stream s; pageable sources go through the pencil's staging at off.
int lm_stage_h2d(lm_pencil *p, void *dst, const void *src, size_t n, size_t off, cudaStream_t s);
bool lm_is_pageable(const void *ptr);
void lm_pencil_release(lm_pencil *p);  // frees without a device-wide synchronisation

// Resumable IRL (irl.cu): the host side of irl_step as a state machine.
// irl_job_advance enqueues the next stretch of device work on the job's stream
// and records the job's event; call it again once that event has completed
// (the first call starts the job). *done = 1 when the result is final.
struct IrlJob;
// reduce (nullable): sum every product over the row shards (irl_step_sharded)
int irl_job_create(lm_pencil *p, const irl_params *prm, double *c_out, double *dtheta_out,
                   double *theta_inout, cudaStream_t s, IrlJob **out,
                   lm_reduce_fn reduce = nullptr, void *reduce_user = nullptr,
                   int reduce_where = LM_REDUCE_HOST);
int irl_job_advance(IrlJob *job, int *done);
cudaEvent_t irl_job_event(const IrlJob *job);
void irl_job_result(const IrlJob *job, irl_result *out);
void irl_job_free(IrlJob *job);

// build.cu
int lm_launch_enumerate(lm_ctx *ctx, int n, int na, int nb, uint64_t *out, int64_t count,
                        cudaStream_t s);
int lm_launch_build(lm_pencil *p, cudaStream_t s);   // rows, then statistics and centring
int lm_launch_build_rows(lm_pencil *p, cudaStream_t s);
int lm_launch_build_prep(lm_pencil *p, cudaStream_t s);
// row shards (lm_shard_*): local maxima of ln psi into p->part[0 .. *nparts),
// raw local sums into p->stats with a given shift, centring with p->stats
int lm_launch_shard_max(lm_pencil *p, cudaStream_t s, int *nparts);
int lm_launch_shard_sums(lm_pencil *p, double lnpsi_max, cudaStream_t s);
int lm_launch_centre(lm_pencil *p, cudaStream_t s);
// streamed pencils: the first statistics pass, and one product (chunk by chunk)
int lm_launch_stream_stats(lm_pencil *p, cudaStream_t s);
int lm_launch_stream_product(lm_pencil *p, const double *v, int sym, int prec, int want_s,
                             double *yH, double *yS, cudaStream_t s);
int lm_launch_connections(lm_ctx *ctx, int n, int na, int nb, const double *h,
                          const double *eri, const uint64_t *rows, int64_t n_rows, int cap,
                          uint64_t *od, int8_t *osg, double *oh, int32_t *cnt, double e_core,
                          cudaStream_t s);

// pencil.cu
// partial products of the pencil over row blocks; y_H into part[b][0..ldp),
// y_S into part[b][ldp..2ldp); FP64 values, or double-float pairs in the same
// 8-byte slots when out_df is set
// reverse: walk each CTA's rows backwards (consecutive Lanczos products
// alternate, so each starts on the rows the previous one left in L2)
int lm_launch_pencil(lm_pencil *p, const double *v, int sym, int prec, int want_s,
                     const int *skip, cudaStream_t s, int out_df = 0,
                     int reverse = 0);
int lm_launch_reduce_partials(lm_pencil *p, int prec, double *yH, double *yS, cudaStream_t s);
// CTAs (= partial vector pairs) of a product of precision prec on pencil p
int lm_pencil_ctas(const lm_pencil *p, int prec);
int lm_launch_df_to_fp64(lm_ctx *ctx, const float2 *src, double *dst, int64_t n, cudaStream_t s);
int lm_pencil_grid(lm_pencil *p);

// block.cu: the tensor-core block product (dbg / descriptor strides for tests)
int lm_launch_pencil_block(lm_pencil *p, const double *V, int ldv, int nvec, double *HV,
                           double *SV, int sym, float *dbg, uint32_t lbo_mn, uint32_t sbo_mn,
                           cudaStream_t s);
void lm_block_release(lm_pencil *p);
// blocklz.cu: the block Lanczos phase (nsteps blocks of 16 vectors on the
// tensor-core product); the Ritz vector of the lowest Ritz value goes to u_out
int lm_launch_block_lanczos(lm_pencil *p, int sym, int nsteps, uint64_t seed, int deflate,
                            double *u_out, cudaStream_t s);

// pencil.cu: the FP64 pencil product on caller-provided scratch (no allocation):
// vpad holds v padded to ldp, part holds grid x 2 ldp partials, flags one int
// that must be zero on entry.
int lm_pencil_fp64_on_scratch(const double *O, const double *G, const double *w, int64_t n_rows,
                              int ldp, int p1, const double *vpad, double *part, int grid, int half,
                              double *yH, double *yS, int smem_optin, int *flags, cudaStream_t s);
