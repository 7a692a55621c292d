/*
 * irlnqs.h — C ABI of the GB300 (sm_103a) library for the data-parallel hot
 * path of the implicitly restarted Lanczos (IRL) optimiser for shallow neural
 * quantum states (arXiv 2601.01437).
 *
 * The path has two halves:
 *   1. lm_build_OG: over bit-packed determinants of a second-quantised
 *      molecular Hamiltonian, build the per-row log-derivative matrix
 *      O_k(x) = d ln psi(x) / d theta_k of an RBM wavefunction and the
 *      Hamiltonian-applied matrix G_k(x) = sum_x' H_xx' psi(x')/psi(x) O_k(x'),
 *      then the weights, the energy E and the centred pencil factors.
 *   2. lm_apply_pencil / irl_step: apply the centred linear-method pencil
 *      matrix-free, y_H = O_c^T W (G'_c v) and y_S = O_c^T W (O_c v), inside
 *      device-resident implicitly restarted Lanczos, and return the lowest
 *      Ritz pair and the parameter update.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Determinants: uint64, bit p = occupation of spin orbital p, blocked order
 *   (spin orbitals 0..n-1 alpha, n..2n-1 beta; spatial orbital p mod n).
 * RBM: ln psi(x) = a.x + sum_j ln(2 cosh(b_j + W_j.x)), M = 2n visible,
 *   Nh hidden, P = M + Nh + M*Nh parameters.
 * Augmented index space (the linear method's basis chi_0 = psi,
 *   chi_k = (O_k - <O_k>) psi; Methods, eqs. rayleigh_quotient/full_gevp):
 *   dimension P+1 = (Nh+1)(M+1), row-major over the grid (r, c), r in [0,Nh],
 *   c in [0,M]. Entry (0,0) is chi_0. theta is this grid without (0,0):
 *   theta[0..M) = a; theta[(j+1)(M+1)-1] = b_j; theta[(j+1)(M+1)+p] = W_jp.
 * Pointers: every input or output array may be host or device memory; the
 *   library detects which with cudaPointerGetAttributes. The caller owns
 *   every pointer it passes; the library owns everything behind a handle.
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   Calls enqueue their work on it; results written to host memory are valid
 *   when the call returns (those calls synchronise the stream).
 * Errors: every function returns an int status (0 = LM_OK). Nothing throws
 *   across the ABI. lm_last_error gives a one-line description of the last
 *   failure on a context.
 * Limits: M = 2*n_orb <= 64, Nh <= 127, P+1 <= 2048, Krylov dimension m <= 64.
 * Tuning overrides (environment, read at each launch; they change reduction
 *   orders, so the last bits of results, within the same parity bars):
 *   IRLNQS_LANCZOS=cluster|coop|split restricts the Lanczos-step kernel
 *   choice; IRLNQS_BUILD_LAYOUT=<slices>:<0|1> fixes the double-float row
 *   build's scatter slices and whether its A table is dropped.
 */
#ifndef IRLNQS_H
#define IRLNQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
    LM_OK = 0,
    LM_ERR_ARG = -1,     /* null pointer, bad enum, rows outside the sector */
    LM_ERR_SIZE = -2,    /* M > 64, N_alpha > n_orb, m > 64, ...            */
    LM_ERR_OOM = -3,     /* device allocation failed                        */
    LM_ERR_CUDA = -4,    /* a CUDA runtime call or kernel launch failed     */
    LM_ERR_TIMEOUT = -5, /* a bounded device wait gave up                   */
    LM_ERR_CALLBACK = -6 /* the caller's reduction callback returned nonzero */
};

/* irl_result.status (Algorithm 1 outcomes and the update's validity) */
enum {
    IRL_OK = 0,                  /* residual below tolerance                  */
    IRL_BREAKDOWN_INVARIANT = 1, /* beta_j ~ 0: invariant subspace, exact Ritz */
    IRL_MAX_RESTARTS = 2,        /* restart budget exhausted (best pair kept) */
    LM_C0_TINY = 3,              /* |c_0| < 1e-8 |c|: no update written       */
    LM_STATIONARY = 4            /* lambda_min > -tol: theta is stationary    */
};

/* Storage of the pencil factors used by the Lanczos products. FP64: the
 * centred factors in FP64. FP32 / BF16: low-precision copies beside the FP64
 * factors (FP32 accumulation; the FP64 factors serve the FP64 continuation,
 * the final refinement and exports). DF64: the centred factors only as
 * double-float FP32 pairs (48-bit significand, products accurate to ~1e-14
 * relative, computed on the FP32 pipes); FP64 product requests, the final
 * refinement and exports are served from them (exports convert). */
typedef enum { LM_FP64 = 0, LM_FP32 = 1, LM_BF16 = 2, LM_DF64 = 3 } lm_precision;

/* symmetrisation of H~' inside the Lanczos operator */
typedef enum {
    LM_SYM_AUTO = 0, /* NONE for the full enumerated sector, HALF otherwise    */
    LM_SYM_NONE = 1, /* y = O_c^T W G'_c v                                     */
    LM_SYM_HALF = 2, /* y = 1/2 (O_c^T W G'_c v + G'_c^T W O_c v)              */
    LM_SYM_ELOC = 3  /* the paper's E_loc estimator of H~' (Methods, eq.
                        matrix_vec_prod): y = O_c^T W diag(E_loc - E) O_c v, i.e.
                        G'_c -> (E_loc - E) O_c, dropping dE_loc/dtheta; reads O_c
                        only, symmetric by construction                          */
} lm_sym;

typedef struct lm_ctx lm_ctx;
typedef struct lm_pencil lm_pencil;

/* Second-quantised Hamiltonian (Methods, "Wave Function Ansatz"):
 * H = sum_{pq,s} h_pq a+_ps a_qs + 1/2 sum_{pqrs,s,t} (pq|rs) a+_ps a+_rt a_st a_qs.
 * h: n_orb x n_orb real symmetric; eri: n_orb^4 chemist (pq|rs) with 8-fold
 * symmetry, index ((p*n+q)*n+r)*n+s. Both are read during lm_build_OG only. */
/* Arithmetic of the row build (lm_build_OG). Both give FP64-level results:
 * DF64 evaluates the per-connection work in double-float (pairs of FP32, a
 * 48-bit significand, relative error ~2^-44 per operation) on the FP32 pipes;
 * FP64 uses native FP64 throughout (GB300 runs FP64 at 1/62 of FP32). */
typedef enum { LM_ARITH_DF64 = 0, LM_ARITH_FP64 = 1 } lm_arith;

typedef struct {
    int n_orb, n_alpha, n_beta, n_hidden;
    const double *h;
    const double *eri;
    double e_core;    /* added to E and E_loc */
    int build_arith;  /* lm_arith; 0 (DF64) by default */
} lm_system;

typedef struct {
    int64_t n_rows;       /* N_s */
    int n_params;         /* P */
    int ld;               /* padded row length of O_c, G'_c (>= P+1, multiple of 8) */
    int precision;        /* lm_precision of the low-precision copy (FP64: none) */
    int sym;              /* resolved lm_sym */
    double energy;        /* E(theta) = sum_x w(x) E_loc(x), including e_core */
    int grid;             /* CTAs of each pencil-product launch (lm_pencil_set_grid) */
} lm_pencil_info;

/* IRL settings (Algorithm 1; the paper uses k = 1, m = 20, tol = 1e-12). */
typedef struct {
    int m;              /* Krylov dimension, k < m <= 64                          */
    int k;              /* kept Ritz pairs per restart (mu = m - k shifts)        */
    double tol;         /* absolute residual tolerance on ||H y - lambda y||      */
    int max_restarts;   /* restart budget (the paper gives none; 200 is typical)  */
    uint64_t seed;      /* SplitMix64 seed of the random start vector             */
    int sym;            /* lm_sym (AUTO resolves as for the pencil)               */
    int precision;      /* lm_precision of the Lanczos operator; a low-precision  */
                        /* solve is refined by FP64 restarts before returning     */
    int deflate_null;   /* 1: remove the particle-number null space of O_c        */
    const double *v0;   /* optional start vector (P+1), NULL = random             */
    int reorth;         /* IRL_REORTH_FULL (0): classical Gram-Schmidt twice      */
                        /* against the whole basis; IRL_REORTH_NONE (1): the      */
                        /* paper's three-term recurrence of Algorithm 2 only      */
    int mode;           /* IRL_MODE_SHEP (0): the paper's S ~ I eigenproblem      */
                        /* (eq. standard_evp); no other mode is accepted          */
    int block;          /* 0: single-vector Lanczos. 16: the low-precision phase  */
                        /* is block Lanczos (m / 16 blocks of 16 vectors, m in    */
                        /* 16..64) on the tensor-core block product; needs a      */
                        /* BF16 pencil and precision LM_BF16. Its Ritz vector     */
                        /* starts the FP64 continuation and refinement.           */
} irl_params;

enum { IRL_REORTH_FULL = 0, IRL_REORTH_NONE = 1 };
enum { IRL_MODE_SHEP = 0 };

typedef struct {
    double lambda;        /* lowest eigenvalue of the SHEP (eq. standard_evp): the  */
                          /* FP64 Rayleigh quotient of the refined Ritz vector      */
    double energy;        /* E(theta)                                             */
    double lambda_gen_rq; /* generalised Rayleigh quotient c^T H~' c / c^T S~ c   */
    double residual;      /* explicit FP64 ||H~' c - lambda c||, |c| = 1          */
    double c0;            /* c[0] of the unit Ritz vector (sign fixed c0 >= 0)    */
    int status;           /* IRL_* / LM_* above                                   */
    int n_matvec;         /* pencil applications (all precisions)                 */
    int n_restart;        /* implicit restarts                                    */
    int n_matvec_lowp;    /* of which in the low-precision phase                  */
} irl_result;

/* ---- context ----------------------------------------------------------- */

/* Context options. struct_size = sizeof(lm_ctx_params) as the caller compiled
 * it (later versions may append fields; fields beyond struct_size keep their
 * defaults). */
typedef struct {
    unsigned struct_size;
    int profile;    /* nonzero: time kernel classes with CUDA events from the
                       start, as lm_stats_reset(ctx, profile) (1: every class;
                       LM_PROF_ONLY | class bits); 0: count launches only    */
    double hbm_gbs; /* streaming rate in GB/s that the grid autotuner of the batch
                       and server engines assumes (its cost model charges each
                       product max(compute, bytes / rate)); 0: 85 % of the
                       device's interface peak (memory clock x bus width)     */
} lm_ctx_params;

/* Create a context on CUDA device `device` (made current for every call).
 * params may be NULL (all defaults). *out receives the handle; free it with
 * lm_destroy. Errors: LM_ERR_CUDA (no such device), LM_ERR_ARG (struct_size
 * smaller than the first two fields, negative hbm_gbs), LM_ERR_OOM. */
int lm_create(lm_ctx **out, int device, const lm_ctx_params *params);
int lm_destroy(lm_ctx *ctx);
/* Description of the last failure on ctx (never NULL; "" after success). */
const char *lm_last_error(const lm_ctx *ctx);

/* ---- the hot path ------------------------------------------------------ */

/*
 * Build the centred pencil factors (Methods: E_loc, O, eqs. heff and
 * centered_hamiltonian; the energy-centring step H' = H - E).
 *   rows    N_s determinants, or NULL to enumerate the whole (N_alpha, N_beta)
 *           sector in ascending order (its size must equal n_rows; pass
 *           n_rows = 0 to let the library size it).
 *   weights N_s non-negative sample weights (e.g. Monte Carlo multiplicities),
 *           normalised by their sum; NULL = |psi(x)|^2 / sum |psi|^2.
 *   prec    FP64 only, or FP64 plus an FP32 / BF16 / DF64 copy of O_c and
 *           G'_c for the Lanczos products.
 * Layout on the device: O_c, G'_c row-major N_s x ld FP64 (columns >= P+1 zero;
 *   DF64 pencils hold them as double-float pairs in the same layout),
 *   O_c(x,0) = 1, G'_c(x,0) = E_loc(x) - E, and for k >= 1
 *   O_c(x,k) = O_k(x) - <O_k>, G'_c(x,k) = G_k(x) - <O_k> E_loc(x) - E O_c(x,k).
 * *inout: NULL to create a pencil, or an existing pencil of the same system
 *   and row count to rebuild in place (buffers are reused).
 * Errors: LM_ERR_SIZE for M > 64 or Nh > 127 or P+1 > 2048 or bad electron counts;
 *   LM_ERR_ARG if a given row lies outside the sector (detected on the device,
 *   reported by this call).
 */
int lm_build_OG(lm_ctx *ctx, const lm_system *sys, const double *theta, const uint64_t *rows,
                const double *weights, int64_t n_rows, lm_precision prec, void *stream,
                lm_pencil **inout);

/*
 * The E_loc estimator's pencil (Methods, eq. matrix_vec_prod, whose H~' uses
 * E_loc(x) in place of the G form of eq. heff): the same build as lm_build_OG
 * with G never formed. Per connection it keeps only the running product of
 * (1 + Z_j) that the coefficient needs (no tanh of the connected
 * configuration, no accumulation into G), and no G'_c or copy of it is
 * allocated. O_c, ln psi, E_loc, the weights and E equal lm_build_OG's.
 * The pencil answers sym = LM_SYM_ELOC (its default, also for LM_SYM_AUTO)
 * and S~ products; lm_apply_pencil and irl_step with LM_SYM_NONE/HALF, a
 * block phase, lm_apply_pencil_block and the export of G'_c return
 * LM_ERR_ARG. Runs in double-float arithmetic (sys->build_arith =
 * LM_ARITH_FP64 returns LM_ERR_ARG). Arguments, layout, ownership and the
 * other errors as lm_build_OG; *inout may only be a pencil from lm_build_O.
 */
int lm_build_O(lm_ctx *ctx, const lm_system *sys, const double *theta, const uint64_t *rows,
               const double *weights, int64_t n_rows, lm_precision prec, void *stream,
               lm_pencil **inout);

/*
 * Matrix-free pencil product (Methods, eq. matrix_vec_prod, with the G form of
 * eq. heff): Hv = H~' v (symmetrised per `sym`), Sv = S~ v, both P+1 FP64.
 * v: P+1 FP64. Either output may be NULL. `prec` selects the FP64 factors or
 * the pencil's low-precision copy (a DF64 pencil answers both from its
 * double-float factors). Reads O_c and G'_c once.
 */
int lm_apply_pencil(lm_pencil *p, const double *v, double *Hv, double *Sv, int sym, int prec,
                    void *stream);

/*
 * Lowest eigenpair of the SHEP H~' c = lambda c (eq. standard_evp) by
 * implicitly restarted Lanczos (Algorithms 1 and 2) with full FP64
 * reorthogonalisation, followed by an explicit residual / Rayleigh
 * refinement in FP64 (with FP64-accurate products: the FP64 factors, or the
 * double-float ones of a DF64 pencil). Writes (all optional, host or device):
 *   c_out      P+1, unit Ritz vector with c[0] >= 0;
 *   dtheta_out P,   the update c[1:]/c[0] (linearised wavefunction, c = [1, v]);
 *   theta_inout P,  theta += dtheta when status is IRL_OK/BREAKDOWN.
 * out receives the result record (host memory). Returns LM_ERR_* on failure;
 * the IRL outcome itself is out->status.
 */
int irl_step(lm_pencil *p, const irl_params *prm, irl_result *out, double *c_out,
             double *dtheta_out, double *theta_inout, void *stream);

int lm_pencil_info_get(lm_pencil *p, lm_pencil_info *out);
int lm_pencil_free(lm_pencil *p);

/* Number of CTAs each pencil-product launch of p uses (default: one per SM),
 * 1 <= ctas <= SM count (LM_ERR_ARG otherwise). The products sum the CTAs'
 * partial vectors in a fixed order, so results depend on this number (in the
 * last bits) and on nothing else about the launch or what runs beside it: an
 * instance run alone with the grid a batch chose reproduces the batch result
 * exactly. */
int lm_pencil_set_grid(lm_pencil *p, int ctas);

/* ---- streamed rows (N_s beyond what O_c and G'_c may occupy) ---------- */

/*
 * A pencil whose O_c and G'_c are never resident (Methods, "Practical
 * Matrix-Free Implementation": every product is a sum of per-row terms, so the
 * rows can be rebuilt when a product needs them). It keeps the rows, weights,
 * ln psi and E_loc (a few numbers per row) and one chunk buffer of chunk_rows
 * rows of O_c and G'_c (and their copy of precision prec). The build makes one
 * pass over the chunks for the statistics (E, <O>, the weights' normaliser; the
 * chunks' sums combined in chunk order with the common ln psi shift); every
 * product -- lm_apply_pencil, each Lanczos step and the refinement of
 * irl_step -- rebuilds, centres and applies the chunks in order and adds their
 * products. Results equal those of lm_build_OG's pencil up to summation
 * order; each product costs one row build. Arguments as lm_build_OG plus
 * chunk_rows >= 1; rows NULL enumerates the sector. O_c and G'_c cannot be
 * exported, and the block product, row shards and the block-Lanczos phase
 * refuse a streamed pencil (LM_ERR_ARG).
 */
int lm_build_streamed(lm_ctx *ctx, const lm_system *sys, const double *theta,
                      const uint64_t *rows, const double *weights, int64_t n_rows,
                      int64_t chunk_rows, lm_precision prec, void *stream, lm_pencil **inout);

/* ---- row shards (one pencil per GPU over a partition of the rows) ------ */

/*
 * The build and the products split by rows (Methods, eqs. heff and
 * centered_hamiltonian: every statistic is a weighted sum over rows, and the
 * matrix-free product of eq. matrix_vec_prod is a sum of per-row terms). Each
 * shard -- typically one GPU of several, each holding its own rows -- runs:
 *   1. lm_shard_build: the row build (ln psi, O, E_loc, G) of the shard's rows;
 *      *lnpsi_max receives the largest ln psi of the shard. The caller takes
 *      the maximum over all shards (it fixes the shift of the |psi|^2
 *      weights; ignored when weights are given).
 *   2. lm_shard_sums(p, lnpsi_max, sums): the shard's unnormalised weights
 *      w = exp(2 (ln psi - lnpsi_max)) (or the given weights) and its P+3 sums
 *      sums[0] = sum w, sums[1] = sum w E_loc, sums[2 + k] = sum w O_k
 *      (k = 0..P; host array). The caller adds them over all shards.
 *   3. lm_shard_centre(p, sums): centring with the summed statistics
 *      (E = sums[1] / sums[0], <O_k> = sums[2 + k] / sums[0], weights
 *      normalised by sums[0]). The pencil is then a shard of the global
 *      pencil: lm_apply_pencil gives this shard's term of the global product,
 *      and the terms of all shards add up to the product of the unsharded
 *      pencil (up to summation order).
 * rows must be given explicitly (lm_enumerate_sector, sliced, for an exact
 * sector); weights NULL means |psi|^2. Host arrays; each call synchronises.
 * irl_step refuses a pencil between steps 1 and 3.
 */
int lm_shard_build(lm_ctx *ctx, const lm_system *sys, const double *theta, const uint64_t *rows,
                   const double *weights, int64_t n_rows, lm_precision prec, void *stream,
                   lm_pencil **inout, double *lnpsi_max);
int lm_shard_sums(lm_pencil *p, double lnpsi_max, double *sums, void *stream);
int lm_shard_centre(lm_pencil *p, const double *sums, void *stream);

/* The caller's sum over shards of a vector of n doubles, in place (one call
 * per pencil product on every shard, in the same order on every shard, with
 * the same n). where = LM_REDUCE_HOST: vec is pinned host memory holding this
 * shard's vector (the stream has been synchronised); the callback returns
 * when vec holds the sum, e.g. after an MPI or gloo all-reduce.
 * where = LM_REDUCE_DEVICE: vec is device memory of this GPU; the callback
 * enqueues an in-place sum on `stream` (a cudaStream_t), e.g. an NCCL
 * all-reduce, and returns. Every shard must receive bitwise the same sum (an
 * all-reduce does), so that the replicated Lanczos work stays identical.
 * A nonzero return aborts the solve with LM_ERR_CALLBACK. */
typedef int (*lm_reduce_fn)(double *vec, int n, void *stream, void *user);
enum { LM_REDUCE_HOST = 0, LM_REDUCE_DEVICE = 1 };

/* irl_step over row shards (Algorithms 1 and 2 with the row-partitioned
 * product): every product is this shard's term of the global product
 * followed by reduce(); the Lanczos vectors, the tridiagonal work and the
 * refinement are replicated on every shard. Each shard calls it with the
 * same prm; results and outputs are those of irl_step on the unsharded
 * pencil, up to the summation order of the products. */
int irl_step_sharded(lm_pencil *p, const irl_params *prm, lm_reduce_fn reduce, void *user,
                     int where, irl_result *out, double *c_out, double *dtheta_out,
                     double *theta_inout, void *stream);

/* ---- block product on the tensor cores --------------------------------- */

/*
 * The pencil product of a block of nvec <= 16 vectors at once (Discussion: the
 * block-Lanczos extension of the method; Methods, eq. matrix_vec_prod per
 * vector): HV = H~' V and SV = S~ V for V = [v_1 .. v_nvec], computed as the
 * two dense tall-skinny contractions O_c^T W (G'_c V) and O_c^T W (O_c V)
 * (HALF: HV = 1/2 (O_c^T W G'_c V + G'_c^T W O_c V)) on the tensor cores with
 * the pencil's BF16 factors, V rounded to BF16 and FP32 accumulation; each
 * factor is read once from HBM per call. Vector k of V, HV, SV starts at
 * k * ldv (P+1 FP64 entries used; ldv >= P+1); all three are device arrays,
 * HV or SV may be NULL. sym: NONE, HALF or AUTO. Needs a pencil built with
 * LM_BF16 and P+1 <= 1920 (LM_ERR_ARG / LM_ERR_SIZE otherwise). Asynchronous
 * on `stream`; a bounded wait that gives up fills HV and SV with NaN.
 */
int lm_apply_pencil_block(lm_pencil *p, const double *V, int ldv, int nvec, double *HV,
                          double *SV, int sym, void *stream);
/* The same with test hooks: dbg (device, nullable) receives the FP32 products
 * O_c V and G'_c V of the first 64 rows ([2][64][16]); lbo_mn, sbo_mn are the
 * shared-memory strides used for the transposed operand (16384 and 1024 in
 * lm_apply_pencil_block). */
int lm_debug_pencil_block(lm_pencil *p, const double *V, int ldv, int nvec, double *HV,
                          double *SV, int sym, float *dbg, unsigned lbo_mn, unsigned sbo_mn,
                          void *stream);

/* ---- inspection (tests and tools; not on the timed path) -------------- */

/* Enumerate the (n_alpha, n_beta) sector in ascending order into out
 * (capacity cap); *count receives the sector size. (Methods, Fock
 * expansion restricted to fixed N_up, N_down.) */
int lm_enumerate_sector(lm_ctx *ctx, int n_orb, int n_alpha, int n_beta, uint64_t *out,
                        int64_t cap, int64_t *count);

/* Connected determinants of each row, as the build kernel enumerates them:
 * for row i, entries [i*cap, i*cap + count[i]) of out_det / out_sign /
 * out_h hold x', the Jordan-Wigner sign of the excitation operator and
 * <x'|H|x>; entry 0 is the diagonal. Slater-Condon rules with parity. */
int lm_debug_connections(lm_ctx *ctx, const lm_system *sys, const uint64_t *rows, int64_t n_rows,
                         int cap, uint64_t *out_det, int8_t *out_sign, double *out_h,
                         int32_t *count);

/* Copy a pencil array out as FP64 (host or device destination):
 * what = 0 O_c (N_s x ld), 1 G'_c (N_s x ld), 2 ln psi (N_s), 3 E_loc (N_s),
 *        4 normalised weights (N_s), 5 mean O (ld), 6 rows (N_s, as uint64 bits). */
int lm_pencil_export(lm_pencil *p, int what, void *dst, void *stream);

/* Per-cycle record of the last irl_step on p (Algorithm 1, step 3: the Ritz
 * values of T_m and the residual test of each cycle): for cycle i (0 = the
 * first Lanczos cycle, then one per implicit restart, a low-precision phase's
 * cycles before its FP64 continuation's), lam[i] is the lowest Ritz value of
 * T_m, res[i] the residual estimate beta_m |e_m^T u| and lowp[i] is 1 if the
 * cycle used the low-precision factors. Up to cap entries are written (any
 * output may be NULL); *n receives the number of cycles recorded (at most
 * 1024). Host memory; call after irl_step has returned. */
int lm_irl_history(lm_pencil *p, double *lam, double *res, int *lowp, int cap, int *n);

/* Test of the timeout path (no counterpart in the paper): run one bounded
 * device wait that nothing ends -- which = 0, the grid barrier of the
 * cooperative Lanczos kernel with a CTA that never arrives; which = 1, an
 * mbarrier phase of the pencil pipeline that no copy completes -- with a wall
 * limit of limit_ns (1 ns .. 2 s; the library's own waits use 2 s). Returns
 * LM_ERR_TIMEOUT when the wait gave up, as it should; the context stays usable.
 * Synchronises the device. */
int lm_debug_wait_timeout(lm_ctx *ctx, int which, int64_t limit_ns);

/* ---- pencil product without allocation -------------------------------- */

/* The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they need a product -- a framework whose
 * caching allocator has reserved the device memory and forbids allocations
 * behind its back, an embedded solver given a fixed memory budget at start-up,
 * or a time-critical loop that cannot afford the synchronisation an
 * allocation or a free may cause.
 *
 * Same product as lm_apply_pencil with FP64 factors, but on the caller's
 * arrays instead of a pencil handle: O_c and G_c are n_rows x ld row-major
 * FP64 (columns >= p1 ignored), w holds the n_rows normalised weights, v has
 * p1 entries, Hv and Sv (either may be NULL, not both) receive p1 entries.
 * sym is LM_SYM_NONE or LM_SYM_HALF. Every array must be memory of the current
 * device (or managed memory), and O_c, G_c 16-byte aligned (LM_ERR_ARG
 * otherwise); ld must be a multiple of 8 and at most LM_NOALLOC_MAX_LD
 * (LM_ERR_SIZE otherwise).
 *
 * It calls no allocator: its scratch (partial products, padded v, a status
 * word) lives in one 4 MiB file-scope device array that every GPU loading the
 * library holds until the process exits. The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress) with the device current;
 * make that first call before any stream capture. All calls share the array
 * and each call overwrites it (the status word and the padded v are cleared
 * or rewritten by every call), so calls that can overlap on a GPU (other
 * streams, other host threads) race and must be serialised by the caller. If
 * a bounded wait inside the kernel gives up, Hv and Sv are filled with NaN.
 * Work is enqueued on `stream`; the call does not synchronise. */
#define LM_NOALLOC_MAX_LD 2048
int lm_apply_pencil_noalloc(const double *O_c, const double *G_c, const double *w, int64_t n_rows,
                            int ld, int p1, const double *v, double *Hv, double *Sv, int sym,
                            void *stream);

/* ---- batched LM steps (many independent systems on one GPU) ----------- */

/* One instance of a batch: one LM step (build of O_c/G'_c, IRL for the lowest
 * Ritz pair, FP64 refinement, update) of an independent system. Pointers may
 * be host or device memory; theta_inout (nullable) is advanced in place by
 * dtheta, dtheta_out (nullable) receives it. */
typedef struct {
    lm_system sys;
    const double *theta;       /* P parameters */
    const uint64_t *rows;      /* NULL: exact sector enumeration; else n_rows samples */
    const double *weights;     /* NULL: |psi|^2 weights; else one weight per row */
    int64_t n_rows;            /* sample count (ignored for exact enumeration) */
    int precision;             /* lm_precision of the stored O/G copies */
    irl_params irl;
    double *dtheta_out;
    double *theta_inout;
} lm_batch_item;

typedef struct lm_batch lm_batch;

/* A batch engine over n_streams CUDA streams (1..64). It keeps one pencil per
 * item index across lm_batch_run calls (device-resident O/G and Lanczos
 * bases; rebuilt in place when the shape is unchanged). autotune = 1 picks,
 * for every new pencil shape, the grid of the products on its stored factors
 * that costs the least shared capacity: with t the duration of a product timed
 * alone once, cost = max(t x CTAs / SMs, bytes streamed / HBM streaming rate);
 * among grids within 3 % of the least cost the fastest is kept. autotune = 0
 * keeps one CTA per SM. FP64 products of a low-precision pencil always use
 * one CTA per SM. */
int lm_batch_create(lm_ctx *ctx, int n_streams, int autotune, lm_batch **out);

/* Run one LM step of every item concurrently (instance i on stream i mod
 * n_streams; no instance waits for another except for GPU resources) and
 * return when all have finished. results[i] is instance i's irl_result;
 * grid_out (nullable, n entries) receives the pencil grid each instance used.
 * Each instance's arithmetic is exactly that of irl_step on the same inputs
 * and grid. Errors: the first failing instance's code (LM_ERR_*); the
 * others' results are still written. */
int lm_batch_run(lm_batch *b, int n, const lm_batch_item *items, irl_result *results,
                 int *grid_out);
int lm_batch_free(lm_batch *b);

/* ---- serving: a request loop with continuous admission ---------------- */

typedef struct lm_server lm_server;

typedef struct {
    int64_t ticket;       /* as returned by lm_server_submit */
    int system_id;
    int status;           /* LM_OK or LM_ERR_* */
    int grid;             /* pencil-product CTAs the request used (lm_pencil_set_grid) */
    irl_result result;
    double t_submit_ms;   /* host steady-clock times of the request */
    double t_admit_ms;
    double t_done_ms;
} lm_response;

/* A server over n_streams streams (at most that many requests in flight)
 * that admits work only while the estimated device footprint of the resident
 * systems stays within hbm_budget_bytes (idle systems are evicted, least
 * recently used first, to make room). */
int lm_server_create(lm_ctx *ctx, size_t hbm_budget_bytes, int n_streams, int autotune,
                     lm_server **out);
/* Register a system: its integrals, rows and weights are copied into the
 * server (host memory); its pencil is created on first admission and stays
 * resident across requests. Returns its id in *system_id. */
int lm_server_add_system(lm_server *srv, const lm_system *sys, const uint64_t *rows,
                         const double *weights, int64_t n_rows, int precision, int *system_id);
/* Queue one LM-step request: theta (host, P entries, copied now), the IRL
 * settings; dtheta_out (host, P, nullable) is written when the request
 * completes. Requests for one system run one at a time, in order. */
int lm_server_submit(lm_server *srv, int system_id, const double *theta,
                     const irl_params *prm, double *dtheta_out, int64_t *ticket);
/* Advance all in-flight work without blocking: admit queued requests that
 * fit, move every in-flight request whose device work has completed to its
 * next stage, and return up to cap finished responses (*n_out of them). */
int lm_server_poll(lm_server *srv, lm_response *out, int cap, int *n_out);
/* Requests submitted but not yet returned by lm_server_poll. */
int lm_server_pending(lm_server *srv, int *n);
int lm_server_free(lm_server *srv);

/* ---- counters (benchmarking; not on the math path) -------------------- */

typedef struct {
    int64_t launches;      /* kernels this context launched since the last reset */
    double build_ms;       /* summed device time of the row-build kernel launches */
    int64_t build_count;
    double pencil_ms;      /* summed device time of the pencil kernel launches    */
    int64_t pencil_count;
    int64_t pencil_rows;   /* rows streamed by those pencil launches               */
    double lanczos_ms;     /* Lanczos step vector kernels (one interval per step)  */
    int64_t lanczos_count;
    double prep_ms;        /* weights, statistics and centring after a build       */
    int64_t prep_count;
    double tri_ms;         /* tridiagonal eigen-solve / shift kernel (per cycle)   */
    int64_t tri_count;
} lm_stats;

/* Kernel classes for lm_stats_reset's profile argument */
#define LM_PROF_ONLY    0x100 /* with class bits: bracket only those classes  */
#define LM_PROF_BUILD   0x01  /* row build                                    */
#define LM_PROF_PENCIL  0x02  /* pencil products                              */
#define LM_PROF_LANCZOS 0x04  /* Lanczos steps                                */
#define LM_PROF_PREP    0x08  /* preparation (weights, statistics, centring)  */
#define LM_PROF_TRI     0x10  /* tridiagonal eigen-solve / shifts             */

/* Reset the counters. profile = 1 also brackets every row-build, pencil,
 * Lanczos-step, preparation and tridiagonal launch (or launch sequence) with
 * CUDA events recorded on the launch stream, until the next reset (at most
 * 2048 intervals per class are timed); profile = LM_PROF_ONLY | class bits
 * brackets only those classes (each event pair adds a few microseconds to the
 * stream, so a caller timing whole steps may want only the class it studies);
 * 0 counts launches only. Timed classes report their timed intervals as
 * counts, the others their launches. lm_stats_get synchronises the device
 * before reading the events. Errors: LM_ERR_ARG (null context, or a profile
 * value other than 0, 1 or LM_PROF_ONLY with class bits). */
int lm_stats_reset(lm_ctx *ctx, int profile);
int lm_stats_get(lm_ctx *ctx, lm_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* IRLNQS_H */
