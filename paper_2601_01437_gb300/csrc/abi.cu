// C ABI of the library: contexts, pencil lifecycle, host/device pointer
// handling and the non-IRL entry points (irl_step lives in irl.cu).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstddef>
#include <cstring>

#include "internal.cuh"

// ---------------------------------------------------------------- helpers
int lm_fail(lm_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int lm_cuda_check(lm_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LM_OK;
    if (e == cudaErrorMemoryAllocation)
        return lm_fail(ctx, LM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return lm_fail(ctx, LM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool lm_is_pageable(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeUnregistered;
}

double *lm_stage_irl(lm_pencil *p, int which) {
    return reinterpret_cast<double *>(p->hstage + p->st_out) + (size_t)which * p->ldp;
}

int lm_stage_h2d(lm_pencil *p, void *dst, const void *src, size_t n, size_t off, cudaStream_t s) {
    if (n == 0) return LM_OK;
    cudaMemcpyKind kind = cudaMemcpyHostToDevice;
    if (lm_is_device_ptr(src)) {
        kind = cudaMemcpyDeviceToDevice;
    } else if (lm_is_pageable(src)) {
        std::memcpy(p->hstage + off, src, n);
        src = p->hstage + off;
    }
    return lm_cuda_check(p->ctx, cudaMemcpyAsync(dst, src, n, kind, s), "input copy");
}

bool lm_is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int lm_read_flags(lm_ctx *ctx, cudaStream_t s, int *flags) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && h) e = cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), s);
    *flags = h;
    return lm_cuda_check(ctx, e, "flag read-back");
}

namespace {

// copy n bytes from a caller pointer (host or device) into device memory
int to_device(lm_ctx *ctx, void *dst, const void *src, size_t n, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(dst, src, n,
                                    lm_is_device_ptr(src) ? cudaMemcpyDeviceToDevice
                                                          : cudaMemcpyHostToDevice,
                                    s);
    return lm_cuda_check(ctx, e, "input copy");
}

// copy from device memory to a caller pointer; returns whether a sync is needed
int from_device(lm_ctx *ctx, void *dst, const void *src, size_t n, cudaStream_t s, bool &host) {
    host = !lm_is_device_ptr(dst);
    cudaError_t e = cudaMemcpyAsync(dst, src, n,
                                    host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
    return lm_cuda_check(ctx, e, "output copy");
}

int64_t binom_host(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t c = 1;
    for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
    return c;
}

template <typename T>
int dalloc(lm_ctx *ctx, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return lm_cuda_check(ctx, cudaMalloc((void **)p, count * sizeof(T)), "cudaMalloc");
}

void pencil_release(lm_pencil *p) {
    if (!p) return;
    void *bufs[] = {p->rows, p->wt,   p->lnpsi, p->eloc, p->O,    p->G,   p->Olo,
                    p->Glo,  p->h,    p->eri,   p->theta, p->tabs, p->stats, p->part,
                    p->V,    p->wvec, p->yvec,  p->hy,   p->sy,   p->tvec, p->dots,
                    p->st,   p->tdf,  p->wlo, p->wel, p->wello, p->bar, p->shv, p->blz,
                    p->cstats, p->rt, p->rt64, p->psim, p->psie};
    for (void *b : bufs)
        if (b) cudaFree(b);
    lm_block_release(p);
    lm_cycle_graphs_release(p);
    if (p->hs) cudaFreeHost(p->hs);
    if (p->hstage) cudaFreeHost(p->hstage);
    delete p;
}

int check_system(lm_ctx *ctx, const lm_system *sys) {
    if (!sys || !sys->h || !sys->eri) return lm_fail(ctx, LM_ERR_ARG, "null system or integrals");
    const int n = sys->n_orb;
    if (n < 1 || 2 * n > LM_MAXM)
        return lm_fail(ctx, LM_ERR_SIZE, "2*n_orb = %d outside [2, 64]", 2 * n);
    if (sys->n_alpha < 0 || sys->n_beta < 0 || sys->n_alpha > n || sys->n_beta > n)
        return lm_fail(ctx, LM_ERR_SIZE, "electron counts (%d, %d) outside [0, %d]", sys->n_alpha,
                       sys->n_beta, n);
    if (sys->n_hidden < 0 || sys->n_hidden > 127)
        return lm_fail(ctx, LM_ERR_SIZE, "n_hidden = %d outside [0, 127]", sys->n_hidden);
    return LM_OK;
}

}  // namespace

// ---------------------------------------------------------------- context
extern "C" int lm_create(lm_ctx **out, int device, const lm_ctx_params *params) {
    if (!out) return LM_ERR_ARG;
    *out = nullptr;
    // the caller's view of the options, fields it did not compile in at their defaults
    lm_ctx_params prm = {sizeof(lm_ctx_params), 0, 0.0};
    if (params) {
        if (params->struct_size < offsetof(lm_ctx_params, hbm_gbs)) return LM_ERR_ARG;
        std::memcpy(&prm, params, std::min<size_t>(params->struct_size, sizeof(prm)));
        if (!(prm.hbm_gbs >= 0.0)) return LM_ERR_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return LM_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return LM_ERR_CUDA;
    lm_ctx *c = new lm_ctx();
    c->device = device;
    c->err[0] = 0;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    {
        // streaming rate: 85 % of the interface's peak (double data rate x bus
        // width), about what a copy kernel sustains on HBM3e
        int khz = 0, bits = 0;
        cudaDeviceGetAttribute(&khz, cudaDevAttrMemoryClockRate, device);
        cudaDeviceGetAttribute(&bits, cudaDevAttrGlobalMemoryBusWidth, device);
        c->hbm_bytes_per_ms = prm.hbm_gbs > 0.0 ? prm.hbm_gbs * 1e6
                                                : 0.85 * 2.0 * (double)khz * (bits / 8);
    }
    cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (cudaMalloc(&c->d_flags, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->d_flags, 0, sizeof(int)) != cudaSuccess) {
        delete c;
        return LM_ERR_OOM;
    }
    if (prm.profile && lm_stats_reset(c, prm.profile) != LM_OK) {
        cudaFree(c->d_flags);
        delete c;
        return LM_ERR_CUDA;
    }
    *out = c;
    return LM_OK;
}

extern "C" int lm_destroy(lm_ctx *ctx) {
    if (!ctx) return LM_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaFree(ctx->d_flags);
    if (ctx->ev_ready)
        for (int c = 0; c < LM_PROF_CLASSES; ++c)
            for (int i = 0; i < LM_PROF_EVENTS; ++i)
                for (int k = 0; k < 2; ++k) cudaEventDestroy(ctx->ev[c][i][k]);
    delete ctx;
    return LM_OK;
}

extern "C" const char *lm_last_error(const lm_ctx *ctx) { return ctx ? ctx->err : "null context"; }

// ---------------------------------------------------------------- build
int lm_build_enqueue(lm_ctx *ctx, const lm_system *sys, const double *theta,
                     const uint64_t *rows, const double *weights, int64_t n_rows,
                     lm_precision prec, void *stream, lm_pencil **inout, int rows_only,
                     int64_t chunk_rows, int gfree) {
    if (!ctx || !inout || !theta) return lm_fail(ctx, LM_ERR_ARG, "null argument");
    ctx->err[0] = 0;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return LM_ERR_CUDA;
    if (int rc = check_system(ctx, sys)) return rc;
    if (prec != LM_FP64 && prec != LM_FP32 && prec != LM_BF16 && prec != LM_DF64)
        return lm_fail(ctx, LM_ERR_ARG, "bad precision %d", (int)prec);
    cudaStream_t s = (cudaStream_t)stream;
    const int n = sys->n_orb, M = 2 * n, nh = sys->n_hidden;
    const int P1 = (nh + 1) * (M + 1);
    const int ldp = (P1 + 7) / 8 * 8;
    if (P1 > 2048) return lm_fail(ctx, LM_ERR_SIZE, "P+1 = %d above 2048", P1);
    const bool enumerate = rows == nullptr;
    if (enumerate) {
        const int64_t cnt = binom_host(n, sys->n_alpha) * binom_host(n, sys->n_beta);
        if (n_rows != 0 && n_rows != cnt)
            return lm_fail(ctx, LM_ERR_SIZE, "n_rows = %lld but the sector has %lld",
                           (long long)n_rows, (long long)cnt);
        n_rows = cnt;
    }
    if (n_rows < 1) return lm_fail(ctx, LM_ERR_SIZE, "no rows");

    lm_pencil *p = *inout;
    if (p) {
        if (p->ctx != ctx || p->n != n || p->na != sys->n_alpha || p->nb != sys->n_beta ||
            p->nh != nh || p->n_rows != n_rows || p->prec != (int)prec || p->gfree != gfree ||
            p->chunk != (chunk_rows > 0 ? std::min(chunk_rows, n_rows) : 0))
            return lm_fail(ctx, LM_ERR_ARG, "pencil shape differs from the requested build");
    } else {
        p = new lm_pencil();
        std::memset(p, 0, sizeof(lm_pencil));
        p->ctx = ctx;
        p->n = n;
        p->na = sys->n_alpha;
        p->nb = sys->n_beta;
        p->nh = nh;
        p->M = M;
        p->M1 = M + 1;
        p->P1 = P1;
        p->ldp = ldp;
        p->n_rows = n_rows;
        p->prec = prec;
        p->gfree = gfree;
        p->g_pencil = lm_pencil_grid(p);
        p->chunk = chunk_rows > 0 ? std::min(chunk_rows, n_rows) : 0;
        const size_t nr = (size_t)n_rows, L = (size_t)ldp;
        // O, G and their copies hold every row, or one chunk of a streamed pencil
        const size_t nrf = p->chunk ? (size_t)p->chunk : nr;
        const int nst = (int)std::min<int64_t>(n_rows, ctx->sms * 2);
        p->part_len = std::max<int64_t>((int64_t)p->g_pencil * 2 * L, 256 + (int64_t)nst * (L + 2));
        int rc = 0;
        rc = rc ? rc : dalloc(ctx, &p->rows, nr);
        rc = rc ? rc : dalloc(ctx, &p->wt, nr);
        rc = rc ? rc : dalloc(ctx, &p->wlo, nr);
        rc = rc ? rc : dalloc(ctx, &p->wel, nr);
        rc = rc ? rc : dalloc(ctx, &p->wello, nr);
        rc = rc ? rc : dalloc(ctx, &p->lnpsi, nr);
        rc = rc ? rc : dalloc(ctx, &p->eloc, nr);
        rc = rc ? rc : dalloc(ctx, &p->O, nrf * L);
        if (!gfree) rc = rc ? rc : dalloc(ctx, &p->G, nrf * L);
        if (!rc && prec != LM_FP64) {
            const size_t es = prec == LM_FP32 ? 4 : (prec == LM_DF64 ? 8 : 2);
            rc = lm_cuda_check(ctx, cudaMalloc(&p->Olo, nrf * L * es), "cudaMalloc");
            if (!gfree)
                rc = rc ? rc : lm_cuda_check(ctx, cudaMalloc(&p->Glo, nrf * L * es), "cudaMalloc");
        }
        if (!rc && p->chunk) {
            const size_t nch = (nr + p->chunk - 1) / p->chunk;
            rc = dalloc(ctx, &p->cstats, nch * (8 + L));
            rc = rc ? rc : dalloc(ctx, &p->shv, 2 * L);
        }
        rc = rc ? rc : dalloc(ctx, &p->h, (size_t)n * n);
        rc = rc ? rc : dalloc(ctx, &p->eri, (size_t)n * n * n * n);
        rc = rc ? rc : dalloc(ctx, &p->theta, L);
        rc = rc ? rc : dalloc(ctx, &p->tabs, (size_t)2 * nh * M + 2 * M + 8);
        rc = rc ? rc
                : dalloc(ctx, &p->tdf, (size_t)2 * nh * M + 2 * M + (size_t)n * n +
                                           (size_t)n * n * n * n + 8);
        rc = rc ? rc : dalloc(ctx, &p->stats, 8 + L);
        rc = rc ? rc : dalloc(ctx, &p->part, (size_t)p->part_len);
        rc = rc ? rc : dalloc(ctx, &p->V, 2 * (LM_MAXKRYLOV + 1) * L);
        rc = rc ? rc : dalloc(ctx, &p->wvec, L);
        rc = rc ? rc : dalloc(ctx, &p->yvec, L);
        rc = rc ? rc : dalloc(ctx, &p->hy, L);
        rc = rc ? rc : dalloc(ctx, &p->sy, L);
        rc = rc ? rc : dalloc(ctx, &p->tvec, L);
        rc = rc ? rc : dalloc(ctx, &p->dots, (size_t)3 * (nh + 1) * (LM_MAXKRYLOV + 8) + L + 64);
        rc = rc ? rc : dalloc(ctx, &p->st, 1);
        rc = rc ? rc : dalloc(ctx, &p->bar, 64);
        if (!rc) rc = lm_cuda_check(ctx, cudaMemsetAsync(p->bar, 0, 64 * sizeof(unsigned), s), "memset");
        if (!rc)
            rc = lm_cuda_check(ctx, cudaMallocHost(&p->hs, sizeof(PencilHost)), "cudaMallocHost");
        if (!rc) {
            const size_t in_fixed = 8 * ((size_t)n * n + (size_t)n * n * n * n + L);
            p->st_in_rows = (in_fixed + 255) / 256 * 256;
            p->st_in_w = p->st_in_rows + (8 * nr + 255) / 256 * 256;
            p->st_out = p->st_in_w + (8 * nr + 255) / 256 * 256;
            rc = lm_cuda_check(ctx, cudaMallocHost(&p->hstage, p->st_out + 4 * 8 * L + 256),
                               "cudaMallocHost");
        }
        if (!rc) {
            p->st_host = &p->hs->st;
            p->d_flags = &p->st->flags;
            rc = lm_cuda_check(ctx, cudaMemsetAsync(p->st, 0, sizeof(IrlState), s), "memset");
        }
        if (rc) {
            pencil_release(p);
            return rc;
        }
        cudaMemsetAsync(p->V, 0, 2 * (LM_MAXKRYLOV + 1) * L * sizeof(double), s);
        *inout = p;
    }
    const bool have_sector = p->enumerated;  // a pencil rebuilt in place keeps its rows
    p->enumerated = enumerate;
    p->given_weights = weights != nullptr;
    p->sym = gfree ? LM_SYM_ELOC : enumerate ? LM_SYM_NONE : LM_SYM_HALF;
    p->e_core = sys->e_core;
    if (sys->build_arith != LM_ARITH_DF64 && sys->build_arith != LM_ARITH_FP64)
        return lm_fail(ctx, LM_ERR_ARG, "bad build_arith %d", sys->build_arith);
    if (gfree && sys->build_arith != LM_ARITH_DF64)
        return lm_fail(ctx, LM_ERR_ARG, "the G-free build runs in double-float arithmetic");
    p->arith = sys->build_arith;
    int rc = 0;
    const size_t nn = (size_t)n * n;
    rc = rc ? rc : lm_stage_h2d(p, p->h, sys->h, sizeof(double) * nn, 0, s);
    rc = rc ? rc : lm_stage_h2d(p, p->eri, sys->eri, sizeof(double) * nn * nn, 8 * nn, s);
    rc = rc ? rc : lm_stage_h2d(p, p->theta, theta, sizeof(double) * (P1 - 1),
                                8 * (nn + nn * nn), s);
    if (rc) return rc;
    if (enumerate) {
        if (!have_sector &&
            (rc = lm_launch_enumerate(ctx, n, sys->n_alpha, sys->n_beta, p->rows, n_rows, s)))
            return rc;
    } else if ((rc = lm_stage_h2d(p, p->rows, rows, sizeof(uint64_t) * n_rows, p->st_in_rows,
                                  s))) {
        return rc;
    }
    if (weights &&
        (rc = lm_stage_h2d(p, p->wt, weights, sizeof(double) * n_rows, p->st_in_w, s)))
        return rc;
    if ((rc = lm_cuda_check(ctx, cudaMemsetAsync(p->d_flags, 0, sizeof(int), s), "memset")))
        return rc;
    p->shard_state = rows_only ? 1 : 0;
    if (p->chunk) {
        if ((rc = lm_launch_stream_stats(p, s))) return rc;
        cudaError_t e = cudaMemcpyAsync(&p->hs->E, p->stats + 1, sizeof(double),
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&p->hs->flags, p->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s);
        return lm_cuda_check(ctx, e, "energy read-back");
    }
    if (rows_only) {
        if ((rc = lm_launch_build_rows(p, s))) return rc;
        return lm_cuda_check(ctx, cudaMemcpyAsync(&p->hs->flags, p->d_flags, sizeof(int),
                                                  cudaMemcpyDeviceToHost, s),
                             "flags read-back");
    }
    if ((rc = lm_launch_build(p, s))) return rc;
    cudaError_t e = cudaMemcpyAsync(&p->hs->E, p->stats + 1, sizeof(double),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&p->hs->flags, p->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    return lm_cuda_check(ctx, e, "energy read-back");
}

int lm_build_finish(lm_pencil *p) {
    p->E_host = p->hs->E;
    if (p->hs->flags & FLAG_ROW_OUTSIDE_SECTOR)
        return lm_fail(p->ctx, LM_ERR_ARG, "a row lies outside the (N_alpha, N_beta) sector");
    if (p->hs->flags & FLAG_TIMEOUT)
        return lm_fail(p->ctx, LM_ERR_TIMEOUT, "a bounded wait of the build timed out");
    return LM_OK;
}

extern "C" int lm_build_OG(lm_ctx *ctx, const lm_system *sys, const double *theta,
                           const uint64_t *rows, const double *weights, int64_t n_rows,
                           lm_precision prec, void *stream, lm_pencil **inout) {
    if (int rc = lm_build_enqueue(ctx, sys, theta, rows, weights, n_rows, prec, stream, inout))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = lm_cuda_check(ctx, cudaStreamSynchronize(s), "build")) return rc;
    return lm_build_finish(*inout);
}

// The E_loc estimator's pencil (Methods, eq. matrix_vec_prod with E_loc in
// place of the G form): the build forms O, ln psi and E_loc, never G.
extern "C" int lm_build_O(lm_ctx *ctx, const lm_system *sys, const double *theta,
                          const uint64_t *rows, const double *weights, int64_t n_rows,
                          lm_precision prec, void *stream, lm_pencil **inout) {
    if (int rc = lm_build_enqueue(ctx, sys, theta, rows, weights, n_rows, prec, stream, inout, 0,
                                  0, 1))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = lm_cuda_check(ctx, cudaStreamSynchronize(s), "build")) return rc;
    return lm_build_finish(*inout);
}

// ---------------------------------------------------------------- streamed rows
extern "C" int lm_build_streamed(lm_ctx *ctx, const lm_system *sys, const double *theta,
                                 const uint64_t *rows, const double *weights, int64_t n_rows,
                                 int64_t chunk_rows, lm_precision prec, void *stream,
                                 lm_pencil **inout) {
    if (chunk_rows < 1) return lm_fail(ctx, LM_ERR_ARG, "chunk_rows must be positive");
    if (int rc = lm_build_enqueue(ctx, sys, theta, rows, weights, n_rows, prec, stream, inout, 0,
                                  chunk_rows))
        return rc;
    if (int rc = lm_cuda_check(ctx, cudaStreamSynchronize((cudaStream_t)stream), "build"))
        return rc;
    return lm_build_finish(*inout);
}

// ---------------------------------------------------------------- row shards
extern "C" int lm_shard_build(lm_ctx *ctx, const lm_system *sys, const double *theta,
                              const uint64_t *rows, const double *weights, int64_t n_rows,
                              lm_precision prec, void *stream, lm_pencil **inout,
                              double *lnpsi_max) {
    if (!lnpsi_max) return lm_fail(ctx, LM_ERR_ARG, "null lnpsi_max");
    if (int rc = lm_build_enqueue(ctx, sys, theta, rows, weights, n_rows, prec, stream, inout, 1))
        return rc;
    lm_pencil *p = *inout;
    cudaStream_t s = (cudaStream_t)stream;
    int nmax = 0;
    if (int rc = lm_launch_shard_max(p, s, &nmax)) return rc;
    if (int rc = lm_cuda_check(ctx, cudaMemcpyAsync(p->hs->xfer, p->part, nmax * sizeof(double),
                                                    cudaMemcpyDeviceToHost, s),
                               "shard max read-back"))
        return rc;
    if (int rc = lm_cuda_check(ctx, cudaStreamSynchronize(s), "lm_shard_build")) return rc;
    p->hs->E = NAN;
    if (int rc = lm_build_finish(p)) return rc;
    double m = -INFINITY;
    for (int i = 0; i < nmax; ++i) m = std::max(m, p->hs->xfer[i]);
    *lnpsi_max = m;
    return LM_OK;
}

extern "C" int lm_shard_sums(lm_pencil *p, double lnpsi_max, double *sums, void *stream) {
    if (!p || !sums) return LM_ERR_ARG;
    lm_ctx *ctx = p->ctx;
    cudaSetDevice(ctx->device);
    if (p->shard_state != 1 && p->shard_state != 2)
        return lm_fail(ctx, LM_ERR_ARG, "lm_shard_sums needs a pencil from lm_shard_build");
    if (!p->given_weights && !std::isfinite(lnpsi_max))
        return lm_fail(ctx, LM_ERR_ARG, "lnpsi_max must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = lm_launch_shard_sums(p, lnpsi_max, s)) return rc;
    if (int rc = lm_cuda_check(ctx, cudaMemcpyAsync(p->hs->xfer, p->stats,
                                                    (8 + p->ldp) * sizeof(double),
                                                    cudaMemcpyDeviceToHost, s),
                               "shard sums read-back"))
        return rc;
    if (int rc = lm_cuda_check(ctx, cudaStreamSynchronize(s), "lm_shard_sums")) return rc;
    const double *st = p->hs->xfer;
    sums[0] = st[0];
    sums[1] = st[1];
    for (int k = 0; k < p->P1; ++k) sums[2 + k] = st[8 + k];
    p->shard_state = 2;
    return LM_OK;
}

extern "C" int lm_shard_centre(lm_pencil *p, const double *sums, void *stream) {
    if (!p || !sums) return LM_ERR_ARG;
    lm_ctx *ctx = p->ctx;
    cudaSetDevice(ctx->device);
    if (p->shard_state != 2)
        return lm_fail(ctx, LM_ERR_ARG, "lm_shard_centre needs lm_shard_sums first");
    if (!(sums[0] > 0.0) || !std::isfinite(sums[0]))
        return lm_fail(ctx, LM_ERR_ARG, "the summed weight must be positive and finite");
    cudaStream_t s = (cudaStream_t)stream;
    // the statistics the unsharded build forms on the device, from the sums of
    // every shard: sum w, E = sum w E_loc / sum w, <O_k> = sum w O_k / sum w
    double *st = p->hs->xfer;
    std::memset(st, 0, (8 + p->ldp) * sizeof(double));
    st[0] = sums[0];
    st[1] = sums[1] / sums[0];
    for (int k = 0; k < p->P1; ++k) st[8 + k] = sums[2 + k] / sums[0];
    if (int rc = lm_cuda_check(ctx, cudaMemcpyAsync(p->stats, st, (8 + p->ldp) * sizeof(double),
                                                    cudaMemcpyHostToDevice, s),
                               "shard statistics"))
        return rc;
    if (int rc = lm_launch_centre(p, s)) return rc;
    if (int rc = lm_cuda_check(ctx, cudaStreamSynchronize(s), "lm_shard_centre")) return rc;
    p->hs->E = sums[1] / sums[0];
    p->E_host = p->hs->E;
    p->shard_state = 0;
    return LM_OK;
}

extern "C" int lm_apply_pencil(lm_pencil *p, const double *v, double *Hv, double *Sv, int sym,
                               int prec, void *stream) {
    if (!p || !v) return LM_ERR_ARG;
    lm_ctx *ctx = p->ctx;
    cudaSetDevice(ctx->device);
    if (sym < 0 || sym > 3 || prec < 0 || prec > 3) return lm_fail(ctx, LM_ERR_ARG, "bad sym/prec");
    if (p->shard_state) return lm_fail(ctx, LM_ERR_ARG, "row shard not centred (lm_shard_centre)");
    cudaStream_t s = (cudaStream_t)stream;
    const int sy = sym == LM_SYM_AUTO ? p->sym : sym;
    if (p->gfree && sy != LM_SYM_ELOC)
        return lm_fail(ctx, LM_ERR_ARG, "a pencil without G'_c answers the E_loc estimator only");
    // the kernels read ldp >= P+1 entries: stage v with zero padding
    const bool v_host = !lm_is_device_ptr(v);
    cudaMemsetAsync(p->tvec, 0, p->ldp * sizeof(double), s);
    if (int rc = to_device(ctx, p->tvec, v, p->P1 * sizeof(double), s)) return rc;
    const double *vd = p->tvec;
    if (p->chunk) {
        if (int rc = lm_launch_stream_product(p, vd, sy, prec, Sv != nullptr, p->hy, p->sy, s))
            return rc;
    } else {
        if (int rc = lm_launch_pencil(p, vd, sy, prec, Sv != nullptr, nullptr, s)) return rc;
        if (int rc = lm_launch_reduce_partials(p, prec, p->hy, p->sy, s)) return rc;
    }
    bool h1 = false, h2 = false;
    if (Hv)
        if (int rc = from_device(ctx, Hv, p->hy, p->P1 * sizeof(double), s, h1)) return rc;
    if (Sv)
        if (int rc = from_device(ctx, Sv, p->sy, p->P1 * sizeof(double), s, h2)) return rc;
    if (h1 || h2 || v_host)
        return lm_cuda_check(ctx, cudaStreamSynchronize(s), "lm_apply_pencil");
    return lm_cuda_check(ctx, cudaGetLastError(), "lm_apply_pencil");
}

extern "C" int lm_pencil_info_get(lm_pencil *p, lm_pencil_info *out) {
    if (!p || !out) return LM_ERR_ARG;
    out->n_rows = p->n_rows;
    out->n_params = p->P1 - 1;
    out->ld = p->ldp;
    out->precision = p->prec;
    out->sym = p->sym;
    out->energy = p->E_host;
    out->grid = p->g_pencil;
    return LM_OK;
}

extern "C" int lm_pencil_set_grid(lm_pencil *p, int ctas) {
    if (!p) return LM_ERR_ARG;
    if (ctas < 1 || ctas > p->ctx->sms)
        return lm_fail(p->ctx, LM_ERR_ARG, "pencil grid %d outside 1..%d", ctas, p->ctx->sms);
    p->g_pencil = ctas;  // the partials buffer holds one vector pair per SM
    return LM_OK;
}

// Device bytes a pencil of this shape holds (the server's admission estimate).
size_t lm_pencil_footprint(lm_ctx *ctx, int n, int nh, int64_t n_rows, int prec) {
    const size_t M = 2 * n, P1 = (nh + 1) * (M + 1), L = (P1 + 7) / 8 * 8, nr = n_rows;
    const size_t es = prec == LM_FP64 ? 0 : (prec == LM_FP32 ? 4 : (prec == LM_DF64 ? 8 : 2));
    size_t b = nr * L * (16 + 2 * es);              // O, G and the low-precision copies
    b += nr * (8 * 7 + 8);                         // rows, weights (x4), ln psi, E_loc
    b += (size_t)n * n * n * n * 16 + 2 * 4 * nh * M * 8;  // integrals and tables
    b += (size_t)ctx->sms * 2 * L * 8;             // partial products
    b += 2 * (LM_MAXKRYLOV + 1) * L * 8 + 16 * L * 8 + (1 << 20);  // bases, vectors, state
    return b;
}

void lm_pencil_release(lm_pencil *p) { pencil_release(p); }

extern "C" int lm_pencil_free(lm_pencil *p) {
    if (!p) return LM_ERR_ARG;
    cudaSetDevice(p->ctx->device);
    cudaDeviceSynchronize();
    pencil_release(p);
    return LM_OK;
}

extern "C" int lm_pencil_export(lm_pencil *p, int what, void *dst, void *stream) {
    if (!p || !dst) return LM_ERR_ARG;
    lm_ctx *ctx = p->ctx;
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const void *src = nullptr;
    size_t bytes = 0;
    const size_t nr = (size_t)p->n_rows;
    if ((what == 0 || what == 1) && p->chunk)
        return lm_fail(ctx, LM_ERR_ARG, "a streamed pencil keeps no O_c, G'_c to export");
    if (what == 1 && p->gfree) return lm_fail(ctx, LM_ERR_ARG, "the pencil has no G'_c");
    if ((what == 0 || what == 1) && p->prec == LM_DF64 && p->Olo) {
        // the centred factors of a double-float pencil exist only as pairs:
        // convert into the (otherwise unused after the build) FP64 buffer
        double *dstd = what == 0 ? p->O : p->G;
        const float2 *srcp = (const float2 *)(what == 0 ? p->Olo : p->Glo);
        if (int rc = lm_launch_df_to_fp64(ctx, srcp, dstd, (int64_t)nr * p->ldp, s)) return rc;
    }
    switch (what) {
        case 0: src = p->O; bytes = nr * p->ldp * sizeof(double); break;
        case 1: src = p->G; bytes = nr * p->ldp * sizeof(double); break;
        case 2: src = p->lnpsi; bytes = nr * sizeof(double); break;
        case 3: src = p->eloc; bytes = nr * sizeof(double); break;
        case 4: src = p->wt; bytes = nr * sizeof(double); break;
        case 5: src = p->stats + 8; bytes = p->ldp * sizeof(double); break;
        case 6: src = p->rows; bytes = nr * sizeof(uint64_t); break;
        default: return lm_fail(ctx, LM_ERR_ARG, "unknown export %d", what);
    }
    bool host = false;
    if (int rc = from_device(ctx, dst, src, bytes, s, host)) return rc;
    return lm_cuda_check(ctx, cudaStreamSynchronize(s), "lm_pencil_export");
}

// ---------------------------------------------------------------- inspection
extern "C" int lm_enumerate_sector(lm_ctx *ctx, int n_orb, int n_alpha, int n_beta,
                                   uint64_t *out, int64_t cap, int64_t *count) {
    if (!ctx || !count) return LM_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (n_orb < 1 || 2 * n_orb > LM_MAXM || n_alpha < 0 || n_beta < 0 || n_alpha > n_orb ||
        n_beta > n_orb)
        return lm_fail(ctx, LM_ERR_SIZE, "bad sector (%d, %d, %d)", n_orb, n_alpha, n_beta);
    const int64_t cnt = binom_host(n_orb, n_alpha) * binom_host(n_orb, n_beta);
    *count = cnt;
    if (!out) return LM_OK;
    if (cap < cnt) return lm_fail(ctx, LM_ERR_SIZE, "capacity %lld < %lld", (long long)cap,
                                  (long long)cnt);
    const bool dev = lm_is_device_ptr(out);
    uint64_t *d = out;
    if (!dev && cudaMalloc(&d, cnt * sizeof(uint64_t)) != cudaSuccess)
        return lm_fail(ctx, LM_ERR_OOM, "cudaMalloc");
    int rc = lm_launch_enumerate(ctx, n_orb, n_alpha, n_beta, d, cnt, 0);
    if (!rc && !dev)
        rc = lm_cuda_check(ctx, cudaMemcpy(out, d, cnt * sizeof(uint64_t), cudaMemcpyDeviceToHost),
                           "copy");
    if (!dev) cudaFree(d);
    if (!rc) rc = lm_cuda_check(ctx, cudaDeviceSynchronize(), "enumerate");
    return rc;
}

extern "C" int lm_debug_connections(lm_ctx *ctx, const lm_system *sys, const uint64_t *rows,
                                    int64_t n_rows, int cap, uint64_t *out_det, int8_t *out_sign,
                                    double *out_h, int32_t *count) {
    if (!ctx || !rows || !out_det || !out_sign || !out_h || !count || cap < 1)
        return lm_fail(ctx, LM_ERR_ARG, "null argument");
    cudaSetDevice(ctx->device);
    if (int rc = check_system(ctx, sys)) return rc;
    const int n = sys->n_orb;
    double *dh = nullptr, *deri = nullptr, *doh = nullptr;
    uint64_t *drows = nullptr, *dod = nullptr;
    int8_t *dsg = nullptr;
    int32_t *dcnt = nullptr;
    const size_t tot = (size_t)n_rows * cap;
    int rc = 0;
    rc = rc ? rc : dalloc(ctx, &dh, (size_t)n * n);
    rc = rc ? rc : dalloc(ctx, &deri, (size_t)n * n * n * n);
    rc = rc ? rc : dalloc(ctx, &drows, (size_t)n_rows);
    rc = rc ? rc : dalloc(ctx, &dod, tot);
    rc = rc ? rc : dalloc(ctx, &dsg, tot);
    rc = rc ? rc : dalloc(ctx, &doh, tot);
    rc = rc ? rc : dalloc(ctx, &dcnt, (size_t)n_rows);
    rc = rc ? rc : to_device(ctx, dh, sys->h, sizeof(double) * n * n, 0);
    rc = rc ? rc : to_device(ctx, deri, sys->eri, sizeof(double) * n * n * n * n, 0);
    rc = rc ? rc : to_device(ctx, drows, rows, sizeof(uint64_t) * n_rows, 0);
    rc = rc ? rc
            : lm_launch_connections(ctx, n, sys->n_alpha, sys->n_beta, dh, deri, drows, n_rows,
                                    cap, dod, dsg, doh, dcnt, sys->e_core, 0);
    bool host;
    rc = rc ? rc : from_device(ctx, out_det, dod, tot * sizeof(uint64_t), 0, host);
    rc = rc ? rc : from_device(ctx, out_sign, dsg, tot, 0, host);
    rc = rc ? rc : from_device(ctx, out_h, doh, tot * sizeof(double), 0, host);
    rc = rc ? rc : from_device(ctx, count, dcnt, n_rows * sizeof(int32_t), 0, host);
    if (!rc) rc = lm_cuda_check(ctx, cudaDeviceSynchronize(), "lm_debug_connections");
    void *bufs[] = {dh, deri, drows, dod, dsg, doh, dcnt};
    for (void *b : bufs)
        if (b) cudaFree(b);
    return rc;
}

// ---------------------------------------------------------------- counters
extern "C" int lm_stats_reset(lm_ctx *ctx, int profile) {
    if (!ctx) return LM_ERR_ARG;
    const int all = (1 << LM_PROF_CLASSES) - 1;
    if (profile != 0 && profile != 1 && (!(profile & LM_PROF_ONLY) || (profile & ~(LM_PROF_ONLY | all))))
        return lm_fail(ctx, LM_ERR_ARG, "profile = %#x: 0, 1 or LM_PROF_ONLY with class bits", profile);
    cudaSetDevice(ctx->device);
    if (profile && !ctx->ev_ready) {
        for (int c = 0; c < LM_PROF_CLASSES; ++c)
            for (int i = 0; i < LM_PROF_EVENTS; ++i)
                for (int k = 0; k < 2; ++k)
                    if (cudaEventCreate(&ctx->ev[c][i][k]) != cudaSuccess)
                        return lm_fail(ctx, LM_ERR_CUDA, "cudaEventCreate");
        ctx->ev_ready = 1;
    }
    ctx->profile = profile != 0;
    ctx->prof_mask = profile == 1 ? all : profile & all;
    ctx->launches = 0;
    ctx->pencil_rows = 0;
    for (int c = 0; c < LM_PROF_CLASSES; ++c) ctx->ev_used[c] = ctx->ev_count[c] = 0;
    return LM_OK;
}

extern "C" int lm_stats_get(lm_ctx *ctx, lm_stats *out) {
    if (!ctx || !out) return LM_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (int rc = lm_cuda_check(ctx, cudaDeviceSynchronize(), "lm_stats_get")) return rc;
    double ms[LM_PROF_CLASSES] = {0.0};
    for (int c = 0; c < LM_PROF_CLASSES; ++c)
        for (int64_t i = 0; i < ctx->ev_used[c]; ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ctx->ev[c][i][0], ctx->ev[c][i][1]) == cudaSuccess) ms[c] += t;
        }
    out->launches = ctx->launches;
    out->build_ms = ms[PROF_BUILD];
    // timed classes report their timed intervals, the others their launches
    auto count = [&](int c) {
        return ctx->profile && ((ctx->prof_mask >> c) & 1) ? ctx->ev_used[c] : ctx->ev_count[c];
    };
    out->build_count = count(PROF_BUILD);
    out->pencil_ms = ms[PROF_PENCIL];
    out->pencil_count = count(PROF_PENCIL);
    out->pencil_rows = ctx->pencil_rows;
    out->lanczos_ms = ms[PROF_LANCZOS];
    out->lanczos_count = count(PROF_LANCZOS);
    out->prep_ms = ms[PROF_PREP];
    out->prep_count = count(PROF_PREP);
    out->tri_ms = ms[PROF_TRI];
    out->tri_count = count(PROF_TRI);
    return LM_OK;
}
