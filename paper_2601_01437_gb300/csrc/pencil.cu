// The hot matvec of the method: the matrix-free application of the centred
// linear-method pencil (arXiv 2601.01437, Methods, "Practical Matrix-Free
// Implementation", eq. matrix_vec_prod, with the G form of eq. heff):
//
//   y_H = O_c^T W (G'_c v)                          (sym NONE)
//   y_H = 1/2 (O_c^T W (G'_c v) + G'_c^T W (O_c v)) (sym HALF)
//   y_S = O_c^T W (O_c v)
//
// One pass over O_c and G'_c. Each CTA owns a contiguous block of rows and
// streams it through shared memory in tiles of R rows with the bulk-copy
// (TMA) engine: one 1-D cp.async.bulk per matrix per tile (a tile of
// consecutive rows of a row-major matrix is one contiguous range), completion
// tracked by an mbarrier per pipeline stage. Each warp owns whole rows: the
// row dot is a 5-step butterfly, and the update of the warp's register-
// resident y uses the same staged row. y_S is a second, O-only pass. Each CTA
// writes its partial y; a second kernel sums the partials in CTA order
// (deterministic).
#include <algorithm>

#include "internal.cuh"

namespace {

constexpr int PT = 256;  // threads per pencil CTA

template <typename T>
struct Acc {
    using type = float;
};
template <>
struct Acc<double> {
    using type = double;
};

template <typename T>
__device__ __forceinline__ typename Acc<T>::type ld_s(const T *p) {
    return (typename Acc<T>::type)(*p);
}
template <>
__device__ __forceinline__ float ld_s<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat162float(*p);
}

enum { MODE_H_NONE = 0, MODE_H_HALF = 1, MODE_S = 2 };

template <typename T>
struct PencilArgs {
    const T *O;
    const T *G;
    const double *w;
    int64_t n_rows;
    int ldp;
    const double *v;
    double *out;    // [gridDim.x][out_ld]: this CTA's partial y
    int out_ld;
    int stages;
    int rows_per_tile;
    const int *skip;
    int *flags;
};

// One warp per row: lane l owns columns l, l+32, ... of the row, so a row dot
// is one 5-step butterfly and the rank-1 update of the warp's y accumulators
// (registers) reuses the staged row. MODE_H_NONE: y += w (G.v) O;
// MODE_H_HALF: y += w/2 ((G.v) O + (O.v) G); MODE_S: y += w (O.v) O (only O
// is staged). At the end the 8 warps' accumulators are summed in warp order.
template <typename T, int NJ, int MODE>
__global__ void __launch_bounds__(PT) k_pencil(PencilArgs<T> a) {
    using AT = typename Acc<T>::type;
    extern __shared__ __align__(128) unsigned char smraw[];
    if (a.skip && *a.skip) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ldp = a.ldp, R = a.rows_per_tile;
    const int nmat = MODE == MODE_S ? 1 : 2;
    const size_t tile_elems = (size_t)R * ldp;
    T *stage_base = reinterpret_cast<T *>(smraw);
    const size_t stage_bytes_all = (size_t)a.stages * nmat * tile_elems * sizeof(T);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smraw + stage_bytes_all);
    AT *vs = reinterpret_cast<AT *>(bars + 8);  // v in the compute type, ldp entries
    __shared__ int s_ok;

    const int64_t r0 = a.n_rows * blockIdx.x / gridDim.x;
    const int64_t r1 = a.n_rows * (blockIdx.x + 1) / gridDim.x;
    const int ntiles = (int)((r1 - r0 + R - 1) / R);
    const int nj = (ldp + 31) >> 5;

    if (tid == 0) {
        for (int s = 0; s < a.stages; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    for (int c = tid; c < ldp; c += PT) vs[c] = (AT)a.v[c];
    __syncthreads();

    auto issue = [&](int i) {
        const int s = i % a.stages;
        const int64_t row = r0 + (int64_t)i * R;
        const int nr = (int)min((int64_t)R, r1 - row);
        const uint32_t bytes = (uint32_t)((size_t)nr * ldp * sizeof(T));
        T *dO = stage_base + (size_t)s * nmat * tile_elems;
        mbar_arrive_expect_tx(&bars[s], nmat * bytes);
        bulk_g2s(dO, a.O + row * ldp, bytes, &bars[s]);
        if (MODE != MODE_S) bulk_g2s(dO + tile_elems, a.G + row * ldp, bytes, &bars[s]);
    };
    if (tid == 0)
        for (int i = 0; i < min(a.stages, ntiles); ++i) issue(i);

    AT y[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) y[j] = 0;

    int consumed = 0;
    bool ok = true;
    for (int i = 0; i < ntiles; ++i) {
        const int s = i % a.stages;
        const uint32_t par = (uint32_t)((i / a.stages) & 1);
        if (tid == 0) s_ok = mbar_wait_bounded(&bars[s], par) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
            ok = false;
            break;
        }
        consumed = i + 1;
        const int64_t row0 = r0 + (int64_t)i * R;
        const int nr = (int)min((int64_t)R, r1 - row0);
        const T *tO = stage_base + (size_t)s * nmat * tile_elems;
        const T *tG = tO + tile_elems;
        for (int r = warp; r < nr; r += PT / 32) {
            const T *ro = tO + (size_t)r * ldp;
            const T *rg = tG + (size_t)r * ldp;
            AT dg = 0, dov = 0;
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                if (j < nj) {
                    const int c = lane + 32 * j;
                    if (c < ldp) {
                        if (MODE != MODE_S) dg += ld_s(rg + c) * vs[c];
                        if (MODE != MODE_H_NONE) dov += ld_s(ro + c) * vs[c];
                    }
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                if (MODE != MODE_S) dg += __shfl_xor_sync(0xffffffffu, dg, off);
                if (MODE != MODE_H_NONE) dov += __shfl_xor_sync(0xffffffffu, dov, off);
            }
            const AT wr = (AT)a.w[row0 + r];
            if (MODE == MODE_H_NONE) {
                const AT cg = wr * dg;
#pragma unroll
                for (int j = 0; j < NJ; ++j)
                    if (j < nj) {
                        const int c = lane + 32 * j;
                        if (c < ldp) y[j] += cg * ld_s(ro + c);
                    }
            } else if (MODE == MODE_H_HALF) {
                const AT cg = (AT)0.5 * wr * dg, co = (AT)0.5 * wr * dov;
#pragma unroll
                for (int j = 0; j < NJ; ++j)
                    if (j < nj) {
                        const int c = lane + 32 * j;
                        if (c < ldp) y[j] += cg * ld_s(ro + c) + co * ld_s(rg + c);
                    }
            } else {
                const AT co = wr * dov;
#pragma unroll
                for (int j = 0; j < NJ; ++j)
                    if (j < nj) {
                        const int c = lane + 32 * j;
                        if (c < ldp) y[j] += co * ld_s(ro + c);
                    }
            }
        }
        __syncthreads();
        if (tid == 0 && i + a.stages < ntiles) issue(i + a.stages);
    }
    if (!ok) {
        // Drain the copies this CTA issued but did not consume before exiting.
        if (tid == 0) {
            atomicOr(a.flags, FLAG_TIMEOUT);
            const int issued = min(ntiles, consumed + a.stages);
            for (int i = consumed; i < issued; ++i)
                (void)mbar_wait_bounded(&bars[i % a.stages], (uint32_t)((i / a.stages) & 1));
        }
        __syncthreads();
        return;
    }
    // Sum the 8 warps' accumulators in warp order (staging buffers are free now).
    double *ys = reinterpret_cast<double *>(smraw);  // [8][ldp] FP64
#pragma unroll
    for (int j = 0; j < NJ; ++j)
        if (j < nj) {
            const int c = lane + 32 * j;
            if (c < ldp) ys[(size_t)warp * ldp + c] = (double)y[j];
        }
    __syncthreads();
    double *out = a.out + (size_t)blockIdx.x * a.out_ld;
    for (int c = tid; c < ldp; c += PT) {
        double t = 0.0;
#pragma unroll
        for (int w8 = 0; w8 < PT / 32; ++w8) t += ys[(size_t)w8 * ldp + c];
        out[c] = t;
    }
}

// y[c] = sum_b part[b][c] in CTA order; 8 warps split b, then a fixed-order sum.
__global__ void k_reduce_partials(const double *part, int nparts, int ldp, double *yH,
                                  double *yS) {
    __shared__ double s[8][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;  // over [0, 2 ldp)
    double acc = 0.0;
    if (c < 2 * ldp)
        for (int b = warp; b < nparts; b += 8) acc += part[(size_t)b * 2 * ldp + c];
    s[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && c < 2 * ldp) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += s[w][lane];
        if (c < ldp) {
            if (yH) yH[c] = t;
        } else if (yS) {
            yS[c - ldp] = t;
        }
    }
}

template <typename T, int NJ, int MODE>
int launch_t(lm_pencil *p, const T *O, const T *G, const double *v, double *out, const int *skip,
             cudaStream_t s) {
    const int nmat = MODE == MODE_S ? 1 : 2;
    const size_t row_bytes = (size_t)nmat * p->ldp * sizeof(T);
    // rows per tile: about 48 KB per pipeline stage, one row per warp when two
    // such stages fit, fewer rows (idle warps) for very long FP64 rows
    const size_t tail = 8 * sizeof(uint64_t) + (size_t)p->ldp * sizeof(typename Acc<T>::type) + 256;
    const size_t budget = (size_t)p->ctx->smem_optin - tail - 2048;
    int R = (int)std::min<size_t>(64, std::max<size_t>(1, 49152 / row_bytes));
    if (R < PT / 32) R = (int)std::max<size_t>(1, std::min<size_t>(PT / 32, budget / (2 * row_bytes)));
    const size_t stage_bytes = R * row_bytes;
    int stages = (int)std::min<size_t>(4, budget / stage_bytes);
    if (stages < 2)
        return lm_fail(p->ctx, LM_ERR_SIZE, "pencil row of %d columns too long", p->ldp);
    size_t smem = stages * stage_bytes + tail;
    smem = std::max(smem, (size_t)(PT / 32) * p->ldp * sizeof(double) + 64);
    PencilArgs<T> a;
    a.O = O;
    a.G = G;
    a.w = p->wt;
    a.n_rows = p->n_rows;
    a.ldp = p->ldp;
    a.v = v;
    a.out = out;
    a.out_ld = 2 * p->ldp;
    a.stages = stages;
    a.rows_per_tile = R;
    a.skip = skip;
    a.flags = p->ctx->d_flags;
    cudaError_t e = cudaFuncSetAttribute(k_pencil<T, NJ, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return lm_cuda_check(p->ctx, e, "pencil smem attribute");
    lm_prof_begin(p->ctx, PROF_PENCIL, s);
    k_pencil<T, NJ, MODE><<<p->g_pencil, PT, smem, s>>>(a);
    lm_prof_end(p->ctx, PROF_PENCIL, s);
    lm_note_launch(p->ctx);
    p->ctx->pencil_rows += p->n_rows;
    return lm_cuda_check(p->ctx, cudaGetLastError(), "k_pencil");
}

template <typename T, int NJ>
int dispatch_mode(lm_pencil *p, const T *O, const T *G, const double *v, int half, int want_s,
                  const int *skip, cudaStream_t s) {
    int rc = half ? launch_t<T, NJ, MODE_H_HALF>(p, O, G, v, p->part, skip, s)
                  : launch_t<T, NJ, MODE_H_NONE>(p, O, G, v, p->part, skip, s);
    if (!rc && want_s) rc = launch_t<T, NJ, MODE_S>(p, O, G, v, p->part + p->ldp, skip, s);
    return rc;
}

template <typename T>
int dispatch_nc(lm_pencil *p, const T *O, const T *G, const double *v, int half, int want_s,
                const int *skip, cudaStream_t s) {
    const int nj = (p->ldp + 31) / 32;
    if (nj <= 8) return dispatch_mode<T, 8>(p, O, G, v, half, want_s, skip, s);
    if (nj <= 16) return dispatch_mode<T, 16>(p, O, G, v, half, want_s, skip, s);
    if (nj <= 28) return dispatch_mode<T, 28>(p, O, G, v, half, want_s, skip, s);
    if (nj <= 40) return dispatch_mode<T, 40>(p, O, G, v, half, want_s, skip, s);
    if (nj <= 52) return dispatch_mode<T, 52>(p, O, G, v, half, want_s, skip, s);
    if (nj <= 64) return dispatch_mode<T, 64>(p, O, G, v, half, want_s, skip, s);
    return lm_fail(p->ctx, LM_ERR_SIZE, "P+1 = %d above the supported 2048", p->P1);
}

}  // namespace

int lm_pencil_grid(lm_pencil *p) { return p->ctx->sms; }

int lm_launch_pencil(lm_pencil *p, const double *v, int sym, int prec, int want_s,
                     const int *skip, cudaStream_t s) {
    const int half = (sym == LM_SYM_HALF);
    if (prec == LM_FP64 || p->prec == LM_FP64 || p->Olo == nullptr)
        return dispatch_nc<double>(p, p->O, p->G, v, half, want_s, skip, s);
    if (p->prec == LM_FP32)
        return dispatch_nc<float>(p, (const float *)p->Olo, (const float *)p->Glo, v, half,
                                  want_s, skip, s);
    return dispatch_nc<__nv_bfloat16>(p, (const __nv_bfloat16 *)p->Olo,
                                      (const __nv_bfloat16 *)p->Glo, v, half, want_s, skip, s);
}

int lm_launch_reduce_partials(lm_pencil *p, double *yH, double *yS, cudaStream_t s) {
    const int blocks = (2 * p->ldp + 31) / 32;
    k_reduce_partials<<<blocks, 256, 0, s>>>(p->part, p->g_pencil, p->ldp, yH, yS);
    lm_note_launch(p->ctx);
    return lm_cuda_check(p->ctx, cudaGetLastError(), "k_reduce_partials");
}

// ---------------------------------------------------------------------------
// Launches on caller-provided scratch (no lm_pencil, no allocation). Used by the
// no-allocation entry point in noalloc.cu; FP64 factors only.
// ---------------------------------------------------------------------------
namespace {

template <int NJ, int MODE>
int raw_launch(const double *O, const double *G, const double *w, int64_t n_rows, int ldp,
               const double *vpad, double *out, int out_ld, int grid, int smem_optin, int *flags,
               cudaStream_t s) {
    const int nmat = MODE == MODE_S ? 1 : 2;
    const size_t row_bytes = (size_t)nmat * ldp * sizeof(double);
    const size_t tail = 8 * sizeof(uint64_t) + (size_t)ldp * sizeof(double) + 256;
    const size_t budget = (size_t)smem_optin - tail - 2048;
    int R = (int)std::min<size_t>(64, std::max<size_t>(1, 49152 / row_bytes));
    if (R < PT / 32) R = (int)std::max<size_t>(1, std::min<size_t>(PT / 32, budget / (2 * row_bytes)));
    const size_t stage_bytes = R * row_bytes;
    const int stages = (int)std::min<size_t>(4, budget / stage_bytes);
    if (stages < 2) return LM_ERR_SIZE;
    size_t smem = stages * stage_bytes + tail;
    smem = std::max(smem, (size_t)(PT / 32) * ldp * sizeof(double) + 64);
    PencilArgs<double> a;
    a.O = O;
    a.G = G;
    a.w = w;
    a.n_rows = n_rows;
    a.ldp = ldp;
    a.v = vpad;
    a.out = out;
    a.out_ld = out_ld;
    a.stages = stages;
    a.rows_per_tile = R;
    a.skip = nullptr;
    a.flags = flags;
    if (cudaFuncSetAttribute(k_pencil<double, NJ, MODE>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LM_ERR_CUDA;
    k_pencil<double, NJ, MODE><<<grid, PT, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

template <int NJ>
int raw_modes(const double *O, const double *G, const double *w, int64_t n_rows, int ldp,
              const double *vpad, double *part, int grid, int half, int want_s, int smem_optin,
              int *flags, cudaStream_t s) {
    int rc = half ? raw_launch<NJ, MODE_H_HALF>(O, G, w, n_rows, ldp, vpad, part, 2 * ldp, grid,
                                                smem_optin, flags, s)
                  : raw_launch<NJ, MODE_H_NONE>(O, G, w, n_rows, ldp, vpad, part, 2 * ldp, grid,
                                                smem_optin, flags, s);
    if (rc == LM_OK && want_s)
        rc = raw_launch<NJ, MODE_S>(O, G, w, n_rows, ldp, vpad, part + ldp, 2 * ldp, grid,
                                    smem_optin, flags, s);
    return rc;
}

// y[c] = sum_b part[b][c] (CTA order); NaN everywhere if a pencil CTA gave up waiting.
__global__ void k_reduce_partials_flagged(const double *part, int nparts, int ldp, int p1,
                                          const int *flags, double *yH, double *yS) {
    __shared__ double s[8][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    double acc = 0.0;
    if (c < 2 * ldp)
        for (int b = warp; b < nparts; b += 8) acc += part[(size_t)b * 2 * ldp + c];
    s[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && c < 2 * ldp) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += s[w][lane];
        if (*flags) t = __longlong_as_double(0x7ff8000000000000ll);
        if (c < ldp) {
            if (yH && c < p1) yH[c] = t;
        } else if (yS && c - ldp < p1) {
            yS[c - ldp] = t;
        }
    }
}

}  // namespace

int lm_pencil_fp64_on_scratch(const double *O, const double *G, const double *w, int64_t n_rows,
                              int ldp, int p1, const double *vpad, double *part, int grid, int half,
                              double *yH, double *yS, int smem_optin, int *flags, cudaStream_t s) {
    const int nj = (ldp + 31) / 32;
    const int want_s = yS != nullptr;
    int rc;
    if (nj <= 8) rc = raw_modes<8>(O, G, w, n_rows, ldp, vpad, part, grid, half, want_s, smem_optin, flags, s);
    else if (nj <= 16) rc = raw_modes<16>(O, G, w, n_rows, ldp, vpad, part, grid, half, want_s, smem_optin, flags, s);
    else if (nj <= 28) rc = raw_modes<28>(O, G, w, n_rows, ldp, vpad, part, grid, half, want_s, smem_optin, flags, s);
    else if (nj <= 40) rc = raw_modes<40>(O, G, w, n_rows, ldp, vpad, part, grid, half, want_s, smem_optin, flags, s);
    else if (nj <= 52) rc = raw_modes<52>(O, G, w, n_rows, ldp, vpad, part, grid, half, want_s, smem_optin, flags, s);
    else if (nj <= 64) rc = raw_modes<64>(O, G, w, n_rows, ldp, vpad, part, grid, half, want_s, smem_optin, flags, s);
    else return LM_ERR_SIZE;
    if (rc != LM_OK) return rc;
    k_reduce_partials_flagged<<<(2 * ldp + 31) / 32, 256, 0, s>>>(part, grid, ldp, p1, flags, yH, yS);
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}
