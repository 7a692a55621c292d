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
// tracked by an mbarrier per pipeline stage. Thread t owns the columns
// t, t+256, ...: it forms its share of every row dot, the dots are finished
// with warp shuffles and a fixed-order cross-warp sum, and the rank-R update
// of the CTA's y accumulators uses the same staged tile. Each CTA writes its
// partial y; a second kernel sums the partials in CTA order (deterministic).
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

template <typename T>
struct PencilArgs {
    const T *O;
    const T *G;
    const double *w;
    int64_t n_rows;
    int ldp;
    const double *v;
    double *part;   // [gridDim.x][2*ldp]
    int half;       // sym HALF
    int want_s;
    int stages;
    const int *skip;
    int *flags;
};

template <typename T, int NC, int R>
__global__ void __launch_bounds__(PT) k_pencil(PencilArgs<T> a) {
    using AT = typename Acc<T>::type;
    extern __shared__ __align__(128) unsigned char smraw[];
    if (a.skip && *a.skip) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ldp = a.ldp;
    const size_t tile_elems = (size_t)R * ldp;
    T *stage_base = reinterpret_cast<T *>(smraw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smraw + (size_t)a.stages * 2 * tile_elems * sizeof(T));
    AT *red = reinterpret_cast<AT *>(bars + a.stages);  // [PT/32][2R]
    __shared__ int s_ok;

    const int64_t r0 = a.n_rows * blockIdx.x / gridDim.x;
    const int64_t r1 = a.n_rows * (blockIdx.x + 1) / gridDim.x;
    const int ntiles = (int)((r1 - r0 + R - 1) / R);

    if (tid == 0) {
        for (int s = 0; s < a.stages; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    __syncthreads();

    auto issue = [&](int i) {
        const int s = i % a.stages;
        const int64_t row = r0 + (int64_t)i * R;
        const int nr = (int)min((int64_t)R, r1 - row);
        const uint32_t bytes = (uint32_t)((size_t)nr * ldp * sizeof(T));
        T *dO = stage_base + (size_t)s * 2 * tile_elems;
        T *dG = dO + tile_elems;
        mbar_arrive_expect_tx(&bars[s], 2 * bytes);
        bulk_g2s(dO, a.O + row * ldp, bytes, &bars[s]);
        bulk_g2s(dG, a.G + row * ldp, bytes, &bars[s]);
    };
    if (tid == 0)
        for (int i = 0; i < min(a.stages, ntiles); ++i) issue(i);

    AT vr[NC], yH[NC], yS[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const int c = tid + q * PT;
        vr[q] = c < ldp ? (AT)a.v[c] : (AT)0;
        yH[q] = 0;
        yS[q] = 0;
    }
    const bool need_o_dot = a.half || a.want_s;
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
        const int64_t row = r0 + (int64_t)i * R;
        const int nr = (int)min((int64_t)R, r1 - row);
        const T *tO = stage_base + (size_t)s * 2 * tile_elems;
        const T *tG = tO + tile_elems;
        AT dG[R], dO[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            dG[r] = 0;
            dO[r] = 0;
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            const int c = tid + q * PT;
            if (c < ldp) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r < nr) {
                        dG[r] += ld_s(tG + (size_t)r * ldp + c) * vr[q];
                        if (need_o_dot) dO[r] += ld_s(tO + (size_t)r * ldp + c) * vr[q];
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            AT g = dG[r], o = dO[r];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                g += __shfl_xor_sync(0xffffffffu, g, off);
                o += __shfl_xor_sync(0xffffffffu, o, off);
            }
            if (lane == 0) {
                red[warp * 2 * R + r] = g;
                red[warp * 2 * R + R + r] = o;
            }
        }
        __syncthreads();
        AT cg[R], co[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            AT g = 0, o = 0;
            for (int w = 0; w < PT / 32; ++w) {
                g += red[w * 2 * R + r];
                o += red[w * 2 * R + R + r];
            }
            const AT wr = r < nr ? (AT)a.w[row + r] : (AT)0;
            cg[r] = wr * g;
            co[r] = wr * o;
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            const int c = tid + q * PT;
            if (c < ldp) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r < nr) {
                        const AT ov = ld_s(tO + (size_t)r * ldp + c);
                        if (a.half) {
                            const AT gv = ld_s(tG + (size_t)r * ldp + c);
                            yH[q] += (AT)0.5 * (cg[r] * ov + co[r] * gv);
                        } else {
                            yH[q] += cg[r] * ov;
                        }
                        if (a.want_s) yS[q] += co[r] * ov;
                    }
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
    double *out = a.part + (size_t)blockIdx.x * 2 * ldp;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const int c = tid + q * PT;
        if (c < ldp) {
            out[c] = (double)yH[q];
            out[ldp + c] = (double)yS[q];
        }
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

template <typename T, int NC, int R>
int launch_t(lm_pencil *p, const T *O, const T *G, const double *v, int half, int want_s,
             const int *skip, int stages, size_t smem, cudaStream_t s) {
    PencilArgs<T> a;
    a.O = O;
    a.G = G;
    a.w = p->wt;
    a.n_rows = p->n_rows;
    a.ldp = p->ldp;
    a.v = v;
    a.part = p->part;
    a.half = half;
    a.want_s = want_s;
    a.stages = stages;
    a.skip = skip;
    a.flags = p->ctx->d_flags;
    cudaError_t e = cudaFuncSetAttribute(k_pencil<T, NC, R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return lm_cuda_check(p->ctx, e, "pencil smem attribute");
    lm_prof_begin(p->ctx, PROF_PENCIL, s);
    k_pencil<T, NC, R><<<p->g_pencil, PT, smem, s>>>(a);
    lm_prof_end(p->ctx, PROF_PENCIL, s);
    lm_note_launch(p->ctx);
    p->ctx->pencil_rows += p->n_rows;
    return lm_cuda_check(p->ctx, cudaGetLastError(), "k_pencil");
}

template <typename T, int NC>
int dispatch_r(lm_pencil *p, const T *O, const T *G, const double *v, int half, int want_s,
               const int *skip, cudaStream_t s) {
    // R rows per tile: about 48 KB of O+G per pipeline stage.
    const size_t row_pair = 2 * (size_t)p->ldp * sizeof(T);
    int R = (int)std::max<size_t>(1, 49152 / row_pair);
    R = R >= 8 ? 8 : R >= 4 ? 4 : R >= 2 ? 2 : 1;
    const size_t stage_bytes = R * row_pair;
    const size_t extra = 64 * sizeof(uint64_t) + (PT / 32) * 2 * 8 * sizeof(double) + 256;
    const size_t budget = (size_t)p->ctx->smem_optin - extra - 2048;
    int stages = (int)std::min<size_t>(4, budget / stage_bytes);
    if (stages < 2)
        return lm_fail(p->ctx, LM_ERR_SIZE, "pencil row of %d columns too long", p->ldp);
    const size_t smem = stages * stage_bytes + extra;
    switch (R) {
        case 8: return launch_t<T, NC, 8>(p, O, G, v, half, want_s, skip, stages, smem, s);
        case 4: return launch_t<T, NC, 4>(p, O, G, v, half, want_s, skip, stages, smem, s);
        case 2: return launch_t<T, NC, 2>(p, O, G, v, half, want_s, skip, stages, smem, s);
        default: return launch_t<T, NC, 1>(p, O, G, v, half, want_s, skip, stages, smem, s);
    }
}

template <typename T>
int dispatch_nc(lm_pencil *p, const T *O, const T *G, const double *v, int half, int want_s,
                const int *skip, cudaStream_t s) {
    const int nc = (p->ldp + PT - 1) / PT;
    if (nc <= 2) return dispatch_r<T, 2>(p, O, G, v, half, want_s, skip, s);
    if (nc <= 4) return dispatch_r<T, 4>(p, O, G, v, half, want_s, skip, s);
    if (nc <= 8) return dispatch_r<T, 8>(p, O, G, v, half, want_s, skip, s);
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
