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
#include <type_traits>

#include "df64.cuh"
#include "internal.cuh"

namespace {



// Arithmetic of the pencil per storage type: A is the accumulator / compute
// type, madd(acc, a, b) forms acc += a b. FP64 storage computes in FP64;
// FP32 and BF16 in FP32; float2 (double-float, h + l) storage computes with
// error-free FP32 transformations and a lazily renormalised accumulator.
template <typename T>
struct PA;
template <>
struct PA<double> {
    using A = double;
    static __device__ __forceinline__ A zero() { return 0.0; }
    static __device__ __forceinline__ A load(const double *p) { return *p; }
    static __device__ __forceinline__ A from_double(double x) { return x; }
    static __device__ __forceinline__ double to_double(A a) { return a; }
    static __device__ __forceinline__ float2 to_df(A a) {
        const df d = df_split_bits(a);
        return make_float2(d.h, d.l);
    }
    static __device__ __forceinline__ void madd(A &acc, A a, A b) { acc = fma(a, b, acc); }
    static __device__ __forceinline__ A add(A a, A b) { return a + b; }
    static __device__ __forceinline__ A mul(A a, A b) { return a * b; }
    static __device__ __forceinline__ A shfl_xor(A a, int off) {
        return __shfl_xor_sync(0xffffffffu, a, off);
    }
    static __device__ __forceinline__ A weight(const double *w, const float2 *, int64_t i) {
        return w[i];
    }
    // 16-byte vector loads: two stored values / two compute values
    static __device__ __forceinline__ void load_vec(const double *p, A *o) {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        o[0] = v.x;
        o[1] = v.y;
    }
    static __device__ __forceinline__ void load_avec(const A *p, A *o) { load_vec(p, o); }
    static __device__ __forceinline__ void store_avec(A *p, const A *o) {
        *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
    }
    static __device__ __forceinline__ void renorm(A &) {}
};
template <>
struct PA<float> {
    using A = float;
    static __device__ __forceinline__ A zero() { return 0.f; }
    static __device__ __forceinline__ A load(const float *p) { return *p; }
    static __device__ __forceinline__ A from_double(double x) { return (float)x; }
    static __device__ __forceinline__ double to_double(A a) { return (double)a; }
    static __device__ __forceinline__ float2 to_df(A a) { return make_float2(a, 0.f); }
    static __device__ __forceinline__ void madd(A &acc, A a, A b) { acc = fmaf(a, b, acc); }
    static __device__ __forceinline__ A add(A a, A b) { return a + b; }
    static __device__ __forceinline__ A mul(A a, A b) { return a * b; }
    static __device__ __forceinline__ A shfl_xor(A a, int off) {
        return __shfl_xor_sync(0xffffffffu, a, off);
    }
    static __device__ __forceinline__ A weight(const double *, const float2 *wl, int64_t i) {
        return wl[i].x;
    }
    // 16-byte vector loads: four stored values / compute values four at a time
    static __device__ __forceinline__ void load_vec(const float *p, A *o) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
    static __device__ __forceinline__ void load_avec(const A *p, A *o) { load_vec(p, o); }
    static __device__ __forceinline__ void store_avec(A *p, const A *o) {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
    static __device__ __forceinline__ void renorm(A &) {}
};
template <>
struct PA<__nv_bfloat16> : PA<float> {
    static __device__ __forceinline__ float load(const __nv_bfloat16 *p) {
        return __bfloat162float(*p);
    }
    // eight stored values in one 16-byte load; compute values in two float4
    static __device__ __forceinline__ void load_vec(const __nv_bfloat16 *p, A *o) {
        const uint4 v = *reinterpret_cast<const uint4 *>(p);
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {  // bf16 -> fp32 is a 16-bit shift
            o[2 * k] = __uint_as_float(w[k] << 16);
            o[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
    static __device__ __forceinline__ void load_avec(const A *p, A *o) {
        PA<float>::load_vec(p, o);
        PA<float>::load_vec(p + 4, o + 4);
    }
    static __device__ __forceinline__ void store_avec(A *p, const A *o) {
        PA<float>::store_avec(p, o);
        PA<float>::store_avec(p + 4, o + 4);
    }
};
template <>
struct PA<float2> {
    using A = df;
    static __device__ __forceinline__ A zero() { return df_make(0.f, 0.f); }
    static __device__ __forceinline__ A load(const float2 *p) {
        const float2 v = *p;
        return df_make(v.x, v.y);
    }
    static __device__ __forceinline__ A from_double(double x) { return df_from_double(x); }
    static __device__ __forceinline__ double to_double(A a) { return df_to_double(a); }
    static __device__ __forceinline__ float2 to_df(A a) { return make_float2(a.h, a.l); }
    // acc += a b: exact head product by FMA, cross terms, head sum by TwoSum,
    // everything else gathered in the (not yet renormalised) tail
    static __device__ __forceinline__ void madd(A &acc, A a, A b) {
        const float p = __fmul_rn(a.h, b.h);
        float e = __fmaf_rn(a.h, b.h, -p);
        e = __fmaf_rn(a.h, b.l, e);
        e = __fmaf_rn(a.l, b.h, e);
        const df s = df_ts(acc.h, p);
        acc.h = s.h;
        acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
    }
    static __device__ __forceinline__ A add(A a, A b) { return df_add(a, b); }
    static __device__ __forceinline__ A mul(A a, A b) { return df_mul(a, b); }
    static __device__ __forceinline__ A shfl_xor(A a, int off) {
        return df_make(__shfl_xor_sync(0xffffffffu, a.h, off),
                       __shfl_xor_sync(0xffffffffu, a.l, off));
    }
    static __device__ __forceinline__ A weight(const double *, const float2 *wl, int64_t i) {
        const float2 v = wl[i];
        return df_make(v.x, v.y);
    }
    static __device__ __forceinline__ void load_vec(const float2 *p, A *o) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = df_make(v.x, v.y);
        o[1] = df_make(v.z, v.w);
    }
    static __device__ __forceinline__ void load_avec(const A *p, A *o) {
        load_vec(reinterpret_cast<const float2 *>(p), o);
    }
    static __device__ __forceinline__ void store_avec(A *p, const A *o) {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0].h, o[0].l, o[1].h, o[1].l);
    }
    // fold the lazily accumulated tail back into the head
    static __device__ __forceinline__ void renorm(A &a) { a = df_fts(a.h, a.l); }
};

enum { MODE_H_NONE = 0, MODE_H_HALF = 1, MODE_S = 2 };

template <typename T>
struct PencilArgs {
    const T *O;
    const T *G;
    const double *w;
    const float2 *wlo;  // the weights as double-float (FP32 / BF16 use .x)
    int64_t n_rows;
    int ldp;
    const double *v;
    double *out;    // [gridDim.x][out_ld]: this CTA's partial y
    int out_ld;
    int stages;
    int rows_per_tile;
    const int *skip;
    int *flags;
    int out_df;     // partials as double-float pairs (same 8-byte slots) instead of FP64
    int reverse;    // take this CTA's tiles last to first
};

// Columns per lane per 16-byte shared-memory access (8 BF16, 4 FP32, 2 FP64 or
// double-float), and the number of 32 x VEC column chunks covering NJ x 32.
template <typename T>
struct VEC {
    static constexpr int value = 16 / (int)sizeof(T);
};
template <typename T, int NJ>
struct NCV {
    static constexpr int value = (NJ + VEC<T>::value - 1) / VEC<T>::value;
};

// One staged row: lane l owns columns k * 32 VEC + l VEC + [0, VEC) of chunk k
// (ldp is a multiple of 8 and so of VEC: in the last, partial chunk a lane
// holds a whole vector or nothing). Row dot(s) by one butterfly,
// then the rank-1 update of the register-resident y:
// MODE_H_NONE: y += w (G.v) O; MODE_H_HALF: y += w/2 ((G.v) O + (O.v) G);
// MODE_S: y += w (O.v) O.
template <typename T, int NJ, int MODE>
__device__ __forceinline__ void consume_row(const T *ro, const T *rg, const typename PA<T>::A *vs,
                                            int ldp, int lane, typename PA<T>::A wr,
                                            typename PA<T>::A (&y)[NCV<T, NJ>::value][VEC<T>::value]) {
    using P = PA<T>;
    using AT = typename PA<T>::A;
    constexpr int W = VEC<T>::value, NC = NCV<T, NJ>::value;
    AT dg = P::zero(), dov = P::zero();
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int c0 = k * 32 * W + lane * W;
        if (c0 < ldp) {
            AT vv[W], x[W];
            P::load_avec(vs + c0, vv);
            if (MODE != MODE_S) {
                P::load_vec(rg + c0, x);
#pragma unroll
                for (int v = 0; v < W; ++v) P::madd(dg, x[v], vv[v]);
            }
            if (MODE != MODE_H_NONE) {
                P::load_vec(ro + c0, x);
#pragma unroll
                for (int v = 0; v < W; ++v) P::madd(dov, x[v], vv[v]);
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        if (MODE != MODE_S) dg = P::add(dg, P::shfl_xor(dg, off));
        if (MODE != MODE_H_NONE) dov = P::add(dov, P::shfl_xor(dov, off));
    }
    AT cg, co;
    if (MODE == MODE_H_HALF) {
        const AT half = P::mul(wr, P::from_double(0.5));
        cg = P::mul(half, dg);
        co = P::mul(half, dov);
    } else {
        cg = P::mul(wr, dg);
        co = P::mul(wr, dov);
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int c0 = k * 32 * W + lane * W;
        if (c0 < ldp) {
            AT x[W];
            P::load_vec(ro + c0, x);
            if (MODE == MODE_S) {
#pragma unroll
                for (int v = 0; v < W; ++v) P::madd(y[k][v], co, x[v]);
            } else {
#pragma unroll
                for (int v = 0; v < W; ++v) P::madd(y[k][v], cg, x[v]);
                if (MODE == MODE_H_HALF) {
                    P::load_vec(rg + c0, x);
#pragma unroll
                    for (int v = 0; v < W; ++v) P::madd(y[k][v], co, x[v]);
                }
            }
        }
    }
}

// Warp-specialised pipeline. Warp NCW (the last) is the producer: its lane 0
// streams this CTA's rows, one row of O (and G) per pipeline stage, into a ring
// of S stages with 1-D bulk copies, re-filling a stage as soon as its
// consumer has released it (full / empty mbarrier pair per stage). Consumer
// warp w takes rows w, w + C, ... (C consuming warps, below): lane l owns columns l, l+32, ..., so a
// row dot is one butterfly and the rank-1 update of the warp's register-
// resident y reuses the staged row. MODE_H_NONE: y += w (G.v) O;
// MODE_H_HALF: y += w/2 ((G.v) O + (O.v) G); MODE_S: y += w (O.v) O (only O
// is staged). At the end the consumer warps' y are summed in warp order.
// Every wait is bounded; a timeout sets FLAG_TIMEOUT and the CTA drains its
// outstanding copies before exiting.
// Consumer warp w waits on full[i % S] with parity (i / S) & 1. That parity
// names phase i / S unambiguously only if the stage's previous fill (tile
// i - S) has already landed when the warp starts to wait. Bulk copies may land
// in any order, so "an earlier tile has landed" does not follow from a later
// one having landed: it holds only for tiles the same warp has itself waited
// for. With C consuming warps taking tiles w, w + C, ..., tile i - S is one of
// warp w's own earlier tiles exactly when S is a multiple of C. So C =
// min(NCW, S) and the launch rounds S down to a multiple of C (with fewer
// stages than warps the extra warps only join the final sum with zero
// accumulators). The producer's waits on `empty` need no such condition: it
// refills a stage only after its own wait on that stage's previous release.
// consumer warps: 16 for rows up to 896 columns, 8 (more registers each) beyond
template <int NJ>
struct Ncw {
    static constexpr int value = NJ <= 28 ? 16 : 8;
};

template <typename T, int NJ, int MODE, int NCW = Ncw<NJ>::value>
__global__ void __launch_bounds__(NCW * 32 + 32, 1) k_pencil(PencilArgs<T> a) {
    using P = PA<T>;
    using AT = typename PA<T>::A;
    extern __shared__ __align__(128) unsigned char smraw[];
    if (a.skip && *a.skip) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ldp = a.ldp, S = a.stages, R = a.rows_per_tile;
    const int ncons = min(NCW, S);  // consuming warps (S is a multiple); see the note above
    const int nmat = MODE == MODE_S ? 1 : 2;
    const size_t row_elems = (size_t)ldp;
    const size_t tile_elems = (size_t)R * row_elems;  // one matrix's rows of a stage
    T *stage_base = reinterpret_cast<T *>(smraw);
    const size_t stage_bytes_all = (size_t)S * nmat * tile_elems * sizeof(T);
    uint64_t *full = reinterpret_cast<uint64_t *>(smraw + stage_bytes_all);
    uint64_t *empty = full + S;
    AT *vs = reinterpret_cast<AT *>(empty + S);  // v in the compute type, ldp entries
    __shared__ int s_abort;

    const int64_t r0 = a.n_rows * blockIdx.x / gridDim.x;
    const int64_t r1 = a.n_rows * (blockIdx.x + 1) / gridDim.x;
    const int nrows = (int)(r1 - r0);
    const int ntiles = (nrows + R - 1) / R;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        s_abort = 0;
        fence_barrier_init();
    }
    for (int c = tid; c < ldp; c += blockDim.x) vs[c] = P::from_double(a.v[c]);
    __syncthreads();

    AT y[NCV<T, NJ>::value][VEC<T>::value];
#pragma unroll
    for (int k = 0; k < NCV<T, NJ>::value; ++k)
#pragma unroll
        for (int v = 0; v < VEC<T>::value; ++v) y[k][v] = P::zero();

    if (warp == NCW) {
        // producer
        if (lane == 0) {
            // stage s = i mod S and round = i / S kept incrementally: a divide
            // converts to and from floating point, at the FP64 rate on this part
            int issued = 0, s = 0, round = 0;
            for (int i = 0; i < ntiles; ++i) {
                if (round > 0 && !mbar_wait_bounded(&empty[s], (uint32_t)((round - 1) & 1))) {
                    atomicOr(a.flags, FLAG_TIMEOUT);
                    atomicExch(&s_abort, 1);
                    break;
                }
                if (*(volatile int *)&s_abort) break;
                // the tile's rows are consecutive in O and in G: one copy per matrix
                const int t = a.reverse ? ntiles - 1 - i : i;
                const int nr = min(R, nrows - t * R);
                const uint32_t bytes = (uint32_t)(nr * row_elems * sizeof(T));
                const int64_t row = r0 + (int64_t)t * R;
                T *dst = stage_base + (size_t)s * nmat * tile_elems;
                mbar_arrive_expect_tx(&full[s], nmat * bytes);
                bulk_g2s(dst, a.O + row * ldp, bytes, &full[s]);
                if (MODE != MODE_S) bulk_g2s(dst + tile_elems, a.G + row * ldp, bytes, &full[s]);
                issued = i + 1;
                if (++s == S) {
                    s = 0;
                    ++round;
                }
            }
            // every issued copy lands before the CTA may exit (bounded)
            const int i0 = max(0, issued - S);
            for (int i = i0, ds = i0 % S, dr = i0 / S; i < issued; ++i) {
                (void)mbar_wait_bounded(&full[ds], (uint32_t)(dr & 1));
                if (++ds == S) {
                    ds = 0;
                    ++dr;
                }
            }
        }
    } else if (warp < ncons) {
        // stage s = i mod S and parity (i / S) & 1, kept incrementally (S is a
        // multiple of ncons, so s wraps at most once per step)
        int s = warp, ph = 0, it = 0;
        for (int i = warp; i < ntiles; i += ncons, ++it) {
            bool ok = true;
            if (lane == 0) ok = mbar_wait_bounded(&full[s], (uint32_t)ph);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok || *(volatile int *)&s_abort) {
                if (lane == 0) {
                    atomicOr(a.flags, FLAG_TIMEOUT);
                    atomicExch(&s_abort, 1);
                }
                break;
            }
            const int t = a.reverse ? ntiles - 1 - i : i;
            const int nr = min(R, nrows - t * R);
            for (int rr = 0; rr < nr; ++rr) {
                const T *ro = stage_base + (size_t)s * nmat * tile_elems + (size_t)rr * row_elems;
                consume_row<T, NJ, MODE>(ro, ro + tile_elems, vs, ldp, lane,
                                         P::weight(a.w, a.wlo, r0 + (int64_t)t * R + rr), y);
            }
            if ((it & 15) == 15)  // fold lazily accumulated tails now and then
#pragma unroll
                for (int k = 0; k < NCV<T, NJ>::value; ++k)
#pragma unroll
                    for (int v = 0; v < VEC<T>::value; ++v) P::renorm(y[k][v]);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            s += ncons;
            if (s >= S) {
                s -= S;
                ph ^= 1;
            }
        }
    }
    __syncthreads();
    if (s_abort) return;
    // Sum the consumer warps' accumulators in warp order, in the accumulator
    // type (the ring is free now); one conversion to FP64 per column.
    AT *ys = reinterpret_cast<AT *>(smraw);  // [NCW][ldp]
    if (warp < NCW) {
        constexpr int W = VEC<T>::value;
#pragma unroll
        for (int k = 0; k < NCV<T, NJ>::value; ++k) {
            const int c0 = k * 32 * W + lane * W;
            if (c0 < ldp) P::store_avec(ys + (size_t)warp * ldp + c0, y[k]);
        }
    }
    __syncthreads();
    double *out = a.out + (size_t)blockIdx.x * a.out_ld;
    for (int c = tid; c < ldp; c += blockDim.x) {
        AT t = ys[c];
#pragma unroll
        for (int w8 = 1; w8 < NCW; ++w8) t = P::add(t, ys[(size_t)w8 * ldp + c]);
        if (a.out_df) reinterpret_cast<float2 *>(out)[c] = P::to_df(t);
        else out[c] = P::to_double(t);
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
int launch_t(lm_pencil *p, const T *O, const T *G, const double *v, double *out,
             const double *w, const float2 *wl, const int *skip, int out_df, cudaStream_t s) {
    const int nmat = MODE == MODE_S ? 1 : 2;
    const size_t row_bytes = (size_t)nmat * p->ldp * sizeof(T);
    // ring of stages filling the shared memory (at most 32). A stage holds R
    // consecutive rows, R chosen so that a stage carries about 16 KB: short rows
    // (BF16, FP32, small P) would otherwise leave the one producer lane issuing
    // copies and barrier operations faster than HBM delivers the rows.
    const int R = (int)std::max<size_t>(1, std::min<size_t>(8, 16384 / row_bytes));
    const size_t tile_bytes = (size_t)R * row_bytes;
    const size_t tail = (size_t)p->ldp * sizeof(typename PA<T>::A) + 256;
    const size_t budget = (size_t)p->ctx->smem_optin - tail - 2048;
    constexpr int NCW = Ncw<NJ>::value;
    int stages = (int)std::min<size_t>(32, budget / (tile_bytes + 2 * sizeof(uint64_t)));
    if (stages < 2)
        return lm_fail(p->ctx, LM_ERR_SIZE, "pencil row of %d columns too long", p->ldp);
    stages -= stages % std::min(NCW, stages);  // a multiple of the consuming warps
    size_t smem = stages * (tile_bytes + 2 * sizeof(uint64_t)) + tail;
    smem = std::max(smem, (size_t)NCW * p->ldp * sizeof(double) + 64);
    PencilArgs<T> a;
    a.O = O;
    a.G = G;
    a.w = w;
    a.wlo = wl;
    a.n_rows = p->n_rows;
    a.ldp = p->ldp;
    a.v = v;
    a.out = out;
    a.out_ld = 2 * p->ldp;
    a.stages = stages;
    a.rows_per_tile = R;
    a.skip = skip;
    a.flags = p->d_flags;
    a.out_df = out_df;
    a.reverse = p->order_rev;
    // the device maximum rather than this launch's size: the attribute is shared
    // by every pencil and read again when a captured IRL cycle replays the launch
    const int dmax = lm_max_dyn_smem((const void *)k_pencil<T, NJ, MODE>, p->ctx->smem_optin);
    cudaError_t e = cudaFuncSetAttribute(k_pencil<T, NJ, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         std::max(dmax, (int)smem));
    if (e != cudaSuccess) return lm_cuda_check(p->ctx, e, "pencil smem attribute");
    lm_prof_begin(p->ctx, PROF_PENCIL, s);
    const int grid = lm_pencil_ctas(p, std::is_same<T, double>::value ? (int)LM_FP64 : p->prec);
    k_pencil<T, NJ, MODE><<<grid, NCW * 32 + 32, smem, s>>>(a);
    lm_prof_end(p->ctx, PROF_PENCIL, s);
    lm_note_launch(p->ctx);
    p->ctx->pencil_rows += p->n_rows;
    return lm_cuda_check(p->ctx, cudaGetLastError(), "k_pencil");
}

// hmode 0: y_H = O_c^T W G'_c v; 1: its symmetrised form; 2: the E_loc
// estimator O_c^T W diag(E_loc - E) O_c v, the S product with weights w (E_loc - E)
template <typename T, int NJ>
int dispatch_mode(lm_pencil *p, const T *O, const T *G, const double *v, int hmode, int want_s,
                  const int *skip, int out_df, cudaStream_t s) {
    int rc;
    if (hmode == 2)
        rc = launch_t<T, NJ, MODE_S>(p, O, G, v, p->part, p->wel, p->wello, skip, out_df, s);
    else if (hmode == 1)
        rc = launch_t<T, NJ, MODE_H_HALF>(p, O, G, v, p->part, p->wt, p->wlo, skip, out_df, s);
    else
        rc = launch_t<T, NJ, MODE_H_NONE>(p, O, G, v, p->part, p->wt, p->wlo, skip, out_df, s);
    if (!rc && want_s)
        rc = launch_t<T, NJ, MODE_S>(p, O, G, v, p->part + p->ldp, p->wt, p->wlo, skip, out_df, s);
    return rc;
}

template <typename T>
int dispatch_nc(lm_pencil *p, const T *O, const T *G, const double *v, int hmode, int want_s,
                const int *skip, int out_df, cudaStream_t s) {
    const int nj = (p->ldp + 31) / 32;
    if (nj <= 8) return dispatch_mode<T, 8>(p, O, G, v, hmode, want_s, skip, out_df, s);
    if (nj <= 16) return dispatch_mode<T, 16>(p, O, G, v, hmode, want_s, skip, out_df, s);
    if (nj <= 28) return dispatch_mode<T, 28>(p, O, G, v, hmode, want_s, skip, out_df, s);
    if (nj <= 40) return dispatch_mode<T, 40>(p, O, G, v, hmode, want_s, skip, out_df, s);
    if (nj <= 52) return dispatch_mode<T, 52>(p, O, G, v, hmode, want_s, skip, out_df, s);
    if (nj <= 64) return dispatch_mode<T, 64>(p, O, G, v, hmode, want_s, skip, out_df, s);
    return lm_fail(p->ctx, LM_ERR_SIZE, "P+1 = %d above the supported 2048", p->P1);
}

}  // namespace

int lm_pencil_grid(lm_pencil *p) { return p->ctx->sms; }

// A product on FP64 factors is bound by the FP64 pipe, not by HBM: its SM time
// hardly depends on the grid, so the FP64 copies of a low-precision pencil (the
// continuation and refinement of a mixed-precision step) always take every SM,
// whatever grid the low-precision products were tuned to.
int lm_pencil_ctas(const lm_pencil *p, int prec) {
    const bool fp64 = (prec == LM_FP64 || p->Olo == nullptr) && p->prec != LM_DF64;
    return fp64 && p->prec != LM_FP64 ? p->ctx->sms : p->g_pencil;
}

int lm_launch_pencil(lm_pencil *p, const double *v, int sym, int prec, int want_s,
                     const int *skip, cudaStream_t s, int out_df, int reverse) {
    const int hmode = sym == LM_SYM_ELOC ? 2 : sym == LM_SYM_HALF ? 1 : 0;  // see dispatch_mode
    p->order_rev = reverse;  // read by the launch below, on this host thread
    // a double-float pencil keeps no centred FP64 factors: FP64-accurate
    // requests use its double-float pairs
    if (p->prec == LM_DF64 && p->Olo)
        return dispatch_nc<float2>(p, (const float2 *)p->Olo, (const float2 *)p->Glo, v, hmode,
                                   want_s, skip, out_df, s);
    if (prec == LM_FP64 || p->prec == LM_FP64 || p->Olo == nullptr)
        return dispatch_nc<double>(p, p->O, p->G, v, hmode, want_s, skip, out_df, s);
    if (p->prec == LM_FP32)
        return dispatch_nc<float>(p, (const float *)p->Olo, (const float *)p->Glo, v, hmode,
                                  want_s, skip, out_df, s);
    if (p->prec == LM_DF64)
        return dispatch_nc<float2>(p, (const float2 *)p->Olo, (const float2 *)p->Glo, v, hmode,
                                   want_s, skip, out_df, s);
    return dispatch_nc<__nv_bfloat16>(p, (const __nv_bfloat16 *)p->Olo,
                                      (const __nv_bfloat16 *)p->Glo, v, hmode, want_s, skip,
                                      out_df, s);
}

int lm_launch_reduce_partials(lm_pencil *p, int prec, double *yH, double *yS, cudaStream_t s) {
    const int blocks = (2 * p->ldp + 31) / 32;
    k_reduce_partials<<<blocks, 256, 0, s>>>(p->part, lm_pencil_ctas(p, prec), p->ldp, yH, yS);
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
    const size_t tail = (size_t)ldp * sizeof(double) + 256;
    const size_t budget = (size_t)smem_optin - tail - 2048;
    constexpr int NCW = Ncw<NJ>::value;
    int stages = (int)std::min<size_t>(32, budget / (row_bytes + 2 * sizeof(uint64_t)));
    const int R = 1;
    if (stages < 2) return LM_ERR_SIZE;
    stages -= stages % std::min(NCW, stages);  // a multiple of the consuming warps
    size_t smem = stages * (row_bytes + 2 * sizeof(uint64_t)) + tail;
    smem = std::max(smem, (size_t)NCW * ldp * sizeof(double) + 64);
    PencilArgs<double> a;
    a.O = O;
    a.G = G;
    a.w = w;
    a.wlo = nullptr;
    a.n_rows = n_rows;
    a.ldp = ldp;
    a.v = vpad;
    a.out = out;
    a.out_ld = out_ld;
    a.stages = stages;
    a.rows_per_tile = R;
    a.skip = nullptr;
    a.flags = flags;
    a.out_df = 0;
    a.reverse = 0;
    // the device maximum (see launch_t): captured IRL cycles replay these kernels
    const int dmax = lm_max_dyn_smem((const void *)k_pencil<double, NJ, MODE>, smem_optin);
    if (cudaFuncSetAttribute(k_pencil<double, NJ, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             std::max(dmax, (int)smem)) != cudaSuccess)
        return LM_ERR_CUDA;
    k_pencil<double, NJ, MODE><<<grid, NCW * 32 + 32, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

template <int NJ>
int raw_modes(const double *O, const double *G, const double *w, int64_t n_rows, int ldp,
              const double *vpad, double *part, int grid, int half, int want_h, int want_s,
              int smem_optin, int *flags, cudaStream_t s) {
    int rc = LM_OK;
    if (want_h)
        rc = half ? raw_launch<NJ, MODE_H_HALF>(O, G, w, n_rows, ldp, vpad, part, 2 * ldp, grid,
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
    const int want_s = yS != nullptr, want_h = yH != nullptr;
    int rc;
    if (nj <= 8) rc = raw_modes<8>(O, G, w, n_rows, ldp, vpad, part, grid, half, want_h, want_s, smem_optin, flags, s);
    else if (nj <= 16) rc = raw_modes<16>(O, G, w, n_rows, ldp, vpad, part, grid, half, want_h, want_s, smem_optin, flags, s);
    else if (nj <= 28) rc = raw_modes<28>(O, G, w, n_rows, ldp, vpad, part, grid, half, want_h, want_s, smem_optin, flags, s);
    else if (nj <= 40) rc = raw_modes<40>(O, G, w, n_rows, ldp, vpad, part, grid, half, want_h, want_s, smem_optin, flags, s);
    else if (nj <= 52) rc = raw_modes<52>(O, G, w, n_rows, ldp, vpad, part, grid, half, want_h, want_s, smem_optin, flags, s);
    else if (nj <= 64) rc = raw_modes<64>(O, G, w, n_rows, ldp, vpad, part, grid, half, want_h, want_s, smem_optin, flags, s);
    else return LM_ERR_SIZE;
    if (rc != LM_OK) return rc;
    k_reduce_partials_flagged<<<(2 * ldp + 31) / 32, 256, 0, s>>>(part, grid, ldp, p1, flags, yH, yS);
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}
