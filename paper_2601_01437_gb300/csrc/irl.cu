// Implicitly restarted Lanczos on the device (arXiv 2601.01437, Methods,
// "The Standard Lanczos Process and Implicit Restart", Algorithms 1 and 2).
//
// Per Lanczos step j (v_j = V[:, j]):
//   w = H~' v_j (pencil kernel, partials per row block)
//   lz_a: w = sum of partials; d1 = V^T w          (CGS pass 1 dots)
//   lz_b: w -= V d1; d2 = V^T w                    (CGS pass 2 dots)
//   lz_c: w -= V d2; alpha_j = d1_j + d2_j; remove the particle-number null
//         space; partial |w|^2
//   lz_d: beta_j = |w|; v_{j+1} = w / beta_j; breakdown test
// The vector kernels use one CTA per row r of the (Nh+1) x (M+1) parameter
// grid, so the null-space projection (which acts within a grid row) needs no
// extra synchronisation. Reductions always run in a fixed order.
//
// After m steps, one CTA (k_tri) finds the Ritz values of T_m (FP32
// multisection for brackets, FP64 Newton on the characteristic polynomial),
// estimates the residual of the lowest pair as beta_m |u_m| with
// u_m^2 = -p_{m-1}(theta)/p_m'(theta), and, if not converged, applies the
// mu = m - k largest Ritz values as shifts by implicit shifted QR sweeps.
// Consecutive bulges are chased concurrently four positions apart; the
// rotations they apply touch disjoint entries, so the result is the same as
// applying the sweeps one after another (the chase is latency bound in FP64).
// k_restart then forms V_k <- V_m Q[:, :k] and the new residual
// f = beta_hat_k V_m Q[:, k] + beta_m Q[m-1, k-1] v_{m+1}.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "df64.cuh"
#include "internal.cuh"

namespace {

constexpr int LT = 256;       // threads of the Lanczos vector kernels
constexpr int DLD = LM_MAXKRYLOV + 8;  // leading dimension of the per-CTA dot buffers

struct LzArgs {
    double *V;          // current basis, column-major ldp x (MAXK+1)
    double *w;          // work vector (ldp)
    const double *part; // pencil partials [nparts][2 ldp]
    int nparts;
    double *dots;       // [3][G2][DLD]
    int ldp, M1, P1, nrow_grid;  // nrow_grid = Nh + 1 = number of CTAs
    int n_orb, na, nb;
    int deflate;
    int three_term;     // IRL_REORTH_NONE: the paper's three-term recurrence, no CGS
    IrlState *st;
    unsigned *bar;      // [0] arrival count, [1] generation (cooperative kernel)
    int *flags;
    // particle-number projection constants as double-float pairs (cluster
    // kernel): 1/n and the inverse Gram matrix [[g22, -g12], [-g12, g11]] / det
    float2 inv_n, gi11, gi12, gi22;
};

__device__ __forceinline__ void cta_range(const LzArgs &a, int &e0, int &e1) {
    e0 = blockIdx.x * a.M1;
    e1 = (blockIdx.x == a.nrow_grid - 1) ? a.ldp : e0 + a.M1;
}

__device__ __forceinline__ bool lz_skip(const IrlState *st) { return st->broke != 0; }

constexpr int LE = 80;  // max entries per CTA: M+1 <= 65 plus the padding of the last row

// Shared-memory working set of one Lanczos vector CTA.
struct LzShared {
    double V[(LM_MAXKRYLOV + 1) * LE];  // V[i][e - e0]
    double w[LE];
    double h[LM_MAXKRYLOV + 1];
    double red[LT];
};

// Stage V[:, 0..j] and w over [e0, e1) into shared memory (one parallel round).
__device__ void load_block(const LzArgs &a, LzShared &S, int e0, int e1, int j, bool with_w) {
    const int E = e1 - e0;
    for (int t = threadIdx.x; t < (j + 1) * E; t += LT) {
        const int i = t / E, e = t % E;
        S.V[i * LE + e] = a.V[(size_t)i * a.ldp + e0 + e];
    }
    if (with_w)
        for (int e = threadIdx.x; e < E; e += LT) S.w[e] = a.w[e0 + e];
}

// dots d[i] = V[:, i] . w over this CTA's entries, i <= j. Warp q handles
// i = q, q+8, ...; lane = entry; the warp's dots are reduced together.
__device__ void block_dots(const LzShared &S, int E, int j, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[(LM_MAXKRYLOV + 8) / 8];
#pragma unroll
    for (int k = 0; k < (LM_MAXKRYLOV + 8) / 8; ++k) {
        const int i = warp + 8 * k;
        double s = 0.0;
        if (i <= j)
            for (int e = lane; e < E; e += 32) s = fma(S.V[i * LE + e], S.w[e], s);
        acc[k] = s;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < (LM_MAXKRYLOV + 8) / 8; ++k)
            acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < (LM_MAXKRYLOV + 8) / 8; ++k) {
            const int i = warp + 8 * k;
            if (i <= j) out[i] = acc[k];
        }
}

// h[i] = sum over CTAs of region[cta][i] (i <= j): 8 interleaved partial sums
// per dot, then a fixed-order sum of the 8.
__device__ void sum_dots(const LzArgs &a, LzShared &S, int region, int j) {
    const double *d = a.dots + (size_t)region * a.nrow_grid * DLD;
    for (int base = 0; base <= j; base += LT / 8) {
        const int i = base + (threadIdx.x >> 3), part = threadIdx.x & 7;
        double s = 0.0;
        if (i <= j)
            for (int b = part; b < a.nrow_grid; b += 8) s += d[(size_t)b * DLD + i];
        S.red[threadIdx.x] = s;
        __syncthreads();
        if (part == 0 && i <= j) {
            double t = 0.0;
            for (int q = 0; q < 8; ++q) t += S.red[threadIdx.x + q];
            S.h[i] = t;
        }
        __syncthreads();
    }
}

// w[e] -= sum_{i<=j} V[i][e] h[i] with the i-sum split over 8 threads per entry.
__device__ void block_update(LzShared &S, int E, int j) {
    const int e = threadIdx.x >> 3, part = threadIdx.x & 7;
    for (int eb = 0; eb < E; eb += LT / 8) {
        const int ee = eb + e;
        double s = 0.0;
        if (ee < E)
            for (int i = part; i <= j; i += 8) s = fma(S.V[i * LE + ee], S.h[i], s);
        S.red[threadIdx.x] = s;
        __syncthreads();
        if (part == 0 && ee < E) {
            double t = 0.0;
            for (int q = 0; q < 8; ++q) t += S.red[threadIdx.x + q];
            S.w[ee] -= t;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(LT) k_lz_a(LzArgs a, int j) {
    if (lz_skip(a.st)) return;
    __shared__ LzShared S;
    int e0, e1;
    cta_range(a, e0, e1);
    const int E = e1 - e0;
    load_block(a, S, e0, e1, j, false);
    // w = sum_b part[b][e]: threads (entry, 1 of 8 slices of b), fixed-order combine
    {
        const int part = threadIdx.x & 7;
        for (int eb = 0; eb < E; eb += LT / 8) {
            const int ee = eb + (threadIdx.x >> 3);
            double acc = 0.0;
            if (ee < E)
                for (int b = part; b < a.nparts; b += 8)
                    acc += a.part[(size_t)b * 2 * a.ldp + e0 + ee];
            S.red[threadIdx.x] = acc;
            __syncthreads();
            if (part == 0 && ee < E) {
                double t = 0.0;
                for (int q = 0; q < 8; ++q) t += S.red[threadIdx.x + q];
                // three-term recurrence (Algorithm 2): w = A v_j - beta_{j-1} v_{j-1}
                if (a.three_term && j > 0) t = fma(-a.st->beta[j - 1], S.V[(j - 1) * LE + ee], t);
                S.w[ee] = t;
                a.w[e0 + ee] = t;
            }
            __syncthreads();
        }
    }
    block_dots(S, E, j, a.dots + (size_t)blockIdx.x * DLD);
}

__global__ void __launch_bounds__(LT) k_lz_b(LzArgs a, int j) {
    if (lz_skip(a.st)) return;
    __shared__ LzShared S;
    int e0, e1;
    cta_range(a, e0, e1);
    const int E = e1 - e0;
    load_block(a, S, e0, e1, j, true);
    sum_dots(a, S, 0, j);
    // three-term recurrence: only alpha_j = v_j . w is removed
    if (a.three_term)
        for (int i = threadIdx.x; i < j; i += LT) S.h[i] = 0.0;
    __syncthreads();
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i <= j; i += LT) a.st->h1[i] = S.h[i];
    block_update(S, E, j);
    for (int e = threadIdx.x; e < E; e += LT) a.w[e0 + e] = S.w[e];
    block_dots(S, E, j, a.dots + ((size_t)a.nrow_grid + blockIdx.x) * DLD);
}

__global__ void __launch_bounds__(LT) k_lz_c(LzArgs a, int j) {
    if (lz_skip(a.st)) return;
    __shared__ LzShared S;
    __shared__ double coef[2];
    int e0, e1;
    cta_range(a, e0, e1);
    const int E = e1 - e0;
    load_block(a, S, e0, e1, j, true);
    if (j >= 0 && a.three_term) {
        if (blockIdx.x == 0 && threadIdx.x == 0) a.st->alpha[j] = a.st->h1[j];
    } else if (j >= 0) {
        sum_dots(a, S, 1, j);
        if (blockIdx.x == 0 && threadIdx.x == 0) a.st->alpha[j] = a.st->h1[j] + S.h[j];
        if (blockIdx.x == 0)
            for (int i = threadIdx.x; i <= j; i += LT) a.st->h2[i] = S.h[i];
        block_update(S, E, j);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (a.deflate) {
        // grid row r = blockIdx.x: entries 1..n alpha, n+1..2n beta, entry 0
        const int r = blockIdx.x, n = a.n_orb;
        if (warp == 0) {
            double sa = 0.0, sb = 0.0;
            for (int c = 1 + lane; c <= 2 * n; c += 32) {
                if (c <= n) sa += S.w[c]; else sb += S.w[c];
            }
            sa = warp_sum(sa);
            sb = warp_sum(sb);
            if (lane == 0) {
                if (r == 0) {
                    coef[0] = sa / n;
                    coef[1] = sb / n;
                } else {
                    // least squares on span{1_alpha - Na e0, 1_beta - Nb e0}
                    const double w0 = S.w[0];
                    const double na = a.na, nb = a.nb;
                    const double g11 = n + na * na, g22 = n + nb * nb, g12 = na * nb;
                    const double r1 = sa - na * w0, r2 = sb - nb * w0;
                    const double det = g11 * g22 - g12 * g12;
                    coef[0] = (g22 * r1 - g12 * r2) / det;
                    coef[1] = (g11 * r2 - g12 * r1) / det;
                }
            }
        }
        __syncthreads();
        for (int c = threadIdx.x; c <= 2 * n; c += LT) {
            if (c == 0) {
                if (r > 0) S.w[0] += coef[0] * a.na + coef[1] * a.nb;
            } else if (c <= n) {
                S.w[c] -= coef[0];
            } else {
                S.w[c] -= coef[1];
            }
        }
        __syncthreads();
    }
    double s2 = 0.0;
    for (int e = threadIdx.x; e < E; e += LT) {
        a.w[e0 + e] = S.w[e];
        s2 = fma(S.w[e], S.w[e], s2);
    }
    s2 = warp_sum(s2);
    if (lane == 0) S.red[warp] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < LT / 32; ++w) t += S.red[w];
        a.dots[((size_t)2 * a.nrow_grid + blockIdx.x) * DLD] = t;
    }
}

// beta = |w| (fixed-order sum of CTA partials), v_{jout} = w / beta.
// mode 0: Lanczos step j (jout = j+1, stores beta_j, breakdown test)
// mode 1: start vector (jout = 0)
// mode 2: restart residual (jout = k, stores beta_{k-1})
__global__ void __launch_bounds__(LT) k_lz_d(LzArgs a, int j, int jout, int mode) {
    if (mode == 0 && lz_skip(a.st)) return;
    __shared__ double red[LT];
    __shared__ double sb;
    __shared__ int sbrk;
    {
        double t = 0.0;
        for (int b = threadIdx.x; b < a.nrow_grid; b += LT)
            t += a.dots[((size_t)2 * a.nrow_grid + b) * DLD];
        red[threadIdx.x] = t;
        __syncthreads();
        for (int h = LT / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        const double beta = sqrt(red[0]);
        int brk = 0;
        if (mode == 0) {
            double tn = fmax(a.st->tnorm, fmax(fabs(a.st->alpha[j]), beta));
            if (j > 0) tn = fmax(tn, fabs(a.st->beta[j - 1]));
            if (beta <= 1e-14 * fmax(tn, 1e-300)) brk = 1;
            if (blockIdx.x == 0) {
                a.st->beta[j] = beta;
                a.st->tnorm = tn;
                if (brk) {
                    a.st->broke = 1;
                    a.st->jend = j + 1;
                }
            }
        } else if (mode == 2 && blockIdx.x == 0) {
            a.st->beta[jout - 1] = beta;
        }
        sb = beta;
        sbrk = brk;
    }
    __syncthreads();
    if (sbrk) return;
    int e0, e1;
    cta_range(a, e0, e1);
    const double inv = sb > 0.0 ? 1.0 / sb : 0.0;
    double *vout = a.V + (size_t)jout * a.ldp;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) vout[e] = a.w[e] * inv;
}

// Grid-wide barrier for the cooperative Lanczos kernel (all CTAs co-resident by
// the cooperative launch). The last CTA to arrive resets the count and bumps
// the generation; the others poll it. The poll gives up after two seconds of
// wall time, sets FLAG_TIMEOUT and lets the CTA continue, so it cannot hang.
__device__ __forceinline__ void grid_barrier(unsigned *bar, int *flags,
                                             uint64_t limit_ns = LM_WAIT_LIMIT_NS) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (*gen == g) {
                if (global_ns() - t0 > limit_ns) {
                    atomicOr(flags, FLAG_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// One Lanczos step's vector work in a single cooperative launch: the bodies of
// k_lz_a, k_lz_b, k_lz_c and k_lz_d (mode 0) separated by grid barriers.
__global__ void __launch_bounds__(LT) k_lz_step(LzArgs a, int j) {
    if (lz_skip(a.st)) return;  // uniform across the grid (written before launch)
    __shared__ LzShared S;
    __shared__ double coef[2];
    __shared__ double sb;
    __shared__ int sbrk;
    int e0, e1;
    cta_range(a, e0, e1);
    const int E = e1 - e0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // (a) w = sum of the pencil partials; pass-1 dots
    load_block(a, S, e0, e1, j, false);
    {
        const int part = threadIdx.x & 7;
        for (int eb = 0; eb < E; eb += LT / 8) {
            const int ee = eb + (threadIdx.x >> 3);
            double acc = 0.0;
            if (ee < E)
                for (int b = part; b < a.nparts; b += 8)
                    acc += a.part[(size_t)b * 2 * a.ldp + e0 + ee];
            S.red[threadIdx.x] = acc;
            __syncthreads();
            if (part == 0 && ee < E) {
                double t = 0.0;
                for (int q = 0; q < 8; ++q) t += S.red[threadIdx.x + q];
                S.w[ee] = t;
            }
            __syncthreads();
        }
    }
    block_dots(S, E, j, a.dots + (size_t)blockIdx.x * DLD);
    grid_barrier(a.bar, a.flags);
    // (b) first projection; pass-2 dots
    sum_dots(a, S, 0, j);
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i <= j; i += LT) a.st->h1[i] = S.h[i];
    const double h1j = S.h[j];
    block_update(S, E, j);
    block_dots(S, E, j, a.dots + ((size_t)a.nrow_grid + blockIdx.x) * DLD);
    grid_barrier(a.bar, a.flags);
    // (c) second projection, alpha_j, null-space deflation, partial |w|^2
    sum_dots(a, S, 1, j);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.st->alpha[j] = h1j + S.h[j];
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i <= j; i += LT) a.st->h2[i] = S.h[i];
    block_update(S, E, j);
    if (a.deflate) {
        const int r = blockIdx.x, n = a.n_orb;
        if (warp == 0) {
            double sa = 0.0, sbe = 0.0;
            for (int c = 1 + lane; c <= 2 * n; c += 32) {
                if (c <= n) sa += S.w[c]; else sbe += S.w[c];
            }
            sa = warp_sum(sa);
            sbe = warp_sum(sbe);
            if (lane == 0) {
                if (r == 0) {
                    coef[0] = sa / n;
                    coef[1] = sbe / n;
                } else {
                    const double w0 = S.w[0];
                    const double na = a.na, nb = a.nb;
                    const double g11 = n + na * na, g22 = n + nb * nb, g12 = na * nb;
                    const double r1 = sa - na * w0, r2 = sbe - nb * w0;
                    const double det = g11 * g22 - g12 * g12;
                    coef[0] = (g22 * r1 - g12 * r2) / det;
                    coef[1] = (g11 * r2 - g12 * r1) / det;
                }
            }
        }
        __syncthreads();
        for (int c = threadIdx.x; c <= 2 * n; c += LT) {
            if (c == 0) {
                if (r > 0) S.w[0] += coef[0] * a.na + coef[1] * a.nb;
            } else if (c <= n) {
                S.w[c] -= coef[0];
            } else {
                S.w[c] -= coef[1];
            }
        }
        __syncthreads();
    }
    {
        double s2 = 0.0;
        for (int e = threadIdx.x; e < E; e += LT) s2 = fma(S.w[e], S.w[e], s2);
        s2 = warp_sum(s2);
        if (lane == 0) S.red[warp] = s2;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < LT / 32; ++w) t += S.red[w];
            a.dots[((size_t)2 * a.nrow_grid + blockIdx.x) * DLD] = t;
        }
    }
    grid_barrier(a.bar, a.flags);
    // (d) beta_j = |w|, breakdown test, v_{j+1} = w / beta_j
    {
        double t = 0.0;
        for (int b = threadIdx.x; b < a.nrow_grid; b += LT)
            t += a.dots[((size_t)2 * a.nrow_grid + b) * DLD];
        S.red[threadIdx.x] = t;
        __syncthreads();
        for (int hh = LT / 2; hh > 0; hh >>= 1) {
            if (threadIdx.x < hh) S.red[threadIdx.x] += S.red[threadIdx.x + hh];
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        const double beta = sqrt(S.red[0]);
        const double alpha = h1j + S.h[j];
        double tn = fmax(a.st->tnorm, fmax(fabs(alpha), beta));
        if (j > 0) tn = fmax(tn, fabs(a.st->beta[j - 1]));
        const int brk = beta <= 1e-14 * fmax(tn, 1e-300);
        sb = beta;
        sbrk = brk;
    }
    grid_barrier(a.bar, a.flags);  // every CTA has read tnorm / beta[j-1] before CTA 0 writes
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.st->beta[j] = sb;
        a.st->tnorm = fmax(a.st->tnorm, fmax(fabs(h1j + S.h[j]), sb));
        if (j > 0) a.st->tnorm = fmax(a.st->tnorm, fabs(a.st->beta[j - 1]));
        if (sbrk) {
            a.st->broke = 1;
            a.st->jend = j + 1;
        }
    }
    if (sbrk) return;
    const double inv = sb > 0.0 ? 1.0 / sb : 0.0;
    double *vout = a.V + (size_t)(j + 1) * a.ldp;
    for (int e = threadIdx.x; e < E; e += LT) vout[e0 + e] = S.w[e] * inv;
}

// ---------------------------------------------------------------- cluster step
// One Lanczos step's vector work in a single thread-block cluster of C = 8 or
// 16 CTAs (the whole grid). CTA q owns the parameter-grid rows
// [q R / C, (q + 1) R / C) (R = Nh + 1), so the particle-number projection
// stays inside a CTA. The three global reductions (pass-1 dots, pass-2 dots,
// |w|^2) are exchanged through distributed shared memory between hardware
// cluster barriers, and every CTA sums the C partials with the same fixed
// tree, so all CTAs hold bit-identical dots and beta. No CTA spins on memory.
//
// The vector arithmetic runs in double-float on the FP32 pipes (GB300 issues
// one FP64 warp instruction per ~16 cycles per SM, which made the FP64 form
// of this latency-bound step slow): the pencil writes its partials as
// double-float pairs, the V slice is split into pairs by integer operations,
// and FP64 remains only for the stored basis vector and the scalars (alpha,
// beta, its square root and reciprocal, the projection coefficients).
constexpr int CT = 512;   // threads per cluster CTA
constexpr int CE = 384;   // entries per CTA: P+1 <= 2048 gives <= 2048/8 + 65 + 31
constexpr int CROWS = 16; // grid rows per CTA: Nh + 1 <= 128 over >= 8 CTAs
constexpr int CW = CT / 32;

__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_sync() {
    cluster_arrive();
    cluster_wait();
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_ncta() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// Generic address of the same shared variable in cluster CTA `rank`.
__device__ __forceinline__ const float2 *peer_ptr(const float2 *local, uint32_t rank) {
    uint64_t r;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(r) : "l"(local), "r"(rank));
    return reinterpret_cast<const float2 *>(r);
}
__device__ __forceinline__ df ldf(const float2 *p) {
    const float2 v = *p;
    return df_make(v.x, v.y);
}
__device__ __forceinline__ void stf(float2 *p, df a) { *p = make_float2(a.h, a.l); }
__device__ __forceinline__ df shfl_df(df a, int off) {
    return df_make(__shfl_xor_sync(0xffffffffu, a.h, off), __shfl_xor_sync(0xffffffffu, a.l, off));
}

struct LcShared {
    float2 w[CE];                  // (the V slice follows in dynamic shared memory)
    float2 pd1[LM_MAXKRYLOV + 1];  // this CTA's pass-1 partial dots (read by peers)
    float2 pd2[LM_MAXKRYLOV + 1];  // pass-2 partial dots (read by peers)
    float2 pn[1];                  // partial |w|^2 (read by peers)
    float2 h[LM_MAXKRYLOV + 1];    // reduced dots
    float2 h1s[LM_MAXKRYLOV + 1];  // reduced pass-1 dots kept for the state (CTA 0)
    float2 red[CT];
    float2 coef[CROWS][2];
};

// sum over the C <= 16 cluster CTAs of x[rank] with one fixed pairwise tree
__device__ __forceinline__ df cluster_tree_sum(const float2 *local, int C) {
    df x[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) x[r] = r < C ? ldf(peer_ptr(local, (uint32_t)r)) : df_make(0.f, 0.f);
#pragma unroll
    for (int h = 8; h > 0; h >>= 1)
#pragma unroll
        for (int r = 0; r < h; ++r) x[r] = df_add(x[r], x[r + h]);
    return x[0];
}

// pd[i] = V[:, i] . w over this CTA's entries, i <= j, from the staged slice
// Vs (leading dimension le): four threads per dot, each over every fourth
// entry, combined by two shuffle levels.
__device__ __forceinline__ void cluster_dots(const float2 *Vs, int le, const LcShared &S, int E,
                                             int j, float2 *pd) {
    const int i = threadIdx.x >> 2, part = threadIdx.x & 3;
    df s0 = df_make(0.f, 0.f), s1 = df_make(0.f, 0.f);
    if (i <= j) {
        const float2 *vi = Vs + (size_t)i * le;
        int e = part;
        for (; e + 4 < E; e += 8) {
            s0 = df_fma(ldf(vi + e), ldf(S.w + e), s0);
            s1 = df_fma(ldf(vi + e + 4), ldf(S.w + e + 4), s1);
        }
        if (e < E) s0 = df_fma(ldf(vi + e), ldf(S.w + e), s0);
    }
    df t = df_add(s0, s1);
    t = df_add(t, shfl_df(t, 1));
    t = df_add(t, shfl_df(t, 2));
    if (part == 0 && i <= j) stf(pd + i, t);
}

// floor(t / d) for 0 <= t, d < 2^22 without a divide (a divide converts to and
// from floating point, and conversions issue at the FP64 rate on this part):
// t and d are exact in FP32 by adding them into the mantissa of 1.5 * 2^23,
// t * (1/d) rounded to an integer is within one of the quotient, and one exact
// integer comparison each way fixes it. rd = __frcp_rn(d as FP32).
__device__ __forceinline__ float small_float(int v) {
    return __fsub_rn(__int_as_float(0x4B400000 + v), 12582912.0f);
}
__device__ __forceinline__ int small_div(int t, int d, float rd) {
    int q = __float_as_int(__fadd_rn(__fmul_rn(small_float(t), rd), 12582912.0f)) - 0x4B400000;
    q -= (q * d > t) ? 1 : 0;
    q += ((q + 1) * d <= t) ? 1 : 0;
    return q;
}

// w[e] -= sum_{i<=j} Vs[i][e] h[i]: thread (g, e) sums i = g, g + ng, ...; the
// ng group sums are combined in group order.
__device__ __forceinline__ void cluster_update(const float2 *Vs, int le, LcShared &S, int E, int EP,
                                               int ng, int j, int g, int e) {
    const int tid = threadIdx.x;
    df s0 = df_make(0.f, 0.f), s1 = df_make(0.f, 0.f);
    if (g < ng && e < E) {
        int i = g;
        for (; i + ng <= j; i += 2 * ng) {
            s0 = df_fma(ldf(Vs + (size_t)i * le + e), ldf(S.h + i), s0);
            s1 = df_fma(ldf(Vs + (size_t)(i + ng) * le + e), ldf(S.h + i + ng), s1);
        }
        if (i <= j) s0 = df_fma(ldf(Vs + (size_t)i * le + e), ldf(S.h + i), s0);
    }
    stf(S.red + tid, df_add(s0, s1));
    __syncthreads();
    if (tid < E) {
        df t = df_make(0.f, 0.f);
        for (int q = 0; q < ng; ++q) t = df_add(t, ldf(S.red + q * EP + tid));
        stf(S.w + tid, df_sub(ldf(S.w + tid), t));
    }
    __syncthreads();
}

__global__ void __launch_bounds__(CT, 1) k_lz_cluster(LzArgs a, int j) {
    if (lz_skip(a.st)) return;  // uniform across the cluster (written before launch)
    __shared__ LcShared S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int C = (int)cluster_ncta(), q = (int)cluster_rank();
    const int R = a.nrow_grid;
    const float rC = __frcp_rn(small_float(C));
    const int rlo = small_div(q * R, C, rC), rhi = small_div((q + 1) * R, C, rC);
    const int e0 = rlo * a.M1;
    const int E = (q == C - 1 ? a.ldp : rhi * a.M1) - e0;
    const int EP = E > 0 ? (E + 31) & ~31 : 32;
    const float rEP = __frcp_rn(small_float(EP));
    const int ng = max(1, min(16, small_div(CT, EP, rEP)));
    const int tg = small_div(tid, EP, rEP), te = tid - tg * EP;
    // state that CTA 0 overwrites at the end, read before the first barrier
    const double tn0 = a.st->tnorm;
    const double bprev = j > 0 ? a.st->beta[j - 1] : 0.0;
    const float tn0f = (float)tn0, bprevf = (float)fabs(bprev);
    // stage V[:, 0..j] over this CTA's entries as double-float pairs (odd
    // leading dimension: the four dot threads of different columns in a warp
    // fall in different banks)
    extern __shared__ float2 Vs[];
    const int le = E | 1;
    {
        const float rE = __frcp_rn(small_float(max(E, 1)));
        for (int t = tid; t < (j + 1) * E; t += CT) {
            const int i = small_div(t, E, rE), e = t - i * E;
            stf(Vs + (size_t)i * le + e, df_split_bits(a.V[(size_t)i * a.ldp + e0 + e]));
        }
    }

    // (a) w = sum over the pencil CTAs' double-float partials: batches of 8
    // independent loads summed pairwise, batches in order, groups in order
    {
        const float2 *part = reinterpret_cast<const float2 *>(a.part);
        const int g = tg, e = te;
        df acc = df_make(0.f, 0.f);
        if (g < ng && e < E) {
            const float2 *src = part + e0 + e;
            const size_t stride = 2 * (size_t)a.ldp;
            // 16 loads in flight per round (zeros past the end), summed pairwise
            for (int b = g; b < a.nparts; b += 16 * ng) {
                df x[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int bb = b + u * ng;
                    x[u] = bb < a.nparts ? ldf(src + (size_t)bb * stride) : df_make(0.f, 0.f);
                }
#pragma unroll
                for (int h = 8; h > 0; h >>= 1)
#pragma unroll
                    for (int u = 0; u < h; ++u) x[u] = df_add(x[u], x[u + h]);
                acc = df_add(acc, x[0]);
            }
        }
        stf(S.red + tid, acc);
        __syncthreads();
        if (tid < E) {
            df t = df_make(0.f, 0.f);
            for (int gg = 0; gg < ng; ++gg) t = df_add(t, ldf(S.red + gg * EP + tid));
            stf(S.w + tid, t);
        }
        __syncthreads();
    }
    // (b) pass 1: h1 = V^T w, w -= V h1
    cluster_dots(Vs, le, S, E, j, S.pd1);
    cluster_sync();
    for (int i = tid; i <= j; i += CT) stf(S.h + i, cluster_tree_sum(S.pd1 + i, C));
    __syncthreads();
    const df h1j = ldf(S.h + j);
    if (q == 0 && tid <= j) stf(S.h1s + tid, ldf(S.h + tid));  // kept for the state
    cluster_update(Vs, le, S, E, EP, ng, j, tg, te);
    // (c) pass 2: h2 = V^T w, w -= V h2; alpha_j = h1_j + h2_j
    cluster_dots(Vs, le, S, E, j, S.pd2);
    cluster_sync();  // also orders the reads of S.h above before it is overwritten
    for (int i = tid; i <= j; i += CT) stf(S.h + i, cluster_tree_sum(S.pd2 + i, C));
    __syncthreads();
    const df alpha = df_add(h1j, ldf(S.h + j));
    cluster_update(Vs, le, S, E, EP, ng, j, tg, te);
    // (d) particle-number null space, per grid row (warp per row); the row sums
    // in double-float, the 2 x 2 solve in FP64 by one lane
    if (a.deflate) {
        const int n = a.n_orb;
        const int nr = rhi - rlo;
        if (warp < nr) {
            const int r = rlo + warp;
            const float2 *wr = S.w + (size_t)warp * a.M1;
            df sa = df_make(0.f, 0.f), sbe = df_make(0.f, 0.f);
            for (int c = 1 + lane; c <= 2 * n; c += 32) {
                if (c <= n) sa = df_add(sa, ldf(wr + c));
                else sbe = df_add(sbe, ldf(wr + c));
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                sa = df_add(sa, shfl_df(sa, off));
                sbe = df_add(sbe, shfl_df(sbe, off));
            }
            if (lane == 0) {
                df c0, c1;
                if (r == 0) {
                    c0 = df_mul(sa, ldf(&a.inv_n));
                    c1 = df_mul(sbe, ldf(&a.inv_n));
                } else {
                    // least squares on span{1_alpha - Na e0, 1_beta - Nb e0}
                    const df w0 = ldf(wr);
                    const float na = (float)a.na, nb = (float)a.nb;  // exact
                    const df r1 = df_sub(sa, df_mul(df_make(na, 0.f), w0));
                    const df r2 = df_sub(sbe, df_mul(df_make(nb, 0.f), w0));
                    c0 = df_add(df_mul(ldf(&a.gi11), r1), df_mul(ldf(&a.gi12), r2));
                    c1 = df_add(df_mul(ldf(&a.gi12), r1), df_mul(ldf(&a.gi22), r2));
                }
                stf(&S.coef[warp][0], c0);
                stf(&S.coef[warp][1], c1);
                // entry 0 of a hidden row moves by Na c0 + Nb c1
                stf(&S.red[warp], df_add(df_mul(df_make((float)a.na, 0.f), c0),
                                         df_mul(df_make((float)a.nb, 0.f), c1)));
            }
        }
        __syncthreads();
        const float rM1 = __frcp_rn(small_float(a.M1));
        for (int t = tid; t < nr * a.M1; t += CT) {
            const int lr = small_div(t, a.M1, rM1), c = t - lr * a.M1;
            float2 *wr = S.w + (size_t)lr * a.M1;
            if (c == 0) {
                if (rlo + lr > 0) stf(wr, df_add(ldf(wr), ldf(&S.red[lr])));
            } else {
                stf(wr + c, df_sub(ldf(wr + c), ldf(&S.coef[lr][c <= n ? 0 : 1])));
            }
        }
        __syncthreads();
    }
    // (e) beta_j = |w| (df: s = |w|^2, y = 1/sqrt(s), beta = s y), breakdown
    // test, v_{j+1} = w y
    {
        df s2 = df_make(0.f, 0.f);
        if (warp * 32 < E) {
            for (int e = tid; e < E; e += CT) {
                const df we = ldf(S.w + e);
                s2 = df_fma(we, we, s2);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s2 = df_add(s2, shfl_df(s2, off));
        }
        __syncthreads();  // the projection's use of S.red is over
        if (lane == 0) stf(S.red + warp, s2);
        __syncthreads();
        if (warp == 0) {
            df t = lane < CW ? ldf(S.red + lane) : df_make(0.f, 0.f);
#pragma unroll
            for (int off = CW / 2; off > 0; off >>= 1) t = df_add(t, shfl_df(t, off));
            if (lane == 0) stf(S.pn, t);
        }
    }
    cluster_sync();
    const df ss = cluster_tree_sum(S.pn, C);
    cluster_arrive();  // this CTA reads no peer memory after this point
    const df y = ss.h > 0.f ? df_rsqrt(ss) : df_make(0.f, 0.f);
    const df beta = df_mul(ss, y);
    // the same decision in every CTA (FP32 threshold on identical values)
    const float tnf = fmaxf(fmaxf(tn0f, fabsf(alpha.h)), fmaxf(beta.h, bprevf));
    const bool brk = !(beta.h > 1e-14f * fmaxf(tnf, 1e-30f));
    if (!brk) {
        double *vout = a.V + (size_t)(j + 1) * a.ldp + e0;
        for (int e = tid; e < E; e += CT) vout[e] = df_to_double(df_mul(ldf(S.w + e), y));
    }
    if (q == 0) {
        if (tid <= j) {
            a.st->h1[tid] = df_to_double(ldf(S.h1s + tid));
            a.st->h2[tid] = df_to_double(ldf(S.h + tid));
        }
        if (tid == 0) {
            const double al = df_to_double(alpha), be = df_to_double(beta);
            double tn = fmax(tn0, fmax(fabs(al), be));
            if (j > 0) tn = fmax(tn, fabs(bprev));
            a.st->alpha[j] = al;
            a.st->beta[j] = be;
            a.st->tnorm = tn;
            if (brk) {
                a.st->broke = 1;
                a.st->jend = j + 1;
            }
        }
    }
    cluster_wait();  // no CTA exits while a peer may still read its shared memory
}

// Random start vector: component e is 2u-1 with u the 53-bit uniform of
// SplitMix64 at counter e (state seed + (e+1) * golden gamma), zero padding.
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t e) {
    uint64_t z = seed + (e + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

__global__ void k_init_start(double *w, int ldp, int P1, uint64_t seed, const double *v0) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ldp; e += gridDim.x * blockDim.x) {
        double x = 0.0;
        if (e < P1) x = v0 ? v0[e] : splitmix_uniform(seed, (uint64_t)e);
        w[e] = x;
    }
}

// ---------------------------------------------------------------- k_tri
constexpr int TT = 1024;

// Sturm count (number of eigenvalues < x) of the scaled tridiagonal, FP32.
__device__ __forceinline__ int sturm_f32(const float *a, const float *b2, int n, float x) {
    const float pivmin = 1e-30f;
    int cnt = 0;
    float q = a[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.0f;
    for (int i = 1; i < n; ++i) {
        q = (a[i] - x) - b2[i - 1] / q;
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += q < 0.0f;
    }
    return cnt;
}

// p_n(x) = det(T - x I) and p_{n-1}(x), p_n'(x) by the three-term recurrence
// (division free), on the scaled matrix.
__device__ __forceinline__ void charpoly(const double *a, const double *b2, int n, double x,
                                         double &pn, double &pn1, double &dpn) {
    double pm2 = 0.0, pm1 = 1.0, dm2 = 0.0, dm1 = 0.0;
    for (int i = 0; i < n; ++i) {
        const double bb = i > 0 ? b2[i - 1] : 0.0;
        const double p = (a[i] - x) * pm1 - bb * pm2;
        const double d = -pm1 + (a[i] - x) * dm1 - bb * dm2;
        pm2 = pm1;
        pm1 = p;
        dm2 = dm1;
        dm1 = d;
    }
    pn = pm1;
    pn1 = pm2;
    dpn = dm1;
}

struct TriArgs {
    IrlState *st;
    int m, k;
    int final_pass;
    double tol;  // absolute tolerance
    double rel;  // floor relative to ||T|| (50 eps for FP64 operators)
};

__global__ void __launch_bounds__(TT) k_tri(TriArgs t) {
    IrlState *st = t.st;
    __shared__ double a[LM_MAXKRYLOV], b[LM_MAXKRYLOV], as[LM_MAXKRYLOV], b2s[LM_MAXKRYLOV];
    __shared__ float af[LM_MAXKRYLOV], b2f[LM_MAXKRYLOV];
    __shared__ double ritz[LM_MAXKRYLOV];
    __shared__ double Q[LM_MAXKRYLOV * LM_MAXKRYLOV];
    __shared__ double rc[LM_MAXKRYLOV], rs[LM_MAXKRYLOV];
    __shared__ int rp[LM_MAXKRYLOV];
    __shared__ double sscale;
    __shared__ int je_s, conv_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        je_s = st->broke ? st->jend : t.m;
        conv_s = 0;
    }
    __syncthreads();
    const int je = je_s;
    for (int i = tid; i < je; i += TT) {
        a[i] = st->alpha[i];
        b[i] = i < je - 1 ? st->beta[i] : 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int i = 0; i < je; ++i) s = fmax(s, fabs(a[i]));
        for (int i = 0; i < je - 1; ++i) s = fmax(s, fabs(b[i]));
        sscale = s > 0.0 ? s : 1.0;
    }
    __syncthreads();
    const double sc = sscale;
    for (int i = tid; i < je; i += TT) {
        as[i] = a[i] / sc;
        af[i] = (float)as[i];
        double bb = i < je - 1 ? b[i] / sc : 0.0;
        b2s[i] = bb * bb;
        b2f[i] = (float)(bb * bb);
    }
    __syncthreads();
    // (1) brackets by 32-way multisection in FP32: warp -> eigenvalue index
    __shared__ float blo[LM_MAXKRYLOV], bhi[LM_MAXKRYLOV];
    for (int i = warp; i < je; i += TT / 32) {
        float lo = -3.0f, hi = 3.0f;  // scaled Gershgorin bound
        for (int round = 0; round < 6; ++round) {
            const float x = lo + (hi - lo) * (float)(lane + 1) / 33.0f;
            const int c = sturm_f32(af, b2f, je, x);
            const unsigned above = __ballot_sync(0xffffffffu, c > i);
            const int L = above ? __ffs(above) - 1 : 32;
            const float nhi = L < 32 ? lo + (hi - lo) * (float)(L + 1) / 33.0f : hi;
            const float nlo = L > 0 ? lo + (hi - lo) * (float)L / 33.0f : lo;
            lo = nlo;
            hi = nhi;
        }
        if (lane == 0) {
            blo[i] = lo;
            bhi[i] = hi;
        }
    }
    __syncthreads();
    // (2) FP64 safeguarded Newton on p_je inside the (widened) bracket
    if (tid < je) {
        const int i = tid;
        double lo = (double)blo[i] - 4e-7, hi = (double)bhi[i] + 4e-7;
        double x = 0.5 * ((double)blo[i] + (double)bhi[i]);
        double pn, pn1, dpn, plo, pl1, dl;
        charpoly(as, b2s, je, lo, plo, pl1, dl);
        double prev = INFINITY;
        for (int it = 0; it < 12; ++it) {
            charpoly(as, b2s, je, x, pn, pn1, dpn);
            if (pn == 0.0) break;
            const double step = dpn != 0.0 ? pn / dpn : 0.0;
            // converged: accept an ulp-sized Newton step before any safeguarding
            if (dpn != 0.0 && fabs(step) <= 4.0 * 2.220446049250313e-16 * fabs(x)) {
                x -= step;
                break;
            }
            // the rounding noise of p near the root: steps below 1e-12 of the scaled
            // norm that no longer halve are noise, not convergence still to come
            if (dpn != 0.0 && fabs(step) <= 1e-12 && fabs(step) > 0.5 * prev) break;
            prev = fabs(step);
            if ((pn > 0.0) == (plo > 0.0)) lo = x; else hi = x;
            double xn = dpn != 0.0 ? x - step : 0.5 * (lo + hi);
            if (!(xn >= lo && xn <= hi)) xn = 0.5 * (lo + hi);
            x = xn;
        }
        ritz[i] = x * sc;
    }
    __syncthreads();
    // (3) eigenvector of the lowest Ritz value by inverse iteration (FP64,
    // tridiagonal elimination with partial pivoting, two sweeps); its last
    // component gives the residual beta_m |u_m| of the Ritz pair.
    __shared__ double us[LM_MAXKRYLOV];
    if (tid == 0) {
        const double lam = ritz[0];
        const double eps = 2.220446049250313e-16 * sc;
        double y[LM_MAXKRYLOV], d[LM_MAXKRYLOV], du[LM_MAXKRYLOV], du2[LM_MAXKRYLOV],
            dl[LM_MAXKRYLOV];
        int piv[LM_MAXKRYLOV];
        for (int i = 0; i < je; ++i) {
            d[i] = a[i] - lam;
            du[i] = i < je - 1 ? b[i] : 0.0;
            dl[i] = i < je - 1 ? b[i] : 0.0;
            du2[i] = 0.0;
            y[i] = 1.0;
        }
        // LU with partial pivoting (the dgttrf layout)
        for (int i = 0; i < je - 1; ++i) {
            if (fabs(d[i]) >= fabs(dl[i])) {
                piv[i] = 0;
                if (d[i] == 0.0) d[i] = eps;
                const double f = dl[i] / d[i];
                dl[i] = f;
                d[i + 1] -= f * du[i];
            } else {
                piv[i] = 1;
                const double f = d[i] / dl[i];
                d[i] = dl[i];
                dl[i] = f;
                const double tmp = du[i];
                du[i] = d[i + 1];
                d[i + 1] = tmp - f * d[i + 1];
                if (i < je - 2) {
                    du2[i] = du[i + 1];
                    du[i + 1] = -f * du[i + 1];
                }
            }
        }
        if (d[je - 1] == 0.0) d[je - 1] = eps;
        // pivot reciprocals once (independent divisions), so the solves are
        // chains of multiply-adds only
        for (int i = 0; i < je; ++i) d[i] = 1.0 / d[i];
        for (int sweep = 0; sweep < 2; ++sweep) {
            for (int i = 0; i < je - 1; ++i) {
                if (piv[i] == 0) {
                    y[i + 1] -= dl[i] * y[i];
                } else {
                    const double tmp = y[i];
                    y[i] = y[i + 1];
                    y[i + 1] = tmp - dl[i] * y[i];
                }
            }
            y[je - 1] *= d[je - 1];
            if (je > 1) y[je - 2] = (y[je - 2] - du[je - 2] * y[je - 1]) * d[je - 2];
            for (int i = je - 3; i >= 0; --i)
                y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) * d[i];
            double nn = 0.0;
            for (int i = 0; i < je; ++i) nn += y[i] * y[i];
            nn = 1.0 / sqrt(nn);
            for (int i = 0; i < je; ++i) y[i] *= nn;
        }
        for (int i = 0; i < je; ++i) us[i] = y[i];
        double tn = 0.0;
        for (int i = 0; i < je; ++i) tn = fmax(tn, fabs(ritz[i]));
        const double tol_eff = fmax(t.tol, t.rel * tn);
        const double bres = st->broke ? 0.0 : fabs(st->beta[je - 1]);
        const double res = bres * fabs(y[je - 1]);
        st->lam = ritz[0];
        st->res = res;
        st->tol_eff = tol_eff;
        st->bnorm = tn;
        const int conv = st->broke || res < tol_eff;
        st->conv = conv;
        conv_s = conv;
    }
    __syncthreads();
    for (int i = tid; i < je; i += TT) st->ritz[i] = ritz[i];
    if (conv_s || t.final_pass) {
        for (int i = tid; i < je; i += TT) st->u[i] = us[i];
        if (tid == 0) st->jend = je;
        return;
    }
    // (4) implicit restart: mu = m - k shifts (largest first), pipelined chase
    const int m = je, k = t.k, mu = m - k;
    for (int e = tid; e < m * m; e += TT) Q[e] = (e % (m + 1) == 0) ? 1.0 : 0.0;
    __syncthreads();
    double bx = 0.0, bz = 0.0;  // per-bulge state (thread q < mu)
    const int nsteps = (m - 1) + 4 * (mu - 1);
    for (int step = 0; step < nsteps; ++step) {
        if (tid < mu) {
            const int q = tid;
            const int p = step - 4 * q;
            if (p >= 0 && p <= m - 2) {
                if (p == 0) {
                    bx = a[0] - ritz[m - 1 - q];
                    bz = b[0];
                }
                // Givens rotation from one reciprocal square root (r = |(x, z)|)
                const double r2 = fma(bx, bx, bz * bz);
                double r = 0.0, c = 1.0, s = 0.0;
                if (r2 > 1e-300) {
                    const double ri = rsqrt(r2);
                    c = bx * ri;
                    s = bz * ri;
                    r = r2 * ri;
                }
                if (p > 0) b[p - 1] = r;
                const double ap = a[p], aq = a[p + 1], bp = b[p];
                a[p] = c * c * ap + 2.0 * c * s * bp + s * s * aq;
                a[p + 1] = s * s * ap - 2.0 * c * s * bp + c * c * aq;
                b[p] = c * s * (aq - ap) + (c * c - s * s) * bp;
                if (p < m - 2) {
                    bz = s * b[p + 1];
                    b[p + 1] = c * b[p + 1];
                    bx = b[p];
                }
                rc[q] = c;
                rs[q] = s;
                rp[q] = p;
            } else {
                rp[q] = -1;
            }
        }
        __syncthreads();
        for (int e = tid; e < mu * m; e += TT) {
            const int q = e / m, i = e % m;
            const int p = rp[q];
            if (p >= 0) {
                const double c = rc[q], s = rs[q];
                const double x0 = Q[p * m + i], x1 = Q[(p + 1) * m + i];
                Q[p * m + i] = c * x0 + s * x1;
                Q[(p + 1) * m + i] = -s * x0 + c * x1;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < m * (k + 1); e += TT) st->Q[e] = Q[e];
    for (int i = tid; i < k; i += TT) st->alpha[i] = a[i];
    for (int i = tid; i < k - 1; i += TT) st->beta[i] = b[i];
    if (tid == 0) {
        st->h1[0] = b[k - 1];                          // beta_hat_k
        st->h2[0] = st->beta[m - 1] * Q[(k - 1) * m + (m - 1)];  // beta_m Q[m-1, k-1]
    }
}

// V_new[:, i] = V[:, :m] Q[:, i] (i < k); w = beta_hat V Q[:, k] + sigma V[:, m];
// per-CTA partial |w|^2 into dots region 2.
__global__ void __launch_bounds__(LT) k_restart(LzArgs a, double *Vnew, int m, int k) {
    __shared__ double Qs[LM_MAXKRYLOV * (LM_MAXKRYLOV + 1)];
    __shared__ double red[LT / 32];
    for (int e = threadIdx.x; e < m * (k + 1); e += blockDim.x) Qs[e] = a.st->Q[e];
    __syncthreads();
    const double bhat = a.st->h1[0], sigma = a.st->h2[0];
    int e0, e1;
    cta_range(a, e0, e1);
    double s2 = 0.0;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        for (int i = 0; i <= k; ++i) {
            double acc = 0.0;
            for (int l = 0; l < m; ++l) acc = fma(a.V[(size_t)l * a.ldp + e], Qs[i * m + l], acc);
            if (i < k) {
                Vnew[(size_t)i * a.ldp + e] = acc;
            } else {
                const double f = fma(sigma, a.V[(size_t)m * a.ldp + e], bhat * acc);
                a.w[e] = f;
                s2 = fma(f, f, s2);
            }
        }
    }
    s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < LT / 32; ++w) t += red[w];
        a.dots[((size_t)2 * a.nrow_grid + blockIdx.x) * DLD] = t;
    }
}

// y = V[:, :jend] u (the Ritz vector)
__global__ void k_ritz_vector(const double *V, const IrlState *st, int ldp, double *y) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ldp; e += gridDim.x * blockDim.x) {
        double acc = 0.0;
        const int n = st->jend;
        for (int l = 0; l < n; ++l) acc = fma(V[(size_t)l * ldp + e], st->u[l], acc);
        y[e] = acc;
    }
}

// One-CTA refinement: Rayleigh quotients, explicit residual, sign of c_0,
// update Delta theta = c[1:]/c[0] (and theta += Delta theta on request).
__global__ void __launch_bounds__(1024) k_refine(double *y, const double *hy, const double *sy,
                                                 IrlState *st, int ldp, int P1, double *c_out,
                                                 double *dth_out, double *theta, double tol,
                                                 int *status_out) {
    __shared__ double red[32][4];
    __shared__ double sv[5];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double yy = 0.0, yh = 0.0, ys = 0.0;
    for (int e = tid; e < P1; e += blockDim.x) {
        yy = fma(y[e], y[e], yy);
        yh = fma(y[e], hy[e], yh);
        ys = fma(y[e], sy[e], ys);
    }
    yy = warp_sum(yy);
    yh = warp_sum(yh);
    ys = warp_sum(ys);
    if (lane == 0) {
        red[warp][0] = yy;
        red[warp][1] = yh;
        red[warp][2] = ys;
    }
    __syncthreads();
    if (tid == 0) {
        double A = 0, B = 0, C = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            A += red[w][0];
            B += red[w][1];
            C += red[w][2];
        }
        sv[0] = A;
        sv[1] = B;
        sv[2] = C;
        sv[3] = y[0] < 0.0 ? -1.0 : 1.0;
        sv[4] = fabs(y[0]);
    }
    __syncthreads();
    const double nrm = sqrt(sv[0]);
    const double lam = sv[1] / sv[0];  // explicit FP64 Rayleigh quotient of the Ritz vector
    const double sgn = sv[3] / nrm;
    double rr = 0.0;
    for (int e = tid; e < P1; e += blockDim.x) {
        const double r = (hy[e] - lam * y[e]) / nrm;
        rr = fma(r, r, rr);
    }
    rr = warp_sum(rr);
    if (lane == 0) red[warp][3] = rr;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][3];
        st->res_explicit = sqrt(t);
        st->rq = sv[1] / sv[0];
        st->lam_ritz = st->lam;
        st->lam = st->rq;
        st->rq_s = sv[1] / sv[2];
        st->c0 = fabs(y[0]) / nrm;
        st->yty = sv[0];
        int status = st->broke ? IRL_BREAKDOWN_INVARIANT : (st->conv ? IRL_OK : IRL_MAX_RESTARTS);
        if (lam > -tol) status = LM_STATIONARY;
        else if (fabs(y[0]) / nrm < 1e-8) status = LM_C0_TINY;
        *status_out = status;
        sv[0] = (double)status;
    }
    __syncthreads();
    const int status = (int)sv[0];
    const bool upd = (status == IRL_OK || status == IRL_BREAKDOWN_INVARIANT);
    const double inv_c0 = 1.0 / (sv[4] / sqrt(sv[0] > 0.0 ? sv[0] : 1.0));
    for (int e = tid; e < ldp; e += blockDim.x) {
        const double c = e < P1 ? sgn * y[e] : 0.0;
        y[e] = c;
        if (c_out && e < P1) c_out[e] = c;
        if (e >= 1 && e < P1) {
            const double d = upd ? c * inv_c0 : 0.0;
            if (dth_out) dth_out[e - 1] = d;
            if (theta && upd) theta[e - 1] += d;
        }
    }
}


// Waits that nothing ends, for tests of the timeout path: which = 0, the grid
// barrier of the cooperative Lanczos kernel with a CTA that leaves without
// arriving (2 CTAs); which = 1, an mbarrier phase that no thread or copy
// completes (the wait of the pencil pipeline). Both give up after limit_ns.
__global__ void k_debug_wait(int which, uint64_t limit_ns, unsigned *bar, int *flags) {
    if (which == 0) {
        if (blockIdx.x != 0) return;
        grid_barrier(bar, flags, limit_ns);
        return;
    }
    __shared__ uint64_t mb;
    if (threadIdx.x == 0) {
        mbar_init(&mb, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&mb, 0, limit_ns)) atomicOr(flags, FLAG_TIMEOUT);
}

}  // namespace

// =========================================================================
// host side
// =========================================================================
namespace {

// How a Lanczos step's vector work is launched.
enum { LZ_SPLIT = 0, LZ_COOP = 1, LZ_CLUSTER = 2 };

struct Run {
    lm_pencil *p;
    cudaStream_t s;
    LzArgs la;
    int m, k, sym, prec;
    int n_matvec, n_restart;
    int lz_mode;   // LZ_*
    int cluster;   // CTAs per cluster for LZ_CLUSTER
    int cluster_emax;  // largest entry count of one cluster CTA
    // row shards: each product is summed over the shards by the caller
    lm_reduce_fn reduce;
    void *reduce_user;
    int reduce_where;
};

// Sum a device vector of n doubles over the row shards with the caller's
// reduction (see irl_step_sharded), in place.
int shard_reduce(Run &R, double *dvec, int n) {
    lm_pencil *p = R.p;
    lm_ctx *ctx = p->ctx;
    if (R.reduce_where == LM_REDUCE_DEVICE) {
        if (int rc = R.reduce(dvec, n, (void *)R.s, R.reduce_user))
            return lm_fail(ctx, LM_ERR_CALLBACK, "reduction callback returned %d", rc);
        return lm_cuda_check(ctx, cudaGetLastError(), "after the reduction callback");
    }
    double *h = p->hs->xfer;
    cudaError_t e = cudaMemcpyAsync(h, dvec, n * sizeof(double), cudaMemcpyDeviceToHost, R.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(R.s);
    if (int rc = lm_cuda_check(ctx, e, "shard vector read-back")) return rc;
    if (int rc = R.reduce(h, n, (void *)R.s, R.reduce_user))
        return lm_fail(ctx, LM_ERR_CALLBACK, "reduction callback returned %d", rc);
    // the next read-back into the same staging is ordered after this copy
    return lm_cuda_check(ctx, cudaMemcpyAsync(dvec, h, n * sizeof(double),
                                              cudaMemcpyHostToDevice, R.s),
                         "shard vector upload");
}

// Dynamic shared memory of k_lz_cluster for Lanczos step j: the V[:, 0..j]
// slice with an odd leading dimension.
size_t cluster_dyn_smem(int j1, int emax) { return (size_t)j1 * (emax | 1) * sizeof(double); }

// Largest entry count and grid-row count of one CTA when R grid rows of M1
// entries (ldp in all) are split over C CTAs the way k_lz_cluster splits them.
void cluster_extent(int R, int M1, int ldp, int C, int &emax, int &rmax) {
    emax = 0;
    rmax = 0;
    for (int q = 0; q < C; ++q) {
        const int rlo = q * R / C, rhi = (q + 1) * R / C;
        const int e = (q == C - 1 ? ldp : rhi * M1) - rlo * M1;
        emax = std::max(emax, e);
        rmax = std::max(rmax, rhi - rlo);
    }
}

// Pick the Lanczos launch: one cluster of 16 (else 8) CTAs when the device can
// place it and the split fits the kernel's shared arrays, else the cooperative
// kernel, else four ordinary launches. IRLNQS_LANCZOS=cluster|coop|split
// restricts the choice (for tests); a mode the device cannot run is skipped.
void choose_lanczos(Run &R, lm_ctx *ctx) {
    const char *env = getenv("IRLNQS_LANCZOS");
    const bool any = !env || !*env;
    R.lz_mode = LZ_SPLIT;
    R.cluster = 0;
    // the cluster step sums the pencil CTAs' double-float partials itself; a
    // sharded solve hands it one reduced FP64 vector instead. The three-term
    // recurrence (no reorthogonalisation) runs in the four-kernel form only.
    if ((any || !strcmp(env, "cluster")) && !R.reduce && !R.la.three_term && !R.p->chunk) {
        for (int C : {16, 8}) {
            int emax = 0, rmax = 0;
            cluster_extent(R.la.nrow_grid, R.la.M1, R.la.ldp, C, emax, rmax);
            if (emax > CE || rmax > CROWS) continue;
            const size_t dyn = cluster_dyn_smem(R.m, emax);
            if (dyn + sizeof(LcShared) > (size_t)ctx->smem_optin) continue;
            if (cudaFuncSetAttribute(k_lz_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)dyn) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (C > 8 && cudaFuncSetAttribute(k_lz_cluster,
                                              cudaFuncAttributeNonPortableClusterSizeAllowed,
                                              1) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(CT);
            cfg.dynamicSmemBytes = dyn;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, k_lz_cluster, &cfg) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (nclusters >= 1) {
                R.lz_mode = LZ_CLUSTER;
                R.cluster = C;
                R.cluster_emax = emax;
                return;
            }
        }
    }
    if ((any || !strcmp(env, "coop")) && !R.la.three_term) {
        // the cooperative step needs all nh+1 CTAs resident at once
        int dev_coop = 0, per_sm = 0;
        cudaDeviceGetAttribute(&dev_coop, cudaDevAttrCooperativeLaunch, ctx->device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lz_step, LT, 0);
        if (dev_coop && (int64_t)per_sm * ctx->sms >= R.la.nrow_grid) R.lz_mode = LZ_COOP;
    }
}

int lanczos_vectors(Run &R, int j);

int lanczos_step(Run &R, int j) {
    lm_pencil *p = R.p;
    R.la.V = p->V;
    const double *vj = p->V + (size_t)j * p->ldp;
    // consecutive steps walk the rows in opposite directions, so each product
    // starts on the rows the previous one left in L2; fixed by j, so a rerun
    // repeats the same order
    if (p->chunk) {
        // streamed pencil: rebuild, centre and apply chunk by chunk into shv
        if (int rc = lm_launch_stream_product(p, vj, R.sym, R.prec, 0, p->shv, nullptr, R.s))
            return rc;
    } else if (int rc = lm_launch_pencil(p, vj, R.sym, R.prec, 0, &p->st->broke, R.s,
                                         R.lz_mode == LZ_CLUSTER, j & 1)) {
        return rc;
    }
    R.n_matvec++;
    if (R.reduce) {
        // this shard's term of the product, summed over the shards
        if (int rc = lm_launch_reduce_partials(p, R.prec, p->shv, nullptr, R.s)) return rc;
        if (int rc = shard_reduce(R, p->shv, p->ldp)) return rc;
    }
    lm_prof_begin(p->ctx, PROF_LANCZOS, R.s);
    const int rc = lanczos_vectors(R, j);
    lm_prof_end(p->ctx, PROF_LANCZOS, R.s);
    return rc;
}

// The vector work of Lanczos step j (after its pencil product).
int lanczos_vectors(Run &R, int j) {
    lm_pencil *p = R.p;
    const int g2 = R.la.nrow_grid;
    if (R.lz_mode == LZ_CLUSTER) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = R.cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(R.cluster);
        cfg.blockDim = dim3(CT);
        cfg.dynamicSmemBytes = cluster_dyn_smem(j + 1, R.cluster_emax);
        cfg.stream = R.s;
        // The limit is an attribute of the kernel, shared by every pencil whose
        // jobs may be in flight at once (batches, the server) and read again when
        // a captured cycle replays this launch: the device maximum.
        const int dmax = lm_max_dyn_smem((const void *)k_lz_cluster, p->ctx->smem_optin);
        if (cudaFuncSetAttribute(k_lz_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 std::max(dmax, (int)cfg.dynamicSmemBytes)) != cudaSuccess)
            return lm_cuda_check(p->ctx, cudaGetLastError(), "cluster smem attribute");
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_lz_cluster, R.la, j);
        lm_note_launch(p->ctx);
        return lm_cuda_check(p->ctx, e, "cluster lanczos step");
    }
    if (R.lz_mode == LZ_COOP) {
        void *args[] = {(void *)&R.la, (void *)&j};
        cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_lz_step, dim3(g2), dim3(LT),
                                                    args, 0, R.s);
        lm_note_launch(p->ctx);
        return lm_cuda_check(p->ctx, e, "cooperative lanczos step");
    }
    k_lz_a<<<g2, LT, 0, R.s>>>(R.la, j);
    k_lz_b<<<g2, LT, 0, R.s>>>(R.la, j);
    k_lz_c<<<g2, LT, 0, R.s>>>(R.la, j);
    k_lz_d<<<g2, LT, 0, R.s>>>(R.la, j, j + 1, 0);
    lm_note_launch(p->ctx, 4);
    return lm_cuda_check(p->ctx, cudaGetLastError(), "lanczos step");
}

// start vector from w (already filled): null projection + normalise into V[:,0]
int start_vector(Run &R) {
    lm_pencil *p = R.p;
    const int g2 = R.la.nrow_grid;
    R.la.V = p->V;
    // reuse k_lz_c with j = -1 (no CGS terms): projection and norm only
    k_lz_c<<<g2, LT, 0, R.s>>>(R.la, -1);
    k_lz_d<<<g2, LT, 0, R.s>>>(R.la, 0, 0, 1);
    lm_note_launch(p->ctx, 2);
    return lm_cuda_check(p->ctx, cudaGetLastError(), "start vector");
}

}  // namespace

// ---------------------------------------------------------------- job
// The host side of one IRL solve as a resumable state machine. Each call of
// advance() enqueues the next stretch of device work on the job's stream and
// records the job's event after it:
//   start of a phase: reset the state, start vector, first Lanczos cycle,
//     tridiagonal solve and the state read-back;
//   after a cycle: either an implicit restart and the next cycle, or the Ritz
//     vector; a low-precision phase then hands its Ritz vector to the FP64 /
//     double-float phase as start vector;
//   refinement: explicit FP64 products, Rayleigh quotients and the update.
// irl_step drives one job synchronously; the batch and server engines poll
// many jobs on many streams. The kernel sequence of a job does not depend on
// what else runs on the device, so its result does not either.
enum { JOB_INIT = 0, JOB_CYCLE = 1, JOB_REFINE = 2, JOB_DONE = 3 };

struct IrlJob {
    Run R;
    lm_pencil *p;
    cudaStream_t s;
    irl_params prm;
    int state;
    bool lowp, dfp, in_lowp;
    int n_lowp, cycle, max_restarts;
    bool block;  // the low-precision phase is block Lanczos
    double rel;
    const double *v0_dev;
    double *c_out, *dtheta_out, *theta_inout, *dth_tmp;
    bool c_dev, d_dev, t_dev;
    cudaEvent_t ev;
};

namespace {

int job_check(IrlJob *J, const char *what) {
    return lm_cuda_check(J->p->ctx, cudaGetLastError(), what);
}

// state read-back (IRL state and flags) on the job's stream, then the event
int job_readback(IrlJob *J) {
    lm_pencil *p = J->p;
    cudaError_t e = cudaMemcpyAsync(p->st_host, p->st, sizeof(IrlState), cudaMemcpyDeviceToHost,
                                    J->s);
    if (e == cudaSuccess) e = cudaEventRecord(J->ev, J->s);
    return lm_cuda_check(p->ctx, e, "IRL state read-back");
}

// Captured cycles. The Lanczos steps j0 .. m-1 of a cycle are the same launches
// with the same arguments every time a pencil runs that cycle (the pencil's
// buffers are rebuilt in place), so a pencil with cycle_graphs set captures
// them once into a CUDA graph and replays it: one graph launch instead of one
// to five kernel launches per step, the same kernels in the same order, so the
// same results bit for bit. Not for row shards (a host reduction between the
// launches) or streamed pencils.
void cycle_key(const Run &R, int j0, int *key) {
    const lm_pencil *p = R.p;
    const int k[LM_CYCLE_KEY] = {j0,           R.m,         R.prec,          R.sym,
                                 R.lz_mode,    R.cluster,   R.la.nparts,     R.la.deflate,
                                 R.la.three_term, p->g_pencil, R.cluster_emax, 0};
    std::memcpy(key, k, sizeof(k));
}

// Launch the captured cycle (capturing it first if needed); *used = false when
// this pencil does not take captured cycles.
int cycle_graph(IrlJob *J, int j0, bool *used) {
    Run &R = J->R;
    lm_pencil *p = J->p;
    lm_ctx *ctx = p->ctx;
    *used = false;
    if (!p->cycle_graphs || R.reduce || p->chunk || j0 >= R.m) return LM_OK;
    if (!p->cg) {
        p->cg = new CycleGraph[LM_CYCLE_GRAPHS];
        std::memset(p->cg, 0, sizeof(CycleGraph) * LM_CYCLE_GRAPHS);
    }
    int key[LM_CYCLE_KEY];
    cycle_key(R, j0, key);
    CycleGraph *slot = nullptr, *victim = &p->cg[0];
    for (int i = 0; i < LM_CYCLE_GRAPHS; ++i) {
        CycleGraph &c = p->cg[i];
        if (c.exec && !std::memcmp(c.key, key, sizeof(key))) slot = &c;
        if (!c.exec || (victim->exec && c.used < victim->used)) victim = &c;
    }
    if (!slot) {
        // capture: no event records (profiling off), the launch counter kept for
        // the first replay below
        const int prof = ctx->profile;
        const long long launches = ctx->launches;
        const int nmv = R.n_matvec;
        ctx->profile = 0;
        cudaError_t e = cudaStreamBeginCapture(R.s, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            ctx->profile = prof;
            return lm_cuda_check(ctx, e, "cycle capture");
        }
        int rc = LM_OK;
        for (int j = j0; j < R.m && !rc; ++j) rc = lanczos_step(R, j);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(R.s, &g);
        ctx->profile = prof;
        ctx->launches = launches;
        R.n_matvec = nmv;
        if (rc || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc ? rc : lm_cuda_check(ctx, e ? e : cudaErrorUnknown, "cycle capture");
        }
        size_t n = 0;
        cudaGraphGetNodes(g, nullptr, &n);
        int kernels = 0;
        if (n) {
            cudaGraphNode_t *nodes = new cudaGraphNode_t[n];
            cudaGraphGetNodes(g, nodes, &n);
            for (size_t i = 0; i < n; ++i) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess &&
                    t == cudaGraphNodeTypeKernel)
                    ++kernels;
            }
            delete[] nodes;
        }
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return lm_cuda_check(ctx, e, "cycle graph instantiate");
        if (victim->exec) cudaGraphExecDestroy(victim->exec);
        slot = victim;
        std::memcpy(slot->key, key, sizeof(key));
        slot->exec = ex;
        slot->kernels = kernels;
    }
    long long top = 0;
    for (int i = 0; i < LM_CYCLE_GRAPHS; ++i) top = std::max(top, p->cg[i].used);
    slot->used = top + 1;
    if (int rc = lm_cuda_check(ctx, cudaGraphLaunch(slot->exec, R.s), "cycle graph launch"))
        return rc;
    lm_note_launch(ctx, slot->kernels);
    R.n_matvec += R.m - j0;
    *used = true;
    return LM_OK;
}

// Lanczos steps j0 .. m-1 and the tridiagonal work of one cycle
int job_cycle(IrlJob *J, int j0) {
    Run &R = J->R;
    lm_pencil *p = J->p;
    bool captured = false;
    if (int rc = cycle_graph(J, j0, &captured)) return rc;
    for (int j = j0; j < R.m && !captured; ++j)
        if (int rc = lanczos_step(R, j)) return rc;
    TriArgs ta;
    ta.st = p->st;
    ta.m = R.m;
    ta.k = R.k;
    ta.final_pass = J->cycle >= J->max_restarts;
    ta.tol = J->prm.tol;
    ta.rel = J->rel;
    lm_prof_begin(p->ctx, PROF_TRI, R.s);
    k_tri<<<1, TT, 0, R.s>>>(ta);
    lm_prof_end(p->ctx, PROF_TRI, R.s);
    lm_note_launch(p->ctx);
    if (int rc = job_check(J, "k_tri")) return rc;
    return job_readback(J);
}

// a phase: reset, start vector from v0 (or the seeded random vector), cycle 0
int job_phase_start(IrlJob *J) {
    Run &R = J->R;
    lm_pencil *p = J->p;
    if (J->in_lowp) {
        R.prec = p->prec;
        J->rel = p->prec == LM_FP32 ? 1e-6 : 1e-3;  // the storage format's resolution
    } else {
        R.prec = J->dfp ? LM_DF64 : LM_FP64;
        J->rel = 50.0 * 2.220446049250313e-16;
        // The FP64 continuation of a low-precision phase starts from a Ritz
        // vector already accurate to the storage's resolution: short cycles
        // (Krylov dimension 8, at least k + 2) reach the tolerance in one or
        // two of them instead of a full m-step cycle.
        if (J->lowp) {
            R.m = std::min(J->prm.m, std::max(8, J->prm.k + 2));
            choose_lanczos(R, p->ctx);
        }
    }
    R.la.nparts = lm_pencil_ctas(p, R.prec);
    if (R.reduce || p->chunk) {
        R.la.part = p->shv;  // the reduced (or chunk-summed) product, one "partial"
        R.la.nparts = 1;
    }
    J->cycle = 0;
    cudaMemsetAsync(p->st, 0, sizeof(IrlState), R.s);
    cudaMemsetAsync(p->bar, 0, 64 * sizeof(unsigned), R.s);
    k_init_start<<<(p->ldp + 255) / 256, 256, 0, R.s>>>(p->wvec, p->ldp, p->P1, J->prm.seed,
                                                         J->v0_dev);
    lm_note_launch(p->ctx);
    if (int rc = job_check(J, "k_init_start")) return rc;
    if (int rc = start_vector(R)) return rc;
    return job_cycle(J, 0);
}

// explicit FP64 refinement: H~' y and S~ y in one pass, Rayleigh quotients,
// residual, update; outputs to the caller's buffers; then the event
int job_refine(IrlJob *J) {
    Run &R = J->R;
    lm_pencil *p = J->p;
    lm_ctx *ctx = p->ctx;
    cudaStream_t s = J->s;
    if (p->chunk) {
        if (int rc = lm_launch_stream_product(p, p->yvec, R.sym, LM_FP64, 1, p->hy, p->sy, s))
            return rc;
    } else {
        if (int rc = lm_launch_pencil(p, p->yvec, R.sym, LM_FP64, 1, nullptr, s)) return rc;
        if (int rc = lm_launch_reduce_partials(p, LM_FP64, p->hy, p->sy, s)) return rc;
    }
    if (R.reduce) {
        if (int rc = shard_reduce(R, p->hy, p->ldp)) return rc;
        if (int rc = shard_reduce(R, p->sy, p->ldp)) return rc;
    }
    R.n_matvec++;
    const size_t stage_vec = (size_t)8 * p->ldp;
    if (J->theta_inout && !J->t_dev)
        if (int rc = lm_stage_h2d(p, p->tvec, J->theta_inout, (p->P1 - 1) * sizeof(double),
                                  p->st_out + LM_STAGE_TIO * stage_vec, s))
            return rc;
    int *status_dev = reinterpret_cast<int *>(&p->st->err);
    k_refine<<<1, 1024, 0, s>>>(p->yvec, p->hy, p->sy, p->st, p->ldp, p->P1,
                                J->c_dev ? J->c_out : nullptr,
                                J->d_dev ? J->dtheta_out : J->dth_tmp,
                                J->theta_inout ? (J->t_dev ? J->theta_inout : p->tvec) : nullptr,
                                J->prm.tol, status_dev);
    lm_note_launch(ctx);
    if (int rc = job_check(J, "k_refine")) return rc;
    // host outputs land in the pinned staging; irl_job_advance copies them out
    if (J->c_out && !J->c_dev)
        cudaMemcpyAsync(lm_stage_irl(p, LM_STAGE_C), p->yvec, p->P1 * sizeof(double),
                        cudaMemcpyDeviceToHost, s);
    if (J->dtheta_out && !J->d_dev)
        cudaMemcpyAsync(lm_stage_irl(p, LM_STAGE_DTH), J->dth_tmp, (p->P1 - 1) * sizeof(double),
                        cudaMemcpyDeviceToHost, s);
    if (J->theta_inout && !J->t_dev)
        cudaMemcpyAsync(lm_stage_irl(p, LM_STAGE_TIO), p->tvec, (p->P1 - 1) * sizeof(double),
                        cudaMemcpyDeviceToHost, s);
    return job_readback(J);
}

}  // namespace

int irl_job_create(lm_pencil *p, const irl_params *prm, double *c_out, double *dtheta_out,
                   double *theta_inout, cudaStream_t s, IrlJob **out, lm_reduce_fn reduce,
                   void *reduce_user, int reduce_where) {
    if (!p || !prm || !out) return LM_ERR_ARG;
    lm_ctx *ctx = p->ctx;
    if (p->shard_state) return lm_fail(ctx, LM_ERR_ARG, "row shard not centred (lm_shard_centre)");
    if (reduce && reduce_where != LM_REDUCE_HOST && reduce_where != LM_REDUCE_DEVICE)
        return lm_fail(ctx, LM_ERR_ARG, "bad reduction location %d", reduce_where);
    if (reduce && p->chunk)
        return lm_fail(ctx, LM_ERR_ARG, "a streamed pencil is not a row shard");
    if (reduce && !p->shv &&
        lm_cuda_check(ctx, cudaMalloc(&p->shv, 2 * (size_t)p->ldp * sizeof(double)),
                      "cudaMalloc"))
        return LM_ERR_OOM;
    if (prm->m > LM_MAXKRYLOV || prm->m < 2 || prm->k < 1 || prm->k >= prm->m || prm->m > p->P1)
        return lm_fail(ctx, LM_ERR_SIZE, "need 1 <= k < m <= min(64, P+1); got k=%d m=%d", prm->k,
                       prm->m);
    if (prm->sym < 0 || prm->sym > 3 || prm->precision < 0 || prm->precision > 3)
        return lm_fail(ctx, LM_ERR_ARG, "bad sym or precision");
    if (prm->reorth != IRL_REORTH_FULL && prm->reorth != IRL_REORTH_NONE)
        return lm_fail(ctx, LM_ERR_ARG, "bad reorth %d", prm->reorth);
    if (prm->mode != IRL_MODE_SHEP)
        return lm_fail(ctx, LM_ERR_ARG, "bad mode %d", prm->mode);
    if (prm->block != 0 &&
        (prm->block != 16 || prm->m % 16 != 0 || prm->m > 64 || p->prec != LM_BF16 ||
         !p->Olo || prm->precision != LM_BF16 || reduce || p->chunk))
        return lm_fail(ctx, LM_ERR_ARG,
                       "block = 16 needs m in {16, 32, 48, 64}, a BF16 pencil, precision BF16 "
                       "and no row shards");
    if (p->gfree && ((prm->sym != LM_SYM_AUTO && prm->sym != LM_SYM_ELOC) || prm->block))
        return lm_fail(ctx, LM_ERR_ARG, "a pencil without G'_c answers the E_loc estimator only");
    IrlJob *J = new IrlJob();
    J->p = p;
    J->s = s;
    J->prm = *prm;
    J->state = JOB_INIT;
    p->n_hist = 0;
    if (cudaEventCreateWithFlags(&J->ev, cudaEventDisableTiming) != cudaSuccess) {
        delete J;
        return lm_fail(ctx, LM_ERR_CUDA, "cudaEventCreate");
    }
    Run &R = J->R;
    R.p = p;
    R.s = s;
    R.m = prm->m;
    R.k = prm->k;
    R.sym = prm->sym == LM_SYM_AUTO ? p->sym : prm->sym;
    R.n_matvec = 0;
    R.n_restart = 0;
    R.reduce = reduce;
    R.reduce_user = reduce_user;
    R.reduce_where = reduce_where;
    R.la.V = p->V;
    R.la.w = p->wvec;
    R.la.part = p->part;
    R.la.dots = p->dots;
    R.la.ldp = p->ldp;
    R.la.M1 = p->M1;
    R.la.P1 = p->P1;
    R.la.nrow_grid = p->nh + 1;
    R.la.n_orb = p->n;
    R.la.na = p->na;
    R.la.nb = p->nb;
    R.la.deflate = prm->deflate_null;
    R.la.three_term = prm->reorth == IRL_REORTH_NONE;
    R.la.st = p->st;
    R.la.bar = p->bar;
    R.la.flags = p->d_flags;
    {
        // projection constants (see k_lz_cluster) as double-float pairs
        const double n = p->n, na = p->na, nb = p->nb;
        const double g11 = n + na * na, g22 = n + nb * nb, g12 = na * nb;
        const double det = g11 * g22 - g12 * g12;
        auto pair = [](double x) {
            const float h = (float)x;
            return make_float2(h, (float)(x - (double)h));
        };
        R.la.inv_n = pair(1.0 / n);
        R.la.gi11 = pair(g22 / det);
        R.la.gi12 = pair(-g12 / det);
        R.la.gi22 = pair(g11 / det);
    }
    choose_lanczos(R, ctx);
    J->max_restarts = prm->max_restarts < 0 ? 0 : prm->max_restarts;
    J->lowp = prm->precision != LM_FP64 && p->Olo != nullptr && p->prec != LM_DF64;
    // double-float factors are accurate to ~1e-14: one phase at the FP64 tolerance
    J->dfp = prm->precision != LM_FP64 && p->Olo != nullptr && p->prec == LM_DF64;
    J->in_lowp = J->lowp;
    J->n_lowp = 0;
    J->block = prm->block == 16;
    if (J->block) J->in_lowp = false;  // the block phase replaces the single-vector one
    J->v0_dev = nullptr;
    J->c_out = c_out;
    J->dtheta_out = dtheta_out;
    J->theta_inout = theta_inout;
    J->c_dev = c_out && lm_is_device_ptr(c_out);
    J->d_dev = dtheta_out && lm_is_device_ptr(dtheta_out);
    J->t_dev = theta_inout && lm_is_device_ptr(theta_inout);
    J->dth_tmp = p->dots + (size_t)3 * (p->nh + 1) * DLD;  // scratch >= ldp
    if (prm->v0) {
        if (lm_is_device_ptr(prm->v0)) {
            J->v0_dev = prm->v0;
        } else {
            if (int rc = lm_stage_h2d(p, p->yvec, prm->v0, p->P1 * sizeof(double),
                                      p->st_out + LM_STAGE_V0 * (size_t)8 * p->ldp, s)) {
                irl_job_free(J);
                return rc;
            }
            J->v0_dev = p->yvec;
        }
    }
    *out = J;
    return LM_OK;
}

int irl_job_advance(IrlJob *J, int *done) {
    *done = 0;
    lm_pencil *p = J->p;
    lm_ctx *ctx = p->ctx;
    Run &R = J->R;
    if (J->state == JOB_INIT) {
        J->state = JOB_CYCLE;
        if (J->block) {
            // block Lanczos on the tensor-core product; its Ritz vector starts
            // the FP64 phase (short cycles, as after any low-precision phase)
            const int nsteps = J->prm.m / 16;
            if (int rc = lm_launch_block_lanczos(p, R.sym, nsteps, J->prm.seed,
                                                 J->prm.deflate_null, p->hy, R.s))
                return rc;
            R.n_matvec += 16 * nsteps;
            J->n_lowp = 16 * nsteps;
            J->v0_dev = p->hy;
        }
        return job_phase_start(J);
    }
    if (J->state == JOB_CYCLE) {
        const IrlState &h = *p->st_host;
        if (h.flags & FLAG_TIMEOUT)
            return lm_fail(ctx, LM_ERR_TIMEOUT, "pencil pipeline wait timed out");
        if (p->n_hist < LM_HIST_MAX) {
            p->hist_lam[p->n_hist] = h.lam;
            p->hist_res[p->n_hist] = h.res;
            p->hist_lowp[p->n_hist] = J->in_lowp ? 1 : 0;
            p->n_hist++;
        }
        if (!(h.conv || h.broke || J->cycle >= J->max_restarts)) {
            // implicit restart, then the next cycle from j = k
            double *Vnew = p->V + (size_t)(LM_MAXKRYLOV + 1) * p->ldp;
            k_restart<<<R.la.nrow_grid, LT, 0, R.s>>>(R.la, Vnew, R.m, R.k);
            lm_note_launch(ctx);
            if (int rc = job_check(J, "k_restart")) return rc;
            // swap halves: the kept vectors now live in Vnew
            cudaMemcpyAsync(p->V, Vnew, (size_t)R.k * p->ldp * sizeof(double),
                            cudaMemcpyDeviceToDevice, R.s);
            R.la.V = p->V;
            k_lz_d<<<R.la.nrow_grid, LT, 0, R.s>>>(R.la, 0, R.k, 2);
            lm_note_launch(ctx);
            if (int rc = job_check(J, "restart normalise")) return rc;
            R.n_restart++;
            J->cycle++;
            return job_cycle(J, R.k);
        }
        k_ritz_vector<<<(p->ldp + 255) / 256, 256, 0, R.s>>>(p->V, p->st, p->ldp, p->yvec);
        lm_note_launch(ctx);
        if (int rc = job_check(J, "k_ritz_vector")) return rc;
        if (J->in_lowp) {
            // the low-precision Ritz vector starts the FP64 phase
            J->n_lowp = R.n_matvec;
            cudaMemcpyAsync(p->hy, p->yvec, p->ldp * sizeof(double), cudaMemcpyDeviceToDevice,
                            R.s);
            J->v0_dev = p->hy;
            J->in_lowp = false;
            return job_phase_start(J);
        }
        J->state = JOB_REFINE;
        return job_refine(J);
    }
    if (J->state == JOB_REFINE) {
        J->state = JOB_DONE;
        if (J->c_out && !J->c_dev)
            std::memcpy(J->c_out, lm_stage_irl(p, LM_STAGE_C), p->P1 * sizeof(double));
        if (J->dtheta_out && !J->d_dev)
            std::memcpy(J->dtheta_out, lm_stage_irl(p, LM_STAGE_DTH),
                        (p->P1 - 1) * sizeof(double));
        if (J->theta_inout && !J->t_dev)
            std::memcpy(J->theta_inout, lm_stage_irl(p, LM_STAGE_TIO),
                        (p->P1 - 1) * sizeof(double));
        *done = 1;
        return LM_OK;
    }
    *done = 1;
    return LM_OK;
}

cudaEvent_t irl_job_event(const IrlJob *J) { return J->ev; }

void irl_job_result(const IrlJob *J, irl_result *out) {
    const IrlState &h = *J->p->st_host;
    out->lambda = h.lam;
    out->energy = J->p->E_host;
    out->lambda_gen_rq = h.rq_s;
    out->residual = h.res_explicit;
    out->c0 = h.c0;
    out->status = h.err;
    out->n_matvec = J->R.n_matvec;
    out->n_restart = J->R.n_restart;
    out->n_matvec_lowp = J->n_lowp;
}

void irl_job_free(IrlJob *J) {
    if (!J) return;
    cudaEventDestroy(J->ev);
    delete J;
}

extern "C" int irl_step(lm_pencil *p, const irl_params *prm, irl_result *out, double *c_out,
                        double *dtheta_out, double *theta_inout, void *stream) {
    if (!p || !prm || !out) return LM_ERR_ARG;
    lm_ctx *ctx = p->ctx;
    cudaSetDevice(ctx->device);
    IrlJob *J = nullptr;
    if (int rc = irl_job_create(p, prm, c_out, dtheta_out, theta_inout, (cudaStream_t)stream, &J))
        return rc;
    int done = 0, rc = LM_OK;
    while (!rc && !done) {
        rc = irl_job_advance(J, &done);
        if (!rc && !done)
            rc = lm_cuda_check(ctx, cudaEventSynchronize(J->ev), "irl_step");
    }
    if (!rc) irl_job_result(J, out);
    irl_job_free(J);
    return rc;
}

extern "C" int irl_step_sharded(lm_pencil *p, const irl_params *prm, lm_reduce_fn reduce,
                                void *user, int where, irl_result *out, double *c_out,
                                double *dtheta_out, double *theta_inout, void *stream) {
    if (!p || !prm || !out || !reduce) return LM_ERR_ARG;
    lm_ctx *ctx = p->ctx;
    cudaSetDevice(ctx->device);
    IrlJob *J = nullptr;
    if (int rc = irl_job_create(p, prm, c_out, dtheta_out, theta_inout, (cudaStream_t)stream, &J,
                                reduce, user, where))
        return rc;
    int done = 0, rc = LM_OK;
    while (!rc && !done) {
        rc = irl_job_advance(J, &done);
        if (!rc && !done)
            rc = lm_cuda_check(ctx, cudaEventSynchronize(J->ev), "irl_step_sharded");
    }
    if (!rc) irl_job_result(J, out);
    irl_job_free(J);
    return rc;
}

extern "C" int lm_irl_history(lm_pencil *p, double *lam, double *res, int *lowp, int cap,
                              int *n) {
    if (!p || !n || cap < 0) return LM_ERR_ARG;
    const int k = std::min(cap, p->n_hist);
    for (int i = 0; i < k; ++i) {
        if (lam) lam[i] = p->hist_lam[i];
        if (res) res[i] = p->hist_res[i];
        if (lowp) lowp[i] = p->hist_lowp[i];
    }
    *n = p->n_hist;
    return LM_OK;
}

extern "C" int lm_debug_wait_timeout(lm_ctx *ctx, int which, int64_t limit_ns) {
    if (!ctx) return LM_ERR_ARG;
    if ((which != 0 && which != 1) || limit_ns < 1 || limit_ns > (int64_t)LM_WAIT_LIMIT_NS)
        return lm_fail(ctx, LM_ERR_ARG, "which must be 0 or 1, limit in [1 ns, 2 s]");
    cudaSetDevice(ctx->device);
    unsigned *buf = nullptr;
    if (cudaMalloc(&buf, 4 * sizeof(unsigned)) != cudaSuccess)
        return lm_fail(ctx, LM_ERR_OOM, "cudaMalloc");
    int rc = lm_cuda_check(ctx, cudaMemset(buf, 0, 4 * sizeof(unsigned)), "memset");
    if (!rc) {
        k_debug_wait<<<which == 0 ? 2 : 1, 32>>>(which, (uint64_t)limit_ns, buf,
                                                 reinterpret_cast<int *>(buf + 2));
        lm_note_launch(ctx);
        rc = lm_cuda_check(ctx, cudaGetLastError(), "k_debug_wait");
    }
    if (!rc) rc = lm_cuda_check(ctx, cudaDeviceSynchronize(), "k_debug_wait");
    int flags = 0;
    if (!rc)
        rc = lm_cuda_check(ctx, cudaMemcpy(&flags, buf + 2, sizeof(int), cudaMemcpyDeviceToHost),
                           "flags");
    cudaFree(buf);
    if (rc) return rc;
    if (flags & FLAG_TIMEOUT)
        return lm_fail(ctx, LM_ERR_TIMEOUT, "the bounded wait gave up (as the test intends)");
    return LM_OK;
}

void lm_cycle_graphs_release(lm_pencil *p) {
    if (!p || !p->cg) return;
    for (int i = 0; i < LM_CYCLE_GRAPHS; ++i)
        if (p->cg[i].exec) cudaGraphExecDestroy(p->cg[i].exec);
    delete[] p->cg;
    p->cg = nullptr;
}
