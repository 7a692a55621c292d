// Block pencil product on the tensor cores (arXiv 2601.01437, Discussion: the
// block-Lanczos extension; Methods, eq. matrix_vec_prod applied to a block of
// vectors): for NV = 16 vectors V (columns of a (P+1) x 16 block),
//   Y_S = O_c^T W (O_c V),
//   Y_H = O_c^T W (G'_c V)                       (sym NONE), or
//   Y_H = 1/2 (O_c^T W (G'_c V) + G'_c^T W (O_c V))   (sym HALF),
// with the pencil's BF16 factors, BF16 V and FP32 accumulation.
//
// Both contractions are dense and tall-skinny, so they run as tcgen05 MMAs
// (M = 128, N = 16, K = 16 per instruction) fed by TMA:
//   phase 1, per tile of 64 rows: [X_O; X_G] = [O_tile; G_tile] V, the tile's
//     O rows stacked over its G rows as one 128-row operand, summed over the
//     row's 128-column chunks into TMEM (FP32);
//   epilogue: X' = W X (the tile's weights), rounded to BF16 into shared
//     memory as the next phase's B operand;
//   phase 2: for every 128-column chunk m, D_S[m] += O_m^T X'_O and
//     D_H[m] += O_m^T X'_G (+ G_m^T X'_O for HALF), the chunks read again
//     (from L2: a tile is 64 rows, so the rows in flight between the two reads
//     stay well inside L2) as MN-major A operands; D stays in TMEM across all
//     the tiles a CTA owns.
// At the end each CTA writes its D as FP32 partials; a second kernel adds the
// partials of all CTAs in CTA order into FP64 outputs (deterministic).
//
// Roles (192 threads): warp 0 issues the TMA loads, warp 1 allocates TMEM and
// one of its threads issues every MMA, warps 2-5 are the epilogue (one TMEM
// lane quarter each). A six-stage ring carries 128-column chunks of the tile's
// O and G (64-column, 128-byte-swizzled boxes, O and G of a chunk back to
// back) with the matching columns of V for phase 1. Round r of the software
// pipeline interleaves, chunk by chunk, phase 2 of tile r - 1 with phase 1 of
// tile r, so the HBM loads of tile r go on while the epilogue turns tile
// r - 1's X into X'. The first read of a tile (phase 1) is loaded with an L2
// evict-last policy and its re-read (phase 2) with evict-first, so the two
// tiles live per SM between the reads stay in L2.
// Every wait is bounded: a timeout sets FLAG_TIMEOUT, every role stops, TMA
// loads still in flight are waited for (bounded), TMEM is freed, and the
// products come back as NaN.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "internal.cuh"

namespace {

// A tile is BM = 64 rows. Phase 1 stacks the tile's 64 rows of O over its 64
// rows of G into one M = 128 operand (both 64-row boxes of a 64-column chunk
// lie back to back), so one MMA yields X_O in TMEM lanes 0-63 and X_G in lanes
// 64-127. Phase 2 takes K = 64 rows per column chunk.
constexpr int BM = 64;                              // rows per tile
constexpr int NV = 16;                              // vectors per block (MMA N)
constexpr int CW = 128;                             // columns per ring stage
constexpr int NSTAGE = 6;
constexpr int BLK_THREADS = 192;
constexpr uint32_t BOX_BYTES = BM * 64 * 2;         // 8 KB: 64 rows x 64 BF16
constexpr uint32_t PAIR_BYTES = 2 * BOX_BYTES;      // O box then G box of one 64-column chunk
constexpr uint32_t VBOX_BYTES = NV * 64 * 2;        // 2 KB: 16 vectors x 64 BF16
constexpr uint32_t STAGE_BYTES = 2 * PAIR_BYTES + 2 * VBOX_BYTES;  // 36 KB: O, G (and V)
constexpr uint32_t RING_BYTES = NSTAGE * STAGE_BYTES;
constexpr uint32_t X_BYTES = NV * BM * 2;           // 2 KB: one X' operand
constexpr int MAX_NCH = 15;                         // TMEM: 16 + 2 * 16 * nch <= 512 columns
constexpr uint32_t TMEM_COLS = 512;

struct BlkArgs {
    const double *w;     // normalised weights, n_rows
    int64_t n_rows;
    int ntiles;          // ceil(n_rows / BM)
    int nch;             // 128-column chunks of a row
    int ldo;             // nch * CW: row length of the partials
    float *part;         // [gridDim.x][2][NV][ldo]
    float hscale;        // 1/2 for HALF, 1 for NONE
    int *flags;
    float *dbg;          // nullable: X_O, X_G (unweighted) of CTA 0's first tile, [2][64][NV]
    uint32_t lbo_mn;     // MN-major A operand: byte stride between 64-column atoms
    uint32_t sbo_mn;     // ... and between 8-row groups
};

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d_hint(uint32_t dst, const CUtensorMap *map, int x,
                                                 int y, uint32_t bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        ".L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_u32(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test_u32(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait (LM_SPIN_LIMIT polls or two seconds); false on timeout.
__device__ __forceinline__ bool mbar_wait_u32(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < LM_SPIN_LIMIT; ++i) {
        if (mbar_test_u32(bar, parity)) return true;
        if ((i & 255u) == 255u && global_ns() - t0 > LM_WAIT_LIMIT_NS) return false;
    }
    return false;
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                       uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// 32 TMEM lanes (the warp's quarter) x 16 consecutive 32-bit columns
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory matrix descriptor: start address, leading / stride byte
// offsets, descriptor version 1 (bit 46), 128-byte swizzle (mode 2, bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}
// Instruction descriptor, kind::f16: FP32 D (bits 4-5 = 1), BF16 A and B (bits
// 7-9 and 10-12 = 1), A K-major or MN-major (bit 15), B K-major, N >> 3 at
// bits 17-22, M >> 4 at bits 24-28 (M = 128 in both phases).
__host__ __device__ constexpr uint32_t mma_idesc(bool a_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) |
           ((uint32_t)(NV >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// ---------------------------------------------------------------- the kernel
template <bool HALF>
__global__ void __launch_bounds__(BLK_THREADS, 1)
    k_pencil_block(const __grid_constant__ CUtensorMap tO, const __grid_constant__ CUtensorMap tG,
                   const __grid_constant__ CUtensorMap tV, BlkArgs a) {
    extern __shared__ unsigned char smem_raw[];
    // the swizzled tiles need 1024-byte alignment
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *sbase = smem_raw + (base - raw);
    const uint32_t sXO = base + RING_BYTES;
    const uint32_t sXG = sXO + X_BYTES;
    unsigned char *pX = sbase + RING_BYTES;  // X'_O, then X'_G
    uint64_t *bars = reinterpret_cast<uint64_t *>(pX + 2 * X_BYTES);
    uint64_t *full = bars, *empty = bars + NSTAGE;
    uint64_t *xready = bars + 2 * NSTAGE, *xfull = xready + 1, *done = xready + 2;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(done + 1);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(xready, 1);
        mbar_init(xfull, 128);
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tD = tmem + 16;  // D_H[m] at tD + 16 m, D_S[m] at tD + 16 (nch + m)
    // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int ntl = (int)blockIdx.x < a.ntiles
                        ? (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                        : 0;

    // Software pipeline over rounds r = 0 .. ntl: round r interleaves, chunk by
    // chunk, phase 2 of tile r - 1 (its re-read, from L2) with phase 1 of tile r
    // (from HBM), so the HBM stream goes on while the epilogue turns tile r - 1's
    // X into X', and a tile is re-read one tile's loads after it was read.
    if (warp == 0) {
        // ---------------- TMA producer (ring order = MMA consumption order)
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            uint32_t pend_ph[NSTAGE];
            bool pend[NSTAGE];
            const uint64_t pol_last = policy_evict_last(), pol_first = policy_evict_first();
            for (int i = 0; i < NSTAGE; ++i) pend[i] = false;
            for (int r = 0; r <= ntl && !*abort_flag; ++r) {
                for (int c = 0; c < a.nch && !*abort_flag; ++c) {
                    for (int ph2 = 1; ph2 >= 0; --ph2) {  // phase 2 of tile r-1, then phase 1 of tile r
                        const bool pass2 = ph2 == 1;
                        if (pass2 ? r < 1 : r >= ntl) continue;
                        const int t = blockIdx.x + (pass2 ? r - 1 : r) * gridDim.x;
                        if (!mbar_wait_u32(smem_u32(empty + s), ph ^ 1u)) {
                            *abort_flag = 1;
                            atomicOr(a.flags, FLAG_TIMEOUT);
                            break;
                        }
                        const uint32_t st = base + s * STAGE_BYTES;
                        const bool wantG = !pass2 || HALF;
                        const uint32_t bytes =
                            2 * BOX_BYTES * (wantG ? 2u : 1u) + (pass2 ? 0u : 2u * VBOX_BYTES);
                        const uint32_t fb = smem_u32(full + s);
                        mbar_expect_tx(fb, bytes);
                        const int x = c * CW, row0 = t * BM;
                        // first read (phase 1): keep in L2; re-read (phase 2): last use
                        const uint64_t pol = pass2 ? pol_first : pol_last;
                        tma_load_2d_hint(st, &tO, x, row0, fb, pol);
                        tma_load_2d_hint(st + PAIR_BYTES, &tO, x + 64, row0, fb, pol);
                        if (wantG) {
                            tma_load_2d_hint(st + BOX_BYTES, &tG, x, row0, fb, pol);
                            tma_load_2d_hint(st + PAIR_BYTES + BOX_BYTES, &tG, x + 64, row0, fb,
                                             pol);
                        }
                        if (!pass2) {
                            tma_load_2d(st + 2 * PAIR_BYTES, &tV, x, 0, fb);
                            tma_load_2d(st + 2 * PAIR_BYTES + VBOX_BYTES, &tV, x + 64, 0, fb);
                        }
                        pend[s] = true;
                        pend_ph[s] = ph;
                        if (++s == NSTAGE) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                }
            }
            // no load may still be landing when the CTA leaves (bounded)
            for (int i = 0; i < NSTAGE; ++i)
                if (pend[i] && !mbar_wait_u32(smem_u32(full + i), pend_ph[i]))
                    atomicOr(a.flags, FLAG_TIMEOUT);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (one thread)
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            constexpr uint32_t id_k = mma_idesc(false), id_mn = mma_idesc(true);
            auto next = [&]() {
                if (++s == NSTAGE) {
                    s = 0;
                    ph ^= 1u;
                }
            };
            auto wait_stage = [&]() {
                if (mbar_wait_u32(smem_u32(full + s), ph)) {
                    tc_fence_after();
                    return true;
                }
                *abort_flag = 1;
                atomicOr(a.flags, FLAG_TIMEOUT);
                return false;
            };
            for (int r = 0; r <= ntl && !*abort_flag; ++r) {
                if (r >= 1) {
                    // the epilogue has read X of tile r - 1 out of TMEM and written X'
                    if (!mbar_wait_u32(smem_u32(xfull), (uint32_t)(r - 1) & 1u)) {
                        *abort_flag = 1;
                        atomicOr(a.flags, FLAG_TIMEOUT);
                        break;
                    }
                    tc_fence_after();
                }
                for (int c = 0; c < a.nch && !*abort_flag; ++c) {
                    if (r >= 1) {
                        // phase 2 of tile r - 1: D_S[c] += O_c^T X'_O,
                        // D_H[c] += O_c^T X'_G (+ G_c^T X'_O)
                        if (!wait_stage()) break;
                        const uint32_t st = base + s * STAGE_BYTES;
                        const uint32_t dH = tD + 16 * c;
                        const uint32_t dS = tD + 16 * a.nch + 16 * c;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t aO = sw128_desc(st + kk * 2048, a.lbo_mn, a.sbo_mn);
                            const uint64_t bXO = sw128_desc(sXO + kk * 32, 16, 1024);
                            const uint64_t bXG = sw128_desc(sXG + kk * 32, 16, 1024);
                            const uint32_t acc = (r == 1 && kk == 0) ? 0u : 1u;
                            tc_mma(dS, aO, bXO, id_mn, acc);
                            tc_mma(dH, aO, bXG, id_mn, acc);
                            if (HALF)
                                tc_mma(dH,
                                       sw128_desc(st + BOX_BYTES + kk * 2048, a.lbo_mn, a.sbo_mn),
                                       bXO, id_mn, 1u);
                        }
                        tc_commit(smem_u32(empty + s));
                        next();
                    }
                    if (r < ntl) {
                        // phase 1 of tile r: [X_O; X_G] += [O_c; G_c] V_c
                        if (!wait_stage()) break;
                        const uint32_t st = base + s * STAGE_BYTES;
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) {
                            const uint32_t koff = (kk >> 2) * PAIR_BYTES + (kk & 3) * 32;
                            const uint32_t voff = (kk >> 2) * VBOX_BYTES + (kk & 3) * 32;
                            tc_mma(tmem, sw128_desc(st + koff, 16, 1024),
                                   sw128_desc(st + 2 * PAIR_BYTES + voff, 16, 1024), id_k,
                                   (c | kk) ? 1u : 0u);
                        }
                        tc_commit(smem_u32(empty + s));
                        next();
                    }
                }
                if (r < ntl && !*abort_flag) tc_commit(smem_u32(xready));
            }
            // completes once every MMA issued above has
            tc_commit(smem_u32(done));
        }
    } else if (warp <= 5) {
        // ---------------- epilogue: warps 2..5, one TMEM lane quarter each;
        // quarters 0-1 hold X_O (rows 0-63), quarters 2-3 hold X_G
        const int q = warp & 3;
        const int which = q >> 1;
        const int r = 32 * (q & 1) + lane;  // row of the tile
        const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
        unsigned char *pXw = pX + which * X_BYTES;
        uint32_t it = 0;
        bool ok = true;
        for (int t = blockIdx.x; it < (uint32_t)ntl; t += gridDim.x, ++it) {
            int w_ok = 1;
            if (lane == 0) w_ok = !*abort_flag && mbar_wait_u32(smem_u32(xready), it & 1u);
            w_ok = __shfl_sync(0xffffffffu, w_ok, 0);
            if (!w_ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    atomicOr(a.flags, FLAG_TIMEOUT);
                }
                ok = false;
                break;
            }
            tc_fence_after();
            float x[16];
            tc_ld16(tmem + lane_addr, x);
            const int64_t row = (int64_t)t * BM + r;
            const float wr = row < a.n_rows ? (float)a.w[row] : 0.f;
            if (a.dbg && blockIdx.x == 0 && it == 0) {
#pragma unroll
                for (int n = 0; n < NV; ++n) a.dbg[(which * BM + r) * NV + n] = x[n];
            }
            // X'[n][k = r], K-major with the 128-byte swizzle (16-byte chunk ^ line % 8)
            const uint32_t kk = (uint32_t)r;
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                const uint32_t off = n * 128u + ((((kk >> 3) ^ (uint32_t)(n & 7))) << 4) + (kk & 7u) * 2u;
                *reinterpret_cast<__nv_bfloat16 *>(pXw + off) = __float2bfloat16_rn(wr * x[n]);
            }
            fence_async_smem();
            tc_fence_before();
            mbar_arrive_u32(smem_u32(xfull));
        }
        // the CTA's D: FP32 partials of its rows
        int d_ok = 1;
        if (lane == 0) d_ok = mbar_wait_u32(smem_u32(done), 0);
        d_ok = __shfl_sync(0xffffffffu, d_ok, 0);
        if (!d_ok && lane == 0) atomicOr(a.flags, FLAG_TIMEOUT);
        if (d_ok) {
            tc_fence_after();
            const int rc = 32 * q + lane;  // column within a 128-column chunk = TMEM lane
            float *pH = a.part + (size_t)blockIdx.x * 2 * NV * a.ldo;
            float *pS = pH + (size_t)NV * a.ldo;
            for (int m = 0; m < a.nch; ++m) {
                float h[16], sv[16];
                tc_ld16(tD + lane_addr + 16 * m, h);
                tc_ld16(tD + lane_addr + 16 * a.nch + 16 * m, sv);
                const int col = m * CW + rc;
#pragma unroll
                for (int n = 0; n < NV; ++n) {
                    pH[(size_t)n * a.ldo + col] = ok ? h[n] * a.hscale : 0.f;
                    pS[(size_t)n * a.ldo + col] = ok ? sv[n] : 0.f;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// V (nvec FP64 vectors of p1 entries, stride ldv) -> BF16 [NV][ldo], zero padded
__global__ void k_block_v(const double *V, int ldv, int nvec, int p1, int ldo,
                          __nv_bfloat16 *Vb) {
    const int total = NV * ldo;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int n = e / ldo, col = e - n * ldo;
        const double v = (n < nvec && col < p1) ? V[(size_t)n * ldv + col] : 0.0;
        Vb[e] = __double2bfloat16(v);
    }
}

// HV, SV [n][col] = sum over CTAs b (in order) of the partials; NaN everywhere
// if a wait of the block kernel gave up
__global__ void k_block_reduce(const float *part, int nparts, int ldo, int p1, int nvec,
                               const int *flags, double *HV, double *SV, int ldv) {
    const int per = nvec * p1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * per;
         e += gridDim.x * blockDim.x) {
        const int which = e >= per;
        const int rem = e - which * per;
        const int n = rem / p1, col = rem - n * p1;
        double acc = 0.0;
        const float *src = part + ((size_t)which * NV + n) * ldo + col;
        for (int b = 0; b < nparts; ++b) acc += (double)src[(size_t)b * 2 * NV * ldo];
        if (*flags & FLAG_TIMEOUT) acc = __longlong_as_double(0x7ff8000000000000ll);
        double *dst = which ? SV : HV;
        if (dst) dst[(size_t)n * ldv + col] = acc;
    }
}

}  // namespace

// ==========================================================================
// host side
// ==========================================================================
struct BlockState {
    CUtensorMap tO, tG, tV;  // 64-byte aligned by their type
    __nv_bfloat16 *Vb;  // NV x ldo
    float *part;        // grid x 2 x NV x ldo
    int *flags;
    int grid, nch, ldo;
};

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D BF16 tensor map over a row-major rows x cols array (row stride ld
// elements), box 64 columns x box_rows rows, 128-byte swizzle, zero fill
// outside the array.
bool encode_2d(CUtensorMap *m, const void *ptr, int64_t rows, int cols, int ld, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t block_smem_bytes() {
    return 1024 + (size_t)RING_BYTES + 2 * X_BYTES + (2 * NSTAGE + 6) * 8;
}

int block_setup(lm_pencil *p) {
    lm_ctx *ctx = p->ctx;
    if (p->blk) return LM_OK;
    const int nch = (p->ldp + CW - 1) / CW;
    const int ntiles = (int)((p->n_rows + BM - 1) / BM);
    BlockState *b = new BlockState();
    b->nch = nch;
    b->ldo = nch * CW;
    b->grid = std::min(ctx->sms, ntiles);
    int rc = lm_cuda_check(ctx, cudaMalloc(&b->Vb, (size_t)NV * b->ldo * 2), "cudaMalloc");
    if (!rc)
        rc = lm_cuda_check(ctx, cudaMalloc(&b->part, (size_t)b->grid * 2 * NV * b->ldo * 4),
                           "cudaMalloc");
    if (!rc) rc = lm_cuda_check(ctx, cudaMalloc(&b->flags, sizeof(int)), "cudaMalloc");
    if (!rc && !(encode_2d(&b->tO, p->Olo, p->n_rows, p->ldp, p->ldp, BM) &&
                 encode_2d(&b->tG, p->Glo, p->n_rows, p->ldp, p->ldp, BM) &&
                 encode_2d(&b->tV, b->Vb, NV, b->ldo, b->ldo, NV)))
        rc = lm_fail(ctx, LM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    if (rc) {
        cudaFree(b->Vb);
        cudaFree(b->part);
        cudaFree(b->flags);
        delete b;
        return rc;
    }
    p->blk = b;
    return LM_OK;
}

}  // namespace

void lm_block_release(lm_pencil *p) {
    if (!p || !p->blk) return;
    cudaFree(p->blk->Vb);
    cudaFree(p->blk->part);
    cudaFree(p->blk->flags);
    delete p->blk;
    p->blk = nullptr;
}

int lm_launch_pencil_block(lm_pencil *p, const double *V, int ldv, int nvec, double *HV,
                           double *SV, int sym, float *dbg, uint32_t lbo_mn, uint32_t sbo_mn,
                           cudaStream_t s) {
    lm_ctx *ctx = p->ctx;
    if (p->prec != LM_BF16 || !p->Olo)
        return lm_fail(ctx, LM_ERR_ARG, "the block product needs a pencil with BF16 factors");
    if (p->shard_state) return lm_fail(ctx, LM_ERR_ARG, "row shard not centred (lm_shard_centre)");
    if (p->chunk) return lm_fail(ctx, LM_ERR_ARG, "the block product needs resident factors");
    if (p->gfree) return lm_fail(ctx, LM_ERR_ARG, "the block product needs G'_c");
    if (nvec < 1 || nvec > NV || ldv < p->P1)
        return lm_fail(ctx, LM_ERR_SIZE, "need 1 <= nvec <= %d and ldv >= P+1", NV);
    const int sy = sym == LM_SYM_AUTO ? p->sym : sym;
    if (sy != LM_SYM_NONE && sy != LM_SYM_HALF)
        return lm_fail(ctx, LM_ERR_ARG, "the block product takes sym NONE or HALF");
    if ((p->ldp + CW - 1) / CW > MAX_NCH)
        return lm_fail(ctx, LM_ERR_SIZE, "P+1 = %d above the block product's %d", p->P1,
                       MAX_NCH * CW);
    if (!lm_is_device_ptr(V) || (HV && !lm_is_device_ptr(HV)) || (SV && !lm_is_device_ptr(SV)))
        return lm_fail(ctx, LM_ERR_ARG, "the block product takes device arrays");
    if (int rc = block_setup(p)) return rc;
    BlockState *b = p->blk;
    const size_t smem = block_smem_bytes();
    if (smem > (size_t)ctx->smem_optin) return lm_fail(ctx, LM_ERR_SIZE, "shared memory");
    k_block_v<<<64, 256, 0, s>>>(V, ldv, nvec, p->P1, b->ldo, b->Vb);
    cudaMemsetAsync(b->flags, 0, sizeof(int), s);
    BlkArgs a;
    a.w = p->wt;
    a.n_rows = p->n_rows;
    a.ntiles = (int)((p->n_rows + BM - 1) / BM);
    a.nch = b->nch;
    a.ldo = b->ldo;
    a.part = b->part;
    a.hscale = sy == LM_SYM_HALF ? 0.5f : 1.0f;
    a.flags = b->flags;
    a.dbg = dbg;
    a.lbo_mn = lbo_mn;
    a.sbo_mn = sbo_mn;
    cudaError_t e;
    if (sy == LM_SYM_HALF) {
        e = cudaFuncSetAttribute(k_pencil_block<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess) {
            lm_prof_begin(ctx, PROF_PENCIL, s);
            k_pencil_block<true><<<b->grid, BLK_THREADS, smem, s>>>(b->tO, b->tG, b->tV, a);
            lm_prof_end(ctx, PROF_PENCIL, s);
        }
    } else {
        e = cudaFuncSetAttribute(k_pencil_block<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            lm_prof_begin(ctx, PROF_PENCIL, s);
            k_pencil_block<false><<<b->grid, BLK_THREADS, smem, s>>>(b->tO, b->tG, b->tV, a);
            lm_prof_end(ctx, PROF_PENCIL, s);
        }
    }
    if (e != cudaSuccess) return lm_cuda_check(ctx, e, "k_pencil_block");
    ctx->pencil_rows += p->n_rows;
    const int tot = 2 * nvec * p->P1;
    k_block_reduce<<<std::min(1024, (tot + 255) / 256), 256, 0, s>>>(
        b->part, b->grid, b->ldo, p->P1, nvec, b->flags, HV, SV, ldv);
    lm_note_launch(ctx, 3);
    return lm_cuda_check(ctx, cudaGetLastError(), "k_pencil_block");
}

extern "C" int lm_apply_pencil_block(lm_pencil *p, const double *V, int ldv, int nvec,
                                     double *HV, double *SV, int sym, void *stream) {
    if (!p || !V) return LM_ERR_ARG;
    cudaSetDevice(p->ctx->device);
    return lm_launch_pencil_block(p, V, ldv, nvec, HV, SV, sym, nullptr, 16384, 1024,
                                  (cudaStream_t)stream);
}

extern "C" int lm_debug_pencil_block(lm_pencil *p, const double *V, int ldv, int nvec,
                                     double *HV, double *SV, int sym, float *dbg,
                                     unsigned lbo_mn, unsigned sbo_mn, void *stream) {
    if (!p || !V) return LM_ERR_ARG;
    cudaSetDevice(p->ctx->device);
    if (lbo_mn % 16 || sbo_mn % 16 || lbo_mn > 65536 || sbo_mn > 65536)
        return lm_fail(p->ctx, LM_ERR_ARG, "descriptor strides");
    return lm_launch_pencil_block(p, V, ldv, nvec, HV, SV, sym, dbg, lbo_mn, sbo_mn,
                                  (cudaStream_t)stream);
}
