// Block Lanczos phase of the IRL solve on the tensor-core block product
// (arXiv 2601.01437, Discussion: block-Lanczos methods as the extension of the
// Standard Lanczos process of Algorithm 2).
//
// With nb = 16 vectors per block and S = m / 16 block steps:
//   Q_0: 16 seeded random vectors (SplitMix64, as the single-vector start),
//        the particle-number null space removed, orthonormalised (CholeskyQR2);
//   step j: AQ_j = H~' Q_j (one tensor-core block product on the BF16
//        factors); W = AQ_j orthogonalised against Q_0..Q_j by classical
//        Gram-Schmidt applied twice (FP64), null space removed, and
//        Q_{j+1} R_j = W (CholeskyQR2, FP64);
//   Rayleigh-Ritz: T = Q^T H~' Q (K = 16 S) from the stored products, its
//        lowest eigenpair by cyclic Jacobi (FP64, one CTA), and the Ritz
//        vector u = Q y.
// u then starts the FP64 IRL continuation, which refines the eigenpair to the
// requested tolerance with FP64-accurate products (as after the single-vector
// low-precision phase). A rank-deficient block (an invariant subspace) ends
// the block steps early; the Rayleigh-Ritz uses the blocks built so far.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace {

constexpr int NB = 16;  // vectors per block

struct BlzState {
    int nblk;    // complete, orthonormal blocks Q_0 .. Q_{nblk-1}
    int broke;   // a block lost rank: no further steps
    double theta;
};

// Q_0[n][e] = 2u - 1 with u the 53-bit SplitMix64 uniform at counter n (P+1) + e
__global__ void k_blz_start(double *Q, int ldp, int P1, uint64_t seed, BlzState *st) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->nblk = 0;
        st->broke = 0;
        st->theta = 0.0;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NB * ldp; i += gridDim.x * blockDim.x) {
        const int n = i / ldp, e = i - n * ldp;
        double v = 0.0;
        if (e < P1) {
            uint64_t z = seed + (uint64_t)((int64_t)n * P1 + e + 1) * 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z = z ^ (z >> 31);
            v = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
        }
        Q[i] = v;
    }
}

// Remove the particle-number null space from nv vectors (grid: (Nh + 1) grid
// rows x nv vectors): within grid row r, the alpha and beta visible entries'
// sums against the null vectors [1_alpha - N_alpha e_0] and [1_beta - N_beta e_0]
// (e_0 only for r > 0), by least squares, as in the single-vector step.
__global__ void k_blz_null(double *W, int ldp, int M1, int n_orb, int na, int nb,
                           const BlzState *st) {
    if (st->broke) return;
    const int r = blockIdx.x, v = blockIdx.y, n = n_orb;
    double *w = W + (size_t)v * ldp + (size_t)r * M1;
    __shared__ double coef[2];
    if (threadIdx.x < 32) {
        double sa = 0.0, sb = 0.0;
        for (int c = 1 + threadIdx.x; c <= 2 * n; c += 32) {
            if (c <= n) sa += w[c]; else sb += w[c];
        }
        sa = warp_sum(sa);
        sb = warp_sum(sb);
        if (threadIdx.x == 0) {
            if (r == 0) {
                coef[0] = sa / n;
                coef[1] = sb / n;
            } else {
                const double w0 = w[0];
                const double g11 = n + (double)na * na, g22 = n + (double)nb * nb,
                             g12 = (double)na * nb;
                const double r1 = sa - na * w0, r2 = sb - nb * w0;
                const double det = g11 * g22 - g12 * g12;
                coef[0] = (g22 * r1 - g12 * r2) / det;
                coef[1] = (g11 * r2 - g12 * r1) / det;
            }
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c <= 2 * n; c += blockDim.x) {
        if (c == 0) {
            if (r > 0) w[0] += coef[0] * na + coef[1] * nb;
        } else if (c <= n) {
            w[c] -= coef[0];
        } else {
            w[c] -= coef[1];
        }
    }
}

// out[a * nbo + b] = sum_{e < P1} X[a][e] Y[b][e] (one warp per output, lanes
// over e, then a fixed butterfly)
__global__ void k_blz_dots(const double *X, int na, const double *Y, int nbo, int ldp, int P1,
                           double *out) {
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (wid >= na * nbo) return;
    const int a = wid / nbo, b = wid - a * nbo;
    const double *x = X + (size_t)a * ldp, *y = Y + (size_t)b * ldp;
    double s = 0.0;
    for (int e = lane; e < P1; e += 32) s = fma(x[e], y[e], s);
    s = warp_sum(s);
    if (lane == 0) out[wid] = s;
}

// out[b][e] = (sub ? out[b][e] : 0) - / + sum_{a < na} X[a][e] C[a * nbo + b]
// (skipped once a block lost rank when skip_broken is set)
__global__ void k_blz_comb(double *out, const double *X, const double *C, int na, int nbo,
                           int ldp, int sub, const BlzState *st, int skip_broken) {
    if (skip_broken && st->broke) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbo * ldp; i += gridDim.x * blockDim.x) {
        const int b = i / ldp, e = i - b * ldp;
        double s = 0.0;
        for (int a = 0; a < na; ++a) s = fma(X[(size_t)a * ldp + e], C[a * nbo + b], s);
        out[i] = sub ? out[i] - s : s;
    }
}

// Cholesky of the 16 x 16 Gram matrix G = R^T R and R^{-1} (upper triangular);
// a pivot below 1e-24 of the largest diagonal marks the block rank-deficient.
__global__ void k_blz_chol(const double *G, double *Rinv, BlzState *st) {
    if (threadIdx.x != 0 || st->broke) return;
    double R[NB][NB], I[NB][NB];
    double dmax = 0.0;
    for (int i = 0; i < NB; ++i) dmax = fmax(dmax, G[i * NB + i]);
    for (int i = 0; i < NB; ++i)
        for (int j = 0; j < NB; ++j) R[i][j] = 0.0;
    for (int j = 0; j < NB; ++j) {
        double d = G[j * NB + j];
        for (int k = 0; k < j; ++k) d -= R[k][j] * R[k][j];
        if (!(d > 1e-24 * dmax)) {
            st->broke = 1;
            return;
        }
        R[j][j] = sqrt(d);
        for (int i = j + 1; i < NB; ++i) {
            double s = G[j * NB + i];
            for (int k = 0; k < j; ++k) s -= R[k][j] * R[k][i];
            R[j][i] = s / R[j][j];
        }
    }
    // R^{-1}: upper triangular, column by column (back substitution)
    for (int j = NB - 1; j >= 0; --j) {
        for (int i = 0; i < NB; ++i) I[i][j] = 0.0;
        I[j][j] = 1.0 / R[j][j];
        for (int i = j - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1; k <= j; ++k) s += R[i][k] * I[k][j];
            I[i][j] = -s / R[i][i];
        }
    }
    for (int i = 0; i < NB; ++i)
        for (int j = 0; j < NB; ++j) Rinv[i * NB + j] = I[i][j];
}

__global__ void k_blz_count(BlzState *st) {
    if (threadIdx.x == 0 && !st->broke) st->nblk++;
}

// Lowest eigenpair of the symmetric K x K matrix T (K = 16 nblk, row stride
// ldt; T symmetrised as (T + T^T) / 2) by cyclic Jacobi in FP64 on one CTA:
// each sweep is K - 1 rounds of K / 2 disjoint rotations (round-robin pairing,
// player 0 fixed), each rotation the symmetric 2 x 2 Schur rotation of
// Golub & Van Loan (tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) /
// (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c), applied to the
// rows, the columns and the accumulated eigenvectors. Stops when the
// off-diagonal norm is below 1e-15 of the matrix norm (at most 40 sweeps).
constexpr int KMAX = 64;
__global__ void __launch_bounds__(256) k_blz_jacobi(const double *T, int ldt, BlzState *st,
                                                    double *y) {
    __shared__ double A[KMAX][KMAX + 1], V[KMAX][KMAX + 1];
    __shared__ double cs[KMAX / 2], sn[KMAX / 2];
    __shared__ int pp[KMAX / 2], qq[KMAX / 2];
    __shared__ double red[256];
    __shared__ int s_done;
    const int K = NB * st->nblk;
    const int tid = threadIdx.x;
    if (K < 1) {
        if (tid == 0) st->theta = NAN;
        return;
    }
    for (int i = tid; i < K * K; i += blockDim.x) {
        const int r = i / K, c = i - r * K;
        A[r][c] = 0.5 * (T[r * ldt + c] + T[c * ldt + r]);
        V[r][c] = r == c ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 40; ++sweep) {
        // convergence: off-diagonal vs total Frobenius norm
        double off = 0.0, tot = 0.0;
        for (int i = tid; i < K * K; i += blockDim.x) {
            const int r = i / K, c = i - r * K;
            const double v = A[r][c] * A[r][c];
            tot += v;
            if (r != c) off += v;
        }
        red[tid] = off;
        __syncthreads();
        for (int h = 128; h > 0; h >>= 1) {
            if (tid < h) red[tid] += red[tid + h];
            __syncthreads();
        }
        const double offs = red[0];
        __syncthreads();
        red[tid] = tot;
        __syncthreads();
        for (int h = 128; h > 0; h >>= 1) {
            if (tid < h) red[tid] += red[tid + h];
            __syncthreads();
        }
        if (tid == 0) s_done = offs <= 1e-30 * red[0];
        __syncthreads();
        if (s_done) break;
        for (int round = 0; round < K - 1; ++round) {
            if (tid < K / 2) {
                const int k = tid;
                const int pos_p = k, pos_q = K - 1 - k;
                const int p = pos_p == 0 ? 0 : ((pos_p - 1 + round) % (K - 1)) + 1;
                const int q = ((pos_q - 1 + round) % (K - 1)) + 1;
                const double apq = A[p][q];
                double c = 1.0, sv = 0.0;
                if (apq != 0.0) {
                    const double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
                    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + t * t);
                    sv = t * c;
                }
                cs[k] = c;
                sn[k] = sv;
                pp[k] = p;
                qq[k] = q;
            }
            __syncthreads();
            // rows p, q of A
            for (int i = tid; i < (K / 2) * K; i += blockDim.x) {
                const int k = i / K, col = i - k * K;
                const int p = pp[k], q = qq[k];
                const double c = cs[k], sv = sn[k];
                const double ap = A[p][col], aq = A[q][col];
                A[p][col] = c * ap - sv * aq;
                A[q][col] = sv * ap + c * aq;
            }
            __syncthreads();
            // columns p, q of A and of V
            for (int i = tid; i < (K / 2) * K; i += blockDim.x) {
                const int k = i / K, row = i - k * K;
                const int p = pp[k], q = qq[k];
                const double c = cs[k], sv = sn[k];
                const double ap = A[row][p], aq = A[row][q];
                A[row][p] = c * ap - sv * aq;
                A[row][q] = sv * ap + c * aq;
                const double vp = V[row][p], vq = V[row][q];
                V[row][p] = c * vp - sv * vq;
                V[row][q] = sv * vp + c * vq;
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        int best = 0;
        for (int i = 1; i < K; ++i)
            if (A[i][i] < A[best][best]) best = i;
        pp[0] = best;
        st->theta = A[best][best];
    }
    __syncthreads();
    for (int i = tid; i < KMAX; i += blockDim.x) y[i] = i < K ? V[i][pp[0]] : 0.0;
}

}  // namespace

// ---------------------------------------------------------------- host side
int lm_launch_block_lanczos(lm_pencil *p, int sym, int nsteps, uint64_t seed, int deflate,
                            double *u_out, cudaStream_t s) {
    lm_ctx *ctx = p->ctx;
    if (nsteps < 1 || nsteps * NB > KMAX)
        return lm_fail(ctx, LM_ERR_SIZE, "block Lanczos takes 1..%d block steps", KMAX / NB);
    const size_t L = (size_t)p->ldp;
    const int K = nsteps * NB;
    if (!p->blz) {
        // Q (K + 16 vectors), AQ (K), W (16), C (K x 16), G, Rinv (16 x 16), T (K x K), y, state
        const size_t nd = (size_t)(2 * KMAX + 2 * NB) * L + (size_t)KMAX * NB + 2 * NB * NB +
                          (size_t)KMAX * KMAX + KMAX + 64;
        if (lm_cuda_check(ctx, cudaMalloc(&p->blz, nd * sizeof(double)), "cudaMalloc"))
            return LM_ERR_OOM;
        p->blz_len = nd;
    }
    double *Q = p->blz;
    double *AQ = Q + (size_t)(KMAX + NB) * L;
    double *W = AQ + (size_t)KMAX * L;
    double *C = W + (size_t)NB * L;
    double *G = C + (size_t)KMAX * NB;
    double *Ri = G + NB * NB;
    double *T = Ri + NB * NB;
    double *y = T + KMAX * KMAX;
    BlzState *st = reinterpret_cast<BlzState *>(y + KMAX);
    if ((size_t)(reinterpret_cast<double *>(st) + 8 - p->blz) > p->blz_len)
        return lm_fail(ctx, LM_ERR_SIZE, "block Lanczos workspace");
    const int P1 = p->P1, g2 = p->nh + 1;
    const int grid = std::min(ctx->sms * 4, (int)((NB * L + 255) / 256));
    auto dots = [&](const double *X, int na, const double *Y, int nbo, double *out) {
        const int nw = na * nbo;
        k_blz_dots<<<(nw + 7) / 8, 256, 0, s>>>(X, na, Y, nbo, (int)L, P1, out);
    };
    auto orth_block = [&](double *X) {  // X (16 vectors) <- X R^{-1}, twice
        for (int pass = 0; pass < 2; ++pass) {
            dots(X, NB, X, NB, G);
            k_blz_chol<<<1, 32, 0, s>>>(G, Ri, st);
            k_blz_comb<<<grid, 256, 0, s>>>(W, X, Ri, NB, NB, (int)L, 0, st, 1);
            cudaMemcpyAsync(X, W, NB * L * sizeof(double), cudaMemcpyDeviceToDevice, s);
        }
    };
    k_blz_start<<<grid, 256, 0, s>>>(Q, (int)L, P1, seed, st);
    if (deflate) k_blz_null<<<dim3(g2, NB), 64, 0, s>>>(Q, (int)L, p->M1, p->n, p->na, p->nb, st);
    orth_block(Q);
    k_blz_count<<<1, 32, 0, s>>>(st);
    for (int j = 0; j < nsteps; ++j) {
        double *Qj = Q + (size_t)j * NB * L, *AQj = AQ + (size_t)j * NB * L;
        if (int rc = lm_launch_pencil_block(p, Qj, (int)L, NB, AQj, nullptr, sym, nullptr, 16384,
                                            1024, s))
            return rc;
        if (j == nsteps - 1) break;
        double *Wn = Q + (size_t)(j + 1) * NB * L;
        cudaMemcpyAsync(Wn, AQj, NB * L * sizeof(double), cudaMemcpyDeviceToDevice, s);
        const int na = (j + 1) * NB;
        for (int pass = 0; pass < 2; ++pass) {
            dots(Q, na, Wn, NB, C);
            k_blz_comb<<<grid, 256, 0, s>>>(Wn, Q, C, na, NB, (int)L, 1, st, 1);
        }
        if (deflate)
            k_blz_null<<<dim3(g2, NB), 64, 0, s>>>(Wn, (int)L, p->M1, p->n, p->na, p->nb, st);
        orth_block(Wn);
        k_blz_count<<<1, 32, 0, s>>>(st);
    }
    // Rayleigh-Ritz on the complete blocks: T = Q^T (H~' Q)
    dots(Q, K, AQ, K, T);
    k_blz_jacobi<<<1, 256, 0, s>>>(T, K, st, y);
    // u = Q y over the first 16 nblk vectors (y is zero beyond them)
    k_blz_comb<<<grid, 256, 0, s>>>(u_out, Q, y, K, 1, (int)L, 0, st, 0);
    lm_note_launch(ctx, 8 * nsteps + 8);
    return lm_cuda_check(ctx, cudaGetLastError(), "block Lanczos");
}
