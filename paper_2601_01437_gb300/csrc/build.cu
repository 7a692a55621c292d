// Build half of the hot path: rows -> O, E_loc, G -> weights, E, <O> -> centred
// O_c and G'_c (arXiv 2601.01437, Methods: E_loc and O definitions, eqs. heff
// and centered_hamiltonian, the energy-centring step H' = H - E).
//
// Layout: one determinant per uint64 (bit p = spin orbital p, alpha block
// then beta block). O and G rows live on the augmented (Nh+1) x (M+1) grid,
// row-major, padded to ldp columns (a multiple of 8, so every row starts on a
// 64-byte boundary for FP64 and on 16 bytes for the low-precision copies).
#include <cstdarg>
#include <cstdlib>
#include <cstring>

#include "df64.cuh"
#include "internal.cuh"

namespace {

// ----------------------------------------------------------------- helpers
__device__ __forceinline__ uint64_t binom_dev(int n, int k) {
    if (k < 0 || n < 0 || k > n) return 0;
    uint64_t c = 1;
    for (int i = 1; i <= k; ++i) c = c * (uint64_t)(n - k + i) / (uint64_t)i;
    return c;
}

// k-subset of [0, n) with colex rank r (ascending bit-mask order).
__device__ __forceinline__ uint64_t unrank_colex(int n, int k, uint64_t r) {
    uint64_t x = 0;
    for (int kk = k; kk >= 1; --kk) {
        int c = kk - 1;
        while (c + 1 < n && binom_dev(c + 1, kk) <= r) ++c;
        x |= (1ull << c);
        r -= binom_dev(c, kk);
    }
    return x;
}

// Division by a fixed divisor d without a divide (which converts to and from
// floating point, and conversions issue at the FP64 rate on this part): with
// l = ceil(log2 d) and m = ceil(2^(31+l) / d) < 2^32, x / d = (x m) >> (31 + l)
// exactly for 0 <= x < 2^31 (Granlund and Montgomery, "Division by invariant
// integers using multiplication", 1994).
struct FastDiv {
    uint32_t m, s, d;
};
inline FastDiv make_fastdiv(int divisor) {
    const uint32_t d = divisor > 0 ? (uint32_t)divisor : 1u;
    uint32_t l = 0;
    while ((1u << l) < d) ++l;
    FastDiv f;
    f.m = (uint32_t)(((1ull << (31 + l)) + d - 1) / d);
    f.s = 31 + l;
    f.d = d;
    return f;
}
__device__ __forceinline__ int fdiv(int x, FastDiv f) {
    return (int)(((uint64_t)(uint32_t)x * f.m) >> f.s);
}

// pair (lo < hi) with colex rank q (q < 2^22): the float of q and the nearest
// integer of the root by exact magic-number arithmetic, then exact corrections
__device__ __forceinline__ void unrank_pair(int q, int &lo, int &hi) {
    const float fq = __fsub_rn(__int_as_float(0x4B400000 + q), 12582912.0f);
    const float r = 0.5f * (1.0f + sqrtf(fmaf(8.0f, fq, 1.0f)));
    int y = __float_as_int(__fadd_rn(r, 12582912.0f)) - 0x4B400000;
    while (y * (y - 1) / 2 > q) --y;
    while ((y + 1) * y / 2 <= q) ++y;
    hi = y;
    lo = q - y * (y - 1) / 2;
}

// parity of the occupied spin orbitals below p, on 32-bit words
__device__ __forceinline__ int parity_below(uint64_t x, int p) {
    const unsigned lo = (unsigned)x, hi = (unsigned)(x >> 32);
    const int c = p < 32 ? __popc(lo & ((1u << p) - 1u))
                         : __popc(lo) + __popc(hi & ((1u << (p - 32)) - 1u));
    return c & 1;
}
// occupation of spin orbital p (p < 64), on 32-bit words
__device__ __forceinline__ bool occ_bit(uint64_t x, int p) {
    return ((p < 32 ? (unsigned)x >> p : (unsigned)(x >> 32) >> (p - 32)) & 1u) != 0u;
}

struct SysView {
    int n, na, nb, nva, nvb;
    int ns_a, ns_b, nd_aa, nd_bb, nd_ab, conn;
    FastDiv fd_nva, fd_nvb, fd_pva, fd_pvb, fd_nbe;  // by nva, nvb, C(nva,2), C(nvb,2), ns_b
    const double *h, *eri;
};

__device__ __forceinline__ double eri4(const SysView &S, int p, int q, int r, int s) {
    return __ldg(S.eri + (((size_t)p * S.n + q) * S.n + r) * S.n + s);
}

// Occupied / empty spin orbitals of one determinant, ascending, per spin.
struct RowLists {
    int oa[32], va[32], ob[32], vb[32];
};

__device__ void make_lists(const SysView &S, uint64_t x, RowLists &L) {
    int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    for (int p = 0; p < S.n; ++p) {
        if (occ_bit(x, p)) L.oa[c0++] = p; else L.va[c1++] = p;
        int q = p + S.n;
        if (occ_bit(x, q)) L.ob[c2++] = q; else L.vb[c3++] = q;
    }
}

struct Exc {
    int i, j, a, b;  // removed i (< j), added a (< b); j = b = -1 for singles
};

// Connection k of the row (0 <= k < conn): singles alpha, singles beta,
// doubles alpha-alpha, beta-beta, alpha-beta, each in a fixed nested order.
__device__ __forceinline__ Exc decode_exc(const SysView &S, const RowLists &L, int k) {
    Exc e;
    e.j = -1;
    e.b = -1;
    if (k < S.ns_a) {
        const int q = fdiv(k, S.fd_nva);
        e.i = L.oa[q];
        e.a = L.va[k - q * S.nva];
        return e;
    }
    k -= S.ns_a;
    if (k < S.ns_b) {
        const int q = fdiv(k, S.fd_nvb);
        e.i = L.ob[q];
        e.a = L.vb[k - q * S.nvb];
        return e;
    }
    k -= S.ns_b;
    int lo, hi;
    if (k < S.nd_aa) {
        const int nvp = S.nva * (S.nva - 1) / 2, q = fdiv(k, S.fd_pva);
        unrank_pair(q, lo, hi);
        e.i = L.oa[lo];
        e.j = L.oa[hi];
        unrank_pair(k - q * nvp, lo, hi);
        e.a = L.va[lo];
        e.b = L.va[hi];
        return e;
    }
    k -= S.nd_aa;
    if (k < S.nd_bb) {
        const int nvp = S.nvb * (S.nvb - 1) / 2, q = fdiv(k, S.fd_pvb);
        unrank_pair(q, lo, hi);
        e.i = L.ob[lo];
        e.j = L.ob[hi];
        unrank_pair(k - q * nvp, lo, hi);
        e.a = L.vb[lo];
        e.b = L.vb[hi];
        return e;
    }
    k -= S.nd_bb;
    const int nbe = S.nb * S.nvb;
    const int sa = fdiv(k, S.fd_nbe), sb = k - sa * nbe;
    const int qa = fdiv(sa, S.fd_nva), qb = fdiv(sb, S.fd_nvb);
    e.i = L.oa[qa];
    e.a = L.va[sa - qa * S.nva];
    e.j = L.ob[qb];
    e.b = L.vb[sb - qb * S.nvb];
    return e;
}

// Apply the excitation to x: x' and the Jordan-Wigner sign of a+_a a_i or
// a+_a a+_b a_j a_i (operators applied right to left).
__device__ __forceinline__ uint64_t apply_exc(uint64_t x, const Exc &e, int &sgn) {
    int par = parity_below(x, e.i);
    x ^= (1ull << e.i);
    if (e.j >= 0) {
        par += parity_below(x, e.j);
        x ^= (1ull << e.j);
        par += parity_below(x, e.b);
        x |= (1ull << e.b);
    }
    par += parity_below(x, e.a);
    x |= (1ull << e.a);
    sgn = (par & 1) ? -1 : 1;
    return x;
}

// <x'|H|x> without the sign (Slater-Condon rules, chemist integrals).
__device__ __forceinline__ double exc_value(const SysView &S, const RowLists &L, const Exc &e) {
    const int n = S.n;
    if (e.j < 0) {
        int sp = e.i >= n;
        int ip = e.i - sp * n, ap = e.a - sp * n;
        double v = __ldg(S.h + ap * n + ip);
        for (int t = 0; t < S.na; ++t) {
            int kp = L.oa[t];
            v += eri4(S, ap, ip, kp, kp);
            if (sp == 0) v -= eri4(S, ap, kp, kp, ip);
        }
        for (int t = 0; t < S.nb; ++t) {
            int kp = L.ob[t] - n;
            v += eri4(S, ap, ip, kp, kp);
            if (sp == 1) v -= eri4(S, ap, kp, kp, ip);
        }
        return v;
    }
    int si = e.i >= n, sj = e.j >= n, sa = e.a >= n, sb = e.b >= n;
    int ip = e.i - si * n, jp = e.j - sj * n, ap = e.a - sa * n, bp = e.b - sb * n;
    double v = 0.0;
    if (sa == si && sb == sj) v += eri4(S, ap, ip, bp, jp);
    if (sa == sj && sb == si) v -= eri4(S, ap, jp, bp, ip);
    return v;
}

// Diagonal <x|H|x> by one warp: sum_I h_II + 1/2 sum_{I,J} [(II|JJ) - d_s (IJ|JI)].
__device__ double diag_value_warp(const SysView &S, const RowLists &L) {
    const int lane = threadIdx.x & 31;
    const int ne = S.na + S.nb;
    double v = 0.0;
    for (int t = lane; t < ne * ne; t += 32) {
        int a = t / ne, b = t % ne;
        int I = a < S.na ? L.oa[a] : L.ob[a - S.na];
        int J = b < S.na ? L.oa[b] : L.ob[b - S.na];
        int sI = I >= S.n, sJ = J >= S.n;
        int ip = I - sI * S.n, jp = J - sJ * S.n;
        double g = eri4(S, ip, ip, jp, jp);
        if (sI == sJ) g -= eri4(S, ip, jp, jp, ip);
        v += 0.5 * g;
    }
    for (int t = lane; t < ne; t += 32) {
        int I = t < S.na ? L.oa[t] : L.ob[t - S.na];
        int ip = I >= S.n ? I - S.n : I;
        v += __ldg(S.h + ip * S.n + ip);
    }
    return warp_sum(v);
}

SysView make_view(int n, int na, int nb, const double *h, const double *eri) {
    SysView S;
    S.n = n;
    S.na = na;
    S.nb = nb;
    S.nva = n - na;
    S.nvb = n - nb;
    S.ns_a = na * S.nva;
    S.ns_b = nb * S.nvb;
    S.nd_aa = (na * (na - 1) / 2) * (S.nva * (S.nva - 1) / 2);
    S.nd_bb = (nb * (nb - 1) / 2) * (S.nvb * (S.nvb - 1) / 2);
    S.nd_ab = S.ns_a * S.ns_b;
    S.conn = S.ns_a + S.ns_b + S.nd_aa + S.nd_bb + S.nd_ab;
    S.fd_nva = make_fastdiv(S.nva);
    S.fd_nvb = make_fastdiv(S.nvb);
    S.fd_pva = make_fastdiv(S.nva * (S.nva - 1) / 2);
    S.fd_pvb = make_fastdiv(S.nvb * (S.nvb - 1) / 2);
    S.fd_nbe = make_fastdiv(S.ns_b);
    S.h = h;
    S.eri = eri;
    return S;
}

// --------------------------------------------------------- K1: enumeration
// Index i = rank_beta * C(n, na) + rank_alpha gives the ascending order of
// x = alpha_bits | beta_bits << n (colex rank = ascending mask order).
__global__ void k_enumerate(int n, int na, int nb, uint64_t *out, int64_t count) {
    const uint64_t ca = binom_dev(n, na);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t ra = (uint64_t)i % ca, rb = (uint64_t)i / ca;
        out[i] = unrank_colex(n, na, ra) | (unrank_colex(n, nb, rb) << n);
    }
}

// ------------------------------------------------------ theta-derived tables
// tabs = [exp(W) (Nh x M) | exp(-W) (Nh x M) | exp(a) (M) | exp(-a) (M)]
__global__ void k_tables(const double *theta, int M, int nh, double *tabs) {
    const int M1 = M + 1;
    const int tot = nh * M + M;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
        double w;
        if (e < nh * M) {
            int j = e / M, p = e % M;
            w = theta[(j + 1) * M1 + p];
            tabs[e] = exp(w);
            tabs[nh * M + e] = exp(-w);
        } else {
            int p = e - nh * M;
            w = theta[p];
            tabs[2 * nh * M + p] = exp(w);
            tabs[2 * nh * M + M + p] = exp(-w);
        }
    }
}

// ------------------------------------------------- K2-K6: fused row build
struct BuildArgs {
    SysView S;
    int nh, M, M1, P1, ldp;
    int ldF, ldS, nslice;
    const double *theta, *tabs;
    const uint64_t *rows;
    int64_t n_rows;
    uint64_t amask, bmask;
    double e_core;
    double *lnpsi, *eloc, *O, *G;
    int *flags;
};

constexpr int BUILD_THREADS = 128;

// One CTA per row (persistent over rows). Per row:
//   z_j = b_j + W_j.x, t_j = tanh z_j, ln psi, O row = [1;t] (x) [1;x];
//   every connection x' (Slater-Condon element with sign) contributes
//   c = H_xx' psi(x')/psi(x), evaluated from tables as
//   psi(x')/psi(x) = exp(a.dx) prod_j cosh(z_j + d_j)/cosh(z_j), with
//   exp(+-d_j) products of exp(+-W_jp) over the moved orbitals, and
//   tanh(z_j + d_j) from the same factors;
//   G row = sum_x' c [1;t'] (x) [1;x'] accumulated sparsely: column 0 gets
//   every term, column p+1 gets terms with x'_p = 1 (all minus those that
//   remove p for occupied p; those that add p for empty p).
__global__ void __launch_bounds__(BUILD_THREADS) k_build_rows(BuildArgs A) {
    extern __shared__ __align__(16) unsigned char smb[];
    const int nh = A.nh, M = A.M, M1 = A.M1;
    const int tid = threadIdx.x;
    const int K = BUILD_THREADS;
    // 16-byte aligned pieces first, then the FP64 arrays
    int4 *sIdx = reinterpret_cast<int4 *>(smb);
    RowLists *sL = reinterpret_cast<RowLists *>(sIdx + K);
    double *sEW = reinterpret_cast<double *>(sL + 1);
    double *sEWi = sEW + nh * M;
    double *sea = sEWi + nh * M;
    double *seai = sea + M;
    double *sP = seai + M;
    double *sQ = sP + nh;
    double *sT = sQ + nh;
    double *sF = sT + nh;
    double *sC = sF + K * A.ldF;
    double *sS = sC + K;
    double *sA = sS + A.nslice * (nh + 1) * A.ldS;
    double *sRed = sA + A.nslice * (nh + 1);
    __shared__ double sDiag, sLn;
    __shared__ int sBad;

    for (int e = tid; e < 2 * nh * M + 2 * M; e += K) sEW[e] = A.tabs[e];
    __syncthreads();

    const int nsl = A.nslice;
    const int sc_r = tid % (nh + 1), sc_s = tid / (nh + 1);
    const bool scatter_thread = sc_s < nsl;

    for (int64_t row = blockIdx.x; row < A.n_rows; row += gridDim.x) {
        const uint64_t x = A.rows[row];
        if (tid == 0) {
            int bad = (__popcll(x & A.amask) != A.S.na) || (__popcll(x & A.bmask) != A.S.nb) ||
                      (x & ~(A.amask | A.bmask)) != 0;
            sBad = bad;
            if (bad) atomicOr(A.flags, FLAG_ROW_OUTSIDE_SECTOR);
            make_lists(A.S, x, *sL);
        }
        __syncthreads();
        if (sBad) {
            __syncthreads();
            continue;
        }
        // hidden pre-activations
        for (int j = tid; j < nh; j += K) {
            double z = A.theta[(j + 1) * M1 - 1];
            for (int p = 0; p < M; ++p)
                if ((x >> p) & 1ull) z += A.theta[(j + 1) * M1 + p];
            double az = fabs(z);
            double e2 = exp(-2.0 * az);
            double inv = 1.0 / (1.0 + e2);
            double big = inv, small = e2 * inv;  // e^{|z|}/(2cosh z), e^{-|z|}/(2cosh z)
            sP[j] = z >= 0.0 ? big : small;       // e^{z} / (2 cosh z)
            sQ[j] = z >= 0.0 ? small : big;       // e^{-z} / (2 cosh z)
            sT[j] = tanh(z);
        }
        for (int e = tid; e < nsl * (nh + 1) * A.ldS; e += K) sS[e] = 0.0;
        __syncthreads();
        if (tid < 32) {
            // ln psi = a.x + sum_j ln(2 cosh z_j), ln(2cosh z) = |z| + log1p(e^{-2|z|})
            double lp = 0.0;
            for (int j = tid; j < nh; j += 32) {
                double zz = A.theta[(j + 1) * M1 - 1];
                for (int p = 0; p < M; ++p)
                    if ((x >> p) & 1ull) zz += A.theta[(j + 1) * M1 + p];
                lp += fabs(zz) + log1p(exp(-2.0 * fabs(zz)));
            }
            for (int p = tid; p < M; p += 32)
                if ((x >> p) & 1ull) lp += A.theta[p];
            lp = warp_sum(lp);
            if (tid == 0) sLn = lp;
        } else if (tid < 64) {
            double d = diag_value_warp(A.S, *sL);
            if (tid == 32) sDiag = d + A.e_core;
        }
        __syncthreads();

        double el_part = 0.0;
        double accA = 0.0;
        const RowLists &L = *sL;
        for (int k0 = 0; k0 < A.S.conn; k0 += K) {
            const int k = k0 + tid;
            if (k < A.S.conn) {
                Exc e = decode_exc(A.S, L, k);
                int sg;
                (void)apply_exc(x, e, sg);
                double hv = sg * exc_value(A.S, L, e);
                const bool dbl = e.j >= 0;
                double ead = sea[e.a] * seai[e.i];
                if (dbl) ead *= sea[e.b] * seai[e.j];
                double r = 1.0;
                double *Frow = sF + tid * A.ldF;
                for (int j = 0; j < nh; ++j) {
                    const double *ew = sEW + j * M;
                    const double *ewi = sEWi + j * M;
                    double ep = ew[e.a] * ewi[e.i];
                    double em = ewi[e.a] * ew[e.i];
                    if (dbl) {
                        ep *= ew[e.b] * ewi[e.j];
                        em *= ewi[e.b] * ew[e.j];
                    }
                    double t1 = ep * sP[j];
                    double q = fma(em, sQ[j], t1);   // cosh(z+d)/cosh(z)
                    double nu = fma(-em, sQ[j], t1); // sinh(z+d)/cosh(z)
                    r *= q;
                    Frow[j] = nu / q;                // tanh(z+d)
                }
                double c = hv * ead * r;
                sC[tid] = c;
                sIdx[tid] = make_int4(e.i, e.j, e.a, e.b);
                el_part += c;
            }
            __syncthreads();
            if (scatter_thread) {
                const int kend = min(K, A.S.conn - k0);
                double *Srow = sS + (sc_s * (nh + 1) + sc_r) * A.ldS;
                for (int kk = sc_s; kk < kend; kk += nsl) {
                    double f = sC[kk];
                    if (sc_r > 0) f *= sF[kk * A.ldF + sc_r - 1];
                    int4 ix = sIdx[kk];
                    accA += f;
                    Srow[ix.x] += f;
                    Srow[ix.z] += f;
                    if (ix.y >= 0) {
                        Srow[ix.y] += f;
                        Srow[ix.w] += f;
                    }
                }
            }
            __syncthreads();
        }
        if (scatter_thread) sA[sc_s * (nh + 1) + sc_r] = accA;
        // E_loc: fixed-order block reduction
        el_part = warp_sum(el_part);
        if ((tid & 31) == 0) sRed[32 + (tid >> 5)] = el_part;
        __syncthreads();
        if (tid == 0) {
            double el = sDiag;
            for (int w = 0; w < K / 32; ++w) el += sRed[32 + w];
            A.eloc[row] = el;
            A.lnpsi[row] = sLn;
        }
        // O row and G row
        double *Orow = A.O + row * (int64_t)A.ldp;
        double *Grow = A.G + row * (int64_t)A.ldp;
        const double hd = sDiag;
        for (int e = tid; e < A.ldp; e += K) {
            double ov = 0.0, gv = 0.0;
            if (e < A.P1) {
                int r = e / M1, c = e % M1;
                double u = (r == 0) ? 1.0 : sT[r - 1];
                double xc = (c == 0) ? 1.0 : (double)((x >> (c - 1)) & 1ull);
                ov = u * xc;
                double at = hd * u;
                for (int s = 0; s < nsl; ++s) at += sA[s * (nh + 1) + r];
                if (c == 0) {
                    gv = at;
                } else {
                    double sv = 0.0;
                    for (int s = 0; s < nsl; ++s) sv += sS[(s * (nh + 1) + r) * A.ldS + c - 1];
                    gv = ((x >> (c - 1)) & 1ull) ? at - sv : sv;
                }
            }
            Orow[e] = ov;
            Grow[e] = gv;
        }
        __syncthreads();
    }
}

// ------------------------------------- K2-K6 in double-float arithmetic
// tdf (float2 = df) = [exp(2W) Nh x M | exp(-2W) Nh x M | h n^2 | (pq|rs) n^4]
__global__ void k_tables_df(const double *theta, const double *h, const double *eri, int M, int nh,
                            int n, float2 *out) {
    const int n_exp = 2 * nh * M, n2 = n * n, n4 = n2 * n2;
    const int tot = n_exp + n2 + n4;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
        double x;
        if (e < n_exp) {
            const int f = e % (nh * M), j = f / M, p = f % M;
            const double w = theta[(j + 1) * (M + 1) + p];
            x = exp(e < nh * M ? 2.0 * w : -2.0 * w);
        } else {
            x = e < n_exp + n2 ? h[e - n_exp] : eri[e - n_exp - n2];
        }
        const df d = df_from_double(x);
        out[e] = make_float2(d.h, d.l);
    }
}

__device__ __forceinline__ df ld_df(const float2 *p) {
    const float2 v = *p;
    return df_make(v.x, v.y);
}
__device__ __forceinline__ df ldg_df(const float2 *p) {
    const float2 v = __ldg(p);
    return df_make(v.x, v.y);
}
__device__ __forceinline__ void st_df(float2 *p, df a) { *p = make_float2(a.h, a.l); }

// Slater-Condon <x'|H|x> (without sign) in double-float, integrals from tdf.
__device__ __forceinline__ df exc_value_df(const SysView &S, const RowLists &L, const Exc &e,
                                           const float2 *hd, const float2 *gd) {
    const int n = S.n;
    auto g4 = [&](int p, int q, int r, int s) {
        return ldg_df(gd + (((size_t)p * n + q) * n + r) * n + s);
    };
    if (e.j < 0) {
        const int sp = e.i >= n;
        const int ip = e.i - sp * n, ap = e.a - sp * n;
        df v = ldg_df(hd + ap * n + ip);
        for (int t = 0; t < S.na; ++t) {
            const int kp = L.oa[t];
            v = df_add(v, g4(ap, ip, kp, kp));
            if (sp == 0) v = df_sub(v, g4(ap, kp, kp, ip));
        }
        for (int t = 0; t < S.nb; ++t) {
            const int kp = L.ob[t] - n;
            v = df_add(v, g4(ap, ip, kp, kp));
            if (sp == 1) v = df_sub(v, g4(ap, kp, kp, ip));
        }
        return v;
    }
    const int si = e.i >= n, sj = e.j >= n, sa = e.a >= n, sb = e.b >= n;
    const int ip = e.i - si * n, jp = e.j - sj * n, ap = e.a - sa * n, bp = e.b - sb * n;
    df v = df_make(0.f, 0.f);
    if (sa == si && sb == sj) v = g4(ap, ip, bp, jp);
    if (sa == sj && sb == si) v = df_sub(v, g4(ap, jp, bp, ip));
    return v;
}

// Keep a running product m * 2^ex with m in [2^-60, 2^60].
__device__ __forceinline__ void df_renorm(df &m, int &ex) {
    const float a = fabsf(m.h);
    if (a > 0x1p60f || a < 0x1p-60f) {
        int k;
        frexpf(m.h, &k);
        m = df_ldexp(m, -k);
        ex += k;
    }
}

// Lazy double-float accumulation acc += f (TwoSum of the heads, tails summed
// unnormalised); df_fts(acc.h, acc.l) renormalises at the end.
__device__ __forceinline__ void df_acc(df &acc, df f) {
    const df s = df_ts(acc.h, f.h);
    acc.h = s.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, f.l));
}
__device__ __forceinline__ df df_norm(df a) { return df_fts(a.h, a.l); }

// 1 + Z for Z >= 0 with the tail left unnormalised (the reciprocal and the
// products that take it are error-free on the head)
__device__ __forceinline__ df df_add1_lazy(df z) {
    const df s = df_ts(z.h, 1.f);
    return df_make(s.h, __fadd_rn(s.l, z.l));
}

// Single excitation s of a row (i -> a): alpha singles first, then beta.
__device__ __forceinline__ void single_of(const SysView &S, const RowLists &L, int s, int &i,
                                          int &a) {
    if (s < S.ns_a) {
        const int q = fdiv(s, S.fd_nva);
        i = L.oa[q];
        a = L.va[s - q * S.nva];
    } else {
        s -= S.ns_a;
        const int q = fdiv(s, S.fd_nvb);
        i = L.ob[q];
        a = L.vb[s - q * S.nvb];
    }
}

// ------------------------------- K2-K6 in double-float, by connection class
// K2-K6 as k_build_rows computes them, in double-float arithmetic on the FP32
// pipes. For hidden unit j let sigma_j = -sign(z_j) (+1 if z_j < 0),
// g_j = exp(2 sigma_j z_j) <= 1 and, for a connection moving orbitals with
// shift d_j of the pre-activation, Z_j = g_j exp(2 sigma_j d_j). Then
//   tanh(z_j + d_j) = sigma_j (1 - 2 u_j),  u_j = 1 / (1 + Z_j),
//   prod_j cosh(z_j+d_j)/cosh(z_j) = exp(-sum_j sigma_j d_j) prod_j (1+Z_j) / prod_j (1+g_j).
// Per row, every single excitation s (i -> a) gets B_s[j] = exp(2 sigma_j d_j),
// A_s[j] = g_j B_s[j] and V_s = exp(a_a - a_i - sum_j sigma_j d_j); a double
// (s1, s2) has Z_j = A_s1[j] B_s2[j] and factor V_s1 V_s2. So the work per
// (connection, hidden unit) is one double-float product (doubles), Z +- 1, a
// division and the running product. Four threads share a connection and
// combine their partial products with shuffles. The G sums are accumulated
// from c u_j rather than c tanh(z_j + d_j): over any connection set Q,
// sum_Q c tanh = sigma_j (sum_Q c - 2 sum_Q c u_j), and sum_Q c is the hidden
// row 0 of the same sums, so the conversion happens once per output element.
//
// The connections of a row, class by class, as row-major grids (R rows x C columns):
//   GC_AA  alpha-alpha doubles: occupied-pair rank x empty-pair rank (colex ranks)
//   GC_BB  beta-beta doubles, the same over the beta orbitals
//   GC_B   beta singles: occupied position x empty position
//   GC_AB  alpha single s x (1 + beta singles): column 0 is the alpha single s
//          itself, column 1 + t the alpha-beta double made of s and beta single t
// A connection moves the orbitals of its row (the occupied pair; the occupied
// orbital; the two orbitals of s) and of its column (the empty pair; the empty
// orbital; the two orbitals of t; none for column 0). Decoding a connection is
// then a division by C and table lookups: the alpha-beta double's integral is
// (a i|b j) at an index that is the sum of a per-single part of s and of t, its
// sign the product of the singles' signs, its Z_j = A_s[j] B_t[j].
// The scatter into the per-orbital sums S[p][j] = sum_{x' moving p} c u_j(x')
// walks each slice's contiguous run of connections: the sum over a run of one
// row stays in a register and goes to the row's orbitals (and to the sum over
// all connections) once per run; only the column's orbitals take one update
// per connection. Each slice owns a private copy of S (no two threads write one
// entry); the copies are added in slice order at the end (bit-reproducible).
enum { GC_AA = 0, GC_BB = 1, GC_B = 2, GC_AB = 3, GC_N = 4 };

constexpr int GDF_THREADS = 256;
constexpr int GDF_TPC = 4;                        // threads per connection
constexpr int GDF_K = GDF_THREADS / GDF_TPC;      // connections per tile

struct GridDfArgs {
    SysView S;
    int nh, M, M1, P1, ldp;
    int ldA;   // stride of the singles' table and the A rows (odd, >= nh)
    int ldF;   // stride of a connection's row [c, c u_0 .. c u_{nh-1}] (odd, >= nh + 1)
    int ldL;   // stride of an orbital-sum row (odd, >= nh + 1)
    int ns;    // singles, alpha then beta
    int nsl;   // scatter slices (each with its own orbital sums; 0 without G)
    int sw;    // threads per scatter slice: n_hidden + 1 rounded up to whole warps
    int gfree; // no G row: O, ln psi and E_loc only (the E_loc estimator's build)
    int lookup; // rows are the sector in enumeration order: read k_row_tables' tables
    const float2 *rt;   // [n_rows][nh] tanh z_j per row (lookup)
    const double *rt64; // [n_rows][nh] the same in FP64 (lookup: the O rows)
    const float2 *psim; // [n_rows] psi mantissa (lookup)
    const int *psie;    // [n_rows] psi exponent (lookup)
    int64_t cA;         // C(n, N_alpha): row index = beta rank * cA + alpha rank
    int R[GC_N], C[GC_N], toff[GC_N];  // toff: class's first row-target entry
    FastDiv fdC[GC_N], fd_nh, fd_nh1, fd_M1;
    int ntab;  // rows of the singles' table (max of the two spins)
    int narow; // A rows one tile of the alpha-beta class can touch
    int ntgt;  // orbital-target entries (rows then columns of every class)
    const double *theta;
    const float2 *tdf;
    const uint64_t *rows;
    int64_t n_rows;
    uint64_t amask, bmask;
    double e_core;
    double *lnpsi, *eloc, *O, *G;
    int *flags;
};

// Byte offsets of the dynamic shared memory (host and device use the same map).
struct GridSmem {
    size_t lists, tgt, tab, F, ix, Sg, arow, ones, V, Hs, Td, Gd, Red, T, Z, L1, Cs, Ve, Sgn, Pi,
        Sig, binom, rk, total;
};
__host__ __device__ inline GridSmem grid_smem(const GridDfArgs &A) {
    GridSmem g;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 15) & ~(size_t)15;
        return at;
    };
    const size_t nh = A.nh, ns = A.ns;
    g.lists = take(sizeof(RowLists));
    g.tgt = take((size_t)A.ntgt * sizeof(int2));
    g.tab = take((size_t)A.ntab * A.ldA * 8);
    // connection rows [c, c u_j]; the lookup form keeps c and the row of x' only
    g.F = take(A.gfree ? 0 : (size_t)GDF_K * (A.lookup ? 1 : A.ldF) * 8);
    g.ix = take(A.gfree || !A.lookup ? 0 : (size_t)GDF_K * 4);
    g.Sg = take((size_t)A.nsl * (A.M + 1) * A.ldL * 8);
    g.arow = take((size_t)2 * A.narow * A.ldA * 8);
    g.ones = take((size_t)A.ldA * 8);
    g.V = take(ns * 8);
    g.Hs = take(ns * 8);
    g.Td = take(nh * 8);
    g.Gd = take(nh * 8);
    g.Red = take((size_t)(GDF_THREADS / 32) * 8);
    g.T = take(nh * 8);
    g.Z = take(nh * 8);
    g.L1 = take(nh * 8);
    g.Cs = take((size_t)2 * A.M * 8);
    g.Ve = take(ns * 4);
    g.Sgn = take(ns * 4);
    g.Pi = take(ns * 4);
    g.Sig = take(nh * 4);
    g.binom = take(A.lookup ? 33 * 33 * 4 : 0);  // C(p, i), p, i <= 32
    g.rk = take(A.lookup ? ns * 4 : 0);          // colex rank of each single's string
    g.total = o;
    return g;
}

// A_s[j] = g_j B_s[j] of alpha single s, from the global exp(+-2W) tables
__device__ __forceinline__ df grid_arow(const GridDfArgs &A, const RowLists &L, int s, int j,
                                        const float2 *e2, const float2 *e2i, const float *sSig,
                                        const float2 *sGd) {
    const int q = fdiv(s, A.S.fd_nva);
    const int i = L.oa[q], a = L.va[s - q * A.S.nva];
    const bool pos = sSig[j] > 0.f;
    const df b = df_mul(ldg_df((pos ? e2 : e2i) + j * A.M + a), ldg_df((pos ? e2i : e2) + j * A.M + i));
    return df_mul(ld_df(sGd + j), b);
}

// B_t[j] of every single of one spin (spin 0: alpha singles, 1: beta)
__device__ __forceinline__ void grid_table(const GridDfArgs &A, const RowLists &L, int spin,
                                           const float2 *e2, const float2 *e2i, const float *sSig,
                                           float2 *sTab) {
    const int nsp = spin ? A.S.ns_b : A.S.ns_a, off = spin ? A.S.ns_a : 0;
    for (int e = threadIdx.x; e < nsp * A.nh; e += GDF_THREADS) {
        const int t = fdiv(e, A.fd_nh), j = e - t * A.nh;
        int i, a;
        single_of(A.S, L, off + t, i, a);
        const bool pos = sSig[j] > 0.f;
        st_df(sTab + t * A.ldA + j, df_mul(ldg_df((pos ? e2 : e2i) + j * A.M + a),
                                           ldg_df((pos ? e2i : e2) + j * A.M + i)));
    }
}

// Orbital targets of target entry e: the rows of each class, then its columns.
__device__ __forceinline__ int2 grid_target(const GridDfArgs &A, const RowLists &L, int e) {
    const SysView &S = A.S;
    int c = GC_N - 1;
    while (c > 0 && e < A.toff[c]) --c;
    int k = e - A.toff[c];
    const bool isrow = k < A.R[c];
    if (!isrow) k -= A.R[c];
    int lo, hi;
    switch (c) {
        case GC_AA:
        case GC_BB: {
            const bool al = c == GC_AA;
            unrank_pair(k, lo, hi);
            if (isrow) return al ? make_int2(L.oa[lo], L.oa[hi]) : make_int2(L.ob[lo], L.ob[hi]);
            return al ? make_int2(L.va[lo], L.va[hi]) : make_int2(L.vb[lo], L.vb[hi]);
        }
        case GC_B:
            return isrow ? make_int2(L.ob[k], -1) : make_int2(L.vb[k], -1);
        default:
            if (isrow) {
                const int q = fdiv(k, S.fd_nva);
                return make_int2(L.oa[q], L.va[k - q * S.nva]);
            }
            if (k == 0) return make_int2(-1, -1);
            {
                const int t = k - 1, q = fdiv(t, S.fd_nvb);
                return make_int2(L.ob[q], L.vb[t - q * S.nvb]);
            }
    }
}

// ------------------------------------------ per-determinant tables (sector rows)
// When the rows are the whole sector in enumeration order, every connected
// determinant x' is itself a row, so tanh(z_j(x')) and psi(x') need computing
// once per determinant, not once per connection pointing to it: k_row_tables
// writes them, and the build (lookup form) reads them by the rank of x'.
//   t[x][j]   tanh z_j(x) as double-float (the connection rows) and in FP64
//             (the row's own O row)
//   psi(x) = m[x] 2^e[x] with m in [1, 2) (double-float) and e an integer, from
//   ln psi(x) = a.x + sum_j |z_j| + ln prod_j (1 + e^{-2|z_j|}) (the ln 2 per
//   cosh cancels in every ratio), which is written to lnpsi as well.
// The transcendental work per (row, hidden unit) runs in double-float on the FP32
// pipes (FP64 issues at 1/64 of the FP32 rate here): e^{-2|z_j|} - 1 by
// df_expm1_neg and tanh as -(e - 1) / (2 + (e - 1)). FP64 keeps what ln psi needs
// to its last bits and costs few instructions: z_j (a sum of theta entries),
// sum_j |z_j|, the product of the 1 + e^{-2|z_j|} (one log per row instead of one
// per hidden unit), a.x and one exp2 per row.
struct RowTabArgs {
    int n, nh, M, M1;
    int R;          // rows per CTA pass
    int ldz;        // stride of a row's per-hidden-unit values in shared memory (odd)
    FastDiv fd_nh;
    const double *theta;
    const uint64_t *rows;
    int64_t n_rows;
    float2 *t;      // [n_rows][nh]
    double *t64;    // [n_rows][nh]
    float2 *psim;   // [n_rows]
    int *psie;      // [n_rows]
    double *lnpsi;  // [n_rows]
};

// e^y - 1 for y <= 0 in double-float (relative error ~1e-14; FP32 emulation over
// y in [-90, 0]). Cody and Waite's reduction y = k ln 2 + r, |r| <= ln 2 / 2, with
// ln 2 in three FP32 parts (the first with 16 significant bits, so k times it is
// exact); r' = r / 32; e^{r'} - 1 by its Taylor series to r'^7 / 7! (Horner; the
// three highest coefficients in FP32, whose terms are below 2^-30 relative);
// five doublings e^{2u} - 1 = (e^u - 1)(2 + e^u - 1); then
// e^y - 1 = 2^k (e^r - 1) + (2^k - 1), both parts exact in double-float. Below
// y = -87 the result is -1 to within 2^-125.
__device__ __forceinline__ df df_expm1_neg(df y) {
    if (y.h < -87.f) return df_make(-1.f, 0.f);
    // k = round(y / ln 2) by the FP32 magic number (no conversion instruction)
    const float kf = __fsub_rn(__fadd_rn(__fmul_rn(y.h, 1.44269504f), 12582912.0f), 12582912.0f);
    const int k = __float_as_int(__fadd_rn(kf, 12582912.0f)) - 0x4B400000;
    const float L1 = 0x1.62e4p-1f, L2 = 0x1.7f7d1cp-20f, L3 = 0x1.ef357ap-45f;
    df r = df_add(y, df_make(-kf * L1, 0.f));  // kf L1 is exact
    const float p2 = __fmul_rn(kf, L2);
    r = df_add(r, df_make(-p2, -__fmaf_rn(kf, L2, -p2)));  // exact k L2
    r = df_add(r, df_make(__fmul_rn(-kf, L3), 0.f));
    const df rs = df_make(r.h * 0x1p-5f, r.l * 0x1p-5f);
    float q = __fmaf_rn(rs.h, 0x1.a01a02p-13f, 0x1.6c16c2p-10f);  // 1/7!, 1/6!
    q = __fmaf_rn(rs.h, q, 0x1.111112p-7f);                        // 1/5!
    df P = df_add(df_make(0x1.555556p-5f, -0x1.555556p-30f), df_mul(rs, df_make(q, 0.f)));  // 1/4!
    P = df_add(df_make(0x1.555556p-3f, -0x1.555556p-28f), df_mul(rs, P));                   // 1/3!
    P = df_add(df_make(0.5f, 0.f), df_mul(rs, P));
    P = df_add(df_make(1.f, 0.f), df_mul(rs, P));
    df E = df_mul(rs, P);
#pragma unroll
    for (int i = 0; i < 5; ++i) E = df_mul(E, df_add(df_make(2.f, 0.f), E));
    // 2^k for k in [-126, 0] from its exponent field
    const float sc = __int_as_float((127 + k) << 23);
    const df B = k >= -24 ? df_make(__fsub_rn(sc, 1.f), 0.f) : df_make(-1.f, sc);
    return df_add(df_make(E.h * sc, E.l * sc), B);
}

// FP32 to FP64 by the exponent field (conversions issue at the FP64 rate here);
// zero and subnormal inputs take the conversion
__device__ __forceinline__ double f2d_bits(float x) {
    const unsigned u = __float_as_uint(x), ex = (u >> 23) & 0xffu;
    if (ex == 0u || ex == 0xffu) return (double)x;
    const unsigned hi = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ double df_to_double_bits(df a) { return f2d_bits(a.h) + f2d_bits(a.l); }

__global__ void __launch_bounds__(256) k_row_tables(RowTabArgs A) {
    extern __shared__ __align__(16) unsigned char smr[];
    const int n = A.n, nh = A.nh, M = A.M, M1 = A.M1, R = A.R, ldz = A.ldz;
    double *sW = reinterpret_cast<double *>(smr);  // [M + nh M1]: a, then b_j, W_j0 .. W_j(M-1)
    double *sAz = sW + M + (size_t)nh * M1;        // [R][ldz] |z_j|
    double *sFc = sAz + (size_t)R * ldz;           // [R][ldz] 1 + e^{-2|z_j|}
    const int tid = threadIdx.x;
    for (int e = tid; e < M + nh * M1; e += blockDim.x) sW[e] = A.theta[e];
    __syncthreads();
    for (int64_t g = blockIdx.x; g * R < A.n_rows; g += gridDim.x) {
        const int64_t r0 = g * R;
        const int nr = A.n_rows - r0 < (int64_t)R ? (int)(A.n_rows - r0) : R;
        // per (row, hidden unit)
        for (int e = tid; e < nr * nh; e += blockDim.x) {
            const int rr = fdiv(e, A.fd_nh), j = e - rr * nh;
            const int64_t row = r0 + rr;
            // z_j = b_j + sum of W_jp over the occupied spin orbitals, alpha then beta
            // in ascending order, in FP64 (ln psi sums the |z_j| of every hidden unit)
            const uint64_t x = A.rows[row];
            const double *wj = sW + M + (size_t)j * M1;
            double za = wj[0], zb = 0.0;
            for (int word = 0; word < 2; ++word) {
                unsigned w = word ? (unsigned)(x >> 32) : (unsigned)x;
                while (w) {
                    const int p = __ffs(w) - 1 + 32 * word;
                    w &= w - 1;
                    if (p < n) za += wj[1 + p];
                    else zb += wj[1 + p];
                }
            }
            const double z = za + zb;
            const df az = df_split_bits(fabs(z));
            const df em = df_expm1_neg(df_make(-2.f * az.h, -2.f * az.l));  // e^{-2|z|} - 1
            const df den = df_add(df_make(2.f, 0.f), em);                   // 1 + e^{-2|z|}
            df t = df_div(df_neg(em), den);
            if (z < 0.0) t = df_neg(t);
            A.t[row * nh + j] = make_float2(t.h, t.l);
            A.t64[row * nh + j] = df_to_double_bits(t);
            sAz[rr * ldz + j] = fabs(z);
            sFc[rr * ldz + j] = df_to_double_bits(den);
        }
        __syncthreads();
        // per row (a thread each): a.x + sum_j |z_j| + ln prod_j (1 + e^{-2|z_j|})
        // (the product stays below 2^255: no rescaling in FP64), then psi = m 2^e
        for (int q = tid; q < nr; q += blockDim.x) {
            const int64_t rw = r0 + q;
            const uint64_t x = A.rows[rw];
            double ax = 0.0;
            for (int word = 0; word < 2; ++word) {
                unsigned w = word ? (unsigned)(x >> 32) : (unsigned)x;
                while (w) {
                    const int p = __ffs(w) - 1 + 32 * word;
                    w &= w - 1;
                    ax += sW[p];
                }
            }
            double sz = 0.0, pr = 1.0;
            for (int jj = 0; jj < nh; ++jj) {
                sz += sAz[q * ldz + jj];
                pr *= sFc[q * ldz + jj];
            }
            const double lp = ax + sz + log(pr);
            A.lnpsi[rw] = lp;
            // psi = 2^(lp / ln 2) = 2^k 2^f, f in [0, 1)
            const double qd = lp * 1.4426950408889634;  // 1 / ln 2
            const double kd = floor(qd);
            const df md = df_from_double(exp2(qd - kd));
            A.psim[rw] = make_float2(md.h, md.l);
            A.psie[rw] = (int)kd;
        }
        __syncthreads();
    }
}

// Colex rank of the k-subset held in the low bits of `bits` (ascending mask
// order: sum over the set positions p_1 < ... < p_k of C(p_i, i)), with C from
// the CTA's table binom[p * 33 + i].
__device__ __forceinline__ uint32_t colex_rank(uint32_t bits, const uint32_t *binom) {
    uint32_t r = 0;
    int i = 1;
    while (bits) {
        const int p = __ffs(bits) - 1;
        bits &= bits - 1;
        r += binom[p * 33 + i];
        ++i;
    }
    return r;
}

// GF: the G-free build of the E_loc estimator (no u_j, no scatter, no G row).
// LK: the lookup form (rows = the sector in enumeration order): a connection's
// psi ratio is m[x'] / m[x] 2^(e[x'] - e[x]) and its row tanh z_j(x') is read
// from k_row_tables' tables at the rank of x', so there is no per-connection
// Z_j, 1 + Z_j, reciprocal or running product, and the sums are of c tanh
// directly (no conversion from sums of c u).
template <bool GF, bool LK>
__global__ void __launch_bounds__(GDF_THREADS) k_build_rows_dg(GridDfArgs A) {
    extern __shared__ __align__(16) unsigned char smb[];
    const int nh = A.nh, M = A.M, M1 = A.M1, NS = A.ns, nh1 = nh + 1;
    const int tid = threadIdx.x, lane = tid & 31;
    const GridSmem lay = grid_smem(A);
    RowLists *sL = reinterpret_cast<RowLists *>(smb + lay.lists);
    int2 *sTgt = reinterpret_cast<int2 *>(smb + lay.tgt);        // [ntgt] orbital targets
    float2 *sTab = reinterpret_cast<float2 *>(smb + lay.tab);    // [ntab][ldA]  B_t[j]
    float2 *sF = reinterpret_cast<float2 *>(smb + lay.F);        // [K][ldF]  c, c u_j (lookup: [K] c)
    int *sIx = reinterpret_cast<int *>(smb + lay.ix);            // lookup: [K] the row of x'
    float2 *sSg = reinterpret_cast<float2 *>(smb + lay.Sg);      // [nsl][M + 1][ldL]
    float2 *sArow = reinterpret_cast<float2 *>(smb + lay.arow);  // [2][narow][ldA]
    float2 *sOne = reinterpret_cast<float2 *>(smb + lay.ones);   // [ldA] ones
    float2 *sV = reinterpret_cast<float2 *>(smb + lay.V);        // [NS]
    float2 *sHs = reinterpret_cast<float2 *>(smb + lay.Hs);      // [NS]
    float2 *sTd = reinterpret_cast<float2 *>(smb + lay.Td);      // [nh] t as df
    float2 *sGd = reinterpret_cast<float2 *>(smb + lay.Gd);      // [nh] g as df
    float2 *sRed = reinterpret_cast<float2 *>(smb + lay.Red);
    double *sT = reinterpret_cast<double *>(smb + lay.T);
    double *sZ = reinterpret_cast<double *>(smb + lay.Z);
    double *sL1 = reinterpret_cast<double *>(smb + lay.L1);
    double *sCs = reinterpret_cast<double *>(smb + lay.Cs);
    int *sVe = reinterpret_cast<int *>(smb + lay.Ve);
    float *sSgn = reinterpret_cast<float *>(smb + lay.Sgn);
    int *sPi = reinterpret_cast<int *>(smb + lay.Pi);
    float *sSig = reinterpret_cast<float *>(smb + lay.Sig);
    uint32_t *sBinom = reinterpret_cast<uint32_t *>(smb + lay.binom);  // lookup form
    int *sRk = reinterpret_cast<int *>(smb + lay.rk);                   // lookup form
    __shared__ double sDiag, sLn, sGinv;
    __shared__ int sGe;
    __shared__ int sBad;
    __shared__ int sRA, sRB, sE;  // lookup form: the row's ranks and psi exponent
    __shared__ float2 sIM;        // lookup form: 1 / psi mantissa of the row
    if (LK) {
        for (int e = threadIdx.x; e < 33 * 33; e += GDF_THREADS) {
            const int pp = e / 33, ii = e % 33;
            sBinom[e] = (uint32_t)binom_dev(pp, ii);
        }
        __syncthreads();
    }

    const float2 *e2 = A.tdf;               // exp(2W) [nh][M]
    const float2 *e2i = e2 + nh * M;        // exp(-2W) [nh][M]
    const float2 *hd = e2 + 2 * nh * M;     // h [n][n]
    const float2 *gd = hd + A.S.n * A.S.n;  // (pq|rs)
    const SysView &S = A.S;
    const int ldL = A.ldL, ldF = A.ldF, ldA = A.ldA;

    // connection kk of a tile is handled by the GDF_TPC lanes kk % CPW, kk % CPW
    // + CPW, ... of warp kk / CPW; the lookup form has no hidden-unit loop to
    // share, so thread kk alone decodes connection kk (warps 0 and 1 the whole
    // tile: a quarter of the decoding's warp instructions)
    constexpr int CPW = 32 / GDF_TPC;
    const int kk = LK ? tid : (tid >> 5) * CPW + (lane % CPW), sub = LK ? 0 : lane / CPW;
    // scatter thread: slice sl, hidden row sr
    const int sl = tid / A.sw, sr = tid - sl * A.sw;
    const bool scatter_thread = sl < A.nsl && sr < nh1;
    float2 *mySg = sSg + (size_t)sl * (M + 1) * ldL + sr;
    auto next_class = [&](int c) -> int {
        for (++c; c < GC_N; ++c)
            if (A.R[c] > 0 && A.C[c] > 0) return c;
        return (int)GC_N;
    };
    auto spin_of = [](int c) { return c == GC_AA ? 0 : 1; };

    for (int64_t row = blockIdx.x; row < A.n_rows; row += gridDim.x) {
        const uint64_t x = A.rows[row];
        if (tid == 0) {
            const int bad = (__popcll(x & A.amask) != S.na) || (__popcll(x & A.bmask) != S.nb) ||
                            (x & ~(A.amask | A.bmask)) != 0;
            sBad = bad;
            if (bad) atomicOr(A.flags, FLAG_ROW_OUTSIDE_SECTOR);
            make_lists(S, x, *sL);
        }
        __syncthreads();
        if (sBad) {
            __syncthreads();
            continue;
        }
        const RowLists &L = *sL;
        // A rows of the first tile of the alpha-beta class (buffer 0)
        auto first_arows = [&]() {
            const int nr = fdiv(min(GDF_K, A.R[GC_AB] * A.C[GC_AB]) - 1, A.fdC[GC_AB]) + 1;
            for (int e = tid; e < nr * nh; e += GDF_THREADS) {
                const int rr = fdiv(e, A.fd_nh), j = e - rr * nh;
                st_df(sArow + rr * ldA + j, grid_arow(A, L, rr, j, e2, e2i, sSig, sGd));
            }
        };
        // per hidden unit (FP64): z_j, g = e^{-2|z|} = 1 + expm1(-2|z|) (no
        // cancellation for small |z|), tanh z = sign(z) (-em) / (2 + em), ln(1 + g)
        // (the lookup form reads the row's own tanh z_j from k_row_tables)
        for (int j = tid; !LK && j < nh; j += GDF_THREADS) {
            const double *wj = A.theta + (size_t)(j + 1) * M1;
            double za = wj[-1], zb = 0.0;
            for (int t = 0; t < S.na; ++t) za += wj[L.oa[t]];
            for (int t = 0; t < S.nb; ++t) zb += wj[L.ob[t]];
            const double z = za + zb;
            sZ[j] = z;
            const double em = expm1(-2.0 * fabs(z));
            const double g = 1.0 + em;
            const double t = copysign(-em / (2.0 + em), z);
            sT[j] = t;
            sL1[j] = log1p(g);
            const df td = df_from_double(t);
            sTd[j] = make_float2(td.h, td.l);
            sSig[j] = z < 0.0 ? 1.f : -1.f;
            const df gdv = df_from_double(g);
            sGd[j] = make_float2(gdv.h, gdv.l);
        }
        {
            // <x'|H|x> of every single (without sign), one warp per single; warps
            // that hold no hidden unit above do this
            const int w0 = (nh + 31) >> 5, warp = tid >> 5;
            for (int sgl = warp - w0; warp >= w0 && sgl < NS; sgl += GDF_THREADS / 32 - w0) {
                int i, a;
                single_of(S, L, sgl, i, a);
                const int n = S.n, sp = i >= n;
                const int ip = i - sp * n, ap = a - sp * n;
                df v = df_make(0.f, 0.f);
                for (int t = lane; t < S.na + S.nb; t += 32) {
                    const bool ta = t < S.na;
                    const int kp = ta ? L.oa[t] : L.ob[t - S.na] - n;
                    const float2 *gk = gd + ((size_t)ap * n + ip) * n * n;
                    v = df_add(v, ldg_df(gk + (size_t)kp * n + kp));
                    if ((ta ? 0 : 1) == sp)
                        v = df_sub(v, ldg_df(gd + (((size_t)ap * n + kp) * n + kp) * n + ip));
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    v = df_add(v, df_make(__shfl_xor_sync(0xffffffffu, v.h, off),
                                          __shfl_xor_sync(0xffffffffu, v.l, off)));
                if (lane == 0) st_df(sHs + sgl, df_add(ldg_df(hd + ap * n + ip), v));
            }
        }
        for (int e = tid; e < A.nsl * (M + 1) * ldL; e += GDF_THREADS) sSg[e] = make_float2(0.f, 0.f);
        for (int e = tid; e < ldA; e += GDF_THREADS) sOne[e] = make_float2(1.f, 0.f);
        for (int e = tid; e < A.ntgt; e += GDF_THREADS) sTgt[e] = grid_target(A, L, e);
        __syncthreads();
        const uint32_t xa = (uint32_t)(x & A.amask), xb = (uint32_t)(x >> S.n);
        if (LK && tid == 0) {
            // lookup form: the row's colex ranks and 1 / its psi mantissa
            sRA = (int)colex_rank(xa, sBinom);
            sRB = (int)colex_rank(xb, sBinom);
            const df im = df_rcp(ldg_df(A.psim + row));
            sIM = make_float2(im.h, im.l);
            sE = A.psie[row];
        } else if (!LK && tid < 32) {
            // ln psi = a.x + sum_j (|z_j| + ln(1 + g_j)) (the ln 2 of each cosh cancels
            // in every ratio and is dropped); prod_j (1 + g_j) = exp(sum_j l1_j)
            double lp = 0.0, lg = 0.0;
            for (int j = tid; j < nh; j += 32) {
                lp += fabs(sZ[j]) + sL1[j];
                lg += sL1[j];
            }
            for (int p = tid; p < M; p += 32)
                if (occ_bit(x, p)) lp += A.theta[p];
            lp = warp_sum(lp);
            lg = warp_sum(lg);
            if (tid == 0) {
                // 1 / prod_j (1 + g_j) = sGinv 2^sGe with sGinv in [0.5, 1)
                sLn = lp;
                int ge = 0;
                sGinv = frexp(exp(-lg), &ge);
                sGe = ge;
            }
        } else if (tid >= 32 && tid < 64) {
            const double d = diag_value_warp(S, L);
            if (tid == 32) sDiag = d + A.e_core;
        } else if (!LK && tid >= 64 && tid - 64 < 2 * M) {
            // sum_j sigma_j W_jp in two interleaved halves (combined where used)
            const int p = (tid - 64) % M, half = (tid - 64) / M;
            double c0 = 0.0, c1 = 0.0;
            int j = half;
            for (; j + 2 < nh; j += 4) {
                const double w0 = A.theta[(size_t)(j + 1) * M1 + p];
                const double w1 = A.theta[(size_t)(j + 3) * M1 + p];
                c0 += sZ[j] < 0.0 ? w0 : -w0;
                c1 += sZ[j + 2] < 0.0 ? w1 : -w1;
            }
            if (j < nh) {
                const double w0 = A.theta[(size_t)(j + 1) * M1 + p];
                c0 += sZ[j] < 0.0 ? w0 : -w0;
            }
            sCs[half * M + p] = c0 + c1;
        }
        __syncthreads();
        // per single: V_s = exp(a_a - a_i - sum_j sigma_j d_j) (FP64 exp), its
        // Jordan-Wigner sign and the index part of an alpha-beta double's integral;
        // the table and A rows of the first class
        for (int s = tid; s < NS; s += GDF_THREADS) {
            int i, a;
            single_of(S, L, s, i, a);
            if (LK) {
                // the colex rank of the single's string (alpha or beta) after i -> a
                const int sh = s < S.ns_a ? 0 : S.n;
                const uint32_t str = (s < S.ns_a ? xa : xb) ^ (1u << (i - sh)) ^ (1u << (a - sh));
                sRk[s] = (int)colex_rank(str, sBinom);
            } else {
                const double csa = sCs[a] + sCs[M + a], csi = sCs[i] + sCs[M + i];
                const double ex = (A.theta[a] - A.theta[i]) - (csa - csi);
                int ve = 0;  // V_s = mantissa * 2^ve, mantissa in [0.5, 1)
                const df v = df_from_double(frexp(exp(ex), &ve));
                sV[s] = make_float2(v.h, v.l);
                sVe[s] = ve;
            }
            const int par = parity_below(x, i) + parity_below(x ^ (1ull << i), a);
            sSgn[s] = (par & 1) ? -1.f : 1.f;
            const int n = S.n;
            sPi[s] = s < S.ns_a ? (a * n + i) * n * n : (a - n) * n + (i - n);
        }
        int cls = next_class(-1);
        if (!LK && cls < GC_N) {
            grid_table(A, L, spin_of(cls), e2, e2i, sSig, sTab);
            if (cls == GC_AB) first_arows();
        }
        __syncthreads();

        df el_part = df_make(0.f, 0.f);
        const df ginv = df_from_double(sGinv);
        for (; cls < GC_N; cls = next_class(cls)) {
            const int C = A.C[cls];
            const FastDiv fdC = A.fdC[cls];
            const int ne = A.R[cls] * C;
            const bool fuse = cls != GC_AB;  // Z carries g_j from sGd
            const int2 *rowT = sTgt + A.toff[cls], *colT = rowT + A.R[cls];
            int tile = 0;
            for (int e0 = 0; e0 < ne; e0 += GDF_K, ++tile) {
                const int e1 = min(ne, e0 + GDF_K);
                const int rf = fdiv(e0, fdC);
                // ---- per connection: u_j = 1 / (1 + Z_j), prod_j (1 + Z_j) and c
                const float2 *arow = sArow + (tile & 1) * A.narow * ldA;
                if (!LK && cls == GC_AB && e1 < ne) {  // A rows of the next tile
                    const int n1 = min(ne, e1 + GDF_K);
                    const int nrf = fdiv(e1, fdC), nrl = fdiv(n1 - 1, fdC);
                    float2 *dst = sArow + ((tile + 1) & 1) * A.narow * ldA;
                    for (int e = tid; e < (nrl - nrf + 1) * nh; e += GDF_THREADS) {
                        const int rr = fdiv(e, A.fd_nh), j = e - rr * nh;
                        st_df(dst + rr * ldA + j, grid_arow(A, L, nrf + rr, j, e2, e2i, sSig, sGd));
                    }
                }
                const int e = e0 + kk;
                const bool active = e < e1;
                int rho = 0, gam = 0;
                const float2 *f1 = sOne, *f2 = sOne;
                int s1 = 0, s2 = -1;  // singles whose V_s the coefficient takes
                int64_t idx = 0;      // lookup form: the row index of x'
                if (active) {
                    rho = fdiv(e, fdC);
                    gam = e - rho * C;
                    if (LK) {
                        if (cls == GC_AB) {
                            s1 = rho;
                            if (gam > 0) s2 = S.ns_a + gam - 1;
                            idx = (int64_t)(gam == 0 ? sRB : sRk[s2]) * A.cA + sRk[rho];
                        } else if (cls == GC_B) {
                            s1 = S.ns_a + e;
                            idx = (int64_t)sRk[s1] * A.cA + sRA;
                        } else {
                            // a same-spin double moves two occupied and two empty
                            // orbitals of one string
                            const bool al = cls == GC_AA;
                            const int sh = al ? 0 : S.n;
                            const int2 o = rowT[rho], v = colT[gam];
                            const uint32_t str = (al ? xa : xb) ^ (1u << (o.x - sh)) ^
                                                 (1u << (o.y - sh)) ^ (1u << (v.x - sh)) ^
                                                 (1u << (v.y - sh));
                            const int r2 = (int)colex_rank(str, sBinom);
                            idx = al ? (int64_t)sRB * A.cA + r2 : (int64_t)r2 * A.cA + sRA;
                        }
                    } else if (cls == GC_AA || cls == GC_BB) {
                        const int nv = cls == GC_AA ? S.nva : S.nvb;
                        const int off = cls == GC_AA ? 0 : S.ns_a;
                        int lo, hi, vlo, vhi;
                        unrank_pair(rho, lo, hi);
                        unrank_pair(gam, vlo, vhi);
                        const int t1 = lo * nv + vlo, t2 = hi * nv + vhi;
                        f1 = sTab + t1 * ldA;
                        f2 = sTab + t2 * ldA;
                        s1 = off + t1;
                        s2 = off + t2;
                    } else if (cls == GC_B) {
                        f1 = sTab + e * ldA;
                        s1 = S.ns_a + e;
                    } else {
                        f1 = arow + (rho - rf) * ldA;
                        s1 = rho;
                        if (gam > 0) {
                            f2 = sTab + (gam - 1) * ldA;
                            s2 = S.ns_a + gam - 1;
                        }
                    }
                }
                // the coefficient's <x'|H|x> and sign (lane 0 of the connection);
                // a double's integrals are fetched before the hidden-unit loop so
                // that their latency hides behind it
                df hv = df_make(0.f, 0.f);
                float sg = 1.f;
                if (active && sub == 0) {
                    if (cls == GC_AA || cls == GC_BB) {
                        const int2 o = rowT[rho], v = colT[gam];
                        Exc ex;
                        ex.i = o.x;
                        ex.j = o.y;
                        ex.a = v.x;
                        ex.b = v.y;
                        int sgi = 1;
                        (void)apply_exc(x, ex, sgi);
                        sg = (float)sgi;
                        hv = exc_value_df(S, L, ex, hd, gd);
                    } else if (s2 < 0) {
                        hv = ld_df(sHs + s1);
                        sg = sSgn[s1];
                    } else {
                        hv = ldg_df(gd + sPi[s1] + sPi[s2]);
                        sg = sSgn[s1] * sSgn[s2];
                    }
                }
                if constexpr (LK) {
                    // c = sign <x'|H|x> psi(x') / psi(x); the scatter forms c tanh z_j(x')
                    // from the row of x' in the table
                    if (active && sub == 0) {
                        if (sg < 0.f) hv = df_neg(hv);
                        const df ratio = df_mul(ldg_df(A.psim + idx), df_make(sIM.x, sIM.y));
                        const df c = df_ldexp(df_mul(hv, ratio), __ldg(A.psie + idx) - sE);
                        if (!GF) {
                            st_df(sF + kk, c);
                            sIx[kk] = (int)idx;
                        }
                        df_acc(el_part, c);
                    }
                } else {
                    float2 *Frow = sF + kk * ldF + 1;
                    df rp = df_make(1.f, 0.f);
                    int re = 0;
                    if (active) {
                        // Z_j = (g_j) f1[j] f2[j]; u = 1 / (1 + Z); the running product of
                        // (1 + Z_j) stays >= 1 and is rescaled past 2^60
                        if (fuse) {
#pragma unroll 2
                            for (int j = sub; j < nh; j += GDF_TPC) {
                                df z = df_mul_lazy(ld_df(sGd + j), ld_df(f1 + j));
                                z = df_mul_lazy(z, ld_df(f2 + j));
                                const df zp = df_add1_lazy(z);
                                if (!GF) st_df(Frow + j, df_rcp_ge1(zp));
                                rp = df_mul_lazy(rp, zp);
                                if (rp.h > 0x1p60f) df_renorm(rp, re);
                            }
                        } else {
#pragma unroll 2
                            for (int j = sub; j < nh; j += GDF_TPC) {
                                const df z = df_mul_lazy(ld_df(f1 + j), ld_df(f2 + j));
                                const df zp = df_add1_lazy(z);
                                if (!GF) st_df(Frow + j, df_rcp_ge1(zp));
                                rp = df_mul_lazy(rp, zp);
                                if (rp.h > 0x1p60f) df_renorm(rp, re);
                            }
                        }
                        rp = df_fts(rp.h, rp.l);
                    }
                    // combine the partial products of the GDF_TPC lanes of a connection
                    // (all lanes take part; inactive ones carry 1 * 2^0)
#pragma unroll
                    for (int off = CPW; off < 32; off <<= 1) {
                        const df o = df_make(__shfl_xor_sync(0xffffffffu, rp.h, off),
                                             __shfl_xor_sync(0xffffffffu, rp.l, off));
                        const int oe = __shfl_xor_sync(0xffffffffu, re, off);
                        rp = df_mul(rp, o);
                        re += oe;
                        df_renorm(rp, re);
                    }
                    df c = df_make(0.f, 0.f);
                    if (active && sub == 0) {
                        if (sg < 0.f) hv = df_neg(hv);
                        df f = df_mul(hv, ld_df(sV + s1));
                        int fe = re + sGe + sVe[s1];
                        if (s2 >= 0) {
                            f = df_mul(f, ld_df(sV + s2));
                            fe += sVe[s2];
                        }
                        c = df_ldexp(df_mul(df_mul(f, ginv), rp), fe);
                        if (!GF) st_df(Frow - 1, c);
                        df_acc(el_part, c);
                    }
                    if (!GF) {
                        // the row of the connection becomes c u_j here, where every thread works
                        c.h = __shfl_sync(0xffffffffu, c.h, lane % CPW);
                        c.l = __shfl_sync(0xffffffffu, c.l, lane % CPW);
                        if (active)
                            for (int j = sub; j < nh; j += GDF_TPC) st_df(Frow + j, df_mul_lazy(c, ld_df(Frow + j)));
                    }
                }
                __syncthreads();
                // ---- scatter: slice sl takes a contiguous run of the tile; the sum over
                // a run of one row goes to the row's orbitals and the all-connections
                // sum, each connection to its column's orbitals
                if (!GF && scatter_thread) {
                    const int len = e1 - e0, per = (len + A.nsl - 1) / A.nsl;
                    const int k0 = sl * per, k1 = min(len, k0 + per);
                    if (k0 < k1) {
                        int r0 = fdiv(e0 + k0, fdC), g = e0 + k0 - r0 * C;
                        df racc = df_make(0.f, 0.f);
                        auto flush = [&](int rr) {
                            const int2 t = rowT[rr];
                            float2 *d = mySg + t.x * ldL;
                            st_df(d, df_add(ld_df(d), racc));
                            if (t.y >= 0) {
                                d = mySg + t.y * ldL;
                                st_df(d, df_add(ld_df(d), racc));
                            }
                            d = mySg + M * ldL;
                            st_df(d, df_add(ld_df(d), racc));
                        };
                        // lookup form: the element of connection k is c_k tanh z(x'_k) at
                        // hidden row sr - 1 (c_k itself at sr = 0); the table rows of the
                        // next two connections are in flight while one is added
                        const float2 *tz = A.rt + (sr > 0 ? sr - 1 : 0);
                        auto trow = [&](int k) {
                            return k < k1 ? ldg_df(tz + (int64_t)sIx[k] * nh) : df_make(1.f, 0.f);
                        };
                        df t0 = df_make(1.f, 0.f), t1 = t0, t2 = t0;
                        if (LK) {
                            t1 = trow(k0);
                            t2 = trow(k0 + 1);
                        }
                        const float2 *fp = sF + k0 * (LK ? 1 : ldF) + (LK ? 0 : sr);
                        for (int k2 = k0; k2 < k1; ++k2, fp += (LK ? 1 : ldF)) {
                            df f = ld_df(fp);
                            if (LK) {
                                t0 = t1;
                                t1 = t2;
                                t2 = trow(k2 + 2);
                                if (sr > 0) f = df_mul_lazy(f, t0);
                            }
                            df_acc(racc, f);
                            const int2 t = colT[g];
                            if (t.x >= 0) {
                                float2 *d = mySg + t.x * ldL;
                                df v = ld_df(d);
                                df_acc(v, f);
                                st_df(d, v);
                            }
                            if (t.y >= 0) {
                                float2 *d = mySg + t.y * ldL;
                                df v = ld_df(d);
                                df_acc(v, f);
                                st_df(d, v);
                            }
                            if (++g == C && k2 + 1 < k1) {
                                racc = df_norm(racc);
                                flush(r0);
                                racc = df_make(0.f, 0.f);
                                g = 0;
                                ++r0;
                            }
                        }
                        racc = df_norm(racc);
                        flush(r0);
                    }
                }
                // the table and A rows of the next class, after its last tile's
                // hidden-unit loop (the scatter reads neither; the lookup form has
                // neither)
                if (!LK && e1 == ne) {
                    const int nc = next_class(cls);
                    if (nc < GC_N) {
                        if (spin_of(nc) != spin_of(cls)) grid_table(A, L, spin_of(nc), e2, e2i, sSig, sTab);
                        if (nc == GC_AB) first_arows();
                    }
                }
                __syncthreads();
            }
        }
        // E_loc: per-warp df sums in lane order, then warps in order
        {
            df v = df_norm(el_part);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const df o = df_make(__shfl_xor_sync(0xffffffffu, v.h, off),
                                     __shfl_xor_sync(0xffffffffu, v.l, off));
                v = df_add(v, o);
            }
            if (lane == 0) st_df(sRed + (tid >> 5), v);
        }
        __syncthreads();
        if (tid == 0) {
            df el = df_from_double(sDiag);
            for (int w = 0; w < GDF_THREADS / 32; ++w) el = df_add(el, ld_df(sRed + w));
            A.eloc[row] = df_to_double(el);
            if (!LK) A.lnpsi[row] = sLn;  // the lookup form's ln psi is k_row_tables'
        }
        // O row and G row; sums of c u_j become sums of c tanh(z_j + d_j):
        // sum c tanh = sigma_j (sum c - 2 sum c u_j)
        double *Orow = A.O + row * (int64_t)A.ldp;
        double *Grow = GF ? nullptr : A.G + row * (int64_t)A.ldp;
        const df hdg = df_from_double(sDiag);
        auto to_tanh = [&](df s0, df su, int r) {
            const df t = df_sub(s0, df_make(2.f * su.h, 2.f * su.l));
            return sSig[r - 1] < 0.f ? df_neg(t) : t;
        };
        // orbital sum p at hidden row r over the slices, in slice order
        auto osum = [&](int p, int r) {
            df a = df_make(0.f, 0.f);
            for (int q = 0; q < A.nsl; ++q) a = df_add(a, df_norm(ld_df(sSg + ((size_t)q * (M + 1) + p) * ldL + r)));
            return a;
        };
        // the row's own tanh z_j: the setup's, or k_row_tables' (lookup form)
        const float2 *ownt = LK ? A.rt + row * nh : sTd;
        for (int e = tid; e < A.ldp; e += GDF_THREADS) {
            double ov = 0.0, gv = 0.0;
            if (e < A.P1) {
                const int r = fdiv(e, A.fd_M1), c = e - r * M1;
                const bool xc = (c == 0) || occ_bit(x, c - 1);
                const double tr = r == 0 ? 1.0 : (LK ? __ldg(A.rt64 + row * nh + r - 1) : sT[r - 1]);
                ov = xc ? tr : 0.0;
            }
            Orow[e] = ov;
            if (GF) continue;
            if (e < A.P1) {
                const int r = fdiv(e, A.fd_M1), c = e - r * M1;
                df a = osum(M, r);
                if (!LK && r > 0) a = to_tanh(osum(M, 0), a, r);
                df at = (r == 0) ? hdg : df_mul(hdg, LK ? ldg_df(ownt + r - 1) : ld_df(sTd + r - 1));
                at = df_add(at, a);
                if (c == 0) {
                    gv = df_to_double(at);
                } else {
                    df sv = osum(c - 1, r);
                    if (!LK && r > 0) sv = to_tanh(osum(c - 1, 0), sv, r);
                    gv = df_to_double(occ_bit(x, c - 1) ? df_sub(at, sv) : sv);
                }
            }
            Grow[e] = gv;
        }
        __syncthreads();
    }
}

// ------------------------------------------------ K7: weights and statistics
// Max of ln psi (for the |psi|^2 weights' shift): per-CTA partial maxima.
__global__ void k_lnpsi_max_partial(const double *lnpsi, int64_t n, double *part) {
    double m = -INFINITY;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, lnpsi[i]);
    m = warp_max(m);
    __shared__ double s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s[w]);
        m = fmax(m, s[0]);
        part[blockIdx.x] = m;
    }
}

// Unnormalised weights, one per row: w = exp(2 (ln psi - max)) (|psi|^2 up to a
// constant) or the given weight.
__global__ void k_weights(const double *lnpsi, const double *given, double *wt, int64_t n,
                          const double *max_part, int n_max_part) {
    __shared__ double sMax;
    if (threadIdx.x == 0) {
        double m = -INFINITY;
        if (!given)
            for (int b = 0; b < n_max_part; ++b) m = fmax(m, max_part[b]);
        sMax = m;
    }
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        wt[r] = given ? given[r] : exp(2.0 * (lnpsi[r] - sMax));
}

// Unnormalised weights with a given shift (row shards: the maximum of ln psi
// over every shard): w = exp(2 (ln psi - lnpsi_max)), or the given weight.
__global__ void k_weights_shift(const double *lnpsi, const double *given, double *wt, int64_t n,
                                double lnpsi_max) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        wt[r] = given ? given[r] : exp(2.0 * (lnpsi[r] - lnpsi_max));
}

// Per-CTA partial sums over a contiguous row chunk: sum w, sum w E_loc,
// sum w O[:, c].
__global__ void k_stats_partial(const double *O, const double *eloc, const double *wt, int64_t n,
                                int ldp, double *part) {
    // column pairs (ldp is a multiple of 8, rows start 64-byte aligned); four
    // independent row chains per thread keep enough loads in flight to stream O
    const int64_t r0 = n * blockIdx.x / gridDim.x, r1 = n * (blockIdx.x + 1) / gridDim.x;
    double *out = part + (int64_t)blockIdx.x * (ldp + 2);
    for (int c = 2 * threadIdx.x; c < ldp; c += 2 * blockDim.x) {
        double2 a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = make_double2(0.0, 0.0);
        int64_t r = r0;
        for (; r + 3 < r1; r += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double2 o = *reinterpret_cast<const double2 *>(O + (r + u) * ldp + c);
                const double w = wt[r + u];
                a[u].x = fma(w, o.x, a[u].x);
                a[u].y = fma(w, o.y, a[u].y);
            }
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            if (r + u < r1) {
                const double2 o = *reinterpret_cast<const double2 *>(O + (r + u) * ldp + c);
                a[u].x = fma(wt[r + u], o.x, a[u].x);
                a[u].y = fma(wt[r + u], o.y, a[u].y);
            }
        }
        out[c] = (a[0].x + a[1].x) + (a[2].x + a[3].x);
        out[c + 1] = (a[0].y + a[1].y) + (a[2].y + a[3].y);
    }
    if (threadIdx.x == 0) {
        double sw = 0.0, se = 0.0;
        for (int64_t r = r0; r < r1; ++r) {
            sw += wt[r];
            se = fma(wt[r], eloc[r], se);
        }
        out[ldp] = sw;
        out[ldp + 1] = se;
    }
}

// stats[0] = sum w, stats[1] = E, stats[8 + c] = <O_c>. CTA b covers columns
// [32 b, 32 b + 32): warp q sums the partials q, q + 8, ... of its lane's
// column, then the 8 warp sums are added in warp order. Every CTA forms sum w
// itself (the same fixed order), so no second pass is needed.
// raw = 1: the sums themselves (stats[1] = sum w E_loc, stats[8 + c] = sum w O_c).
__global__ void __launch_bounds__(256) k_stats_final(const double *part, int nparts, int ldp,
                                                      double *stats, int raw) {
    __shared__ double red[8][33];
    __shared__ double s_sw;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t ld2 = ldp + 2;
    {
        double a = 0.0, b = 0.0;
        for (int q = threadIdx.x; q < nparts; q += 256) {
            a += part[q * ld2 + ldp];
            b += part[q * ld2 + ldp + 1];
        }
        a = warp_sum(a);
        b = warp_sum(b);
        if (lane == 0) {
            red[warp][0] = a;
            red[warp][1] = b;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double ta = 0.0, tb = 0.0;
            for (int w = 0; w < 8; ++w) {
                ta += red[w][0];
                tb += red[w][1];
            }
            s_sw = ta;
            if (blockIdx.x == 0) {
                stats[0] = ta;
                stats[1] = raw ? tb : tb / ta;
            }
        }
        __syncthreads();
    }
    const int c = blockIdx.x * 32 + lane;
    double a0 = 0.0, a1 = 0.0;
    if (c < ldp) {
        int q = warp;
        for (; q + 8 < nparts; q += 16) {
            a0 += part[q * ld2 + c];
            a1 += part[(q + 8) * ld2 + c];
        }
        if (q < nparts) a0 += part[q * ld2 + c];
    }
    red[warp][lane] = a0 + a1;
    __syncthreads();
    if (warp == 0 && c < ldp) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w][lane];
        stats[8 + c] = raw ? t : t / s_sw;
    }
}

template <typename TL>
__device__ __forceinline__ TL to_low(double x) {
    return (TL)x;
}
template <>
__device__ __forceinline__ __nv_bfloat16 to_low<__nv_bfloat16>(double x) {
    return __double2bfloat16(x);
}

// Centre in place (FP64) and write the optional low-precision copies:
//   O_c(x,0) = 1, G'_c(x,0) = E_loc - E,
//   O_c(x,k) = O - <O_k>, G'_c(x,k) = G - <O_k> E_loc - E O_c(x,k),
// and normalise the weights. One warp per row, lanes over column pairs (16-byte
// loads and stores; ldp is a multiple of 8 and rows start 64-byte aligned).
template <typename TL>
__device__ __forceinline__ void store_low2(TL *p, double a, double b) {
    p[0] = to_low<TL>(a);
    p[1] = to_low<TL>(b);
}
template <>
__device__ __forceinline__ void store_low2<float>(float *p, double a, double b) {
    *reinterpret_cast<float2 *>(p) = make_float2((float)a, (float)b);
}
template <>
__device__ __forceinline__ void store_low2<__nv_bfloat16>(__nv_bfloat16 *p, double a, double b) {
    __nv_bfloat162 v;
    v.x = __double2bfloat16(a);
    v.y = __double2bfloat16(b);
    *reinterpret_cast<__nv_bfloat162 *>(p) = v;
}

template <typename TL>
__global__ void k_centre(double *__restrict__ O, double *__restrict__ G,
                         const double *__restrict__ eloc, double *__restrict__ wt,
                         const double *__restrict__ stats, int64_t n, int ldp, int P1,
                         double e_core, TL *__restrict__ Olo, TL *__restrict__ Glo,
                         float2 *__restrict__ wlo) {
    const double E = stats[1];
    const double isw = 1.0 / stats[0];
    const int lane = threadIdx.x & 31, hp = ldp / 2;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += nw) {
        const double el = eloc[r];  // E_loc already includes e_core
        double *Or = O + r * ldp, *Gr = G ? G + r * ldp : nullptr;  // G null: no G'_c
        for (int c = 2 * lane; c < 2 * hp; c += 64) {
            const double2 o = *reinterpret_cast<const double2 *>(Or + c);
            const double2 g = Gr ? *reinterpret_cast<const double2 *>(Gr + c) : make_double2(0.0, 0.0);
            const double2 ob = *reinterpret_cast<const double2 *>(stats + 8 + c);
            double oc[2], gc[2];
            const double ov[2] = {o.x, o.y}, gv[2] = {g.x, g.y}, bv[2] = {ob.x, ob.y};
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int cc = c + u;
                if (cc == 0) {
                    oc[u] = 1.0;
                    gc[u] = el - E;
                } else if (cc < P1) {
                    oc[u] = ov[u] - bv[u];
                    gc[u] = fma(-E, oc[u], fma(-bv[u], el, gv[u]));
                } else {
                    oc[u] = 0.0;
                    gc[u] = 0.0;
                }
            }
            *reinterpret_cast<double2 *>(Or + c) = make_double2(oc[0], oc[1]);
            if (Gr) *reinterpret_cast<double2 *>(Gr + c) = make_double2(gc[0], gc[1]);
            if (Olo) store_low2<TL>(Olo + r * ldp + c, oc[0], oc[1]);
            if (Glo) store_low2<TL>(Glo + r * ldp + c, gc[0], gc[1]);
        }
        if (lane == 0) {
            const double wn = wt[r] * isw;
            wt[r] = wn;
            const df d = df_from_double(wn);
            wlo[r] = make_float2(d.h, d.l);
        }
    }
}

// Centring for double-float pencils: the same formulas in double-float
// arithmetic on the FP32 pipes (inputs split by integer operations), stored
// only as double-float pairs. The FP64 buffers keep the uncentred build output;
// GB300's FP64 pipe would otherwise bound this pass (three FP64 operations per
// element).
__global__ void k_centre_df(const double *__restrict__ O, const double *__restrict__ G,
                            const double *__restrict__ eloc, double *__restrict__ wt,
                            const double *__restrict__ stats, int64_t n, int ldp, int P1,
                            float2 *__restrict__ Olo, float2 *__restrict__ Glo,
                            float2 *__restrict__ wlo) {
    const df E = df_split_bits(stats[1]);
    const double isw = 1.0 / stats[0];
    const int lane = threadIdx.x & 31, hp = ldp / 2;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += nw) {
        const df el = df_split_bits(eloc[r]);  // E_loc already includes e_core
        const df g0 = df_sub(el, E);
        const double *Or = O + r * ldp, *Gr = G ? G + r * ldp : nullptr;  // G null: no G'_c
        for (int c = 2 * lane; c < 2 * hp; c += 64) {
            const double2 o = *reinterpret_cast<const double2 *>(Or + c);
            const double2 g = Gr ? *reinterpret_cast<const double2 *>(Gr + c) : make_double2(0.0, 0.0);
            const double2 ob = *reinterpret_cast<const double2 *>(stats + 8 + c);
            df oc[2], gc[2];
            const double ov[2] = {o.x, o.y}, gv[2] = {g.x, g.y}, bv[2] = {ob.x, ob.y};
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int cc = c + u;
                if (cc == 0) {
                    oc[u] = df_make(1.f, 0.f);
                    gc[u] = g0;
                } else if (cc < P1) {
                    const df b = df_split_bits(bv[u]);
                    oc[u] = df_sub(df_split_bits(ov[u]), b);
                    gc[u] = df_sub(df_sub(df_split_bits(gv[u]), df_mul(b, el)), df_mul(E, oc[u]));
                } else {
                    oc[u] = df_make(0.f, 0.f);
                    gc[u] = df_make(0.f, 0.f);
                }
            }
            *reinterpret_cast<float4 *>(Olo + r * ldp + c) = make_float4(oc[0].h, oc[0].l, oc[1].h, oc[1].l);
            if (Glo)
                *reinterpret_cast<float4 *>(Glo + r * ldp + c) = make_float4(gc[0].h, gc[0].l, gc[1].h, gc[1].l);
        }
        if (lane == 0) {
            const double wn = wt[r] * isw;
            wt[r] = wn;
            const df d = df_from_double(wn);
            wlo[r] = make_float2(d.h, d.l);
        }
    }
}

// Streamed pencils: slot[2] = the chunk's largest ln psi (from the per-CTA maxima)
__global__ void k_chunk_max(const double *part, int nparts, double *slot) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double m = -INFINITY;
    for (int b = 0; b < nparts; ++b) m = fmax(m, part[b]);
    slot[2] = m;
}

// Streamed pencils: combine the chunks' raw sums (slot c: [0] sum w, [1] sum w
// E_loc, [2] the chunk's ln psi shift, [8 + k] sum w O_k, each with weights
// exp(2 (ln psi - shift_c)) or the given weights) in chunk order, with the
// common shift M = max_c shift_c: stats[1] = E, stats[8 + k] = <O_k>,
// stats[2] = M, stats[3] = the total weight, stats[0] = 1 (the weights are
// normalised once, by k_stream_weights, so later centrings leave them alone).
__global__ void k_stream_combine(const double *cst, int nchunks, int ldp, int given,
                                 double *stats) {
    const int ld = 8 + ldp;
    __shared__ double sM, sW;
    if (threadIdx.x == 0) {
        double M = 0.0;
        if (!given) {
            M = -INFINITY;
            for (int c = 0; c < nchunks; ++c) M = fmax(M, cst[(size_t)c * ld + 2]);
        }
        double w = 0.0, we = 0.0;
        for (int c = 0; c < nchunks; ++c) {
            const double f = given ? 1.0 : exp(2.0 * (cst[(size_t)c * ld + 2] - M));
            w += f * cst[(size_t)c * ld];
            we += f * cst[(size_t)c * ld + 1];
        }
        sM = M;
        sW = w;
        stats[0] = 1.0;
        stats[1] = we / w;
        stats[2] = M;
        stats[3] = w;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ldp; k += blockDim.x) {
        double a = 0.0;
        for (int c = 0; c < nchunks; ++c) {
            const double f = given ? 1.0 : exp(2.0 * (cst[(size_t)c * ld + 2] - sM));
            a += f * cst[(size_t)c * ld + 8 + k];
        }
        stats[8 + k] = a / sW;
    }
}

// Streamed pencils: the normalised weights of every row, once:
// w = exp(2 (ln psi - M)) / W, or the given weight / W (in place)
__global__ void k_stream_weights(const double *lnpsi, double *wt, int64_t n, int given,
                                 const double *stats) {
    const double M = stats[2], iw = 1.0 / stats[3];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        wt[r] = (given ? wt[r] : exp(2.0 * (lnpsi[r] - M))) * iw;
}

// y (+)= sum of the CTA partials (CTA order): streamed products add chunk by chunk
__global__ void k_reduce_partials_add(const double *part, int nparts, int ldp, double *yH,
                                      double *yS, int first) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * ldp) return;
    double t = 0.0;
    for (int b = 0; b < nparts; ++b) t += part[(size_t)b * 2 * ldp + e];
    double *y = e < ldp ? yH : yS;
    const int i = e < ldp ? e : e - ldp;
    if (y) y[i] = first ? t : y[i] + t;
}

// Weights of the E_loc-estimator product: w(x) (E_loc(x) - E), FP64 and
// double-float (both E_loc and E include the core energy)
__global__ void k_eloc_weights(const double *__restrict__ wt, const double *__restrict__ eloc,
                               const double *__restrict__ stats, int64_t n,
                               double *__restrict__ wel, float2 *__restrict__ wello) {
    const double E = stats[1];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const double we = wt[r] * (eloc[r] - E);
        wel[r] = we;
        const df d = df_split_bits(we);
        wello[r] = make_float2(d.h, d.l);
    }
}

// FP64 copy of double-float pairs (exports of a double-float pencil)
__global__ void k_df_to_fp64(const float2 *__restrict__ src, double *__restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = src[i];
        dst[i] = (double)v.x + (double)v.y;
    }
}

// ------------------------------------------------ debug: connection lists
__global__ void k_connections(SysView S, const uint64_t *rows, int64_t n_rows, int cap,
                              uint64_t *od, int8_t *osg, double *oh, int32_t *cnt,
                              double e_core) {
    __shared__ RowLists L;
    for (int64_t row = blockIdx.x; row < n_rows; row += gridDim.x) {
        const uint64_t x = rows[row];
        if (threadIdx.x == 0) make_lists(S, x, L);
        __syncthreads();
        if (threadIdx.x < 32) {
            double d = diag_value_warp(S, L);
            if (threadIdx.x == 0) {
                od[row * cap] = x;
                osg[row * cap] = 1;
                oh[row * cap] = d + e_core;
                cnt[row] = min(S.conn + 1, cap);
            }
        }
        for (int k = threadIdx.x; k < S.conn; k += blockDim.x) {
            if (k + 1 >= cap) break;
            Exc e = decode_exc(S, L, k);
            int sg;
            uint64_t y = apply_exc(x, e, sg);
            od[row * cap + k + 1] = y;
            osg[row * cap + k + 1] = (int8_t)sg;
            oh[row * cap + k + 1] = sg * exc_value(S, L, e);
        }
        __syncthreads();
    }
}

}  // namespace

// ==========================================================================
// host launchers
// ==========================================================================
int lm_launch_enumerate(lm_ctx *ctx, int n, int na, int nb, uint64_t *out, int64_t count,
                        cudaStream_t s) {
    int blocks = (int)std::min<int64_t>((count + 255) / 256, (int64_t)ctx->sms * 8);
    if (blocks < 1) blocks = 1;
    k_enumerate<<<blocks, 256, 0, s>>>(n, na, nb, out, count);
    lm_note_launch(ctx);
    return lm_cuda_check(ctx, cudaGetLastError(), "k_enumerate");
}

static size_t build_smem_bytes(int nh, int M, int ldF, int ldS, int nslice) {
    size_t d = (size_t)2 * nh * M + 2 * M + 3 * nh + (size_t)BUILD_THREADS * ldF + BUILD_THREADS +
               (size_t)nslice * (nh + 1) * ldS + (size_t)nslice * (nh + 1) + 64;
    return d * sizeof(double) + BUILD_THREADS * sizeof(int4) + sizeof(RowLists) + 64;
}

// The double-float row build by connection class (k_build_rows_dg): class
// shapes, target table, scatter slices, shared-memory map and launch.
static int launch_build_grid(lm_pencil *p, const BuildArgs &A, cudaStream_t s) {
    lm_ctx *ctx = p->ctx;
    GridDfArgs G;
    G.S = A.S;
    G.nh = p->nh;
    G.M = p->M;
    G.M1 = p->M1;
    G.P1 = p->P1;
    G.ldp = p->ldp;
    G.ldA = p->nh | 1;
    G.ldF = (p->nh + 1) | 1;
    G.ldL = (p->nh + 1) | 1;
    G.ns = A.S.ns_a + A.S.ns_b;
    const SysView &S = A.S;
    G.R[GC_AA] = S.na * (S.na - 1) / 2;
    G.C[GC_AA] = S.nva * (S.nva - 1) / 2;
    G.R[GC_BB] = S.nb * (S.nb - 1) / 2;
    G.C[GC_BB] = S.nvb * (S.nvb - 1) / 2;
    G.R[GC_B] = S.nb;
    G.C[GC_B] = S.nvb;
    G.R[GC_AB] = S.ns_a;
    G.C[GC_AB] = S.ns_b + 1;
    int ntgt = 0;
    for (int c = 0; c < GC_N; ++c) {
        G.toff[c] = ntgt;
        ntgt += G.R[c] + G.C[c];
        G.fdC[c] = make_fastdiv(std::max(1, G.C[c]));
    }
    G.ntgt = ntgt;
    G.fd_nh = make_fastdiv(p->nh);
    G.fd_nh1 = make_fastdiv(p->nh + 1);
    G.fd_M1 = make_fastdiv(p->M1);
    // the lookup form: the rows are the sector in enumeration order (enumerated by
    // the library, all of them resident), so every connection is a row
    // (row indices of the lookup form are held as int)
    // k_row_tables: R rows per CTA pass (one thread per row for the per-row FP64
    // steps); theta and the per-row values in shared memory, up to 32 rows in 96 KB
    // for the latter (the form is not taken where it would not fit)
    const int tab_ldz = p->nh | 1;
    const int tab_R = (int)std::max<int64_t>(1, std::min<int64_t>(32, 96 * 1024 / (16 * (int64_t)tab_ldz)));
    const size_t tsm = ((size_t)p->M + (size_t)p->nh * p->M1 + 2 * (size_t)tab_R * tab_ldz) * sizeof(double);
    const bool lookup = p->enumerated && !p->chunk && !p->shard_state && p->n_rows < INT32_MAX &&
                        tsm <= (size_t)ctx->smem_optin;
    G.lookup = lookup;
    G.ntab = lookup ? 0 : std::max(1, std::max(S.ns_a, S.ns_b));
    G.narow = lookup ? 0 : (GDF_K + G.C[GC_AB] - 2) / G.C[GC_AB] + 1;
    G.rt = nullptr;
    G.rt64 = nullptr;
    G.psim = nullptr;
    G.psie = nullptr;
    G.cA = 1;  // C(n, N_alpha)
    for (int i = 1; i <= p->na; ++i) G.cA = G.cA * (p->n - p->na + i) / i;
    if (lookup) {
        const size_t nr = (size_t)p->n_rows;
        if (!p->rt && lm_cuda_check(ctx, cudaMalloc(&p->rt, nr * p->nh * sizeof(float2)), "cudaMalloc"))
            return LM_ERR_OOM;
        if (!p->psim && lm_cuda_check(ctx, cudaMalloc(&p->psim, nr * sizeof(float2)), "cudaMalloc"))
            return LM_ERR_OOM;
        if (!p->rt64 && lm_cuda_check(ctx, cudaMalloc(&p->rt64, nr * p->nh * sizeof(double)), "cudaMalloc"))
            return LM_ERR_OOM;
        if (!p->psie && lm_cuda_check(ctx, cudaMalloc(&p->psie, nr * sizeof(int)), "cudaMalloc"))
            return LM_ERR_OOM;
        RowTabArgs T;
        T.n = p->n;
        T.nh = p->nh;
        T.M = p->M;
        T.M1 = p->M1;
        T.theta = p->theta;
        T.rows = p->rows;
        T.n_rows = p->n_rows;
        T.t = p->rt;
        T.t64 = p->rt64;
        T.psim = p->psim;
        T.psie = p->psie;
        T.lnpsi = p->lnpsi;
        T.ldz = tab_ldz;
        T.R = tab_R;
        T.fd_nh = make_fastdiv(p->nh);
        if (tsm > 48 * 1024) {
            cudaError_t ea = cudaFuncSetAttribute(k_row_tables, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)tsm);
            if (ea != cudaSuccess) return lm_cuda_check(ctx, ea, "row tables smem attribute");
        }
        const int blocks = (int)std::min<int64_t>((p->n_rows + T.R - 1) / T.R, (int64_t)ctx->sms * 8);
        k_row_tables<<<std::max(blocks, 1), 256, tsm, s>>>(T);
        lm_note_launch(ctx);
        if (int rc = lm_cuda_check(ctx, cudaGetLastError(), "k_row_tables")) return rc;
        G.rt = p->rt;
        G.rt64 = p->rt64;
        G.psim = p->psim;
        G.psie = p->psie;
    }
    G.theta = p->theta;
    G.tdf = p->tdf;
    G.rows = p->rows;
    G.n_rows = p->n_rows;
    G.amask = A.amask;
    G.bmask = A.bmask;
    G.e_core = p->e_core;
    G.lnpsi = p->lnpsi;
    G.eloc = p->eloc;
    G.O = p->O;
    G.G = p->G;
    G.flags = p->d_flags;
    G.gfree = p->gfree;
    // 228 KB of shared memory per SM, 1 KB of it reserved per CTA. Scatter slices
    // q against CTAs per SM: the most CTAs x min(q, 3); on a tie the fewest slices
    // at 4 or more CTAs per SM (other CTAs fill the scatter's barrier waits, so its
    // instruction count decides) and the most below (its critical path decides).
    // Measured (ms per build): F2-shaped rows, products formed per connection,
    // q = 1..6 at 4,4,4,3,3,2 CTAs/SM: 4.06, 3.21, 2.80, 3.13, 3.09, 3.55;
    // F2-shaped rows in the lookup form, q = 2..6 at 5,5,5,5,4: 2.35, 1.95, 2.20,
    // 2.16, 2.12; LiCl-shaped (65,536 rows) q = 1..4 at 3,2,2,2: 111.9, 106.3,
    // 93.1, 84.0.
    auto kern = p->gfree ? (lookup ? k_build_rows_dg<true, true> : k_build_rows_dg<true, false>)
                         : (lookup ? k_build_rows_dg<false, true> : k_build_rows_dg<false, false>);
    // CTAs per SM that the registers allow (the kernels differ: 46 to 56 per thread)
    int reg_cap = 4;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&reg_cap, kern, GDF_THREADS, 0) != cudaSuccess ||
        reg_cap < 1)
        return lm_fail(ctx, LM_ERR_CUDA, "df64 build kernel occupancy query failed");
    auto per_sm_of = [&](size_t bytes) {
        return std::min(reg_cap, (int)(233472 / (bytes + 1024 + 64)));
    };
    const int max_sl = std::max(1, GDF_THREADS / (p->nh + 1));
    int best = 1, best_key = -1;
    for (int q = 1; q <= max_sl; ++q) {
        G.nsl = q;
        const size_t b = grid_smem(G).total;
        if (b > (size_t)ctx->smem_optin) break;
        const int cta = per_sm_of(b);
        const int key = (cta * std::min(q, 3)) * 256 + (cta >= 4 ? 255 - q : q);
        if (key > best_key) {
            best_key = key;
            best = q;
        }
    }
    // IRLNQS_BUILD_SLICES overrides the choice (tuning runs)
    if (const char *env = getenv("IRLNQS_BUILD_SLICES")) {
        const int q = atoi(env);
        if (q >= 1 && q <= max_sl) best = q;
    }
    G.nsl = p->gfree ? 0 : best;
    // Slices packed back to back, unless giving each slice whole warps of its own
    // takes no more warps (then no warp holds two slices' connections): LiCl-shaped
    // rows (57 threads a slice, 4 slices) 81.8 against 83.3 ms at 65,536 rows;
    // F2-shaped ones (41 threads, 3 slices) would take 6 warps instead of 4.
    {
        const int nh1 = p->nh + 1, wps = (nh1 + 31) / 32, q = std::max(G.nsl, 1);
        const bool own = q * wps * 32 <= GDF_THREADS && q * wps == (q * nh1 + 31) / 32;
        G.sw = own ? wps * 32 : nh1;
    }
    const size_t dsm = grid_smem(G).total;
    if (dsm > (size_t)ctx->smem_optin)
        return lm_fail(ctx, LM_ERR_SIZE, "df64 build kernel needs %zu B shared memory", dsm);
    cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    if (e2 != cudaSuccess) return lm_cuda_check(ctx, e2, "df64 build smem attribute");
    const int per_sm = std::max(1, per_sm_of(dsm));
    int64_t grid = std::min<int64_t>(p->n_rows, (int64_t)ctx->sms * per_sm);
    // many rows per resident CTA: one CTA per row instead, so that other streams'
    // kernels can be scheduled as rows finish
    if (p->n_rows > 64 * grid) grid = std::min<int64_t>(p->n_rows, 0x7fffffff);
    if (grid < 1) grid = 1;
    lm_prof_begin(ctx, PROF_BUILD, s);
    kern<<<(unsigned)grid, GDF_THREADS, dsm, s>>>(G);
    lm_prof_end(ctx, PROF_BUILD, s);
    lm_note_launch(ctx);
    return lm_cuda_check(ctx, cudaGetLastError(), "k_build_rows_dg");
}

int lm_launch_build(lm_pencil *p, cudaStream_t s) {
    if (int rc = lm_launch_build_rows(p, s)) return rc;
    return lm_launch_build_prep(p, s);
}

// K2-K6: ln psi, O, E_loc and G of every row (uncentred)
int lm_launch_build_rows(lm_pencil *p, cudaStream_t s) {
    lm_ctx *ctx = p->ctx;
    BuildArgs A;
    A.S = make_view(p->n, p->na, p->nb, p->h, p->eri);
    A.nh = p->nh;
    A.M = p->M;
    A.M1 = p->M1;
    A.P1 = p->P1;
    A.ldp = p->ldp;
    A.ldF = p->nh | 1;
    A.ldS = p->M | 1;
    A.nslice = std::max(1, BUILD_THREADS / (p->nh + 1));
    A.theta = p->theta;
    A.tabs = p->tabs;
    A.rows = p->rows;
    A.n_rows = p->n_rows;
    A.amask = (p->n >= 64) ? ~0ull : ((1ull << p->n) - 1ull);
    A.bmask = A.amask << p->n;
    A.e_core = p->e_core;
    A.lnpsi = p->lnpsi;
    A.eloc = p->eloc;
    A.O = p->O;
    A.G = p->G;
    A.flags = p->d_flags;
    if (p->nh + 1 > BUILD_THREADS)
        return lm_fail(ctx, LM_ERR_SIZE, "n_hidden + 1 = %d exceeds %d", p->nh + 1,
                       BUILD_THREADS);
    const size_t smem = build_smem_bytes(p->nh, p->M, A.ldF, A.ldS, A.nslice);
    if (p->arith == LM_ARITH_FP64) {
        if (smem > (size_t)ctx->smem_optin)
            return lm_fail(ctx, LM_ERR_SIZE, "build kernel needs %zu B shared memory", smem);
        cudaError_t e = cudaFuncSetAttribute(k_build_rows,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return lm_cuda_check(ctx, e, "build smem attribute");
    }

    int tb = 256;
    k_tables<<<(p->nh * p->M + p->M + tb - 1) / tb, tb, 0, s>>>(p->theta, p->M, p->nh, p->tabs);
    lm_note_launch(ctx);
    if (int rc = lm_cuda_check(ctx, cudaGetLastError(), "k_tables")) return rc;

    if (p->arith == LM_ARITH_FP64) {
        int per_sm = std::max(1, (int)(200 * 1024 / smem));
        per_sm = std::min(per_sm, 8);
        int64_t grid = std::min<int64_t>(p->n_rows, (int64_t)ctx->sms * per_sm);
        if (grid < 1) grid = 1;
        lm_prof_begin(ctx, PROF_BUILD, s);
        k_build_rows<<<(unsigned)grid, BUILD_THREADS, smem, s>>>(A);
        lm_prof_end(ctx, PROF_BUILD, s);
        lm_note_launch(ctx);
        if (int rc = lm_cuda_check(ctx, cudaGetLastError(), "k_build_rows")) return rc;
    } else {
        const int n = p->n;
        const int ntab = 2 * p->nh * p->M + n * n + n * n * n * n;
        k_tables_df<<<std::min(1024, (ntab + 255) / 256), 256, 0, s>>>(p->theta, p->h, p->eri, p->M,
                                                                       p->nh, n, p->tdf);
        lm_note_launch(ctx);
        if (int rc = lm_cuda_check(ctx, cudaGetLastError(), "k_tables_df")) return rc;
        return launch_build_grid(p, A, s);
    }

    return LM_OK;
}

// K7: weights, E, <O>, then the centring
int lm_launch_build_prep(lm_pencil *p, cudaStream_t s) {
    lm_ctx *ctx = p->ctx;
    const int nmax = std::max(1, std::min(ctx->sms, (int)((p->n_rows + 255) / 256)));
    double *maxpart = p->part;  // reuse the partials buffer (nmax doubles first)
    double *given = p->given_weights ? p->wt : nullptr;
    lm_prof_begin(ctx, PROF_PREP, s);
    if (!given) {
        k_lnpsi_max_partial<<<nmax, 256, 0, s>>>(p->lnpsi, p->n_rows, maxpart);
        lm_note_launch(ctx);
        if (int rc = lm_cuda_check(ctx, cudaGetLastError(), "k_lnpsi_max")) return rc;
    }
    const int nst = (int)std::max<int64_t>(1, std::min<int64_t>(p->n_rows, ctx->sms * 2));
    double *spart = p->part + 256;
    k_weights<<<(int)std::min<int64_t>((p->n_rows + 255) / 256, ctx->sms * 4), 256, 0, s>>>(
        p->lnpsi, given, p->wt, p->n_rows, maxpart, nmax);
    lm_note_launch(ctx);
    k_stats_partial<<<nst, 256, 0, s>>>(p->O, p->eloc, p->wt, p->n_rows, p->ldp, spart);
    lm_note_launch(ctx);
    if (int rc = lm_cuda_check(ctx, cudaGetLastError(), "k_stats_partial")) return rc;
    k_stats_final<<<(p->ldp + 31) / 32, 256, 0, s>>>(spart, nst, p->ldp, p->stats, 0);
    lm_note_launch(ctx);
    if (int rc = lm_cuda_check(ctx, cudaGetLastError(), "k_stats_final")) return rc;
    const int rc = lm_launch_centre(p, s);
    lm_prof_end(ctx, PROF_PREP, s);
    return rc;
}

// Local statistics of a row shard: the per-CTA maxima of ln psi into
// part[0 .. nmax) (returns nmax).
int lm_launch_shard_max(lm_pencil *p, cudaStream_t s, int *nparts) {
    lm_ctx *ctx = p->ctx;
    const int nmax = std::max(1, std::min(ctx->sms, (int)((p->n_rows + 255) / 256)));
    k_lnpsi_max_partial<<<nmax, 256, 0, s>>>(p->lnpsi, p->n_rows, p->part);
    lm_note_launch(ctx);
    *nparts = nmax;
    return lm_cuda_check(ctx, cudaGetLastError(), "k_lnpsi_max");
}

// Unnormalised weights of a row shard with the shift lnpsi_max shared by all
// shards (or the caller's weights), and the shard's raw sums into stats:
// stats[0] = sum w, stats[1] = sum w E_loc, stats[8 + c] = sum w O_c.
int lm_launch_shard_sums(lm_pencil *p, double lnpsi_max, cudaStream_t s) {
    lm_ctx *ctx = p->ctx;
    double *given = p->given_weights ? p->wt : nullptr;
    const int nst = (int)std::max<int64_t>(1, std::min<int64_t>(p->n_rows, ctx->sms * 2));
    double *spart = p->part + 256;
    lm_prof_begin(ctx, PROF_PREP, s);
    k_weights_shift<<<(int)std::min<int64_t>((p->n_rows + 255) / 256, ctx->sms * 4), 256, 0, s>>>(
        p->lnpsi, given, p->wt, p->n_rows, lnpsi_max);
    lm_note_launch(ctx);
    k_stats_partial<<<nst, 256, 0, s>>>(p->O, p->eloc, p->wt, p->n_rows, p->ldp, spart);
    lm_note_launch(ctx);
    k_stats_final<<<(p->ldp + 31) / 32, 256, 0, s>>>(spart, nst, p->ldp, p->stats, 1);
    lm_prof_end(ctx, PROF_PREP, s);
    lm_note_launch(ctx);
    return lm_cuda_check(ctx, cudaGetLastError(), "shard sums");
}

// Centring with the statistics in p->stats (stats[0] = sum w over every row of
// every shard, stats[1] = E, stats[8 + c] = <O_c>): O_c, G'_c, the normalised
// weights and the E_loc-estimator weights.
int lm_launch_centre(lm_pencil *p, cudaStream_t s) {
    lm_ctx *ctx = p->ctx;
    int cgrid = (int)std::min<int64_t>((p->n_rows + 7) / 8, (int64_t)ctx->sms * 16);
    if (p->prec == LM_FP32)
        k_centre<float><<<cgrid, 256, 0, s>>>(p->O, p->G, p->eloc, p->wt, p->stats, p->n_rows,
                                              p->ldp, p->P1, p->e_core, (float *)p->Olo,
                                              (float *)p->Glo, p->wlo);
    else if (p->prec == LM_DF64)
        k_centre_df<<<cgrid, 256, 0, s>>>(p->O, p->G, p->eloc, p->wt, p->stats, p->n_rows, p->ldp,
                                          p->P1, (float2 *)p->Olo, (float2 *)p->Glo, p->wlo);
    else if (p->prec == LM_BF16)
        k_centre<__nv_bfloat16><<<cgrid, 256, 0, s>>>(
            p->O, p->G, p->eloc, p->wt, p->stats, p->n_rows, p->ldp, p->P1, p->e_core,
            (__nv_bfloat16 *)p->Olo, (__nv_bfloat16 *)p->Glo, p->wlo);
    else
        k_centre<double><<<cgrid, 256, 0, s>>>(p->O, p->G, p->eloc, p->wt, p->stats, p->n_rows,
                                               p->ldp, p->P1, p->e_core, (double *)nullptr,
                                               (double *)nullptr, p->wlo);
    lm_note_launch(ctx);
    if (int rc = lm_cuda_check(ctx, cudaGetLastError(), "k_centre")) return rc;
    k_eloc_weights<<<(int)std::max<int64_t>(1, std::min<int64_t>((p->n_rows + 255) / 256,
                                                                 ctx->sms * 4)),
                     256, 0, s>>>(p->wt, p->eloc, p->stats, p->n_rows, p->wel, p->wello);
    lm_note_launch(ctx);
    return lm_cuda_check(ctx, cudaGetLastError(), "k_eloc_weights");
}

// A chunk of a streamed pencil: the same pencil with its per-row arrays
// offset to rows [r0, r0 + n) (O, G and their copies are the chunk buffers)
static lm_pencil chunk_view(const lm_pencil *p, int64_t r0, int64_t n) {
    lm_pencil v = *p;
    v.rows += r0;
    v.wt += r0;
    v.wlo += r0;
    v.wel += r0;
    v.wello += r0;
    v.lnpsi += r0;
    v.eloc += r0;
    v.n_rows = n;
    return v;
}

// First pass over a streamed pencil: per chunk, the row build, the chunk's
// ln psi shift and raw sums; then the combined statistics and the normalised
// weights of every row.
int lm_launch_stream_stats(lm_pencil *p, cudaStream_t s) {
    lm_ctx *ctx = p->ctx;
    const int64_t C = p->chunk;
    const int nch = (int)((p->n_rows + C - 1) / C);
    const int ld = 8 + p->ldp;
    lm_prof_begin(ctx, PROF_PREP, s);
    for (int c = 0; c < nch; ++c) {
        const int64_t r0 = (int64_t)c * C, n = std::min(C, p->n_rows - r0);
        lm_pencil v = chunk_view(p, r0, n);
        if (int rc = lm_launch_build_rows(&v, s)) return rc;
        double *slot = p->cstats + (size_t)c * ld;
        const int nmax = std::max(1, std::min(ctx->sms, (int)((n + 255) / 256)));
        double *given = p->given_weights ? v.wt : nullptr;
        if (!given) {
            k_lnpsi_max_partial<<<nmax, 256, 0, s>>>(v.lnpsi, n, p->part);
            k_chunk_max<<<1, 32, 0, s>>>(p->part, nmax, slot);
            lm_note_launch(ctx, 2);
        }
        k_weights<<<(int)std::min<int64_t>((n + 255) / 256, ctx->sms * 4), 256, 0, s>>>(
            v.lnpsi, given, v.wt, n, p->part, nmax);
        const int nst = (int)std::max<int64_t>(1, std::min<int64_t>(n, ctx->sms * 2));
        k_stats_partial<<<nst, 256, 0, s>>>(v.O, v.eloc, v.wt, n, p->ldp, p->part + 256);
        // raw sums into the slot (its [2] keeps the shift written above)
        k_stats_final<<<(p->ldp + 31) / 32, 256, 0, s>>>(p->part + 256, nst, p->ldp, p->stats, 1);
        cudaMemcpyAsync(slot, p->stats, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(slot + 8, p->stats + 8, p->ldp * sizeof(double), cudaMemcpyDeviceToDevice,
                        s);
        lm_note_launch(ctx, 3);
        if (int rc = lm_cuda_check(ctx, cudaGetLastError(), "stream statistics")) return rc;
    }
    k_stream_combine<<<1, 256, 0, s>>>(p->cstats, nch, p->ldp, p->given_weights, p->stats);
    k_stream_weights<<<(int)std::min<int64_t>((p->n_rows + 255) / 256, ctx->sms * 4), 256, 0, s>>>(
        p->lnpsi, p->wt, p->n_rows, p->given_weights, p->stats);
    lm_prof_end(ctx, PROF_PREP, s);
    lm_note_launch(ctx, 2);
    (void)ld;
    return lm_cuda_check(ctx, cudaGetLastError(), "stream statistics");
}

// A product on a streamed pencil: per chunk, rebuild the rows, centre them
// with the pencil's statistics, apply the pencil (partials) and add the
// chunk's product into yH / yS (chunk order).
int lm_launch_stream_product(lm_pencil *p, const double *v, int sym, int prec, int want_s,
                             double *yH, double *yS, cudaStream_t s) {
    lm_ctx *ctx = p->ctx;
    const int64_t C = p->chunk;
    const int nch = (int)((p->n_rows + C - 1) / C);
    for (int c = 0; c < nch; ++c) {
        const int64_t r0 = (int64_t)c * C, n = std::min(C, p->n_rows - r0);
        lm_pencil w = chunk_view(p, r0, n);
        if (int rc = lm_launch_build_rows(&w, s)) return rc;
        if (int rc = lm_launch_centre(&w, s)) return rc;
        if (int rc = lm_launch_pencil(&w, v, sym, prec, want_s, nullptr, s)) return rc;
        k_reduce_partials_add<<<(2 * p->ldp + 255) / 256, 256, 0, s>>>(
            p->part, lm_pencil_ctas(&w, prec), p->ldp, yH, want_s ? yS : nullptr, c == 0);
        lm_note_launch(ctx);
        if (int rc = lm_cuda_check(ctx, cudaGetLastError(), "stream product")) return rc;
    }
    return LM_OK;
}

int lm_launch_df_to_fp64(lm_ctx *ctx, const float2 *src, double *dst, int64_t n, cudaStream_t s) {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, ctx->sms * 8));
    k_df_to_fp64<<<blocks, 256, 0, s>>>(src, dst, n);
    lm_note_launch(ctx);
    return lm_cuda_check(ctx, cudaGetLastError(), "k_df_to_fp64");
}

int lm_launch_connections(lm_ctx *ctx, int n, int na, int nb, const double *h, const double *eri,
                          const uint64_t *rows, int64_t n_rows, int cap, uint64_t *od,
                          int8_t *osg, double *oh, int32_t *cnt, double e_core, cudaStream_t s) {
    SysView S = make_view(n, na, nb, h, eri);
    int grid = (int)std::min<int64_t>(n_rows, (int64_t)ctx->sms * 4);
    if (grid < 1) return LM_OK;
    k_connections<<<grid, 256, 0, s>>>(S, rows, n_rows, cap, od, osg, oh, cnt, e_core);
    lm_note_launch(ctx);
    return lm_cuda_check(ctx, cudaGetLastError(), "k_connections");
}
