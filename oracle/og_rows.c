/*
 * Oracle: TEST INFRASTRUCTURE ONLY. Only tests/, the package smoke check and
 * the benchmark's CPU-baseline leg may load this code. It shares no code with
 * the CUDA path.
 *
 * Plain FP64 per-row evaluation, written directly from the definitions:
 *
 *   Hamiltonian (Methods, "Wave Function Ansatz", the second-quantised H):
 *     H = sum_{pq,s} h_pq a+_{ps} a_{qs}
 *       + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}
 *   with chemist-notation integrals (pq|rs) and Jordan-Wigner ordering signs:
 *   a_q|x> = (-1)^{#occupied spin orbitals below q} |x - e_q>.
 *   Matrix elements between determinants follow the Slater-Condon rules.
 *
 *   Fock basis (Methods, Fock expansion): a determinant is a uint64, bit p is
 *   the occupation of spin orbital p; blocked order (alpha 0..n-1, beta n..2n-1).
 *
 *   RBM amplitude: ln psi(x) = a.x + sum_j ln(2 cosh(b_j + W_j.x)).
 *   Log-derivatives (Methods, definition of O): O_k(x) = d ln psi / d theta_k,
 *   laid out on the augmented (Nh+1) x (M+1) grid as [1; tanh z] (x) [1; x];
 *   entry (0,0) = 1 is the psi basis function of the linear method.
 *   Local energy (Methods, E_loc = (H psi)(x) / psi(x)).
 *   G_k(x) = sum_x' H_xx' psi(x')/psi(x) O_k(x'), the Hamiltonian applied to the
 *   derivative basis functions chi_k = O_k psi (Methods, H_eff definition).
 *
 * Every connected determinant's ln psi, tanh and O row is evaluated from
 * scratch; no incremental updates, no tables, no reordering of the sums.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n, na, nb, nh, m, p1;
    const double *h, *eri, *theta;
} osys;

static int spin_of(const osys *s, int p) { return p >= s->n; }
static int spatial(const osys *s, int p) { return p >= s->n ? p - s->n : p; }

/* spin-orbital one-electron integral t_PQ = delta(spin) h_pq */
static double t1(const osys *s, int P, int Q) {
    if (spin_of(s, P) != spin_of(s, Q)) return 0.0;
    return s->h[spatial(s, P) * s->n + spatial(s, Q)];
}

/* spin-orbital chemist integral (PQ|RS) = delta(sP,sQ) delta(sR,sS) (pq|rs) */
static double g2(const osys *s, int P, int Q, int R, int S) {
    if (spin_of(s, P) != spin_of(s, Q) || spin_of(s, R) != spin_of(s, S)) return 0.0;
    int n = s->n;
    int p = spatial(s, P), q = spatial(s, Q), r = spatial(s, R), t = spatial(s, S);
    return s->eri[((p * n + q) * n + r) * n + t];
}

static int popc(uint64_t v) {
    int c = 0;
    while (v) { v &= v - 1; c++; }
    return c;
}

/* Jordan-Wigner annihilation of spin orbital q: returns the sign, 0 if empty */
static int jw_ann(uint64_t *x, int q) {
    if (!((*x >> q) & 1ULL)) return 0;
    int sg = (popc(*x & ((1ULL << q) - 1ULL)) & 1) ? -1 : 1;
    *x ^= (1ULL << q);
    return sg;
}

/* Jordan-Wigner creation of spin orbital p: returns the sign, 0 if occupied */
static int jw_cre(uint64_t *x, int p) {
    if ((*x >> p) & 1ULL) return 0;
    int sg = (popc(*x & ((1ULL << p) - 1ULL)) & 1) ? -1 : 1;
    *x |= (1ULL << p);
    return sg;
}

/*
 * All determinants connected to x by H (the diagonal first, then singles
 * I->A, then doubles I<J -> A<B, each only if it conserves N_alpha and
 * N_beta), with <x'|H|x> and the Jordan-Wigner sign of the excitation
 * operator a+_A a_I (singles) or a+_A a+_B a_J a_I (doubles).
 * Returns the count, or -1 if it would exceed cap.
 */
static int connections(const osys *s, uint64_t x, int cap, uint64_t *od, double *oh, int *osg) {
    int m = s->m;
    int occ[64], vir[64], no = 0, nv = 0;
    for (int p = 0; p < m; p++) {
        if ((x >> p) & 1ULL) occ[no++] = p; else vir[nv++] = p;
    }
    int cnt = 0;
    /* diagonal: sum_I t_II + 1/2 sum_{I,J} [(II|JJ) - (IJ|JI)] */
    double d = 0.0;
    for (int a = 0; a < no; a++) {
        int I = occ[a];
        d += t1(s, I, I);
        for (int b = 0; b < no; b++) {
            int J = occ[b];
            d += 0.5 * (g2(s, I, I, J, J) - g2(s, I, J, J, I));
        }
    }
    if (cnt >= cap) return -1;
    od[cnt] = x; oh[cnt] = d; osg[cnt] = 1; cnt++;
    /* singles: <x'|H|x> = sign * [t_AI + sum_{K occ} ((AI|KK) - (AK|KI))] */
    for (int a = 0; a < no; a++) {
        int I = occ[a];
        for (int b = 0; b < nv; b++) {
            int A = vir[b];
            if (spin_of(s, A) != spin_of(s, I)) continue;
            uint64_t y = x;
            int sg = jw_ann(&y, I);
            sg *= jw_cre(&y, A);
            double v = t1(s, A, I);
            for (int c = 0; c < no; c++) {
                int K = occ[c];
                v += g2(s, A, I, K, K) - g2(s, A, K, K, I);
            }
            if (cnt >= cap) return -1;
            od[cnt] = y; oh[cnt] = sg * v; osg[cnt] = sg; cnt++;
        }
    }
    /* doubles: <x'|H|x> = sign * [<AB|IJ> - <AB|JI>] = sign * [(AI|BJ) - (AJ|BI)] */
    for (int a1 = 0; a1 < no; a1++) {
        for (int a2 = a1 + 1; a2 < no; a2++) {
            int I = occ[a1], J = occ[a2];
            for (int b1 = 0; b1 < nv; b1++) {
                for (int b2 = b1 + 1; b2 < nv; b2++) {
                    int A = vir[b1], B = vir[b2];
                    int sin_ = spin_of(s, I) + spin_of(s, J);
                    int sout = spin_of(s, A) + spin_of(s, B);
                    if (sin_ != sout) continue;
                    uint64_t y = x;
                    int sg = jw_ann(&y, I);
                    sg *= jw_ann(&y, J);
                    sg *= jw_cre(&y, B);
                    sg *= jw_cre(&y, A);
                    double v = g2(s, A, I, B, J) - g2(s, A, J, B, I);
                    if (cnt >= cap) return -1;
                    od[cnt] = y; oh[cnt] = sg * v; osg[cnt] = sg; cnt++;
                }
            }
        }
    }
    return cnt;
}

/* theta layout: augmented (Nh+1) x (M+1) row-major grid without entry (0,0) */
static double th_a(const osys *s, int p) { return s->theta[p]; }
static double th_b(const osys *s, int j) { return s->theta[(j + 1) * (s->m + 1) - 1]; }
static double th_w(const osys *s, int j, int p) { return s->theta[(j + 1) * (s->m + 1) + p]; }

/* ln psi(x) = a.x + sum_j ln(2 cosh z_j), z_j = b_j + W_j.x ; tanh z_j into t */
static double rbm_lnpsi(const osys *s, uint64_t x, double *t) {
    double lp = 0.0;
    for (int p = 0; p < s->m; p++)
        if ((x >> p) & 1ULL) lp += th_a(s, p);
    for (int j = 0; j < s->nh; j++) {
        double z = th_b(s, j);
        for (int p = 0; p < s->m; p++)
            if ((x >> p) & 1ULL) z += th_w(s, j, p);
        /* ln(2 cosh z) = |z| + ln(1 + exp(-2|z|)) */
        lp += fabs(z) + log1p(exp(-2.0 * fabs(z)));
        t[j] = tanh(z);
    }
    return lp;
}

/* O row on the augmented grid: O[r*(M+1)+c] = u_r * v_c, u = [1; t], v = [1; x] */
static void rbm_orow(const osys *s, uint64_t x, const double *t, double *o) {
    int m1 = s->m + 1;
    for (int r = 0; r <= s->nh; r++) {
        double u = (r == 0) ? 1.0 : t[r - 1];
        for (int c = 0; c <= s->m; c++) {
            double v = (c == 0) ? 1.0 : (double)((x >> (c - 1)) & 1ULL);
            o[r * m1 + c] = u * v;
        }
    }
}

static int max_conn(int n, int na, int nb) {
    /* generous bound: every pair of (occupied, empty) pairs */
    int m = 2 * n, ne = na + nb, nv = m - ne;
    return 1 + ne * nv + (ne * (ne - 1) / 2) * (nv * (nv - 1) / 2) + 16;
}

static int check_sys(int n, int na, int nb, int nh) {
    if (n <= 0 || 2 * n > 64 || na < 0 || nb < 0 || na > n || nb > n || nh < 0) return -1;
    return 0;
}

/* Connected determinants of one row; returns the count or a negative error. */
int oracle_connections(int n_orb, int n_alpha, int n_beta, const double *h, const double *eri,
                       uint64_t det, int cap, uint64_t *out_det, double *out_h, int *out_sign) {
    if (check_sys(n_orb, n_alpha, n_beta, 0)) return -1;
    osys s = {n_orb, n_alpha, n_beta, 0, 2 * n_orb, 0, h, eri, NULL};
    return connections(&s, det, cap, out_det, out_h, out_sign);
}

/*
 * Per-row ln psi, O row, E_loc and G row for n_rows determinants.
 * O and G are n_rows x (Nh+1)(M+1) row-major (either may be NULL).
 * Rows are independent, so the loop over rows runs in parallel; each row's
 * sums are taken in the fixed connection order above.
 */
int oracle_rows(int n_orb, int n_alpha, int n_beta, int n_hidden, const double *h,
                const double *eri, const double *theta, const uint64_t *rows, int64_t n_rows,
                double *lnpsi, double *O, double *eloc, double *G) {
    if (check_sys(n_orb, n_alpha, n_beta, n_hidden)) return -1;
    int m = 2 * n_orb;
    int p1 = (n_hidden + 1) * (m + 1);
    osys s = {n_orb, n_alpha, n_beta, n_hidden, m, p1, h, eri, theta};
    int cap = max_conn(n_orb, n_alpha, n_beta);
    int err = 0;
#pragma omp parallel
    {
        uint64_t *cd = (uint64_t *)malloc(sizeof(uint64_t) * cap);
        double *ch = (double *)malloc(sizeof(double) * cap);
        int *cs = (int *)malloc(sizeof(int) * cap);
        double *t = (double *)malloc(sizeof(double) * (n_hidden + 1));
        double *tp = (double *)malloc(sizeof(double) * (n_hidden + 1));
        double *orow = (double *)malloc(sizeof(double) * p1);
        double *grow = (double *)malloc(sizeof(double) * p1);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n_rows; i++) {
            uint64_t x = rows[i];
            double lp = rbm_lnpsi(&s, x, t);
            if (lnpsi) lnpsi[i] = lp;
            if (O) {
                rbm_orow(&s, x, t, orow);
                memcpy(O + i * (int64_t)p1, orow, sizeof(double) * p1);
            }
            if (!eloc && !G) continue;
            int nc = connections(&s, x, cap, cd, ch, cs);
            if (nc < 0) {
#pragma omp atomic write
                err = -2;
                continue;
            }
            double el = 0.0;
            for (int c = 0; c < p1; c++) grow[c] = 0.0;
            for (int k = 0; k < nc; k++) {
                double lpk = rbm_lnpsi(&s, cd[k], tp);
                double ck = ch[k] * exp(lpk - lp);  /* H_xx' psi(x')/psi(x) */
                el += ck;
                if (G) {
                    rbm_orow(&s, cd[k], tp, orow);
                    for (int c = 0; c < p1; c++) grow[c] += ck * orow[c];
                }
            }
            if (eloc) eloc[i] = el;
            if (G) memcpy(G + i * (int64_t)p1, grow, sizeof(double) * p1);
        }
        free(cd); free(ch); free(cs); free(t); free(tp); free(orow); free(grow);
    }
    return err;
}

/*
 * First-order rounding scale of every O_k(x): for hidden unit j,
 * O = tanh(z_j) x_c with z_j = b_j + sum_p W_jp x_p, and a relative change u
 * of every term of z_j moves tanh(z_j) by at most u (1 - tanh^2) S_j with
 * S_j = |b_j| + sum_p |W_jp| x_p; so the scale is (|t_j| + (1 - t_j^2) S_j) x_c
 * (x_0 = 1). Visible-unit entries (0/1) and entry (0,0) are exact: scale |O|.
 */
static void rbm_oscale(const osys *s, uint64_t x, uint64_t occ, double *oa) {
    /* hidden factors from x, visible factors from the occupation mask occ */
    int m1 = s->m + 1;
    for (int c = 0; c <= s->m; c++)
        oa[c] = (c == 0) ? 1.0 : (double)((occ >> (c - 1)) & 1ULL);
    for (int j = 0; j < s->nh; j++) {
        double z = th_b(s, j), sz = fabs(th_b(s, j));
        for (int p = 0; p < s->m; p++)
            if ((x >> p) & 1ULL) {
                z += th_w(s, j, p);
                sz += fabs(th_w(s, j, p));
            }
        double t = tanh(z);
        double u = fabs(t) + (1.0 - t * t) * sz;
        for (int c = 0; c <= s->m; c++) {
            double v = (c == 0) ? 1.0 : (double)((occ >> (c - 1)) & 1ULL);
            oa[(j + 1) * m1 + c] = u * v;
        }
    }
}

/*
 * Condition scales of the per-row sums, for componentwise error bars: with
 * c_x' = H_xx' psi(x')/psi(x) and the scale Oa_k(x') above,
 * eloc_abs[i] = sum_x' |c_x'|, G_abs[i][k] = sum_x' |c_x'| Oa_k(x'), and
 * O_abs[i][k] = Oa_k(x): a relative change u in every rounded quantity moves
 * E_loc, G and O by at most about u times these.
 * union_occ = 1: in G_abs, the visible factor of Oa_k(x') is 1 when orbital k
 * is occupied in x or in x' (the scale of a G formed, for orbitals occupied in
 * x, as a sum over all connections minus the sum over those that empty k).
 */
int oracle_rows_abs(int n_orb, int n_alpha, int n_beta, int n_hidden, const double *h,
                    const double *eri, const double *theta, const uint64_t *rows, int64_t n_rows,
                    double *eloc_abs, double *G_abs, double *O_abs, int union_occ) {
    if (check_sys(n_orb, n_alpha, n_beta, n_hidden)) return -1;
    int m = 2 * n_orb;
    int p1 = (n_hidden + 1) * (m + 1);
    osys s = {n_orb, n_alpha, n_beta, n_hidden, m, p1, h, eri, theta};
    int cap = max_conn(n_orb, n_alpha, n_beta);
    int err = 0;
#pragma omp parallel
    {
        uint64_t *cd = (uint64_t *)malloc(sizeof(uint64_t) * cap);
        double *ch = (double *)malloc(sizeof(double) * cap);
        int *cs = (int *)malloc(sizeof(int) * cap);
        double *t = (double *)malloc(sizeof(double) * (n_hidden + 1));
        double *tp = (double *)malloc(sizeof(double) * (n_hidden + 1));
        double *orow = (double *)malloc(sizeof(double) * p1);
        double *grow = (double *)malloc(sizeof(double) * p1);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n_rows; i++) {
            uint64_t x = rows[i];
            double lp = rbm_lnpsi(&s, x, t);
            if (O_abs) rbm_oscale(&s, x, x, O_abs + i * (int64_t)p1);
            int nc = connections(&s, x, cap, cd, ch, cs);
            if (nc < 0) {
#pragma omp atomic write
                err = -2;
                continue;
            }
            double el = 0.0;
            for (int c = 0; c < p1; c++) grow[c] = 0.0;
            for (int k = 0; k < nc; k++) {
                double lpk = rbm_lnpsi(&s, cd[k], tp);
                double ck = fabs(ch[k] * exp(lpk - lp));
                el += ck;
                if (G_abs) {
                    rbm_oscale(&s, cd[k], union_occ ? (cd[k] | x) : cd[k], orow);
                    for (int c = 0; c < p1; c++) grow[c] += ck * orow[c];
                }
            }
            if (eloc_abs) eloc_abs[i] = el;
            if (G_abs) memcpy(G_abs + i * (int64_t)p1, grow, sizeof(double) * p1);
        }
        free(cd); free(ch); free(cs); free(t); free(tp); free(orow); free(grow);
    }
    return err;
}
