/*
 * vegasp_oracle.c -- plain, slow, FP64 CPU restatement of one vegas+ iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs use it.  It shares no code, header, table or
 * constant generator with the CUDA path: the Philox generator, the map, the
 * integrands, the estimate, the reallocation and the grid refinement below are
 * written independently from the paper (Lepage, "Adaptive Multidimensional
 * Integration: vegas Enhanced", arXiv:2009.05112) and from the published
 * definition of Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
 *
 * Everything is FP64, sequential, in the order the paper states it.  Compiled
 * with -ffp-contract=off so that no multiply-add is fused behind our back (the
 * result must not depend on the host CPU: x86-64 here, aarch64 on the GPU host).
 *
 * Readings of points the paper leaves open are marked "reading:"; they are the
 * same readings the library states.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 5: the Philox S-P network).      */
/* Each round: two 32x32->64 products of counter words 0 and 2 with the       */
/* round multipliers; the high halves are xored with the other two counter    */
/* words and the round key, the low halves pass through.  The key is bumped by */
/* the two Weyl increments before every round but the first.                  */
/* ------------------------------------------------------------------------ */
#define OR_PHILOX_MUL_A 0xD2511F53u
#define OR_PHILOX_MUL_B 0xCD9E8D57u
#define OR_PHILOX_WEYL_A 0x9E3779B9u
#define OR_PHILOX_WEYL_B 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += OR_PHILOX_WEYL_A;
            k1 += OR_PHILOX_WEYL_B;
        }
        uint64_t pa = (uint64_t)OR_PHILOX_MUL_A * (uint64_t)c0;
        uint64_t pb = (uint64_t)OR_PHILOX_MUL_B * (uint64_t)c2;
        uint32_t pa_hi = (uint32_t)(pa >> 32), pa_lo = (uint32_t)pa;
        uint32_t pb_hi = (uint32_t)(pb >> 32), pb_lo = (uint32_t)pb;
        uint32_t n0 = pb_hi ^ c1 ^ k0;
        uint32_t n1 = pb_lo;
        uint32_t n2 = pa_hi ^ c3 ^ k1;
        uint32_t n3 = pa_lo;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Stratification count, §3 Eq. (Nst_vegasp): N_st = floor((N_ev/4)^(1/D)),  */
/* or classic vegas's §3 Eq. (Nst): floor((N_ev/2)^(1/D)) -- the divisor div.  */
/* reading: evaluated exactly as the largest integer n >= 1 with               */
/* div n^D <= N_ev (the real power is only a starting guess).                 */
/* ------------------------------------------------------------------------ */
static int or_pow_le(int64_t n, int d, int64_t limit) { /* 1 if n^d <= limit */
    int64_t p = 1;
    for (int i = 0; i < d; ++i) {
        if (p > limit / n) return 0;
        p *= n;
    }
    return p <= limit;
}

int64_t or_nstrat_div(int dim, int64_t n_ev, int div) {
    if (dim < 1 || n_ev < div) return 1;
    int64_t n = (int64_t)floor(pow((double)n_ev / (double)div, 1.0 / (double)dim));
    if (n < 1) n = 1;
    while (n > 1 && !or_pow_le(n, dim, n_ev / div)) --n;
    while (or_pow_le(n + 1, dim, n_ev / div)) ++n;
    return n;
}

int64_t or_nstrat(int dim, int64_t n_ev) { return or_nstrat_div(dim, n_ev, 4); }

/* ------------------------------------------------------------------------ */
/* §3.2 (Limitations and a Variation): the mixed stratification -- N_st + 1   */
/* strata in the first d directions and N_st in the others, N_st from         */
/* Eq. (Nst_vegasp) and d the largest value that still allows 4 samples per   */
/* hypercube, i.e. 4 (N_st + 1)^d N_st^(D - d) <= N_ev (exact integers).       */
/* ------------------------------------------------------------------------ */
void or_nstrat_mixed_div(int dim, int64_t n_ev, int div, int64_t *nst_ax) {
    const int64_t n = or_nstrat_div(dim, n_ev, div);
    const int64_t limit = n_ev / div;
    int d = 0;
    for (int k = 1; k <= dim; ++k) { /* largest k with (n+1)^k n^(dim-k) <= N_ev/4 */
        int64_t p = 1;
        int ok = 1;
        for (int mu = 0; mu < dim && ok; ++mu) {
            const int64_t s = mu < k ? n + 1 : n;
            if (p > limit / s) ok = 0;
            else p *= s;
        }
        if (ok && p <= limit) d = k;
        else break;
    }
    for (int mu = 0; mu < dim; ++mu) nst_ax[mu] = mu < d ? n + 1 : n;
}

void or_nstrat_mixed(int dim, int64_t n_ev, int64_t *nst_ax) {
    or_nstrat_mixed_div(dim, n_ev, 4, nst_ax);
}

/* ------------------------------------------------------------------------ */
/* Integrands (the paper's example families, written out in FP64).           */
/* Parameter blob layouts (doubles):                                          */
/*  kind 0 gaussian peaks  §2.4 Eq. (easy):  [K, {a, w, c[D]} x K]            */
/*         f = sum_k a_k exp(-sum_mu (x_mu - c_k,mu)^2 / w_k^2)               */
/*  kind 1 balls           §2.4 Eq. (balls): [K, {a, r, c[D]} x K]            */
/*         f = sum_k a_k Theta(|x - c_k| < r_k)                                */
/*  kind 2 exp-norm peaks  §3.1 Eq. (exponentials): [K, {a, s, c[D]} x K]     */
/*         f = sum_k a_k exp(-s_k |x - c_k|)                                   */
/*  kind 3 posterior       App. B Eqs. (posterior, prior):                     */
/*         [n, P, G, sigma_y, prior_width, log_ref, y[n], A[n][P]], D = P + G; */
/*         x = (c_0..c_{P-1}, w_0..w_{G-1}); model_i = sum_m A[i][m] c_m;     */
/*         point i has the outlier weight w = w_{i mod G} (G = 1: one shared   */
/*         w, the first example of App. B; one per point: its second);        */
/*         P_i = (1-w)/(sqrt(2pi) s) e^{-r^2/2s^2} + w/(sqrt(2pi) 10 s) e^{-r^2/200 s^2} */
/*         f = exp(sum_i log P_i - sum_m c_m^2 / (2 pw^2) - log_ref)           */
/* ------------------------------------------------------------------------ */
double or_integrand(int kind, int dim, const double *prm, const double *x) {
    if (kind == 0 || kind == 1 || kind == 2) {
        int npk = (int)prm[0];
        const double *p = prm + 1;
        double f = 0.0;
        for (int k = 0; k < npk; ++k) {
            double a = p[0], w = p[1];
            const double *c = p + 2;
            double r2 = 0.0;
            for (int mu = 0; mu < dim; ++mu) {
                double dx = x[mu] - c[mu];
                r2 += dx * dx;
            }
            if (kind == 0) f += a * exp(-r2 / (w * w));
            else if (kind == 1) f += (r2 < w * w) ? a : 0.0;   /* w holds the radius */
            else f += a * exp(-w * sqrt(r2));                   /* w holds the slope s */
            p += 2 + dim;
        }
        return f;
    }
    if (kind == 3) {
        int n = (int)prm[0], npar = (int)prm[1], ngrp = (int)prm[2];
        double sy = prm[3], pw = prm[4], log_ref = prm[5];
        const double *y = prm + 6;
        const double *A = prm + 6 + n;
        const double two_pi = 6.283185307179586476925286766559;
        double logl = 0.0;
        for (int i = 0; i < n; ++i) {
            double w = x[npar + i % ngrp];
            double model = 0.0;
            for (int m = 0; m < npar; ++m) model += A[i * npar + m] * x[m];
            double r = y[i] - model;
            double narrow = (1.0 - w) / (sqrt(two_pi) * sy) * exp(-r * r / (2.0 * sy * sy));
            double wide = w / (sqrt(two_pi) * 10.0 * sy) * exp(-r * r / (200.0 * sy * sy));
            logl += log(narrow + wide);
        }
        double logprior = 0.0;
        for (int m = 0; m < npar; ++m) logprior -= x[m] * x[m] / (2.0 * pw * pw);
        return exp(logl + logprior - log_ref);
    }
    return NAN;
}

/* The integrand at n points X[n][dim] (row-major), for quadrature checks. */
void or_integrand_many(int kind, int dim, const double *prm, int64_t n, const double *X,
                       double *out) {
    for (int64_t p = 0; p < n; ++p) out[p] = or_integrand(kind, dim, prm, X + p * dim);
}

/* ------------------------------------------------------------------------ */
/* One sample: §3 (stratified y in hypercube h), §2.2 Eqs. (y), (jac),        */
/* §2.4 Eq. (y-Dspace).                                                       */
/* reading (counter layout): Philox key = (seed_lo, seed_hi); counter =       */
/*   (j*ceil(D/4) + q, h, t, integral_id); lanes 0..3 of call q give axes     */
/*   4q..4q+3.                                                                */
/* reading (uniform): u = (r + 1/2) 2^-32 from one 32-bit word r, so          */
/*   0 < u < 1 strictly, as §2.4 requires of y.                                */
/* The grid for axis mu is edges[mu*(N_g+1) + 0..N_g], edges[0] = a,          */
/* edges[N_g] = b.                                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dim;
    int n_g;
    const int64_t *nst_ax; /* strata per axis (§3; §3.2 allows them to differ) */
    uint64_t seed;
    uint32_t integral_id;
    const double *edges;
    int kind;
    const double *prm;
} or_problem;

/* Fills x[dim], idx[dim]; returns J and writes f. */
static double or_sample(const or_problem *P, uint32_t t, uint64_t h, uint32_t j,
                        double *x, int *idx, double *f_out) {
    int dim = P->dim, n_g = P->n_g;
    uint32_t calls = (uint32_t)((dim + 3) / 4);
    uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};
    double jac = 1.0;
    uint64_t rest = h; /* mixed-radix digits of h: axis 0 least significant */
    for (uint32_t q = 0; q < calls; ++q) {
        uint32_t ctr[4] = {j * calls + q, (uint32_t)h, t, P->integral_id};
        uint32_t r[4];
        or_philox4x32_10(ctr, key, r);
        for (int lane = 0; lane < 4; ++lane) {
            int mu = (int)(4 * q) + lane;
            if (mu >= dim) break;
            const uint64_t s_mu = (uint64_t)P->nst_ax[mu];
            int64_t k_mu = (int64_t)(rest % s_mu);
            rest /= s_mu;
            double u = ((double)r[lane] + 0.5) * (1.0 / 4294967296.0);
            double y = ((double)k_mu + u) / (double)s_mu; /* point in stratum k_mu of axis mu */
            double yng = y * (double)n_g;
            int i = (int)floor(yng); /* i(y) = floor(y N_g) */
            if (i > n_g - 1) i = n_g - 1;
            double delta = yng - (double)i; /* delta(y) = y N_g - i(y) */
            const double *e = P->edges + (size_t)mu * (size_t)(n_g + 1);
            double dx = e[i + 1] - e[i];
            x[mu] = e[i] + dx * delta;          /* Eq. (y) */
            jac *= (double)n_g * dx;            /* Eq. (jac), product over axes */
            idx[mu] = i;
        }
    }
    *f_out = or_integrand(P->kind, dim, P->prm, x);
    return jac;
}

/* Per-sample inspection: x[dim], idx[dim], jac, f for sample j of hypercube h. */
void or_eval_sample(int dim, int n_g, const int64_t *nst_ax, uint64_t seed, uint32_t integral_id,
                    const double *edges, int kind, const double *prm, uint32_t t,
                    uint64_t h, uint32_t j, double *x, int *idx, double *jac, double *f) {
    or_problem P = {dim, n_g, nst_ax, seed, integral_id, edges, kind, prm};
    *jac = or_sample(&P, t, h, j, x, idx, f);
}

/* ------------------------------------------------------------------------ */
/* Steps a1-a5 of one iteration (§2.3, §2.4, §3 step 2): for every hypercube h */
/* in order and every sample j < n_h in order, accumulate                     */
/*   S1_h = sum J f,  S2_h = sum (J f)^2                        (§3 step 2)   */
/*   hsum[mu][i] += (J f)^2,  hcnt[mu][i] += 1                  (§2.4, d_i^mu) */
/* or, with d_weighted (reading: each sample weighted by its hypercube's      */
/* y-volume per sample, Omega_h / n_h, Omega_h being the same for every        */
/* hypercube and dropped since d is normalised), hsum[mu][i] += (J f)^2 / n_h, */
/* an estimate of the slab integral of J^2 f^2 whatever the allocation (§3:   */
/* the optimal map does not depend on the allocation of samples).             */
/* All outputs are overwritten.                                               */
/* ------------------------------------------------------------------------ */
int or_sample_iteration(int dim, int n_g, const int64_t *nst_ax, uint64_t seed,
                        uint32_t integral_id, const double *edges, int kind, const double *prm,
                        uint32_t t, const uint32_t *n_h, double *s1, double *s2, double *hsum,
                        double *hcnt, int d_weighted) {
    or_problem P = {dim, n_g, nst_ax, seed, integral_id, edges, kind, prm};
    int64_t n_hc = 1;
    for (int mu = 0; mu < dim; ++mu) n_hc *= nst_ax[mu];
    memset(hsum, 0, sizeof(double) * (size_t)dim * (size_t)n_g);
    memset(hcnt, 0, sizeof(double) * (size_t)dim * (size_t)n_g);
    double x[64];
    int idx[64];
    if (dim > 64) return -1;
    for (int64_t h = 0; h < n_hc; ++h) {
        double a1 = 0.0, a2 = 0.0;
        for (uint32_t j = 0; j < n_h[h]; ++j) {
            double f;
            double jac = or_sample(&P, t, (uint64_t)h, j, x, idx, &f);
            double jf = jac * f;
            a1 += jf;
            a2 += jf * jf;
            const double w = d_weighted ? jf * jf / (double)n_h[h] : jf * jf;
            for (int mu = 0; mu < dim; ++mu) {
                hsum[(size_t)mu * n_g + idx[mu]] += w;
                hcnt[(size_t)mu * n_g + idx[mu]] += 1.0;
            }
        }
        s1[h] = a1;
        s2[h] = a2;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* App. B (several integrals from the same samples): outputs k = 0 .. M-1  */
/* v_k = J f g_k(x), g_k(x) = x^a x^b for the pair (a, b) = mono[2k], mono[2k+1] */
/* (a or b < 0: that factor is 1; output 0 is f itself, mono = (-1, -1)).      */
/* Per hypercube, in sample order:                                             */
/*   X1_h[k] = sum_j v_k,   X2_h[k,l] = sum_j v_k v_l  (k <= l)                */
/* X2 is stored as the upper triangle row by row: T = M (M + 1) / 2 entries,   */
/* (k, l) at k M - k (k - 1) / 2 + (l - k).  Overwrites x1 [n_hc][M] and      */
/* x2 [n_hc][T].                                                              */
/* ------------------------------------------------------------------------ */
static int or_tri(int M, int k, int l) { return k * M - k * (k - 1) / 2 + (l - k); }
double or_tree_sum(const double *v, int64_t n); /* below: the fixed summation order */

int or_sample_multi(int dim, int n_g, const int64_t *nst_ax, uint64_t seed, uint32_t integral_id,
                    const double *edges, int kind, const double *prm, uint32_t t,
                    const uint32_t *n_h, int M, const int32_t *mono, double *x1, double *x2) {
    or_problem P = {dim, n_g, nst_ax, seed, integral_id, edges, kind, prm};
    int64_t n_hc = 1;
    for (int mu = 0; mu < dim; ++mu) n_hc *= nst_ax[mu];
    const int T = M * (M + 1) / 2;
    double x[64], v[64];
    int idx[64];
    if (dim > 64 || M > 64) return -1;
    for (int64_t h = 0; h < n_hc; ++h) {
        double *a1 = x1 + (size_t)h * M, *a2 = x2 + (size_t)h * T;
        for (int k = 0; k < M; ++k) a1[k] = 0.0;
        for (int q = 0; q < T; ++q) a2[q] = 0.0;
        for (uint32_t j = 0; j < n_h[h]; ++j) {
            double f;
            double jf = or_sample(&P, t, (uint64_t)h, j, x, idx, &f) * f;
            for (int k = 0; k < M; ++k) {
                const int a = mono[2 * k], b = mono[2 * k + 1];
                const double g = (a >= 0 ? x[a] : 1.0) * (b >= 0 ? x[b] : 1.0);
                v[k] = jf * g;
            }
            for (int k = 0; k < M; ++k) {
                a1[k] += v[k];
                for (int l = k; l < M; ++l) a2[or_tri(M, k, l)] += v[k] * v[l];
            }
        }
    }
    return 0;
}

/* App. B with §2.1 Eq. (sigest) in its several-variable form, per hypercube, and */
/* §3 Eq. (sumI) over hypercubes:                                            */
/*   I[k]     = sum_h Omega X1_h[k] / n_h                                    */
/*   C[k][l]  = sum_h Omega^2 (X2_h[k,l]/n_h - (X1_h[k]/n_h)(X1_h[l]/n_h))   */
/*                      / (n_h - 1)                                          */
/* each sum in the fixed order of or_tree_sum; the diagonal terms clamped at   */
/* zero as the scalar variance is (reading).  out_c is M x M, symmetric.      */
void or_estimate_multi(int64_t n_hc, double omega, int M, const double *x1, const double *x2,
                       const uint32_t *n_h, double *work, double *out_i, double *out_c) {
    const int T = M * (M + 1) / 2;
    for (int k = 0; k < M; ++k) {
        for (int64_t h = 0; h < n_hc; ++h)
            work[h] = omega * (x1[(size_t)h * M + k] / (double)n_h[h]);
        out_i[k] = or_tree_sum(work, n_hc);
    }
    for (int k = 0; k < M; ++k)
        for (int l = k; l < M; ++l) {
            for (int64_t h = 0; h < n_hc; ++h) {
                const double n = (double)n_h[h];
                const double mk = x1[(size_t)h * M + k] / n, ml = x1[(size_t)h * M + l] / n;
                double c = x2[(size_t)h * T + or_tri(M, k, l)] / n - mk * ml;
                if (k == l && c < 0.0) c = 0.0;
                work[h] = omega * omega * c / (n - 1.0);
            }
            out_c[k * M + l] = out_c[l * M + k] = or_tree_sum(work, n_hc);
        }
}

/* S1_h, S2_h of one hypercube h with n samples (for spot checks at sizes  */
/* where a whole iteration is too slow on the CPU).                          */
void or_hcube_moments(int dim, int n_g, const int64_t *nst_ax, uint64_t seed,
                      uint32_t integral_id, const double *edges, int kind, const double *prm,
                      uint32_t t, uint64_t h, uint32_t n, double *s1, double *s2) {
    or_problem P = {dim, n_g, nst_ax, seed, integral_id, edges, kind, prm};
    double x[64];
    int idx[64];
    double a1 = 0.0, a2 = 0.0;
    for (uint32_t j = 0; j < n; ++j) {
        double f;
        double jf = or_sample(&P, t, h, j, x, idx, &f) * f;
        a1 += jf;
        a2 += jf * jf;
    }
    *s1 = a1;
    *s2 = a2;
}

/* ------------------------------------------------------------------------ */
/* reading (summation order): every sum over hypercubes is taken in one fixed */
/* order -- blocks of 1024 consecutive terms, each summed by pairwise halving */
/* (term i += term i+s for s = 512, 256, ..., 1; missing terms are zero), and  */
/* the block sums combined by an adjacent pairwise tree: P leaves, P the least */
/* power of two >= the number of blocks, leaves past the last block zero,      */
/* level by level (leaf 2i += leaf 2i+1, then 4i += 4i+2, ...).  This order    */
/* makes sum_h d_h, and hence the integer n_h, reproducible bit for bit.      */
/* ------------------------------------------------------------------------ */
double or_tree_sum(const double *v, int64_t n) {
    if (n <= 0) return 0.0;
    const int64_t nb = (n + 1023) / 1024;
    int64_t P = 1;
    while (P < nb) P <<= 1;
    double *bs = (double *)calloc((size_t)P, sizeof(double));
    double blk[1024];
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t base = b * 1024;
        for (int i = 0; i < 1024; ++i) blk[i] = (base + i < n) ? v[base + i] : 0.0;
        for (int s = 512; s >= 1; s >>= 1)
            for (int i = 0; i < s; ++i) blk[i] = blk[i] + blk[i + s];
        bs[b] = blk[0];
    }
    for (int64_t w = 1; w < P; w <<= 1)
        for (int64_t i = 0; i < P; i += 2 * w) bs[i] = bs[i] + bs[i + w];
    const double total = bs[0];
    free(bs);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Step a6: the iteration's estimate (§3 Eq. (sumI), with the per-hypercube   */
/* simple-MC estimates of §2.1 Eqs. (MCIy), (sigest) applied inside each      */
/* hypercube of y-volume Omega = N_st^-D):                                    */
/*   dI_h  = Omega S1_h / n_h                                                 */
/*   var_h = Omega^2 (S2_h/n_h - (S1_h/n_h)^2) / (n_h - 1)                    */
/*   I = sum_h dI_h,  sigma^2 = sum_h var_h                                   */
/* reading: var_h is clamped at zero against rounding; n_h >= 2 always.       */
/* ------------------------------------------------------------------------ */
void or_estimate(int64_t n_hc, double omega, const double *s1, const double *s2,
                 const uint32_t *n_h, double *work, double *out_i, double *out_var) {
    for (int64_t h = 0; h < n_hc; ++h) work[h] = omega * (s1[h] / (double)n_h[h]);
    *out_i = or_tree_sum(work, n_hc);
    for (int64_t h = 0; h < n_hc; ++h) {
        double n = (double)n_h[h];
        double m1 = s1[h] / n, m2 = s2[h] / n;
        double v = m2 - m1 * m1;
        if (v < 0.0) v = 0.0;
        work[h] = omega * omega * v / (n - 1.0);
    }
    *out_var = or_tree_sum(work, n_hc);
}

/* §3 step 2: sigma_h(Jf) from the same samples,                              */
/*   sigma_h^2 = Omega^2/n_h sum (Jf)^2 - (Omega/n_h sum Jf)^2 (clamped >= 0). */
void or_sigma(int64_t n_hc, double omega, const double *s1, const double *s2,
              const uint32_t *n_h, double *sigma) {
    for (int64_t h = 0; h < n_hc; ++h) {
        double n = (double)n_h[h];
        double a = omega * omega / n * s2[h];
        double b = omega / n * s1[h];
        double v = a - b * b;
        sigma[h] = v > 0.0 ? sqrt(v) : 0.0;
    }
}

/* §3 step 3, Eq. (dh): d_h = sigma_h^beta (beta = 0 gives d_h = 1, beta = 1   */
/* gives d_h = sigma_h, both exactly).                                         */
/* reading: the powers 1/2 and 3/4 (the paper's default beta) are taken as     */
/* correctly rounded IEEE square roots, sigma^(1/2) = sqrt(sigma) and          */
/* sigma^(3/4) = sqrt(sigma * sqrt(sigma)) (two roots, one product, each       */
/* rounded once), so that the result is one fixed IEEE sequence on every       */
/* machine; any other beta goes through pow.                                   */
void or_damp(int64_t n_hc, double beta, const double *sigma, double *d) {
    for (int64_t h = 0; h < n_hc; ++h) {
        if (beta == 0.0) d[h] = 1.0;
        else if (beta == 1.0) d[h] = sigma[h];
        else if (beta == 0.5) d[h] = sqrt(sigma[h]);
        else if (beta == 0.75) {
            double r = sqrt(sigma[h]);
            d[h] = sqrt(sigma[h] * r);
        } else d[h] = pow(sigma[h], beta);
    }
}

/* §3 step 4, Eq. (nh): n_h = max(2, N_ev d_h / sum d)  (plus2 = 0), or the    */
/* alternative n_h = N_ev d_h / sum d + 2 (plus2 = 1).                         */
/* reading: the real quotient is formed as (N_ev * d_h) / sum_d in IEEE FP64   */
/* and floored, except that a quotient within 2^-50 q below the next integer   */
/* counts as that integer (a quotient that is an integer in exact arithmetic,  */
/* e.g. N_ev when there is one hypercube, must not be decided by the last bit  */
/* of d_h); if sum_d is zero every hypercube gets max(2, floor(N_ev/N_h)).     */
/* Offsets are the exclusive prefix sums of n_h; offsets[N_h] = samples used.  */
/* Returns 1 if a d_h or sum_d is not finite (nothing written), else 0.       */
int or_allocate(int64_t n_hc, int64_t n_ev, int plus2, const double *d, uint32_t *n_h,
                uint64_t *offsets) {
    double sum_d = or_tree_sum(d, n_hc);
    if (!isfinite(sum_d)) return 1;
    for (int64_t h = 0; h < n_hc; ++h) {
        double q;
        if (sum_d > 0.0) {
            q = (double)n_ev * d[h];
            q = q / sum_d;
        } else {
            q = (double)n_ev / (double)n_hc;
        }
        double fl = floor(q);
        if ((fl + 1.0) - q <= q * 8.8817841970012523e-16) fl = fl + 1.0; /* 2^-50 q */
        int64_t n;
        if (plus2) n = (int64_t)fl + 2;
        else n = fl > 2.0 ? (int64_t)fl : 2;
        n_h[h] = (uint32_t)n;
    }
    uint64_t run = 0;
    for (int64_t h = 0; h < n_hc; ++h) {
        offsets[h] = run;
        run += n_h[h];
    }
    offsets[n_hc] = run;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Step a8: refinement of one axis's grid, §2.3, in the paper's order.        */
/* ------------------------------------------------------------------------ */

/* d_i = hsum_i / hcnt_i (reading: 0 when the increment got no sample; with   */
/* d_weighted, hsum_i itself: its samples are already weighted), then         */
/* the smoothing (7,1)/8, (1,6,1)/8, (1,7)/8 with division by sum_i d_i, then  */
/* the compression d_i -> ((1 - d_i)/ln(1/d_i))^alpha (reading: 1 at d_i = 1;  */
/* a smoothed d_i of zero is raised to the smallest normal double first, so    */
/* that, as for alpha -> 0 "no refinement", an increment nobody sampled keeps  */
/* a small nonzero share instead of vanishing from the grid).  Returns 0, or 1 */
/* when every d_i is zero (or the sum is not finite): nothing to refine.       */
/* Needs n_g >= 2.                                                             */
int or_smooth_compress(int n_g, const double *hsum, const double *hcnt, double alpha,
                       double *out, double *work, int d_weighted) {
    double *d = work;
    double sum_d = 0.0;
    for (int i = 0; i < n_g; ++i) {
        d[i] = hcnt[i] > 0.0 ? (d_weighted ? hsum[i] : hsum[i] / hcnt[i]) : 0.0;
        sum_d += d[i];
    }
    if (!(sum_d > 0.0) || !isfinite(sum_d)) return 1;
    out[0] = (7.0 * d[0] + d[1]) / 8.0;
    for (int i = 1; i < n_g - 1; ++i) out[i] = (d[i - 1] + 6.0 * d[i] + d[i + 1]) / 8.0;
    out[n_g - 1] = (d[n_g - 2] + 7.0 * d[n_g - 1]) / 8.0;
    for (int i = 0; i < n_g; ++i) out[i] = out[i] / sum_d;
    for (int i = 0; i < n_g; ++i) {
        double v = out[i];
        if (v <= 0.0) v = 2.2250738585072014e-308; /* smallest normal double */
        if (v == 1.0) out[i] = 1.0;
        else out[i] = pow((1.0 - v) / log(1.0 / v), alpha);
    }
    return 0;
}

/* The four-step re-gridding of §2.3: new increments each holding an equal    */
/* share delta_d = sum_i d_i / N_g of d, with d_i spread uniformly over the    */
/* old increment i; walks i (new edge), j (old edge) and S_d as the paper      */
/* does.  x and x_new hold N_g + 1 edges and may not alias.                    */
void or_regrid(int n_g, const double *x, const double *d, double *x_new) {
    /* Step 1 */
    double total = 0.0;
    for (int i = 0; i < n_g; ++i) total += d[i];
    double delta_d = total / (double)n_g;
    x_new[0] = x[0];
    x_new[n_g] = x[n_g];
    int i = 0, j = 0;
    double s_d = 0.0;
    for (;;) {
        i += 1; /* Step 2 */
        if (i >= n_g) break;
        while (s_d < delta_d && j < n_g) { /* Step 3 */
            s_d += d[j];
            j += 1;
        }
        s_d -= delta_d; /* Step 4 */
        x_new[i] = x[j] - (s_d / d[j - 1]) * (x[j] - x[j - 1]);
    }
}

/* ------------------------------------------------------------------------ */
/* §4.2 (preconditioned integrators): the map trained on sample data          */
/* {x, f(x)} given before integrating.  The inverse map y(x): on axis mu, the */
/* increment i with x_i <= x < x_{i+1} (the last increment also takes x = b), */
/* y = (i + (x - x_i) / dx_i) / N_g; J(y(x)) is Eq. (jac) there, the product  */
/* over axes of N_g dx_i.  The data histogram is that of §2.3/§2.4 with the   */
/* sum over the data in place of the sum over samples:                        */
/*   hsum[mu][i] += J^2 f^2 = (J f)^2,  hcnt[mu][i] += 1                       */
/* (overwrites hsum, hcnt; x [n][dim] inside the box).                        */
/* ------------------------------------------------------------------------ */
static int or_increment(int n_g, const double *e, double x) {
    int lo = 0, hi = n_g; /* e[lo] <= x < e[hi], or x = e[n_g] */
    if (x >= e[n_g]) return n_g - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (e[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

void or_inverse_map(int dim, int n_g, const double *edges, const double *x, int *idx,
                    double *y, double *jac) {
    double J = 1.0;
    for (int mu = 0; mu < dim; ++mu) {
        const double *e = edges + (size_t)mu * (size_t)(n_g + 1);
        const int i = or_increment(n_g, e, x[mu]);
        const double dx = e[i + 1] - e[i];
        idx[mu] = i;
        y[mu] = ((double)i + (x[mu] - e[i]) / dx) / (double)n_g;
        J *= (double)n_g * dx;
    }
    *jac = J;
}

void or_precondition_hist(int dim, int n_g, const double *edges, int64_t n, const double *x,
                          const double *f, double *hsum, double *hcnt) {
    int idx[64];
    double y[64];
    memset(hsum, 0, sizeof(double) * (size_t)dim * (size_t)n_g);
    memset(hcnt, 0, sizeof(double) * (size_t)dim * (size_t)n_g);
    if (dim > 64) return;
    for (int64_t p = 0; p < n; ++p) {
        double jac;
        or_inverse_map(dim, n_g, edges, x + (size_t)p * dim, idx, y, &jac);
        const double jf = jac * f[p];
        for (int mu = 0; mu < dim; ++mu) {
            hsum[(size_t)mu * n_g + idx[mu]] += jf * jf;
            hcnt[(size_t)mu * n_g + idx[mu]] += 1.0;
        }
    }
}

/* The whole refinement of one axis.  alpha = 0 means no refinement (§2.3);   */
/* N_g = 1 or all-zero d_i leave the grid unchanged (reading).  work holds     */
/* 2 N_g doubles.                                                             */
void or_refine_axis(int n_g, const double *edges_in, const double *hsum, const double *hcnt,
                    double alpha, double *edges_out, double *work, int d_weighted) {
    for (int i = 0; i <= n_g; ++i) edges_out[i] = edges_in[i];
    if (alpha == 0.0 || n_g < 2) return;
    double *sm = work + n_g;
    if (or_smooth_compress(n_g, hsum, hcnt, alpha, sm, work, d_weighted) != 0) return;
    or_regrid(n_g, edges_in, sm, edges_out);
}
