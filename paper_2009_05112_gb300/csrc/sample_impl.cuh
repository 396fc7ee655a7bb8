// sample_impl.cuh -- the fused sampling kernel of one vegas+ iteration
// (steps a1-a5) and its per-sample inspection twin.
//
// Per sample j of hypercube h (§3: N_st strata per axis, h = sum_mu k_mu N_st^mu):
//   a1  y^mu = (k_mu + u^mu) / N_st, u from Philox4x32-10 with counter
//       (j ceil(D/4) + q, h, t, integral_id): no per-sample memory traffic;
//   a2  i = floor(y N_g), delta = y N_g - i, x = x_i + dx_i delta,
//       J = prod_mu N_g dx_i   (§2.2 Eqs. y, jac; §2.4 Eq. y-Dspace);
//   a3  f(x) (integrand family, device functor);
//   a4  S1_h += J f, S2_h += (J f)^2 (§3 step 2), accumulated per thread over
//       its run of consecutive samples (Kahan-compensated in FP32) and flushed
//       to FP64 with one atomic add per hypercube touched;
//   a5  hsum[mu][i] += (J f)^2, hcnt[mu][i] += 1 (§2.3 d_i, §2.4 d_i^mu), in a
//       per-CTA shared-memory copy flushed with global atomics when the CTA
//       moves to another integral or finishes.
//
// Work decomposition: a persistent grid pulls chunks of C = blockDim.x * R
// consecutive samples from a device queue; each thread owns R consecutive
// samples of its chunk, so per-hypercube sums stay in registers and the
// hypercube index is found once per run.  Samples of an integral are laid out
// hypercube by hypercube through the offsets off[h] (a7), so chunks are equal
// in samples however uneven n_h is.
#pragma once

#include <cooperative_groups.h>

#include "vp_internal.cuh"

namespace vp {

// Histogram layouts of the sampling kernels:
//   kHistGlobal   FP64 sums and counts with global atomics per sample;
//   kHistShared   per CTA in shared memory, per bin an FP64 sum (FP64 path) or
//                 an FP32 sum and an FP32 tiny-term sum (FP32 path), and a
//                 count: 12 B;
//   kHistCompact  (one-integral kernel, FP32) an FP32 sum and a count, 8 B;
//                 tiny terms go to the global FP64 sums.
constexpr int kHistGlobal = 0, kHistShared = 1, kHistCompact = 2;
// dynamic shared memory the one-integral kernel may use (one CTA per SM)
constexpr size_t kOneSmemMax = 220 * 1024;

// Launch arguments when the launch serves several integrals (tasks).
struct SampleArgs {
    const Desc *desc;          // [n_int] descriptors of the whole set
    const uint32_t *members;   // [n_group] set indices served by this launch
    const uint64_t *chunk_base;// [n_group + 1] prefix of tasks
    uint32_t *head;            // queue head (tasks)
    uint32_t *exit_count;      // CTAs finished; the last one resets head and itself
    int n_group;
    int r;                     // samples per thread per warp chunk
    uint32_t task;             // samples per task
    int hist_shared;           // histograms privatised in shared memory
    int hist_words;            // dim * n_g bins reserved in shared memory
    int prm_words;             // 4-byte words reserved for integrand constants
};

template <bool F64> struct Real;
template <> struct Real<true> { typedef double T; };
template <> struct Real<false> { typedef float T; };

// ---------------------------------------------------------------------------
// Integrands.  FP64 versions follow the blob (see vegasp.h) in IEEE-rounded
// steps; FP32 versions use constants prepared on the host (prm32):
//  GAUSS    per peak {a, log2(e)/w^2, 0, 0, c[D], pad}  f = sum a 2^(-k |x-c|^2)
//  BALL     per peak {a, r^2, 0, 0, c[D], pad}          f = sum a [|x-c|^2 < r^2]
//  EXPNORM  per peak {a, s log2(e), 0, 0, c[D], pad}    f = sum a 2^(-k |x-c|)
//           (peaks padded to a multiple of 4 floats for 16-byte shared loads)
//  POSTERIOR {n, P, G, kN, kW, lcN, lcW, kprior, logref2, y[n], A[n][P]} in log2 units
// ---------------------------------------------------------------------------
template <int DMAX>
__device__ __forceinline__ double f_peaks64(int kind, const double *p, int K, int dim,
                                            const double (&x)[DMAX]) {
    double f = 0.0;
    for (int k = 0; k < K; ++k) {
        const double a = p[0], w = p[1];
        const double *c = p + 2;
        double r2 = 0.0;
#pragma unroll
        for (int mu = 0; mu < DMAX; ++mu) {
            if (mu < dim) {
                double dx = __dsub_rn(x[mu], c[mu]);
                r2 = __dadd_rn(r2, __dmul_rn(dx, dx));
            }
        }
        if (kind == VP_GAUSS) f += a * exp(__ddiv_rn(-r2, __dmul_rn(w, w)));
        else if (kind == VP_BALL) f += (r2 < __dmul_rn(w, w)) ? a : 0.0;
        else f += a * exp(-w * sqrt(r2));
        p += 2 + dim;
    }
    return f;
}

template <int DMAX>
__device__ __forceinline__ float f_peaks32(int kind, const float *p, int K, int dim,
                                           const float (&x)[DMAX]) {
    // per peak: {a, k, 0, 0, c_0 .. c_{D-1}, pad to 4} in shared memory
    const int stride = 4 + ((dim + 3) & ~3);
    float f = 0.0f;
    for (int k = 0; k < K; ++k, p += stride) {
        const float4 hd = *(const float4 *)p;
        float r2 = 0.0f;
#pragma unroll
        for (int m4 = 0; m4 < DMAX; m4 += 4) {
            if (m4 < dim) {
                const float4 c = *(const float4 *)(p + 4 + m4);
                const float cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    if (m4 + l < DMAX && m4 + l < dim) {
                        const float dx = x[m4 + l] - cc[l];
                        r2 = fmaf(dx, dx, r2);
                    }
                }
            }
        }
        if (kind == VP_GAUSS) f = fmaf(hd.x, ex2_approx(-hd.y * r2), f);
        else if (kind == VP_BALL) f += (r2 < hd.y) ? hd.x : 0.0f;
        else f = fmaf(hd.x, ex2_approx(-hd.y * sqrtf(r2)), f);
    }
    return f;
}

// Peak families with their constants in the kernel parameters (one-integral
// kernel, FP32, K <= kParamPeaks): per peak {a, k, c_0 .. c_{kMaxDim-1}} at a
// fixed stride, read as constant-bank operands (every index is a compile-time
// constant once the loops are unrolled), with the same operations in the same
// order as f_peaks32.
constexpr int kParamPeaks = 8;
constexpr int kParamStride = 2 + kMaxDim;

template <int DMAX, int KIND>
__device__ __forceinline__ float f_peaks32_param(const float *kp, int K, int dim,
                                                 const float (&x)[DMAX]) {
    float f = 0.0f;
#pragma unroll
    for (int k = 0; k < kParamPeaks; ++k) {
        if (k < K) {
            const float *p = kp + k * kParamStride;
            float r2 = 0.0f;
#pragma unroll
            for (int mu = 0; mu < DMAX; ++mu) {
                if (mu < dim) {
                    const float dx = x[mu] - p[2 + mu];
                    r2 = fmaf(dx, dx, r2);
                }
            }
            if (KIND == VP_GAUSS) f = fmaf(p[0], ex2_approx(-p[1] * r2), f);
            else if (KIND == VP_BALL) f += (r2 < p[1]) ? p[0] : 0.0f;
            else f = fmaf(p[0], ex2_approx(-p[1] * sqrtf(r2)), f);
        }
    }
    return f;
}

template <int DMAX>
__device__ __forceinline__ double f_post64(const double *p, int dim, const double (&x)[DMAX]) {
    const int n = (int)p[0], npar = (int)p[1], ngrp = (int)p[2];
    const double sy = p[3], pw = p[4], log_ref = p[5];
    const double *y = p + 6;
    const double *A = p + 6 + n;
    const double s2pi = sqrt(6.283185307179586476925286766559);  // sqrt(2 pi)
    double logl = 0.0;
    int g = 0;  // i mod G
    for (int i = 0; i < n; ++i) {
        double w = 0.0;
#pragma unroll
        for (int mu = 0; mu < DMAX; ++mu)
            if (mu == npar + g) w = x[mu];
        double model = 0.0;
#pragma unroll
        for (int m = 0; m < DMAX; ++m)
            if (m < npar) model += A[i * npar + m] * x[m];
        const double r = y[i] - model;
        const double nar = (1.0 - w) / (s2pi * sy) * exp(-r * r / (2.0 * sy * sy));
        const double wid = w / (s2pi * 10.0 * sy) * exp(-r * r / (200.0 * sy * sy));
        logl += log(nar + wid);
        if (++g == ngrp) g = 0;
    }
    double lp = 0.0;
#pragma unroll
    for (int m = 0; m < DMAX; ++m)
        if (m < npar) lp -= x[m] * x[m] / (2.0 * pw * pw);
    (void)dim;
    return exp(logl + lp - log_ref);
}

// FP32: the points are visited group by group (points g, g + G, g + 2G, ...
// share the weight w_g), so that each w_g is read from a fixed register.
// Returns log2 f: a posterior's values span hundreds of binary orders below
// its maximum (a sharp 21-parameter one integrates to ~1e-28), far beyond the
// FP32 range, so f is formed by the caller as a mantissa and an exponent.
template <int DMAX>
__device__ __forceinline__ float f_post32_log2(const float *p, int dim, const float (&x)[DMAX]) {
    const int n = (int)p[0], npar = (int)p[1], ngrp = (int)p[2];
    const float kN = p[3], kW = p[4], lcN = p[5], lcW = p[6], kpr = p[7], lref = p[8];
    const float *y = p + 9;
    const float *A = p + 9 + n;
    float acc = 0.0f;
#pragma unroll
    for (int mu = 1; mu < DMAX; ++mu) {
        if (mu < npar || mu >= npar + ngrp) continue;
        const float w = x[mu];
        const float lw1 = lg2_approx(1.0f - w), lw = lg2_approx(w);
        for (int i = mu - npar; i < n; i += ngrp) {
            const float *a = A + i * npar;
            float model = 0.0f;
#pragma unroll
            for (int m = 0; m < DMAX; ++m)
                if (m < npar) model = fmaf(a[m], x[m], model);
            const float r = y[i] - model;
            const float r2 = r * r;
            const float nar = ex2_approx(fmaf(-kN, r2, lcN + lw1));
            const float wid = ex2_approx(fmaf(-kW, r2, lcW + lw));
            acc += lg2_approx(nar + wid);
        }
    }
    float c2 = 0.0f;
#pragma unroll
    for (int m = 0; m < DMAX; ++m)
        if (m < npar) c2 = fmaf(x[m], x[m], c2);
    (void)dim;
    return fmaf(-kpr, c2, acc - lref);
}

// ---------------------------------------------------------------------------
// One sample: a1-a3.  Returns J and f; x[] and idx[] are filled.
// digits kd[] hold k_mu of hypercube h as the real type.
// ---------------------------------------------------------------------------
// FP32 Jacobians of adapted high-dimensional maps leave the FP32 range (e.g.
// 20 axes of N_g dx ~ 3e-3 give 3e-51), so the FP32 path carries J as a
// mantissa in [1, 2) and a separate integer exponent, renormalised after
// every group of four axes (four factors dx_i cannot leave the range: each is
// at least ~ulp(x) and at most b - a).
__device__ __forceinline__ void renorm(float &m, int &e) {
    const int b = __float_as_int(m);
    const int ex = (b >> 23) & 0xff;
    if (ex != 0) {  // zero stays zero
        e += ex - 127;
        m = __int_as_float((b & 0x807fffff) | 0x3f800000);
    }
}

// x * 2^n for any int n, by two exact power-of-two multiplies.
__device__ __forceinline__ float scale2(float x, int n) {
    const int n1 = max(-126, min(127, n));
    const int n2 = max(-126, min(127, n - n1));
    return x * __int_as_float((n1 + 127) << 23) * __int_as_float((n2 + 127) << 23);
}

// Per-integral constants of the sampling loop, read once into registers.
struct Loop {
    int dim, n_g, K;
    uint32_t nst_magic;
    int nst_shift;
    uint32_t n_st, calls, iid, t;
    int dw;                     // the grid's d_i from samples weighted by 1/n_h
    uint32_t rk0[10], rk1[10];  // Philox round keys
    float c32;                  // N_g / N_st
    float ngm1;                 // N_g - 1
    float ngD_m;                // N_g^D = ngD_m 2^ngD_e
    int ngD_e;
    double nst, ng;
    const float2 *tab;
    const double *edges;
};

__device__ __forceinline__ Loop make_loop(const Desc *dp, uint32_t t) {
    Loop L;
    L.dim = __ldg(&dp->dim);
    L.n_g = __ldg(&dp->n_g);
    L.K = __ldg(&dp->n_peaks);
    L.n_st = __ldg(&dp->n_st);
    L.nst_magic = __ldg(&dp->nst_magic);
    L.nst_shift = __ldg(&dp->nst_shift);
    L.calls = (uint32_t)((L.dim + 3) >> 2);
    L.iid = __ldg(&dp->integral_id);
    L.dw = __ldg(&dp->d_weighted);
    L.t = t;
    uint32_t k0 = __ldg(&dp->key0), k1 = __ldg(&dp->key1);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        L.rk0[r] = k0;
        L.rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    L.c32 = __ldg(&dp->ng_over_nst);
    L.ngm1 = (float)(L.n_g - 1);
    L.ngD_m = __ldg(&dp->ngD_m);
    L.ngD_e = __ldg(&dp->ngD_e);
    L.nst = (double)L.n_st;
    L.ng = (double)L.n_g;
    L.tab = (const float2 *)__ldg((const unsigned long long *)&dp->tab);
    L.edges = (const double *)__ldg((const unsigned long long *)&dp->edges);
    return L;
}

// The dynamic tail of the one-integral kernel is split into kTailQueues
// equal queues, each with its own counter on its own 256-byte line: warps
// start at queue (warp mod kTailQueues) and move on when it runs dry, so that
// no single counter takes every warp's atomic (atomics on one address are
// served one at a time).
constexpr uint32_t kTailQueues = 32, kQueueStride = 64;

// Launch arguments when the launch serves one integral: its constants travel
// in the kernel parameters (constant bank), not in registers.
struct SampleOne {
    Loop L;                    // t is read from the device state at launch
    State *st;
    const uint64_t *off;
    const uint32_t *n_h;
    double *s1, *s2, *hsum;    // double-buffered bases
    uint32_t *hcnt;
    const float *prm32;
    const double *prm;
    uint64_t n_hc;
    uint32_t *head;            // the dynamic tail's kTailQueues counters, kQueueStride apart
    uint32_t *exit_count;      // CTAs finished; the last one resets the counters and itself
    int r;                     // samples per lane in a chunk of the dynamic tail
    // the share of the samples split statically over the warps, in 16ths
    // (16: all of them); the rest is pulled by warps in chunks of 32 r samples
    int static16;
    int hist_shared;           // kHist* layout of the histograms
    int bins;
    int prm_words;
    int kp_peaks;              // > 0: the peak constants are in kp (FP32 peak families)
    float kp[kParamPeaks * kParamStride];
    Strata S;                  // strata per axis (read as constants by the unrolled loops)
    // several integrals from the same samples (App. B; FP64 path): M outputs,
    // g_k = x^a x^b with (a, b) = mono[2k], mono[2k + 1]; output 0 is f
    int n_out;
    int32_t mono[2 * kMaxOut];
    double *x1, *x2;           // double-buffered bases [2][n_hc][M], [2][n_hc][M (M+1)/2]
    // one integral over several devices: this launch samples part `part` of
    // n_parts equal, contiguous ranges of the iteration's samples (n_parts <= 1:
    // all of them)
    int part, n_parts;
};

// Fire-and-forget global reductions.
__device__ __forceinline__ void red_add(double *p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add(uint32_t *p, uint32_t v) {
    asm volatile("red.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Philox4x32-10 with precomputed round keys (same function as philox4x32_10).
__device__ __forceinline__ U4 philox_rk(U4 c, const uint32_t (&k0)[10], const uint32_t (&k1)[10]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        const uint32_t hi0 = __umulhi(m0, c.a), lo0 = m0 * c.a;
        const uint32_t hi1 = __umulhi(m1, c.c), lo1 = m1 * c.c;
        U4 n;
        n.a = hi1 ^ c.b ^ k0[r];
        n.b = lo1;
        n.c = hi0 ^ c.d ^ k1[r];
        n.d = lo0;
        c = n;
    }
    return c;
}

// The strata constants of axis mu: per axis (AX, from S) or the one count
// every axis shares (from L).
template <bool AX>
__device__ __forceinline__ float c32_of(const Loop &L, const Strata *S, int mu) {
    return AX ? S->c32[mu] : L.c32;
}

// FP32 per-hypercube offsets kc[mu] = (k_mu - 1 + 2^-24) N_g/s_mu so that
// y N_g = (1 + m 2^-23) N_g/s_mu + kc with m = r >> 9, i.e. u = (m + 1/2) 2^-23.
template <int DMAX, bool AX>
__device__ __forceinline__ void hcube_offsets(const Loop &L, const Strata *S,
                                              const uint32_t (&kd)[DMAX], float (&kc)[DMAX]) {
#pragma unroll
    for (int mu = 0; mu < DMAX; ++mu)
        kc[mu] = ((float)kd[mu] - 0.99999994039535522461f) * c32_of<AX>(L, S, mu);
}

// ---------------------------------------------------------------------------
// One sample, FP32 path (a1-a3): x[], idx[], J = Jm 2^Je, f.
// ---------------------------------------------------------------------------
template <int DMAX, bool EXACT, int KIND, bool KP, bool AX>
__device__ __forceinline__ void point32(const Loop &L, const Strata *S, const float *prm,
                                        uint32_t h, uint32_t j,
                                        const float (&kc)[DMAX], float (&x)[DMAX],
                                        int (&idx)[DMAX], float &Jm, int &Je, float &f,
                                        int &fe) {
    const int dim = EXACT ? DMAX : L.dim;
    const uint32_t calls = EXACT ? (uint32_t)((DMAX + 3) / 4) : L.calls;
    float J = L.ngD_m;
    int e = L.ngD_e;
#pragma unroll
    for (int q = 0; q < (DMAX + 3) / 4; ++q) {
        if (q < (int)calls) {
            U4 c = {j * calls + (uint32_t)q, h, L.t, L.iid};
            const U4 r = philox_rk(c, L.rk0, L.rk1);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int mu = 4 * q + l;
                if (mu < DMAX && mu < dim) {
                    const uint32_t w = lane_of(r, l);
                    // (1 + m 2^-23) from the top 23 bits, no int->float conversion
                    const float one_m = __int_as_float(0x3f800000 | (w >> 9));
                    const float tt = fmaf(one_m, c32_of<AX>(L, S, mu), kc[mu]);  // y N_g
                    // floor(tt) for 0 <= tt < 2^22 by a round-down add of 1.5 2^23
                    const float big = __fadd_rd(tt, 12582912.0f);
                    int i = __float_as_int(big) - 0x4B400000;
                    float fl = big - 12582912.0f;
                    i = min(i, L.n_g - 1);
                    fl = fminf(fl, L.ngm1);
                    const float delta = tt - fl;
                    const float2 ed = __ldg(L.tab + mu * L.n_g + i);  // {x_i, dx_i}
                    x[mu] = fmaf(ed.y, delta, ed.x);
                    J *= ed.y;
                    idx[mu] = i;
                }
            }
            renorm(J, e);
        }
    }
    Jm = J;
    Je = e;
    fe = 0;  // the integrand is f 2^fe
    if (KIND == VP_POSTERIOR) {
        // f = 2^lf as a mantissa in [1, 2) and an integer exponent (f = 0
        // when log2 f is -inf or below any exponent that can matter)
        const float lf = f_post32_log2<DMAX>(prm, dim, x);
        if (lf > -1.0e9f) {
            const float fl = floorf(lf);
            f = ex2_approx(lf - fl);
            fe = (int)fl;
        } else {
            f = 0.0f;
        }
    } else if (KP) {
        f = f_peaks32_param<DMAX, KIND>(prm, L.K, dim, x);
    } else {
        f = f_peaks32<DMAX>(KIND, prm, L.K, dim, x);
    }
}

// ---------------------------------------------------------------------------
// One sample, FP32 path, an integrand of one peak with its constants in the
// kernel parameters (a1-a3, and the counts of a5): the same operations as
// point32 followed by f_peaks32_param, reordered so that no per-axis array of
// x is kept -- the peak's squared distance is accumulated axis by axis as each
// x_mu is formed (the same sum in the same order), the sample's count goes to
// its increment on every axis as soon as the increment is known, and the
// increment indices are kept two to a register for the histogram sums.
// Fewer live registers, so more warps per SM.
// ---------------------------------------------------------------------------
template <int DMAX, int KIND, int HM>
__device__ __forceinline__ void point32_p1(const Loop &L, const Strata *S, const float *kp,
                                           uint32_t h, uint32_t j, const float (&kc)[DMAX],
                                           uint32_t (&ip)[DMAX / 2], float &Jm, int &Je,
                                           float &f, uint32_t *hc, uint32_t *HC) {
    constexpr uint32_t calls = (uint32_t)((DMAX + 3) / 4);
    float J = L.ngD_m;
    int e = L.ngD_e;
    float r2 = 0.0f;
#pragma unroll
    for (int q = 0; q < (DMAX + 3) / 4; ++q) {
        U4 c = {j * calls + (uint32_t)q, h, L.t, L.iid};
        const U4 r = philox_rk(c, L.rk0, L.rk1);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int mu = 4 * q + l;
            if (mu < DMAX) {
                const uint32_t w = lane_of(r, l);
                const float one_m = __int_as_float(0x3f800000 | (w >> 9));
                const float tt = fmaf(one_m, S->c32[mu], kc[mu]);  // y N_g
                const float big = __fadd_rd(tt, 12582912.0f);
                int i = __float_as_int(big) - 0x4B400000;
                float fl = big - 12582912.0f;
                i = min(i, L.n_g - 1);
                fl = fminf(fl, L.ngm1);
                const float delta = tt - fl;
                const uint32_t bin = (uint32_t)mu * (uint32_t)L.n_g + (uint32_t)i;
                const float2 ed = __ldg(L.tab + bin);  // {x_i, dx_i}
                const float x = fmaf(ed.y, delta, ed.x);
                J *= ed.y;
                const float dx = x - kp[2 + mu];
                r2 = fmaf(dx, dx, r2);
                if (HM != kHistGlobal) atomicAdd(hc + bin, 1u);
                else red_add(HC + bin, 1u);
                if (mu & 1) ip[mu >> 1] |= (uint32_t)i << 16;
                else ip[mu >> 1] = (uint32_t)i;
            }
        }
        renorm(J, e);
    }
    Jm = J;
    Je = e;
    if (KIND == VP_GAUSS) f = fmaf(kp[0], ex2_approx(-kp[1] * r2), 0.0f);
    else if (KIND == VP_BALL) f = 0.0f + ((r2 < kp[1]) ? kp[0] : 0.0f);
    else f = fmaf(kp[0], ex2_approx(-kp[1] * sqrtf(r2)), 0.0f);
}

// ---------------------------------------------------------------------------
// One sample, FP64 path (a1-a3), the oracle's IEEE sequence step by step.
// ---------------------------------------------------------------------------
template <int DMAX, int KIND, bool AX>
__device__ __forceinline__ void point64(const Loop &L, const Strata *S, const double *prm,
                                        uint32_t h, uint32_t j,
                                        const uint32_t (&kd)[DMAX], double (&x)[DMAX],
                                        int (&idx)[DMAX], double &J, double &f) {
    J = 1.0;
#pragma unroll
    for (int q = 0; q < (DMAX + 3) / 4; ++q) {
        if (q < (int)L.calls) {
            U4 c = {j * L.calls + (uint32_t)q, h, L.t, L.iid};
            const U4 r = philox_rk(c, L.rk0, L.rk1);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int mu = 4 * q + l;
                if (mu < DMAX && mu < L.dim) {
                    const double u = u01_f64(lane_of(r, l));
                    const double y =
                        __ddiv_rn(__dadd_rn((double)kd[mu], u), AX ? S->nd[mu] : L.nst);
                    const double yng = __dmul_rn(y, L.ng);
                    int i = (int)floor(yng);
                    i = i > L.n_g - 1 ? L.n_g - 1 : i;
                    const double delta = __dsub_rn(yng, (double)i);
                    const double *e = L.edges + (size_t)mu * (size_t)(L.n_g + 1);
                    const double e0 = __ldg(e + i), e1 = __ldg(e + i + 1);
                    const double dx = __dsub_rn(e1, e0);
                    x[mu] = __dadd_rn(e0, __dmul_rn(dx, delta));
                    J = __dmul_rn(J, __dmul_rn(L.ng, dx));
                    idx[mu] = i;
                }
            }
        }
    }
    if (KIND == VP_POSTERIOR) f = f_post64<DMAX>(prm, L.dim, x);
    else f = f_peaks64<DMAX>(KIND, prm + 1, L.K, L.dim, x);
}

// h / N_st by multiply and shifts (Granlund & Montgomery, "Division by
// Invariant Integers using Multiplication", PLDI 1994); exact for all 32-bit h.
__device__ __forceinline__ uint32_t div_nst(uint32_t h, uint32_t magic, int shift) {
    if (shift == 0) return h;  // N_st = 1
    const uint32_t t = __umulhi(magic, h);
    return (t + ((h - t) >> 1)) >> (shift - 1);
}

// Mixed-radix digits of h: k_mu = (h / prod_{nu < mu} s_nu) mod s_mu.
template <int DMAX, bool AX>
__device__ __forceinline__ void decode_digits(uint32_t h, const Loop &L, const Strata *S, int dim,
                                              uint32_t (&kd)[DMAX]) {
#pragma unroll
    for (int mu = 0; mu < DMAX; ++mu) {
        if (mu < dim) {
            const uint32_t q = AX ? div_nst(h, S->magic[mu], S->shift[mu])
                                  : div_nst(h, L.nst_magic, L.nst_shift);
            kd[mu] = h - q * (AX ? S->n[mu] : L.n_st);
            h = q;
        } else {
            kd[mu] = 0u;
        }
    }
}

// h -> h + 1 on the digits (carry propagation).
template <int DMAX, bool AX>
__device__ __forceinline__ void next_digits(const Loop &L, const Strata *S, int dim,
                                            uint32_t (&kd)[DMAX]) {
    bool carry = true;
#pragma unroll
    for (int mu = 0; mu < DMAX; ++mu) {
        if (carry && mu < dim) {
            const uint32_t v = kd[mu] + 1u;
            if (v >= (AX ? S->n[mu] : L.n_st)) {
                kd[mu] = 0u;
            } else {
                kd[mu] = v;
                carry = false;
            }
        }
    }
}

// Largest g in [0, n) with a[g] <= key (a[0] <= key assumed).
__device__ __forceinline__ int upper_index(const uint64_t *a, int n, uint64_t key) {
    int lo = 0, hi = n;  // a[lo] <= key < a[hi] (a[n] = +inf)
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(a + mid) <= key) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint64_t find_hcube(const uint64_t *off, uint64_t n_hc, uint64_t s) {
    uint64_t lo = 0, hi = n_hc;  // off[lo] <= s < off[hi]
    while (hi - lo > 1) {
        uint64_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= s) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Kahan accumulation (FP32 path); plain sums on the FP64 path.
template <bool F64> struct Acc;
template <> struct Acc<true> {
    double s1, s2;
    __device__ __forceinline__ void reset() { s1 = 0.0; s2 = 0.0; }
    __device__ __forceinline__ void add(double v, double v2) { s1 += v; s2 += v2; }
    __device__ __forceinline__ void add_tiny(double, double) {}  // (FP32 path only)
    // the sums, unscaled by 2^-sexp
    __device__ __forceinline__ void values(int sexp, double &d1, double &d2) const {
        const double u = pow2d(-sexp);
        d1 = s1 * u;
        d2 = s2 * (u * u);
    }
    // adds them to the hypercube's FP64 accumulators
    template <bool SPLIT = true>
    __device__ __forceinline__ void flush(double *p1, double *p2, int sexp) const {
        double d1, d2;
        values(sexp, d1, d2);
        red_add(p1, d1);
        red_add(p2, d2);
    }
    __device__ __forceinline__ void shfl_down(Acc &o, int s) const {
        o.s1 = __shfl_down_sync(0xffffffffu, s1, s);
        o.s2 = __shfl_down_sync(0xffffffffu, s2, s);
    }
    __device__ __forceinline__ void combine(const Acc &o) {
        s1 += o.s1;
        s2 += o.s2;
    }
};
// FP32 samples whose v = J f 2^sexp lies far below the iteration's scale
// (2^-163 <= |v| < 2^-60; most samples of a narrow peak's tails) are summed
// apart, scaled by 2^kTinyShift, so that v^2 stays a normal FP32 number: t1, t2
// and the "tiny" shared histogram (plain FP32 sums: such terms only matter
// where nothing larger falls).
constexpr int kTinyShift = 100;

template <> struct Acc<false> {
    float s1, c1, s2, c2;
    float t1, t2;  // sums of v 2^kTinyShift and v^2 2^(2 kTinyShift)
    __device__ __forceinline__ void reset() { s1 = c1 = s2 = c2 = t1 = t2 = 0.0f; }
    __device__ __forceinline__ static void kahan(float &s, float &c, float v) {
        const float y = __fsub_rn(v, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ void add(float v, float v2) {
        kahan(s1, c1, v);
        kahan(s2, c2, v2);
    }
    __device__ __forceinline__ void add_tiny(float vt, float vt2) {
        t1 += vt;
        t2 += vt2;
    }
    // adds the compensated sums s - c and the tiny sums, unscaled exactly, to
    // the hypercube's FP64 accumulators.  SPLIT: each nonzero term reduced on
    // its own (FP64 arithmetic is scarce on this part: the conversions are
    // integer operations and the memory system adds the terms); else the terms
    // added in FP64 first and two reductions issued.  (Measured: the split
    // form is faster for the 20-D kernels, slower for the 64-register ones up
    // to D = 8.)
    template <bool SPLIT = true>
    __device__ __forceinline__ void flush(double *p1, double *p2, int sexp) const {
        if (!SPLIT) {
            red_add(p1, (f2d_pow2(s1, -sexp) - f2d_pow2(c1, -sexp)) +
                            f2d_pow2(t1, -sexp - kTinyShift));
            red_add(p2, (f2d_pow2(s2, -2 * sexp) - f2d_pow2(c2, -2 * sexp)) +
                            f2d_pow2(t2, -2 * (sexp + kTinyShift)));
            return;
        }
        if (s1 != 0.0f) red_add(p1, f2d_pow2(s1, -sexp));
        if (c1 != 0.0f) red_add(p1, f2d_pow2(-c1, -sexp));
        if (t1 != 0.0f) red_add(p1, f2d_pow2(t1, -sexp - kTinyShift));
        if (s2 != 0.0f) red_add(p2, f2d_pow2(s2, -2 * sexp));
        if (c2 != 0.0f) red_add(p2, f2d_pow2(-c2, -2 * sexp));
        if (t2 != 0.0f) red_add(p2, f2d_pow2(t2, -2 * (sexp + kTinyShift)));
    }
    __device__ __forceinline__ void shfl_down(Acc &o, int s) const {
        o.s1 = __shfl_down_sync(0xffffffffu, s1, s);
        o.c1 = __shfl_down_sync(0xffffffffu, c1, s);
        o.s2 = __shfl_down_sync(0xffffffffu, s2, s);
        o.c2 = __shfl_down_sync(0xffffffffu, c2, s);
        o.t1 = __shfl_down_sync(0xffffffffu, t1, s);
        o.t2 = __shfl_down_sync(0xffffffffu, t2, s);
    }
    // (s, c) + (os, oc), both meaning s - c: the sum s + os split exactly into
    // t + e (Knuth's two-sum), the compensations carried as c + oc - e
    __device__ __forceinline__ static void add_pair(float &s, float &c, float os, float oc) {
        const float t = __fadd_rn(s, os);
        const float bb = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(os, bb));
        c = __fsub_rn(__fadd_rn(c, oc), e);
        s = t;
    }
    __device__ __forceinline__ void combine(const Acc &o) {
        add_pair(s1, c1, o.s1, o.c1);
        add_pair(s2, c2, o.s2, o.c2);
        t1 += o.t1;
        t2 += o.t2;
    }
};

// A lane's last partial sums of a run, handed back instead of flushed, so that
// the lanes of a warp whose runs end in the same hypercube add them first
// (warp_flush): a hypercube holding many samples -- up to most of an
// iteration's -- otherwise receives reductions from every lane, all on the
// same addresses.
template <bool F64> struct RunTail {
    uint64_t h;  // ~0: none
    Acc<F64> acc;
};

// The outputs of several integrals from the same samples (App. B), summed per
// hypercube in registers (FP64): m1[k] = sum v_k, m2[k,l] = sum v_k v_l with
// v_k = J f g_k(x), the same IEEE sequence per sample as the oracle's
// (v_k = (J f)(x^a x^b), products and sums unfused).  MAcc<false> is empty.
template <bool MO> struct MAcc {
    __device__ __forceinline__ void reset() {}
    template <int DMAX>
    __device__ __forceinline__ void add(const SampleOne &, const double (&)[DMAX], double) {}
    __device__ __forceinline__ void flush(const SampleOne &, double *, double *) const {}
};
template <> struct MAcc<true> {
    double m1[kMaxOut], m2[kMaxTri];  // m2 by rows of the kMaxOut triangle
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int k = 0; k < kMaxOut; ++k) m1[k] = 0.0;
#pragma unroll
        for (int q = 0; q < kMaxTri; ++q) m2[q] = 0.0;
    }
    template <int DMAX>
    __device__ __forceinline__ void add(const SampleOne &a, const double (&x)[DMAX], double jf) {
        const int M = a.n_out;
        double v[kMaxOut];
#pragma unroll
        for (int k = 0; k < kMaxOut; ++k) {
            v[k] = 0.0;
            if (k < M) {
                const int p = a.mono[2 * k], r = a.mono[2 * k + 1];
                double xp = 1.0, xr = 1.0;  // x^p, x^r by selects (no indexed registers)
#pragma unroll
                for (int mu = 0; mu < DMAX; ++mu) {
                    xp = mu == p ? x[mu] : xp;
                    xr = mu == r ? x[mu] : xr;
                }
                v[k] = __dmul_rn(jf, __dmul_rn(xp, xr));
            }
        }
        int q = 0;
#pragma unroll
        for (int k = 0; k < kMaxOut; ++k) {
            if (k < M) m1[k] = __dadd_rn(m1[k], v[k]);
#pragma unroll
            for (int l = k; l < kMaxOut; ++l, ++q)
                if (l < M) m2[q] = __dadd_rn(m2[q], __dmul_rn(v[k], v[l]));
        }
    }
    // adds the sums to hypercube h's rows p1 = X1 + h M, p2 = X2 + h M (M+1)/2
    __device__ __forceinline__ void flush(const SampleOne &a, double *p1, double *p2) const;
};

// Integrand constants for this CTA: FP32 path copies them to shared memory
// (read with broadcast loads in the sample loop); FP64 path reads the blob.
__device__ __forceinline__ void load_prm32(const Desc *dp, float *sprm, int words) {
    const float *src = (const float *)__ldg((const unsigned long long *)&dp->prm32);
    for (int i = threadIdx.x; i < words; i += blockDim.x) sprm[i] = __ldg(src + i);
}

// Per-integral device pointers of the sampling loop.
struct Ptrs {
    const uint64_t *off;
    const uint32_t *nh;  // n_h = off[h + 1] - off[h]
    double *S1, *S2, *HS;
    uint32_t *HC;
    uint64_t n_hc, n_total;
};

// Samples [s_begin, s_end) of one integral, consecutive, by one thread:
// per-hypercube sums in registers, flushed with one FP64 atomic pair per
// hypercube touched; histograms into shared memory (or global).
// Hypercube of sample `base` (the warp chunk's first), by a 32-ary search of
// the offsets: every lane probes one point per round (4 rounds for 2^20
// hypercubes).  Warp-uniform result.
__device__ __forceinline__ uint64_t warp_find_hcube(const uint64_t *off, uint64_t n_hc,
                                                    uint64_t base, int lane) {
    uint64_t lo = 0, hi = n_hc;  // off[lo] <= base < off[hi]
    while (hi - lo > 1) {
        const uint64_t step = (hi - lo + 31) / 32;
        const uint64_t p = lo + (uint64_t)(lane + 1) * step;
        const bool le = p < hi && __ldg(off + p) <= base;
        const int c = __popc(__ballot_sync(0xffffffffu, le));  // probes are increasing
        const uint64_t nlo = lo + (uint64_t)c * step;
        hi = min(hi, nlo + step);
        lo = nlo;
    }
    return lo;
}

// Each lane's hypercube h (off[h] <= s < off[h + 1]) for its first sample s,
// walking windows of 32 consecutive boundaries from the chunk's hypercube.
// All shuffles run on every lane (no divergent collectives); the loop ends
// once every active lane has found its hypercube, at the latest when the
// window passes the last boundary.  Returns h; *lo_off = off[h],
// *hi_off = off[h + 1].
__device__ __forceinline__ uint64_t lane_find_hcube(const uint64_t *off, uint64_t n_hc,
                                                    uint64_t h_base, uint64_t s, bool active,
                                                    int lane, uint64_t *lo_off,
                                                    uint64_t *hi_off) {
    uint64_t win = h_base;  // off[win] <= every active lane's s
    uint64_t h = h_base;
    bool done = !active;
    for (;;) {
        const uint64_t pi = win + 1 + (uint64_t)lane;  // boundaries off[win + 1 .. win + 32]
        const uint64_t bnd = pi <= n_hc ? __ldg(off + pi) : ~0ull;
        int lo = -1, hi = 31;  // smallest m in (lo, hi] with boundary m > s (if any)
#pragma unroll
        for (int st = 0; st < 5; ++st) {
            const int mid = (lo + hi) >> 1;
            const uint64_t bm = __shfl_sync(0xffffffffu, bnd, mid < 0 ? 0 : mid);
            if (hi - lo > 1) {
                if (bm > s) hi = mid;
                else lo = mid;
            }
        }
        const uint64_t bh = __shfl_sync(0xffffffffu, bnd, hi);
        const uint64_t bl = __shfl_sync(0xffffffffu, bnd, hi > 0 ? hi - 1 : 0);
        if (!done && bh > s) {
            h = win + (uint64_t)hi;
            *hi_off = bh;
            *lo_off = hi > 0 ? bl : __ldg(off + win);
            done = true;
        }
        if (__all_sync(0xffffffffu, done)) break;
        win += 32;
    }
    return h;
}

__device__ __forceinline__ void MAcc<true>::flush(const SampleOne &a, double *p1,
                                                  double *p2) const {
    const int M = a.n_out;
    int q = 0, qm = 0;  // index in the kMaxOut triangle, in the M triangle
#pragma unroll
    for (int k = 0; k < kMaxOut; ++k) {
        if (k < M && m1[k] != 0.0) red_add(p1 + k, m1[k]);
#pragma unroll
        for (int l = k; l < kMaxOut; ++l, ++q)
            if (l < M) {
                if (m2[q] != 0.0) red_add(p2 + qm, m2[q]);
                ++qm;
            }
    }
}

// (HM: the histogram layout, kHist*; a template parameter so that the
// per-axis updates carry no branch on it)
// (P1: an FP32 integrand of one peak through point32_p1 -- counts added as
// each axis is formed, no digit array kept: the digits of the next hypercube
// are decoded from its index)
template <int DMAX, bool EXACT, bool F64, int KIND, bool KP, int HM, bool AX, bool MO,
          bool P1 = false>
__device__ __forceinline__ void run_samples_t(const Loop &L, const Strata *S, const Ptrs &P,
                                              const SampleOne *A, double *X1, double *X2,
                                              const void *prm,
                                              uint64_t s_begin, uint64_t s_end, uint64_t h,
                                              uint64_t lo_off, uint64_t next,
                                              typename Real<F64>::T *hs, float *hs_t,
                                              uint32_t *hc, int sexp, RunTail<F64> *tail) {
    constexpr bool hist_shared = HM != kHistGlobal;
    constexpr bool compact = HM == kHistCompact;
    static_assert(!P1 || (!F64 && KP && EXACT && !MO && KIND != VP_POSTERIOR), "P1 path");
    typedef typename Real<F64>::T T;
    const int dim = EXACT ? DMAX : L.dim;
    uint32_t j = (uint32_t)(s_begin - lo_off);
    uint32_t kd[P1 ? 1 : DMAX];
    float kc[DMAX];
    if constexpr (P1) {
        uint32_t kd1[DMAX];
        decode_digits<DMAX, AX>((uint32_t)h, L, S, dim, kd1);
        hcube_offsets<DMAX, AX>(L, S, kd1, kc);
    } else {
        decode_digits<DMAX, AX>((uint32_t)h, L, S, dim, kd);
        if (!F64) hcube_offsets<DMAX, AX>(L, S, kd, kc);
    }
    Acc<F64> acc;
    acc.reset();
    MAcc<MO> macc;  // (several outputs, App. B: FP64 path only)
    macc.reset();
    const uint64_t MM = MO ? (uint64_t)A->n_out : 0u, MT = MM * (MM + 1) / 2;
    // 32-bit counters (an iteration has fewer than 2^32 samples): samples left
    // in the run, and before the next hypercube (n_h >= 2, so at most one
    // boundary per sample)
    uint32_t to_next = (uint32_t)(next - s_begin);
    // the grid's d_i weighted per sample by 1/n_h of its hypercube (L.dw), or
    // the plain mean (weight 1, an exact multiply)
    uint32_t nh_cur = L.dw ? __ldg(P.nh + h) : 1u;
    float hw32 = L.dw ? __frcp_rn((float)nh_cur) : 1.0f;
    // above D = 8 (fewer warps per SM to hide latency): n_h of the next
    // hypercube loaded one hypercube ahead, its latency hidden behind the
    // current hypercube's samples
    constexpr bool kPrefetch = DMAX > 8;
    const uint32_t left0 = (uint32_t)(s_end - s_begin);
    uint32_t nh_next =
        (kPrefetch && to_next < left0 && h + 1 < P.n_hc) ? __ldg(P.nh + h + 1) : 0u;
    for (uint32_t left = left0; left > 0; --left) {
        if (to_next == 0u) {
            acc.template flush<(DMAX > 8)>(P.S1 + h, P.S2 + h, sexp);
            acc.reset();
            if (MO) {
                macc.flush(*A, X1 + h * MM, X2 + h * MT);
                macc.reset();
            }
            ++h;
            if (kPrefetch) {
                to_next = nh_next;
                // (n_h >= 2: the run reaches the next boundary only if more
                // than n_h samples are left)
                nh_next = (to_next < left && h + 1 < P.n_hc) ? __ldg(P.nh + h + 1) : 0u;
            } else {
                to_next = __ldg(P.nh + h);
            }
            if (L.dw) {
                nh_cur = to_next;
                hw32 = __frcp_rn((float)nh_cur);
            }
            j = 0;
            if constexpr (P1) {
                uint32_t kd1[DMAX];
                decode_digits<DMAX, AX>((uint32_t)h, L, S, dim, kd1);
                hcube_offsets<DMAX, AX>(L, S, kd1, kc);
            } else {
                next_digits<DMAX, AX>(L, S, dim, kd);
                if (!F64) hcube_offsets<DMAX, AX>(L, S, kd, kc);
            }
        }
        --to_next;
        int idx[P1 ? 1 : DMAX];
        uint32_t ip[P1 ? DMAX / 2 : 1];  // (P1: increment indices, two to a register)
        T v;
        // FP32: v = J f 2^sexp in [2^-60, 2^60) is summed as is, tiny v in
        // [2^-163, 2^-60) scaled by 2^kTinyShift (see Acc); beyond those (v^2
        // would leave FP32, e.g. in the first iteration, before the scale has
        // adapted) a sample takes exact FP64 terms of its own
        bool big = false, tiny = false;
        double vbig = 0.0, vbig2 = 0.0, hbig = 0.0;
        if constexpr (F64) {
            double x[DMAX], J, f;
            if (MO) {  // (the outputs' selects read every entry)
#pragma unroll
                for (int mu = 0; mu < DMAX; ++mu) x[mu] = 0.0;
            }
            point64<DMAX, KIND, AX>(L, S, (const double *)prm, (uint32_t)h, j, kd, x, idx, J, f);
            v = (T)(J * f * pow2d(sexp));
            if (MO) macc.template add<DMAX>(*A, x, __dmul_rn(J, f));
        } else {
            float Jm, f;
            int Je;
            if constexpr (P1) {
                point32_p1<DMAX, KIND, HM>(L, S, (const float *)prm, (uint32_t)h, j, kc, ip, Jm,
                                           Je, f, hc, P.HC);
            } else {
                float x[DMAX];
                int fe;
                point32<DMAX, EXACT, KIND, KP, AX>(L, S, (const float *)prm, (uint32_t)h, j, kc, x,
                                                   idx, Jm, Je, f, fe);
                Je += fe;  // J f = (Jm f) 2^(Je + fe)
            }
            float jf = Jm * f;  // Jm in [1, 2); the last multiply-add of f may leave it subnormal
            if (((__float_as_int(jf) & 0x7f800000) == 0) && jf != 0.0f) {  // renormalise (exact)
                jf *= 16777216.0f;
                Je -= 24;
            }
            const int ej = ((__float_as_int(jf) >> 23) & 0xff) - 127;
            const int ev = ej + Je + sexp;  // exponent of v
            const bool nz = jf != 0.0f && isfinite(jf);
            if (nz && (ev >= 60 || ev < -163)) {
                big = true;
                const float m = __int_as_float((__float_as_int(jf) & 0x807fffff) | 0x3f800000);
                vbig = f2d_pow2(jf, Je);                    // J f, unscaled
                vbig2 = f2d_pow2(m * m, 2 * (ej + Je));     // (J f)^2
                red_add(P.S1 + h, vbig);
                red_add(P.S2 + h, vbig2);
                hbig = L.dw ? vbig2 / (double)nh_cur : vbig2;  // (rare: only here)
                v = (T)0;
            } else {
                tiny = nz && ev < -60;
                // the scaled v has exponent ev (+ kTinyShift if tiny), in
                // [-63, 60): a normal number, so the power of two goes straight
                // into the exponent field (exact, as a multiply would be); zero,
                // inf and NaN pass unchanged
                const int sh = Je + sexp + (tiny ? kTinyShift : 0);
                v = (T)(nz ? __int_as_float(__float_as_int(jf) + (sh << 23)) : jf);
            }
        }
        const T v2 = v * v;
        if (F64) {
            acc.add(v, v2);
        } else {
            acc.add(tiny ? (T)0 : v, tiny ? (T)0 : v2);
            acc.add_tiny(tiny ? (float)v : 0.0f, tiny ? (float)v2 : 0.0f);
        }
        T *hdst = hs;
        int hexp = -2 * sexp;
        if (!F64 && tiny) {
            hdst = (T *)hs_t;
            hexp -= 2 * kTinyShift;
        }
        // the histogram term: (J f)^2, or (J f)^2 / n_h for the weighted d_i
        // (FP64: the oracle's division; FP32: times the rounded 1/n_h)
        T hv = v2;
        if (F64) {
            if (L.dw) hv = (T)__ddiv_rn((double)v2, (double)nh_cur);
        } else {
            hv = v2 * (T)hw32;
        }
        // (the branches are taken once per sample, not per axis: the axis
        // loops below are plain runs of atomics)
        int bin[DMAX];
#pragma unroll
        for (int mu = 0; mu < DMAX; ++mu) {
            if constexpr (P1) bin[mu] = mu * L.n_g + (int)((ip[mu >> 1] >> (16 * (mu & 1))) & 0xffffu);
            else bin[mu] = mu * L.n_g + idx[mu];
        }
        if (big) {
#pragma unroll
            for (int mu = 0; mu < DMAX; ++mu)
                if (mu < dim) red_add(P.HS + bin[mu], hbig);
        } else if (hv != (T)0) {
            if (hist_shared && !(compact && tiny)) {
#pragma unroll
                for (int mu = 0; mu < DMAX; ++mu)
                    if (mu < dim) atomicAdd(hdst + bin[mu], hv);
            } else {  // global sums (and, compact, the FP32 tiny sums)
                const double hg = F64 ? (double)hv * pow2d(hexp) : f2d_pow2((float)hv, hexp);
#pragma unroll
                for (int mu = 0; mu < DMAX; ++mu)
                    if (mu < dim) red_add(P.HS + bin[mu], hg);
            }
        }
        if (P1) {
            // (the counts were added as the axes were formed)
        } else if (hist_shared) {
#pragma unroll
            for (int mu = 0; mu < DMAX; ++mu)
                if (mu < dim) atomicAdd(hc + bin[mu], 1u);
        } else {
#pragma unroll
            for (int mu = 0; mu < DMAX; ++mu)
                if (mu < dim) red_add(P.HC + bin[mu], 1u);
        }
        ++j;
    }
    if (tail && !MO) {  // (the caller adds it with the warp's others)
        tail->h = h;
        tail->acc = acc;
    } else {
        acc.template flush<(DMAX > 8)>(P.S1 + h, P.S2 + h, sexp);
    }
    if (MO) macc.flush(*A, X1 + h * MM, X2 + h * MT);
}

// The warp's run tails, added per hypercube before they reach global memory:
// lanes hold consecutive samples, so lanes with the same hypercube are
// contiguous; a segmented tree of shuffles leaves each segment's sum in its
// lowest lane, which issues the two reductions.  Every lane of the warp calls
// it (tail.h = ~0 for a lane without samples).
template <bool F64>
__device__ __forceinline__ void warp_flush(const Ptrs &P, RunTail<F64> t, int lane, int sexp) {
    const uint64_t ph = __shfl_up_sync(0xffffffffu, t.h, 1);
    const bool head = lane == 0 || ph != t.h;  // the lowest lane of its hypercube
    if (!__all_sync(0xffffffffu, head)) {  // (else every lane its own: nothing to add)
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const uint64_t oh = __shfl_down_sync(0xffffffffu, t.h, s);
            Acc<F64> o;
            t.acc.shfl_down(o, s);
            if (lane + s < 32 && oh == t.h) t.acc.combine(o);
        }
    }
    if (t.h != ~0ull && head) t.acc.flush(P.S1 + t.h, P.S2 + t.h, sexp);
}

template <int DMAX, bool EXACT, bool F64, int KIND, bool KP, bool AX, bool MO = false,
          bool P1 = false>
__device__ __forceinline__ void run_samples(const Loop &L, const Strata *S, const Ptrs &P,
                                            const void *prm, uint64_t s_begin, uint64_t s_end,
                                            uint64_t h, uint64_t lo_off, uint64_t next,
                                            typename Real<F64>::T *hs, float *hs_t, uint32_t *hc,
                                            int hist_mode, int sexp,
                                            const SampleOne *A = nullptr, double *X1 = nullptr,
                                            double *X2 = nullptr, RunTail<F64> *tail = nullptr) {
    if (hist_mode == kHistShared)
        run_samples_t<DMAX, EXACT, F64, KIND, KP, kHistShared, AX, MO, P1>(
            L, S, P, A, X1, X2, prm, s_begin, s_end, h, lo_off, next, hs, hs_t, hc, sexp, tail);
    else if (!F64 && hist_mode == kHistCompact)
        run_samples_t<DMAX, EXACT, F64, KIND, KP, kHistCompact, AX, MO, P1>(
            L, S, P, A, X1, X2, prm, s_begin, s_end, h, lo_off, next, hs, hs_t, hc, sexp, tail);
    else
        run_samples_t<DMAX, EXACT, F64, KIND, KP, kHistGlobal, AX, MO, P1>(
            L, S, P, A, X1, X2, prm, s_begin, s_end, h, lo_off, next, hs, hs_t, hc, sexp, tail);
}

// ---------------------------------------------------------------------------
// The fused sampling kernel (a1-a5), one integral per launch.
//
// The N samples of the iteration are split evenly over the warps of the grid
// (every CTA is resident at once), warp w taking [w N / W, (w + 1) N / W) and
// lane l a run of consecutive samples within it, so the work is balanced to a
// sample and nothing is queued.  The CTAs of a thread-block cluster then add
// their shared-memory histograms through distributed shared memory, each CTA
// reducing one slice of the bins, so the global flush is one reduction per bin
// and cluster.
// Shared memory: [prm: prm_words x 4 B][hist sums: bins x 8 B (FP64 sum, or FP32 sum and FP32
// tiny sum)][hist count: bins x 4 B]
// ---------------------------------------------------------------------------
// Largest CTA of the one-integral kernel: the autotuner also tries one CTA per
// SM (one shared-memory histogram per SM instead of one per 256 threads).
// The bound sets the register budget: 64 for FP32 with D <= 8 (1024 threads,
// no spills: a third more warps than 768 threads at 80 registers), the 256 x 2
// shape's for FP32 with D > 8 and the 256 x 1 shape's for FP64.
// The single-peak FP32 form (P1), which keeps fewer registers, takes 768
// threads above D = 8.
__host__ __device__ constexpr int one_max_threads(int dmax, bool f64, bool p1 = false) {
    return f64 ? 256 : (dmax <= 8 ? 1024 : (p1 ? 768 : 512));
}

// Sum of the cluster's CS copies of bins [b0, b1) of the histograms, added to
// the global FP64 histograms (one reduction per bin and cluster).
template <int CS, bool F64>
__device__ __forceinline__ void cluster_flush(cooperative_groups::cluster_group &cl,
                                              typename Real<F64>::T *hs, float *hs_t,
                                              uint32_t *hc, const Ptrs &P, int b0, int b1,
                                              int sexp, bool tiny_sums) {
    typedef typename Real<F64>::T T;
    // each cluster starts at its own bin of the slice (in whole warps), so
    // that the clusters' global reductions do not queue on the same addresses
    const int n_cl = (int)(gridDim.x / CS), cid = (int)(blockIdx.x / CS);
    const int len = max(b1 - b0, 0);
    const int rot = (int)(((uint32_t)cid * (uint32_t)len / (uint32_t)n_cl) & ~31u);
    for (int q = threadIdx.x; q < len; q += blockDim.x) {
        const int b = b0 + (q + rot < len ? q + rot : q + rot - len);
        T vs[CS];
        float vt[CS];
        uint32_t vc[CS];
#pragma unroll
        for (int r = 0; r < CS; ++r) {  // the remote loads of a bin issued together
            vs[r] = *cl.map_shared_rank(hs + b, r);
            vt[r] = (F64 || !tiny_sums) ? 0.0f : *cl.map_shared_rank(hs_t + b, r);
            vc[r] = *cl.map_shared_rank(hc + b, r);
        }
        // (the FP32 path adds the CTAs' FP32 sums in FP32, like each CTA's own)
        T sum = (T)0;
        float sum_t = 0.0f;
        uint32_t cnt = 0;
#pragma unroll
        for (int r = 0; r < CS; ++r) {
            sum += vs[r];
            sum_t += vt[r];
            cnt += vc[r];
        }
        if (cnt) {
            double d = F64 ? (double)sum * pow2d(-2 * sexp) : f2d_pow2((float)sum, -2 * sexp);
            if (sum_t != 0.0f) d += f2d_pow2(sum_t, -2 * (sexp + kTinyShift));
            red_add(P.HS + b, d);
            red_add(P.HC + b, cnt);
        }
    }
}

template <int DMAX, bool EXACT, bool F64, int KIND, bool MO = false, bool P1 = false>
__global__ void __launch_bounds__(one_max_threads(DMAX, F64, P1), 1)
    k_sample_one(const __grid_constant__ SampleOne a) {
    typedef typename Real<F64>::T T;
    namespace cg = cooperative_groups;
    // FP32 peak families read their constants from the parameters
    constexpr bool KP = !F64 && KIND != VP_POSTERIOR;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint8_t s_tried[32];  // per warp: tail queues found empty
    float *sprm = (float *)smem;
    // histograms: sums (FP64, or FP32 and -- unless compact -- the FP32 tiny
    // sums), then counts
    const bool compact = a.hist_shared == kHistCompact;
    T *hs = (T *)(smem + (size_t)a.prm_words * 4);
    float *hs_t = (float *)(smem + (size_t)a.prm_words * 4 + (size_t)a.bins * 4);
    uint32_t *hc =
        (uint32_t *)(smem + (size_t)a.prm_words * 4 + (size_t)a.bins * (compact ? 4 : 8));
    const int lane = threadIdx.x & 31;
    if (a.hist_shared) {  // (no dependence on earlier kernels: before the wait)
        for (int b = threadIdx.x; b < a.bins; b += blockDim.x) {
            hs[b] = (T)0;
            if (!F64 && !compact) hs_t[b] = 0.0f;
            hc[b] = 0u;
        }
    }
    pdl_wait();

    const uint32_t t_it = __ldcg(&a.st->t);
    // the FP64 path sums J f and (J f)^2 unscaled, the oracle's IEEE sequence
    // (where (J f)^2 leaves the normal range, as in a sharply peaked
    // posterior's far tails, scaled squares would round differently, and the
    // grid's compression weighs those tiny d_i by their logarithm)
    const int sexp = F64 ? 0 : __ldcg(&a.st->scale_exp);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.st->hist_par = (t_it & 1u) | (a.L.dw ? 2u : 0u);
    Loop L = a.L;
    L.t = t_it;
    Ptrs P;
    const uint64_t par = t_it & 1u;  // accumulators of this iteration: buffer t & 1
    P.off = a.off;
    P.nh = a.n_h;
    P.n_hc = a.n_hc;
    P.n_total = __ldcg(a.off + a.n_hc);
    P.S1 = a.s1 + par * a.n_hc;
    P.S2 = a.s2 + par * a.n_hc;
    P.HS = a.hsum + par * (uint64_t)a.bins;
    P.HC = a.hcnt + par * (uint64_t)a.bins;
    const void *prm;
    if (F64) {
        prm = (const void *)a.prm;
    } else if (KP) {
        prm = (const void *)a.kp;
    } else {
        for (int i = threadIdx.x; i < a.prm_words; i += blockDim.x) sprm[i] = __ldg(a.prm32 + i);
        prm = (const void *)sprm;
    }
    __syncthreads();
    {
        // this warp's share of the samples (the first n mod W warps take one
        // more), then this lane's run within it.  32-bit arithmetic: the
        // samples of an iteration number below 2^32, and a 64-bit division
        // by a runtime value would run on the scarce FP64 units.
        const uint32_t W = gridDim.x * (blockDim.x >> 5);
        const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        uint32_t n_tot = (uint32_t)P.n_total, lo = 0u;
        if (a.n_parts > 1) {  // samples [T p / P, T (p + 1) / P) of the T in the iteration
            const uint64_t T = P.n_total;
            lo = (uint32_t)(T * (uint64_t)a.part / (uint64_t)a.n_parts);
            n_tot = (uint32_t)(T * (uint64_t)(a.part + 1) / (uint64_t)a.n_parts) - lo;
        }
        // the static head: the first n_st samples of the range, split evenly
        // over the warps (the costs of samples differ -- hypercube changes,
        // nonzero integrand values -- so a dynamic tail evens out the end)
        const uint32_t n_st =
            a.static16 >= 16 ? n_tot : (uint32_t)(((uint64_t)n_tot * (uint32_t)a.static16) >> 4);
        double *X1 = MO ? a.x1 + par * a.n_hc * (uint64_t)a.n_out : nullptr;
        double *X2 = MO ? a.x2 + par * a.n_hc * (uint64_t)(a.n_out * (a.n_out + 1) / 2) : nullptr;
        // (sample indices are 32-bit: an iteration has fewer than 2^32 samples)
        const uint32_t per_w = n_st / W, extra = n_st - per_w * W;
        const uint32_t wb = lo + w * per_w + min(w, extra);
        const uint32_t we = wb + per_w + (w < extra ? 1u : 0u);
        // the dynamic tail: chunks of 32 r samples, each warp pulling the next
        // one from the queue as it finishes
        const uint32_t C = 32u * (uint32_t)a.r;
        const uint32_t n_ch = (n_tot - n_st + C - 1) / C;
        // work items of this warp: its static range, then the chunks it pulls;
        // lane l takes `per` consecutive samples of an item (one call site of
        // the sample loop, so that it is inlined once)
        uint32_t base = wb, end = we, per = (we - wb + 31) / 32;
        // (lane 0: queues found empty so far, kept in shared memory rather
        // than in a register of the sample loop)
        if (lane == 0) s_tried[threadIdx.x >> 5] = 0u;
        for (bool first = true;; first = false) {
            if (!first) {
                uint32_t c = n_ch;
                if (lane == 0) {
                    uint32_t tried = s_tried[threadIdx.x >> 5];
                    while (n_st < n_tot && tried < kTailQueues) {
                        const uint32_t qu = (w + tried) % kTailQueues;
                        const uint32_t q0 = (uint32_t)((uint64_t)n_ch * qu / kTailQueues);
                        const uint32_t q1 = (uint32_t)((uint64_t)n_ch * (qu + 1) / kTailQueues);
                        const uint32_t k = atomicAdd(a.head + kQueueStride * qu, 1u);
                        if (k < q1 - q0) {
                            c = q0 + k;
                            break;
                        }
                        ++tried;  // this queue is done: the next one
                    }
                    s_tried[threadIdx.x >> 5] = (uint8_t)min(tried, kTailQueues);
                }
                c = __shfl_sync(0xffffffffu, c, 0);
                if (c >= n_ch) break;
                base = lo + n_st + c * C;
                end = min(base + C, lo + n_tot);
                per = (uint32_t)a.r;
            }
            if (base >= end) continue;  // (warp-uniform: an empty static range)
            const uint32_t c0 = min(base + (uint32_t)lane * per, end);
            const uint32_t c1 = min(c0 + per, end);
            const uint64_t hb = warp_find_hcube(P.off, P.n_hc, base, lane);
            uint64_t lo_off = 0, hi_off = 0;
            const uint64_t h =
                lane_find_hcube(P.off, P.n_hc, hb, c0, c0 < c1, lane, &lo_off, &hi_off);
            RunTail<F64> tail;
            if (c0 < c1) {  // (the strata per axis: constants of the parameter bank)
                run_samples<DMAX, EXACT, F64, KIND, KP, true, MO, P1>(
                    L, &a.S, P, prm, c0, c1, h, lo_off, hi_off, hs, hs_t, hc, a.hist_shared,
                    sexp, &a, X1, X2, MO ? nullptr : &tail);
            } else {  // (set here, not before the loop: no registers held across it)
                tail.h = ~0ull;
                tail.acc.reset();
            }
            // (measured: the 64-register kernels up to D = 8 run the eight-D
            // four-peak workload slower with the warp's combine, the larger
            // ones gain from it where one hypercube holds many samples)
            if (!MO) {
                if (DMAX > 8) warp_flush<F64>(P, tail, lane, sexp);
                else if (tail.h != ~0ull)
                    tail.acc.template flush<false>(P.S1 + tail.h, P.S2 + tail.h, sexp);
            }
        }
    }
    __syncthreads();
    if (a.static16 < 16 && threadIdx.x == 0) {
        // the last CTA out resets the queue for the next launch (every other
        // CTA has left its tail loop, so none reads the head again)
        __threadfence();
        if (atomicAdd(a.exit_count, 1u) == gridDim.x - 1) {
            for (uint32_t q = 0; q < kTailQueues; ++q) a.head[kQueueStride * q] = 0u;
            *a.exit_count = 0u;
            __threadfence();
        }
    }
    if (a.hist_shared) {
        // cluster-wide reduction of the CTAs' histograms, one slice per CTA
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        const int cs = (int)cl.num_blocks(), rank = (int)cl.block_rank();
        const int per = (a.bins + cs - 1) / cs;
        const int b0 = rank * per, b1 = min(a.bins, b0 + per);
        switch (cs) {
            case 1: cluster_flush<1, F64>(cl, hs, hs_t, hc, P, b0, b1, sexp, !compact); break;
            case 2: cluster_flush<2, F64>(cl, hs, hs_t, hc, P, b0, b1, sexp, !compact); break;
            case 4: cluster_flush<4, F64>(cl, hs, hs_t, hc, P, b0, b1, sexp, !compact); break;
            default: cluster_flush<8, F64>(cl, hs, hs_t, hc, P, b0, b1, sexp, !compact); break;
        }
        cl.sync();  // keep this CTA's shared memory until every remote read is done
    }
}

// ---------------------------------------------------------------------------
// The fused sampling kernel (a1-a5) for several integrals per launch: a CTA
// pulls tasks (an integral and a range of `task` samples, big integrals
// first) and its warps pull warp chunks of the task from a shared counter; the
// CTA's histograms are flushed when it moves to another integral.
// ---------------------------------------------------------------------------
// (AX: the strata per axis from each integral's descriptor, for sets with
// integrals whose strata differ between axes, §3.2; a separate instantiation
// so that the other sets keep the one count in registers)
template <int DMAX, bool EXACT, bool F64, int KIND, bool AX = false>
__global__ void __launch_bounds__(256, 2) k_sample_many(SampleArgs a) {
    typedef typename Real<F64>::T T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_task, s_wc;
    float *sprm = (float *)smem;
    // histograms: sums (FP64, or FP32 and the FP32 tiny sums), then counts
    T *hs = (T *)(smem + (size_t)a.prm_words * 4);
    float *hs_t = (float *)(smem + (size_t)a.prm_words * 4 + (size_t)a.hist_words * 4);
    uint32_t *hc = (uint32_t *)(smem + (size_t)a.prm_words * 4 + (size_t)a.hist_words * 8);
    const int lane = threadIdx.x & 31;
    const uint32_t wchunk = 32u * (uint32_t)a.r;
    pdl_wait();

    int cur = -1;
    Loop L;
    Ptrs P;
    const void *prm = nullptr;
    int bins = 0, sexp = 0;
    const Strata *S = nullptr;

    auto flush_hist = [&]() {
        // each CTA starts at its own bin (in whole warps), so that the CTAs'
        // global reductions do not all queue on the same addresses at once
        const int rot = (int)(((uint32_t)blockIdx.x * (uint32_t)bins / gridDim.x) & ~31u);
        for (int q = threadIdx.x; q < bins; q += blockDim.x) {
            const int b = q + rot < bins ? q + rot : q + rot - bins;
            const uint32_t n = hc[b];
            if (n) {
                double d = F64 ? (double)hs[b] * pow2d(-2 * sexp) : f2d_pow2((float)hs[b], -2 * sexp);
                if (!F64 && hs_t[b] != 0.0f) d += f2d_pow2(hs_t[b], -2 * (sexp + kTinyShift));
                red_add(P.HS + b, d);
                red_add(P.HC + b, n);
            }
        }
    };
    auto enter = [&](int g) {  // all threads; caller synchronises afterwards
        cur = g;
        const Desc *dp = a.desc + __ldg(a.members + g);
        State *st = (State *)__ldg((const unsigned long long *)&dp->st);
        const uint32_t t_it = __ldcg(&st->t);
        if (threadIdx.x == 0)  // every CTA of the integral writes the same
            st->hist_par = (t_it & 1u) | (__ldg(&dp->d_weighted) ? 2u : 0u);
        L = make_loop(dp, t_it);
        if (AX) S = &dp->strata;
        sexp = F64 ? 0 : __ldcg(&st->scale_exp);  // (FP64: unscaled, as in k_sample_one)
        bins = L.dim * L.n_g;
        P.off = (const uint64_t *)__ldg((const unsigned long long *)&dp->off);
        P.nh = (const uint32_t *)__ldg((const unsigned long long *)&dp->n_h);
        P.n_hc = __ldg(&dp->n_hc);
        P.n_total = __ldcg(P.off + P.n_hc);
        // accumulators of this iteration: buffer (t & 1) of the double-buffered pairs
        const uint64_t par = t_it & 1u;
        P.S1 = (double *)__ldg((const unsigned long long *)&dp->s1) + par * P.n_hc;
        P.S2 = (double *)__ldg((const unsigned long long *)&dp->s2) + par * P.n_hc;
        P.HS = (double *)__ldg((const unsigned long long *)&dp->hsum) + par * bins;
        P.HC = (uint32_t *)__ldg((const unsigned long long *)&dp->hcnt) + par * bins;
        if (F64) {
            prm = (const void *)__ldg((const unsigned long long *)&dp->prm);
        } else {
            load_prm32(dp, sprm, a.prm_words);
            prm = (const void *)sprm;
        }
        if (a.hist_shared) {
            for (int b = threadIdx.x; b < bins; b += blockDim.x) {
                hs[b] = (T)0;
                if (!F64) hs_t[b] = 0.0f;
                hc[b] = 0u;
            }
        }
    };

    const uint64_t total = __ldg(a.chunk_base + a.n_group);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_task = atomicAdd(a.head, 1u);
            s_wc = 0u;
        }
        __syncthreads();
        const uint64_t task = s_task;
        if (task >= total) break;
        const int g = upper_index(a.chunk_base, a.n_group, task);
        if (g != cur) {
            if (cur >= 0 && a.hist_shared) {
                flush_hist();
                __syncthreads();
            }
            enter(g);
            __syncthreads();
        }
        const uint64_t t0 = (task - __ldg(a.chunk_base + g)) * (uint64_t)a.task;
        const uint64_t t1 = min(t0 + (uint64_t)a.task, P.n_total);
        const uint32_t n_wc = ((uint32_t)(t1 - t0) + wchunk - 1) / wchunk;  // 32-bit (no FP64 units)
        for (;;) {
            uint32_t c = 0;
            if (lane == 0) c = atomicAdd(&s_wc, 1u);
            c = __shfl_sync(0xffffffffu, c, 0);
            if (c >= n_wc) break;
            const uint64_t base = t0 + (uint64_t)c * wchunk;
            const uint64_t s0 = base + (uint64_t)lane * a.r;
            const uint64_t s1 = min(s0 + (uint64_t)a.r, t1);
            const uint64_t hb = warp_find_hcube(P.off, P.n_hc, base, lane);
            uint64_t lo_off = 0, hi_off = 0;
            const uint64_t h =
                lane_find_hcube(P.off, P.n_hc, hb, s0, s0 < s1, lane, &lo_off, &hi_off);
            if (s0 < s1)
                run_samples<DMAX, EXACT, F64, KIND, false, AX>(
                    L, S, P, prm, s0, s1, h, lo_off, hi_off, hs, hs_t, hc,
                    a.hist_shared ? kHistShared : kHistGlobal, sexp);
        }
    }
    if (cur >= 0 && a.hist_shared) flush_hist();
    // the last CTA out resets the queue for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.exit_count, 1u) == gridDim.x - 1) {
            *a.head = 0u;
            *a.exit_count = 0u;
            __threadfence();
        }
    }
}

// Per-sample inspection: the same device code as k_sample, on listed samples.
template <int DMAX, bool EXACT, bool F64, int KIND>
__global__ void k_eval(const Desc *desc, int member, int64_t n, const uint64_t *hs,
                       const uint32_t *js, uint32_t t, double *xo, int32_t *io, double *jo,
                       double *fo, int prm_words) {
    extern __shared__ __align__(16) unsigned char smem[];
    float *sprm = (float *)smem;
    const Desc *dp = desc + member;
    const Loop L = make_loop(dp, t);
    const Strata *S = &dp->strata;
    const int dim = EXACT ? DMAX : L.dim;
    if (!F64) load_prm32(dp, sprm, prm_words);
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        uint32_t kd[DMAX];
        int idx[DMAX];
        decode_digits<DMAX, true>((uint32_t)hs[k], L, S, dim, kd);
        double xd[DMAX], jac, f;
        if (F64) {
            point64<DMAX, KIND, true>(L, S, (const double *)__ldg((const unsigned long long *)&dp->prm),
                                (uint32_t)hs[k], js[k], kd, xd, idx, jac, f);
        } else {
            float kc[DMAX], x[DMAX], Jm, ff;
            int Je;
            hcube_offsets<DMAX, true>(L, S, kd, kc);
            int fe;
            point32<DMAX, EXACT, KIND, false, true>(L, S, sprm, (uint32_t)hs[k], js[k], kc, x, idx,
                                                    Jm, Je, ff, fe);
#pragma unroll
            for (int mu = 0; mu < DMAX; ++mu) xd[mu] = (double)x[mu];
            jac = ldexp((double)Jm, Je);
            f = ldexp((double)ff, fe);
        }
#pragma unroll
        for (int mu = 0; mu < DMAX; ++mu) {
            if (mu < dim) {
                xo[k * dim + mu] = xd[mu];
                io[k * dim + mu] = idx[mu];
            }
        }
        jo[k] = jac;
        fo[k] = f;
    }
}

// §4.2 (preconditioned integrators): the data histogram of the map's training
// on sample data {x, f(x)}.  Per data point (one thread each): on every axis
// the increment i holding x (x_i <= x < x_{i+1}, the last one also taking
// x = b), i.e. the inverse map y(x); J(y(x)) = prod N_g dx_i; f from the data
// or from the integrand (FP64); then (J f)^2 and a count added to increment i
// of every axis, in histogram buffer `buf` (the oracle's IEEE sequence).
template <int DMAX, int KIND>
__global__ void __launch_bounds__(256) k_precondition(const Desc *desc, int member, int64_t n,
                                                      const double *xs, const double *fs,
                                                      uint32_t buf) {
    const Desc *dp = desc + member;
    const int dim = __ldg(&dp->dim), n_g = __ldg(&dp->n_g), K = __ldg(&dp->n_peaks);
    const double *edges = (const double *)__ldg((const unsigned long long *)&dp->edges);
    const double *prm = (const double *)__ldg((const unsigned long long *)&dp->prm);
    const size_t bins = (size_t)dim * n_g;
    double *HS = (double *)__ldg((const unsigned long long *)&dp->hsum) + buf * bins;
    uint32_t *HC = (uint32_t *)__ldg((const unsigned long long *)&dp->hcnt) + buf * bins;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double x[DMAX];
        int idx[DMAX];
        double J = 1.0;
#pragma unroll
        for (int mu = 0; mu < DMAX; ++mu) {
            x[mu] = 0.0;
            idx[mu] = 0;
            if (mu < dim) {
                const double xv = __ldg(xs + p * dim + mu);
                const double *e = edges + (size_t)mu * (size_t)(n_g + 1);
                int lo = 0, hi = n_g;  // e[lo] <= x < e[hi]
                if (xv >= __ldg(e + n_g)) {
                    lo = n_g - 1;
                } else {
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (__ldg(e + mid) <= xv) lo = mid;
                        else hi = mid;
                    }
                }
                const double dx = __dsub_rn(__ldg(e + lo + 1), __ldg(e + lo));
                J = __dmul_rn(J, __dmul_rn((double)n_g, dx));
                x[mu] = xv;
                idx[mu] = lo;
            }
        }
        double f;
        if (fs) f = __ldg(fs + p);
        else if (KIND == VP_POSTERIOR) f = f_post64<DMAX>(prm, dim, x);
        else f = f_peaks64<DMAX>(KIND, prm + 1, K, dim, x);
        const double jf = __dmul_rn(J, f);
        const double w = __dmul_rn(jf, jf);
#pragma unroll
        for (int mu = 0; mu < DMAX; ++mu) {
            if (mu < dim) {
                if (w != 0.0) red_add(HS + (size_t)mu * n_g + idx[mu], w);
                red_add(HC + (size_t)mu * n_g + idx[mu], 1u);
            }
        }
    }
}

// Launch dispatch (one translation unit per precision instantiates these).
// bucket b serves D <= kBucketDim[b]; exact: D == kBucketDim[b] (no dimension guards)
constexpr int kNumBuckets = 6;
__host__ __device__ constexpr int bucket_dim(int b) {
    return b == 0 ? 4 : b == 1 ? 8 : b == 2 ? 12 : b == 3 ? 16 : b == 4 ? 20 : 24;
}
// Several integrals (tasks) / one integral (cluster launch of cs CTAs per cluster).
// (ax: the task kernel with the strata per axis from the descriptors, §3.2)
cudaError_t launch_sample_f32(int bucket, bool exact, int kind, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, const SampleArgs &a, bool ax = false);
cudaError_t launch_sample_f64(int bucket, bool exact, int kind, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, const SampleArgs &a, bool ax = false);
cudaError_t launch_sample_one_f32(int bucket, bool exact, int kind, dim3 grid, dim3 block,
                                  size_t smem, int cs, cudaStream_t s, const SampleOne &a);
cudaError_t launch_sample_one_f64(int bucket, bool exact, int kind, dim3 grid, dim3 block,
                                  size_t smem, int cs, cudaStream_t s, const SampleOne &a);
cudaError_t launch_eval_f32(int bucket, bool exact, int kind, cudaStream_t s, const Desc *desc,
                            int member, int64_t n, const uint64_t *h, const uint32_t *j,
                            uint32_t t, double *x, int32_t *idx, double *jac, double *f, int pw);
cudaError_t launch_eval_f64(int bucket, bool exact, int kind, cudaStream_t s, const Desc *desc,
                            int member, int64_t n, const uint64_t *h, const uint32_t *j,
                            uint32_t t, double *x, int32_t *idx, double *jac, double *f, int pw);
// (p1: the one-integral kernel's single-peak form, chosen at launch when the
// FP32 integrand has one peak and the bucket is dimension-exact)
cudaError_t sample_smem_config_f32(int bucket, bool exact, int kind, bool one, int max_smem,
                                   bool ax = false, bool p1 = false);
// §4.2: the data histogram of the map's training (buffer buf; f NULL: the integrand).
cudaError_t launch_precondition(int bucket, int kind, cudaStream_t s, const Desc *desc, int member,
                                int64_t n, const double *x, const double *f, uint32_t buf);
// (mo: the FP64 one-integral kernel with several outputs, App. B)
cudaError_t sample_smem_config_f64(int bucket, bool exact, int kind, bool one, int max_smem,
                                   bool mo = false, bool ax = false);
int sample_occupancy_f32(int bucket, bool exact, int kind, bool one, int threads, size_t smem,
                         bool ax = false, bool p1 = false);
int sample_occupancy_f64(int bucket, bool exact, int kind, bool one, int threads, size_t smem,
                         bool mo = false, bool ax = false);
// Resident CTAs of the one-integral kernel with clusters of cs CTAs (0 if it cannot run).
int sample_cluster_ctas_f32(int bucket, bool exact, int kind, int cs, int grid, int threads,
                            size_t smem, bool p1 = false);
int sample_cluster_ctas_f64(int bucket, bool exact, int kind, int cs, int grid, int threads,
                            size_t smem, bool mo = false);

}  // namespace vp
