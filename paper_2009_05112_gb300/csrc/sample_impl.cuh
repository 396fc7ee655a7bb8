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

#include "vp_internal.cuh"

namespace vp {

struct SampleArgs {
    const Desc *desc;          // [n_int] descriptors of the whole set
    const uint32_t *members;   // [n_group] set indices served by this launch
    const uint64_t *chunk_base;// [n_group + 1]
    uint32_t *head;            // queue head
    int n_group;
    int R;                     // samples per thread per chunk
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
//  GAUSS    per peak {a, log2(e)/w^2, c[D]}     f = sum a 2^(-k |x-c|^2)
//  BALL     per peak {a, r^2, c[D]}             f = sum a [|x-c|^2 < r^2]
//  EXPNORM  per peak {a, s log2(e), c[D]}       f = sum a 2^(-k |x-c|)
//  POSTERIOR {n, P, kN, kW, lcN, lcW, kprior, logref2, y[n], A[n][P]} in log2 units
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
    float f = 0.0f;
    for (int k = 0; k < K; ++k) {
        const float a = p[0], kk = p[1];
        const float *c = p + 2;
        float r2 = 0.0f;
#pragma unroll
        for (int mu = 0; mu < DMAX; ++mu) {
            if (mu < dim) {
                float dx = x[mu] - c[mu];
                r2 = fmaf(dx, dx, r2);
            }
        }
        if (kind == VP_GAUSS) f += a * ex2_approx(-kk * r2);
        else if (kind == VP_BALL) f += (r2 < kk) ? a : 0.0f;
        else f += a * ex2_approx(-kk * sqrtf(r2));
        p += 2 + dim;
    }
    return f;
}

template <int DMAX>
__device__ __forceinline__ double f_post64(const double *p, int dim, const double (&x)[DMAX]) {
    const int n = (int)p[0], npar = (int)p[1];
    const double sy = p[2], pw = p[3], log_ref = p[4];
    const double *y = p + 5;
    const double *A = p + 5 + n;
    const double s2pi = sqrt(6.283185307179586476925286766559);  // sqrt(2 pi)
    double w = 0.0;
#pragma unroll
    for (int mu = 0; mu < DMAX; ++mu)
        if (mu == npar) w = x[mu];
    double logl = 0.0;
    for (int i = 0; i < n; ++i) {
        double model = 0.0;
#pragma unroll
        for (int m = 0; m < DMAX; ++m)
            if (m < npar) model += A[i * npar + m] * x[m];
        const double r = y[i] - model;
        const double nar = (1.0 - w) / (s2pi * sy) * exp(-r * r / (2.0 * sy * sy));
        const double wid = w / (s2pi * 10.0 * sy) * exp(-r * r / (200.0 * sy * sy));
        logl += log(nar + wid);
    }
    double lp = 0.0;
#pragma unroll
    for (int m = 0; m < DMAX; ++m)
        if (m < npar) lp -= x[m] * x[m] / (2.0 * pw * pw);
    (void)dim;
    return exp(logl + lp - log_ref);
}

template <int DMAX>
__device__ __forceinline__ float f_post32(const float *p, int dim, const float (&x)[DMAX]) {
    const int n = (int)p[0], npar = (int)p[1];
    const float kN = p[2], kW = p[3], lcN = p[4], lcW = p[5], kpr = p[6], lref = p[7];
    const float *y = p + 8;
    const float *A = p + 8 + n;
    float w = 0.0f;
#pragma unroll
    for (int mu = 0; mu < DMAX; ++mu)
        if (mu == npar) w = x[mu];
    const float lw1 = lg2_approx(1.0f - w), lw = lg2_approx(w);
    float acc = 0.0f;
    for (int i = 0; i < n; ++i) {
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
    float c2 = 0.0f;
#pragma unroll
    for (int m = 0; m < DMAX; ++m)
        if (m < npar) c2 = fmaf(x[m], x[m], c2);
    (void)dim;
    return ex2_approx(fmaf(-kpr, c2, acc - lref));
}

// ---------------------------------------------------------------------------
// One sample: a1-a3.  Returns J and f; x[] and idx[] are filled.
// digits kd[] hold k_mu of hypercube h as the real type.
// ---------------------------------------------------------------------------
// FP32 Jacobians of adapted high-dimensional maps leave the FP32 range (e.g.
// 20 axes of N_g dx ~ 3e-3 give 3e-51), so the FP32 path carries J as a
// mantissa in [1, 2) and a separate integer exponent, renormalised after
// every group of four axes (four factors cannot leave the range: each is at
// least ~N_g ulp(x) and at most N_g (b - a)).
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

template <int DMAX, bool F64, int KIND>
__device__ __forceinline__ void sample_point(const Desc &d, const void *prm, uint32_t t,
                                             uint32_t h, uint32_t j,
                                             const typename Real<F64>::T (&kd)[DMAX],
                                             typename Real<F64>::T (&x)[DMAX],
                                             int (&idx)[DMAX],
                                             typename Real<F64>::T &jac, int &jexp,
                                             typename Real<F64>::T &f) {
    typedef typename Real<F64>::T T;
    const int dim = d.dim, n_g = d.n_g;
    const uint32_t calls = (uint32_t)((dim + 3) >> 2);
    T J = (T)1;
    int Je = 0;
#pragma unroll
    for (int q = 0; q < (DMAX + 3) / 4; ++q) {
        if (q < (int)calls) {
            U4 c = {j * calls + (uint32_t)q, h, t, d.integral_id};
            U4 r = philox4x32_10(c, d.key0, d.key1);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int mu = 4 * q + l;
                if (mu < DMAX && mu < dim) {
                    const uint32_t word = lane_of(r, l);
                    if (F64) {
                        const double u = u01_f64(word);
                        const double y = __ddiv_rn(__dadd_rn((double)kd[mu], u), (double)d.n_st);
                        const double yng = __dmul_rn(y, (double)n_g);
                        int i = (int)floor(yng);
                        i = i > n_g - 1 ? n_g - 1 : i;
                        const double delta = __dsub_rn(yng, (double)i);
                        const double *e = d.edges + (size_t)mu * (size_t)(n_g + 1);
                        const double e0 = __ldg(e + i), e1 = __ldg(e + i + 1);
                        const double dx = __dsub_rn(e1, e0);
                        x[mu] = (T)__dadd_rn(e0, __dmul_rn(dx, delta));
                        J = (T)__dmul_rn((double)J, __dmul_rn((double)n_g, dx));
                        idx[mu] = i;
                    } else {
                        const float u = u01_f32(word);
                        const float tt = ((float)kd[mu] + u) * d.ng_over_nst;
                        int i = (int)tt;
                        i = i > n_g - 1 ? n_g - 1 : i;
                        const float delta = tt - (float)i;
                        const float2 e = __ldg(d.tab + (size_t)mu * (size_t)n_g + i);
                        x[mu] = (T)fmaf(e.y, delta * d.inv_ng, e.x);
                        J = (T)((float)J * e.y);
                        idx[mu] = i;
                    }
                }
            }
            if (!F64) {
                float m = (float)J;
                renorm(m, Je);
                J = (T)m;
            }
        }
    }
    jac = J;
    jexp = Je;
    if (F64) {
        const double *p = (const double *)prm;
        double xv[DMAX];
#pragma unroll
        for (int mu = 0; mu < DMAX; ++mu) xv[mu] = (double)x[mu];
        if (KIND == VP_POSTERIOR) f = (T)f_post64<DMAX>(p, dim, xv);
        else f = (T)f_peaks64<DMAX>(KIND, p + 1, (int)p[0], dim, xv);
    } else {
        const float *p = (const float *)prm;
        float xv[DMAX];
#pragma unroll
        for (int mu = 0; mu < DMAX; ++mu) xv[mu] = (float)x[mu];
        if (KIND == VP_POSTERIOR) f = (T)f_post32<DMAX>(p, dim, xv);
        else f = (T)f_peaks32<DMAX>(KIND, p, d.n_peaks, dim, xv);
    }
}

// Mixed-radix digits of h: k_mu = (h / N_st^mu) mod N_st.
template <int DMAX, typename T>
__device__ __forceinline__ void decode_digits(uint32_t h, uint32_t n_st, int dim, T (&kd)[DMAX]) {
#pragma unroll
    for (int mu = 0; mu < DMAX; ++mu) {
        if (mu < dim) {
            uint32_t q = h / n_st;
            kd[mu] = (T)(h - q * n_st);
            h = q;
        } else {
            kd[mu] = (T)0;
        }
    }
}

// h -> h + 1 on the digits (carry propagation).
template <int DMAX, typename T>
__device__ __forceinline__ void next_digits(uint32_t n_st, int dim, T (&kd)[DMAX]) {
    bool carry = true;
#pragma unroll
    for (int mu = 0; mu < DMAX; ++mu) {
        if (carry && mu < dim) {
            T v = kd[mu] + (T)1;
            if (v >= (T)n_st) {
                kd[mu] = (T)0;
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
    __device__ __forceinline__ void add(double v) { s1 += v; s2 += v * v; }
    __device__ __forceinline__ double m1() const { return s1; }
    __device__ __forceinline__ double m2() const { return s2; }
};
template <> struct Acc<false> {
    float s1, c1, s2, c2;
    __device__ __forceinline__ void reset() { s1 = c1 = s2 = c2 = 0.0f; }
    __device__ __forceinline__ static void kahan(float &s, float &c, float v) {
        float y = __fsub_rn(v, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ void add(float v) {
        kahan(s1, c1, v);
        kahan(s2, c2, __fmul_rn(v, v));
    }
    __device__ __forceinline__ double m1() const { return (double)s1 - (double)c1; }
    __device__ __forceinline__ double m2() const { return (double)s2 - (double)c2; }
};

// ---------------------------------------------------------------------------
// The fused sampling kernel.
// Shared memory: [prm_words x 4 B][hist sum: hist_words x (4|8) B][hist count: hist_words x 4 B]
// ---------------------------------------------------------------------------
template <int DMAX, bool F64, int KIND>
__global__ void __launch_bounds__(256) k_sample(SampleArgs a) {
    typedef typename Real<F64>::T T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_chunk;
    uint32_t *sprm = (uint32_t *)smem;
    T *hs = (T *)(smem + (size_t)a.prm_words * 4);
    uint32_t *hc = (uint32_t *)(smem + (size_t)a.prm_words * 4 + (size_t)a.hist_words * sizeof(T));

    const uint64_t total = a.chunk_base[a.n_group];
    const uint32_t C = blockDim.x * (uint32_t)a.R;
    int cur = -1;
    const Desc *dp = nullptr;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_chunk = atomicAdd(a.head, 1u);
        __syncthreads();
        const uint64_t c = s_chunk;
        if (c >= total) break;
        const int g = upper_index(a.chunk_base, a.n_group, c);
        if (g != cur) {
            // leaving integral cur: flush its privatised histograms
            if (cur >= 0 && a.hist_shared) {
                const int bins = dp->dim * dp->n_g;
                const double unscale = ldexp(1.0, -2 * dp->st->scale_exp);
                for (int b = threadIdx.x; b < bins; b += blockDim.x) {
                    if (hc[b]) {
                        atomicAdd(dp->hsum + b, (double)hs[b] * unscale);
                        atomicAdd(dp->hcnt + b, hc[b]);
                    }
                }
                __syncthreads();
            }
            cur = g;
            dp = a.desc + a.members[g];
            if (a.hist_shared) {
                const int bins = dp->dim * dp->n_g;
                for (int b = threadIdx.x; b < bins; b += blockDim.x) {
                    hs[b] = (T)0;
                    hc[b] = 0u;
                }
            }
            __syncthreads();
        }
        const Desc &d = *dp;
        const int dim = d.dim;
        const uint64_t n_total = __ldcg(d.off + d.n_hc);
        const uint64_t c0 = (c - a.chunk_base[g]) * (uint64_t)C;
        const uint64_t c_end = min(c0 + (uint64_t)C, n_total);
        const uint64_t s_begin = c0 + (uint64_t)threadIdx.x * (uint64_t)a.R;
        const uint64_t s_end = min(s_begin + (uint64_t)a.R, c_end);
        if (s_begin >= s_end) continue;

        const uint32_t t = __ldcg(&d.st->t);
        const int sexp = __ldcg(&d.st->scale_exp);
        const T scale = (T)ldexp(1.0, sexp);
        const double unscale = ldexp(1.0, -sexp);
        const void *prm = F64 ? (const void *)d.prm : (const void *)d.prm32;

        uint64_t h = find_hcube(d.off, d.n_hc, s_begin);
        uint64_t next = __ldg(d.off + h + 1);
        uint32_t j = (uint32_t)(s_begin - __ldg(d.off + h));
        T kd[DMAX];
        decode_digits<DMAX, T>((uint32_t)h, d.n_st, dim, kd);
        Acc<F64> acc;
        acc.reset();
        for (uint64_t s = s_begin; s < s_end; ++s) {
            if (s == next) {
                atomicAdd(d.s1 + h, acc.m1() * unscale);
                atomicAdd(d.s2 + h, acc.m2() * unscale * unscale);
                acc.reset();
                ++h;
                next = __ldg(d.off + h + 1);
                j = 0;
                next_digits<DMAX, T>(d.n_st, dim, kd);
            }
            T x[DMAX];
            int idx[DMAX];
            T jac, f;
            int jexp;
            sample_point<DMAX, F64, KIND>(d, prm, t, (uint32_t)h, j, kd, x, idx, jac, jexp, f);
            T v;
            if (F64) v = jac * f * scale;
            else v = (T)scale2((float)(jac * f), jexp + sexp);
            acc.add(v);
            const T v2 = v * v;
#pragma unroll
            for (int mu = 0; mu < DMAX; ++mu) {
                if (mu < dim) {
                    const int b = mu * d.n_g + idx[mu];
                    if (a.hist_shared) {
                        if (v2 != (T)0) atomicAdd(hs + b, v2);
                        atomicAdd(hc + b, 1u);
                    } else {
                        if (v2 != (T)0) atomicAdd(d.hsum + b, (double)v2 * unscale * unscale);
                        atomicAdd(d.hcnt + b, 1u);
                    }
                }
            }
            ++j;
        }
        atomicAdd(d.s1 + h, acc.m1() * unscale);
        atomicAdd(d.s2 + h, acc.m2() * unscale * unscale);
    }
    if (cur >= 0 && a.hist_shared) {
        __syncthreads();
        const int bins = dp->dim * dp->n_g;
        const double unscale = ldexp(1.0, -2 * dp->st->scale_exp);
        for (int b = threadIdx.x; b < bins; b += blockDim.x) {
            if (hc[b]) {
                atomicAdd(dp->hsum + b, (double)hs[b] * unscale);
                atomicAdd(dp->hcnt + b, hc[b]);
            }
        }
    }
}

// Per-sample inspection: the same device code as k_sample, on listed samples.
template <int DMAX, bool F64, int KIND>
__global__ void k_eval(const Desc *desc, int member, int64_t n, const uint64_t *hs,
                       const uint32_t *js, uint32_t t, double *xo, int32_t *io, double *jo,
                       double *fo) {
    typedef typename Real<F64>::T T;
    const Desc &d = desc[member];
    const void *prm = F64 ? (const void *)d.prm : (const void *)d.prm32;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        T kd[DMAX], x[DMAX], jac, f;
        int idx[DMAX], jexp;
        decode_digits<DMAX, T>((uint32_t)hs[k], d.n_st, d.dim, kd);
        sample_point<DMAX, F64, KIND>(d, prm, t, (uint32_t)hs[k], js[k], kd, x, idx, jac, jexp, f);
        for (int mu = 0; mu < d.dim; ++mu) {
            xo[k * d.dim + mu] = (double)x[mu];
            io[k * d.dim + mu] = idx[mu];
        }
        jo[k] = ldexp((double)jac, jexp);
        fo[k] = (double)f;
    }
}

// Launch dispatch (one translation unit per precision instantiates these).
cudaError_t launch_sample_f32(int bucket, int kind, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, const SampleArgs &a);
cudaError_t launch_sample_f64(int bucket, int kind, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, const SampleArgs &a);
cudaError_t launch_eval_f32(int bucket, int kind, cudaStream_t s, const Desc *desc, int member,
                            int64_t n, const uint64_t *h, const uint32_t *j, uint32_t t,
                            double *x, int32_t *idx, double *jac, double *f);
cudaError_t launch_eval_f64(int bucket, int kind, cudaStream_t s, const Desc *desc, int member,
                            int64_t n, const uint64_t *h, const uint32_t *j, uint32_t t,
                            double *x, int32_t *idx, double *jac, double *f);
cudaError_t sample_smem_config_f32(int bucket, int kind, int max_smem);
cudaError_t sample_smem_config_f64(int bucket, int kind, int max_smem);
int sample_occupancy_f32(int bucket, int kind, int threads, size_t smem);
int sample_occupancy_f64(int bucket, int kind, int threads, size_t smem);

}  // namespace vp
