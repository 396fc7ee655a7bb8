// adapt.cu -- the per-hypercube and per-axis kernels of one vegas+ iteration:
//
//   k_chunks    prefix of sample chunks over the integrals of a launch group
//               (the sampling kernel's work queue);
//   k_estimate  step a6 and the first half of a7: per hypercube
//               dI_h = Omega S1_h / n_h, var_h = Omega^2 (S2_h/n_h - (S1_h/n_h)^2)/(n_h - 1)
//               (§3 Eq. sumI with §2.1 Eqs. MCIy, sigest inside each hypercube),
//               sigma_h = Omega sqrt(S2_h/n_h - (S1_h/n_h)^2) (§3 step 2) and
//               d_h = sigma_h^beta (§3 Eq. dh); sums over h in the library's
//               fixed order (blocks of 1024 hypercubes, pairwise halving inside
//               a block, the block sums by an adjacent pairwise tree), so
//               sum_h d_h -- and with it every integer n_h -- is reproducible
//               bit for bit;
//   k_alloc     a7: n_h = max(2, floor(N_ev d_h / sum d)) (§3 Eq. nh; or + 2;
//               a quotient within 2^-50 q below an integer counts as that
//               integer; the first allocation is always the equal split),
//               sums of n_h over kSubH hypercubes, then (last CTA) their offsets;
//   k_offsets   a7: exclusive offsets off[h] = sum_{h' < h} n_h';
//   k_refine    a8 on one axis (§2.3): d_i = hsum_i / hcnt_i, smoothing
//               (7,1)/(1,6,1)/(1,7) over 8, normalisation by sum d_i,
//               compression ((1 - d)/ln(1/d))^alpha (a zero d first raised to
//               the smallest normal double), then the equal-share
//               re-gridding as an inverse of the cumulative d: new edge k is
//               where the cumulative reaches k sum(d)/N_g, d spread uniformly
//               over each old increment (the same points the paper's four-step
//               walk produces, up to rounding).
//
// The per-hypercube kernels are memory-bound streams over N_h elements; the
// refinement is one CTA per (integral, axis) and latency-bound at N_g <= 4096.
#include <algorithm>
#include <cooperative_groups.h>
#include <cstdio>

#include "vp_internal.cuh"

namespace vp {

// Maps a flat block index to (integral, block within it) through a prefix
// array base[n + 1] held in device memory.
__device__ __forceinline__ int owner_of(const uint32_t *base, int n, uint32_t blk) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(base + mid) <= blk) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// k_chunks: chunk_base[g + 1] = chunk_base[g] + ceil(N_b / C) over the group
// members; resets the queue head.  One CTA.
// ---------------------------------------------------------------------------
__global__ void k_chunks(const Desc *desc, const uint32_t *members, int n_group,
                         uint64_t *chunk_base, uint32_t *head, uint32_t C) {
    __shared__ uint64_t s_cnt[1024];
    __shared__ uint64_t s_carry;
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0) {
        s_carry = 0;
        chunk_base[0] = 0;
        *head = 0u;
    }
    __syncthreads();
    for (int base = 0; base < n_group; base += blockDim.x) {
        const int g = base + threadIdx.x;
        uint64_t cnt = 0;
        if (g < n_group) {
            const Desc &d = desc[members[g]];
            const uint64_t n = d.off[d.n_hc];
            const uint32_t n32 = (uint32_t)n;  // n < 2^32; 32-bit division (no FP64 units)
            cnt = n32 / C + (n32 % C != 0u ? 1u : 0u);
        }
        s_cnt[threadIdx.x] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t run = s_carry;
            const int m = min((int)blockDim.x, n_group - base);
            for (int i = 0; i < m; ++i) {
                run += s_cnt[i];
                chunk_base[base + i + 1] = run;
            }
            s_carry = run;
        }
        __syncthreads();
    }
}

struct D3 { double a, b, c; };

// d_h = sigma_h^beta (§3 Eq. dh); beta = 0 and 1 exactly; 1/2 and 3/4 (the
// paper's default) as correctly rounded square roots, sqrt(sigma) and
// sqrt(sigma * sqrt(sigma)) -- each operation rounded once, the library's
// reading of these two powers, so that d_h (and every n_h) is reproducible
// bit for bit from sigma_h; other beta through pow.
__device__ __forceinline__ double damp(double sigma, double beta) {
    if (beta == 0.0) return 1.0;
    if (beta == 1.0) return sigma;
    if (beta == 0.5) return __dsqrt_rn(sigma);
    if (beta == 0.75) return __dsqrt_rn(__dmul_rn(sigma, __dsqrt_rn(sigma)));
    return pow(sigma, beta);
}

// d_h on the FP32 path: sigma_h^beta = 2^(beta/2 log2 var + beta log2 Omega)
// (§3 Eq. dh), log2 var from the exponent and mantissa bits of var with the
// FP32 log2 unit, the power's integer part put into the exponent field and its
// fraction through the FP32 exp2 unit (relative error ~1e-6; the FP64 path
// takes damp()).  On this part three FP64 square roots per hypercube would
// cost more than the sampling of a few of its samples, and the result is
// formed without an FP64 instruction.  var >= 0 and finite.
__device__ __forceinline__ double damp_var32(double var, const Desc &d) {
    if ((uint64_t)__double_as_longlong(d.beta) == 0ull) return 1.0;  // beta = 0: d = 1
    uint64_t b = (uint64_t)__double_as_longlong(var);
    if (b == 0ull) return 0.0;
    int E = (int)((b >> 52) & 0x7ffu);
    if (E == 0x7ff) return var;  // inf or NaN propagates (the iteration is flagged)
    if (E == 0) {  // subnormal: normalise the mantissa (integer operations)
        const int sh = __clzll((long long)(b & ((1ull << 52) - 1ull))) - 11;
        b = (b << sh) & ((1ull << 52) - 1ull);
        E = 1 - sh;
    }
    E -= 1023;
    const float m = __uint_as_float(0x3f800000u | (uint32_t)((b >> 29) & 0x7fffffu));  // [1, 2)
    const float Ef = (float)E;                            // exact
    const float p = d.half_beta_hi * Ef;
    const float err = fmaf(d.half_beta_hi, Ef, -p);       // p + err = hi E exactly
    const float fl = floorf(p);                           // exact (|p| < 2^23)
    const float y =
        (p - fl) + err + fmaf(d.half_beta_lo, Ef, d.half_beta_hi * lg2_approx(m)) + d.lob_f;
    return f2d_pow2(ex2_approx(y), (int)fl + d.lob_i);
}

// The same from t = n_h var and log2 n_h = L.x + L.y (a float pair from the
// table): d_h = 2^(beta/2 (log2 t - log2 n_h) + beta log2 Omega), so that var
// itself is never formed (one FP64 product less per hypercube).  The
// integer parts of beta/2 log2 t and beta/2 log2 n_h go into the exponent
// field, their fractions (whose difference is exact) through the exp2 unit.
// t >= 0 and finite.
__device__ __forceinline__ double damp_tn32(double t, float2 L, const Desc &d) {
    if ((uint64_t)__double_as_longlong(d.beta) == 0ull) return 1.0;  // beta = 0: d = 1
    uint64_t b = (uint64_t)__double_as_longlong(t);
    if (b == 0ull) return 0.0;
    int E = (int)((b >> 52) & 0x7ffu);
    if (E == 0x7ff) return t;  // inf or NaN propagates (the iteration is flagged)
    if (E == 0) {  // subnormal: normalise the mantissa (integer operations)
        const int sh = __clzll((long long)(b & ((1ull << 52) - 1ull))) - 11;
        b = (b << sh) & ((1ull << 52) - 1ull);
        E = 1 - sh;
    }
    E -= 1023;
    const float m = __uint_as_float(0x3f800000u | (uint32_t)((b >> 29) & 0x7fffffu));  // [1, 2)
    const float Ef = (float)E;                            // exact
    const float p = d.half_beta_hi * Ef;
    const float err = fmaf(d.half_beta_hi, Ef, -p);       // p + err = hi E exactly
    const float fl = floorf(p);
    const float q = d.half_beta_hi * L.x;
    const float qe = fmaf(d.half_beta_hi, L.x, -q);       // q + qe = hi L.x exactly
    const float fq = floorf(q);
    const float frac = (p - fl) - (q - fq);               // exact: both fractions on a 2^-21 grid
    const float small = fmaf(d.half_beta_lo, Ef, -fmaf(d.half_beta_hi, L.y, d.half_beta_lo * L.x));
    const float y = (frac + (err - qe)) + fmaf(d.half_beta_hi, lg2_approx(m), small) + d.lob_f;
    return f2d_pow2(ex2_approx(y), (int)fl - (int)fq + d.lob_i);
}

// ---------------------------------------------------------------------------
// k_estimate.  mode 0: from the moments (a6 + sigma_h + d_h), records the
// iteration; mode 1: dh[] holds sigma_h, turn it into d_h and sum; mode 2:
// dh[] holds d_h, sum only.
// Four CTAs (256 threads each) serve one block of 1024 hypercubes, so the
// per-hypercube FP64 work spreads over four SMs.  CTA q holds the terms
// 4t + q: the fixed-order tree's halving levels 512 .. 4 join terms of one
// residue class mod 4, so each CTA runs them on its own terms as levels
// 128 .. 1 and stores its class's sum; the last CTA of the integral takes the
// last two levels (classes 0 + 2 and 1 + 3, then their sum) for every block
// before the tree over the blocks -- the same additions in the same order,
// with no exchange between the CTAs of a block.
// ---------------------------------------------------------------------------
constexpr int kEstCtas = 4;

// The state fields the last step reads, loaded early by every CTA's thread 0
// (they change only in that step, so the loads overlap the sums instead of
// queueing behind one another at the end).
struct EstPre {
    uint32_t t, status;
    uint64_t n_samples, n_eval_total;
};
__device__ void finish_estimate(const Desc &d, double I, double V, double Sd, int mode,
                                const EstPre &pre);
__device__ __forceinline__ void block_levels(const Desc &d, uint64_t dst, double *red);
__device__ __forceinline__ void estimate_last_cta(const Desc &d, uint32_t n_cta, int mode,
                                                  const EstPre &pre, double *red, bool *s_last,
                                                  bool residues = false);

// 1/n for n beyond the table (rare: a call, so that none of its FP64 work is
// hoisted into the common path)
__device__ __noinline__ double recip_u32(uint32_t n) { return 1.0 / u32_to_f64(n); }

// (PREC: -1 the descriptor's precision at run time, else VP_FP64 / VP_FP32
// for a set whose integrals all take that path: one path compiled)
template <int PREC = -1>
__device__ __forceinline__ D3 hcube_terms(const Desc &d, uint64_t h, int mode, uint32_t par) {
    D3 v = {0.0, 0.0, 0.0};
    if (h >= d.n_hc) return v;
    if (mode == 0) {
        // (reciprocals of the small integer n_h come from the set's table, one
        // 32-byte entry per n: 1/n, 1/(n (n-1)), log2 n)
        const uint32_t nh = d.n_h[h];
        const bool in_tab = nh < (uint32_t)kInvTab;
        double2 e01 = make_double2(0.0, 0.0);
        float2 e2 = make_float2(0.0f, 0.0f);
        if (in_tab) {
            const double2 *e = (const double2 *)(d.inv_tab + 4 * (size_t)nh);
            e01 = __ldg(e);
            const double2 w = __ldg(e + 1);
            e2 = make_float2(__uint_as_float((uint32_t)__double_as_longlong(w.x)),
                             __uint_as_float((uint32_t)((uint64_t)__double_as_longlong(w.x) >> 32)));
        }
        const double inv_n = in_tab ? e01.x : recip_u32(nh);
        const uint64_t ph = (uint64_t)par * d.n_hc + h;
        const double s1 = d.s1[ph], s2 = d.s2[ph];
        // the other buffer collects the next iteration's sums
        const uint64_t qh = (uint64_t)(par ^ 1u) * d.n_hc + h;
        d.s1[qh] = 0.0;
        d.s2[qh] = 0.0;
        // FP64 is scarce on this part: m1 = S1 / n_h, t = S2 - S1 m1 (one fused
        // multiply-add; t = n_h var) and, on the FP32 path, var / (n_h - 1) as
        // t / (n_h (n_h - 1)) from the table and d_h from t and log2 n_h: three
        // FP64 operations (four beyond the table and on the FP64 path, which
        // forms var = t / n_h); Omega and Omega^2 multiply the two totals
        // (finish_estimate)
        const bool fp32 = PREC < 0 ? d.prec == VP_FP32 : PREC == VP_FP32;
        const double m1 = s1 * inv_n;
        double t = __fma_rn(-s1, m1, s2);
        {  // a rounding-negative variance (or -0) is zero; a NaN stays NaN
            const long long tb = __double_as_longlong(t);
            if (tb < 0ll && (tb & 0x7fffffffffffffffll) <= 0x7ff0000000000000ll) t = 0.0;
        }
        v.a = m1;
        if (fp32 && in_tab) {
            v.b = t * e01.y;
            v.c = damp_tn32(t, e2, d);
        } else {
            const double inv_n1 =
                nh - 1 < (uint32_t)kInvTab ? __ldg(d.inv_tab + 4 * (size_t)(nh - 1)) : recip_u32(nh - 1);
            const double var = t * inv_n;
            v.b = var * inv_n1;
            v.c = fp32 ? damp_var32(var, d) : damp(d.omega * sqrt(var), d.beta);
        }
        d.dh[h] = v.c;
    } else if (mode == 1) {
        v.c = damp(d.dh[h], d.beta);
        d.dh[h] = v.c;
    } else {
        v.c = d.dh[h];
    }
    return v;
}

__global__ void __launch_bounds__(256, 4)
    k_estimate(const Desc *desc, const uint32_t *tree_base, int n_int, int mode) {
    __shared__ double red[3 * 256];
    __shared__ bool s_last;
    pdl_wait();
    pdl_trigger();
    const int q = (int)(blockIdx.x % kEstCtas);  // residue class of this CTA
    const uint32_t tb = blockIdx.x / kEstCtas;
    const int b = owner_of(tree_base, n_int, tb);
    const Desc &d = desc[b];
    const uint32_t k = tb - tree_base[b];
    const int t = threadIdx.x;
    const uint32_t par = d.st->t & 1u;  // buffer of the iteration being estimated
    EstPre pre = {0u, 0u, 0ull, 0ull};
    if (t == 0) {
        pre.t = d.st->t;
        pre.status = d.st->status;
        pre.n_samples = d.st->n_samples;
        pre.n_eval_total = d.st->n_eval_total;
    }
    const D3 v = hcube_terms(d, (uint64_t)k * kTreeBlock + 4 * t + q, mode, par);
    if (mode == 0) {  // clear the other histogram buffer, spread over this integral's CTAs
        const int bins = d.dim * d.n_g;
        double *hs = d.hsum + (size_t)(par ^ 1u) * bins;
        uint32_t *hc = d.hcnt + (size_t)(par ^ 1u) * bins;
        const int stride = (int)d.n_tree * kEstCtas * 256;
        for (int i = (int)(k * kEstCtas + q) * 256 + t; i < bins; i += stride) {
            hs[i] = 0.0;
            hc[i] = 0u;
        }
    }
    red[t] = v.a;
    red[256 + t] = v.b;
    red[512 + t] = v.c;
    // the halving levels 512 .. 4 of the block join terms of one residue class
    // mod 4 (term i and term i + s, s a multiple of 4): on this CTA's terms
    // 4t + q they are the levels 128 .. 1 over t; the last two levels (2, 1)
    // join the four classes' sums, in the last CTA
    block_levels(d, 3 * (uint64_t)d.n_tree + 12 * (uint64_t)k + 3 * (uint64_t)q, red);
    estimate_last_cta(d, d.n_tree * kEstCtas, mode, pre, red, &s_last, true);
}

// A pairwise halving over 256 values, one CTA of 256 threads: red[c][t]
// (red = 3 x 256 doubles in shared memory) holds value t of series c -- in
// the wide form the sum of terms t, t + 256, t + 512, t + 768 of a block (its
// first two halving levels), in the four-CTA form the term 4t + q; the
// levels 128 .. 1 leave the sum in part[dst + c] (block_levels).  Then, once
// per CTA, the ticket and in the last CTA of the integral the block sums in
// the fixed tree order and the iteration's bookkeeping (estimate_last_cta).
__device__ __forceinline__ void block_levels(const Desc &d, uint64_t dst, double *red) {
    const int t = threadIdx.x;
    double *r0 = red, *r1 = red + 256, *r2 = red + 512;
    __syncthreads();
    for (int s = 128; s >= 64; s >>= 1) {
        if (t < s) {
            r0[t] = __dadd_rn(r0[t], r0[t + s]);
            r1[t] = __dadd_rn(r1[t], r1[t + s]);
            r2[t] = __dadd_rn(r2[t], r2[t + s]);
        }
        __syncthreads();
    }
    // levels 32 .. 1: one warp per sum, the three in parallel (a chain of
    // dependent FP64 additions is slow on this part)
    const int w = t >> 5, l = t & 31;
    if (w < 3) {
        const double *r = w == 0 ? r0 : (w == 1 ? r1 : r2);
        double x = __dadd_rn(r[l], r[l + 32]);
        for (int s = 16; s >= 1; s >>= 1) x = __dadd_rn(x, __shfl_down_sync(0xffffffffu, x, s));
        if (l == 0) d.part[dst + w] = x;
    }
}

__device__ __forceinline__ void estimate_last_cta(const Desc &d, uint32_t n_cta, int mode,
                                                  const EstPre &pre, double *red, bool *s_last,
                                                  bool residues) {
    const int t = threadIdx.x;
    if (t < 96 && (t & 31) == 0) __threadfence();  // (the writers of part[]: lane 0 of warps 0-2)
    __syncthreads();
    if (t == 0) {
        const uint32_t ticket = atomicAdd(&d.st->done_est, 1u);
        *s_last = (ticket == n_cta - 1);
    }
    __syncthreads();
    if (!*s_last) return;
    // last CTA of this integral: the block sums in the fixed tree order
    __threadfence();
    __syncthreads();
    if (residues) {
        // the block sums from their residue classes: the last two halving
        // levels (term 0 += term 2, 1 += 3; then 0 += 1)
        const double *r4 = d.part + 3 * (size_t)d.n_tree;
        for (uint32_t i = t; i < 3 * d.n_tree; i += blockDim.x) {
            const uint32_t k = i / 3, c = i - 3 * k;
            const double *q = r4 + 12 * (size_t)k + c;
            d.part[i] = __dadd_rn(__dadd_rn(__ldcg(q), __ldcg(q + 6)),
                                  __dadd_rn(__ldcg(q + 3), __ldcg(q + 9)));
        }
        __threadfence_block();
        __syncthreads();
    }
    double tot[3];
    block_tree_sum<3>(d.part, d.n_tree, red, tot);
    if (t != 0) return;
    d.st->done_est = 0u;
    finish_estimate(d, tot[0], tot[1], tot[2], mode, pre);
}

// k_estimate for many blocks (large N_h): one CTA of 256 threads per block of
// 1024 hypercubes, each thread four of them (t, t + 256, t + 512, t + 768),
// so that more loads are in flight per thread; the first two halving levels
// are the thread's own (t + 512 joins t, t + 768 joins t + 256, then t + 256
// joins t), the same tree as the cluster form's.
template <int PREC>
__global__ void __launch_bounds__(256, 4)
    k_estimate_wide(const Desc *desc, const uint32_t *tree_base, int n_int, int mode, int group) {
    __shared__ double red[3 * 256];
    __shared__ bool s_last;
    pdl_wait();
    pdl_trigger();
    // blocks k0 .. k0 + group - 1 of one integral (group > 1 only for one integral)
    const uint32_t tb = blockIdx.x;
    const int b = group > 1 ? 0 : owner_of(tree_base, n_int, tb);
    const Desc &d = desc[b];
    const uint32_t k0 = group > 1 ? tb * (uint32_t)group : tb - tree_base[b];
    const uint32_t k1 = min(k0 + (uint32_t)group, d.n_tree);
    const int t = threadIdx.x;
    const uint32_t par = d.st->t & 1u;
    EstPre pre = {0u, 0u, 0ull, 0ull};
    if (t == 0) {
        pre.t = d.st->t;
        pre.status = d.st->status;
        pre.n_samples = d.st->n_samples;
        pre.n_eval_total = d.st->n_eval_total;
    }
    if (mode == 0) {  // clear the other histogram buffer, spread over this integral's CTAs
        const int bins = d.dim * d.n_g;
        double *hs = d.hsum + (size_t)(par ^ 1u) * bins;
        uint32_t *hc = d.hcnt + (size_t)(par ^ 1u) * bins;
        const uint32_t n_cta = (d.n_tree + (uint32_t)group - 1u) / (uint32_t)group;
        const int stride = (int)n_cta * 256;
        for (int i = (int)(k0 / (uint32_t)group) * 256 + t; i < bins; i += stride) {
            hs[i] = 0.0;
            hc[i] = 0u;
        }
    }
    for (uint32_t k = k0; k < k1; ++k) {
        const uint64_t h0 = (uint64_t)k * kTreeBlock + t;
        const D3 v0 = hcube_terms<PREC>(d, h0, mode, par);
        const D3 v1 = hcube_terms<PREC>(d, h0 + 256, mode, par);
        const D3 v2 = hcube_terms<PREC>(d, h0 + 512, mode, par);
        const D3 v3 = hcube_terms<PREC>(d, h0 + 768, mode, par);
        __syncthreads();  // (the previous block's last reads of red are done)
        red[t] = __dadd_rn(__dadd_rn(v0.a, v2.a), __dadd_rn(v1.a, v3.a));
        red[256 + t] = __dadd_rn(__dadd_rn(v0.b, v2.b), __dadd_rn(v1.b, v3.b));
        red[512 + t] = __dadd_rn(__dadd_rn(v0.c, v2.c), __dadd_rn(v1.c, v3.c));
        block_levels(d, 3 * (uint64_t)k, red);
    }
    estimate_last_cta(d, (d.n_tree + (uint32_t)group - 1u) / (uint32_t)group, mode, pre, red,
                      &s_last);
}

// The iteration's totals I_j, sigma_j^2 and sum d recorded in the state (one
// thread): history, the FP32 path's scale, the iteration count and, for a
// served request, the stop rule.
__device__ void finish_estimate(const Desc &d, double I, double V, double Sd, int mode,
                                const EstPre &pre) {
    State *st = d.st;
    I *= d.omega;  // (the per-hypercube terms leave Omega and Omega^2 to the totals)
    V *= d.omega2;
    st->sum_d = Sd;
    st->inv_sum_d = Sd > 0.0 ? 1.0 / Sd : 0.0;
    {
        const double c = d.n_ev_d * st->inv_sum_d;
        const bool normal = Sd >= 2.2250738585072014e-308 && c >= 2.2250738585072014e-308 &&
                            c <= 1.7976931348623157e308;
        st->alloc_c = normal ? c : 0.0;
        // d_h >= 2^-1021 keeps N_ev d_h normal for every N_ev >= 1 (a constant:
        // no FP64 division in this serial step; the rare d_h below it take the
        // exact quotient)
        st->alloc_dmin = 4.4501477170144028e-308;
    }
    if (mode == 0) {
        const uint32_t tt = pre.t;
        if (tt < (uint32_t)d.hist_cap) {
            d.hist_i[tt] = I;
            d.hist_var[tt] = V;
        }
        st->last_i = I;
        st->last_var = V;
        st->n_eval_total = pre.n_eval_total + pre.n_samples;
        if (!isfinite(I) || !isfinite(V)) st->status = pre.status | kStatusNonFinite;
        // keep J f 2^scale_exp near one in the next iteration: the mean of J f
        // over y-space is the integral (an exact power-of-two rescaling).
        if (isfinite(I) && I != 0.0) {
            int e = ilogb(fabs(I));
            e = e > 120 ? 120 : (e < -120 ? -120 : e);
            st->scale_exp = -e;
        }
        st->t = tt + 1;
        if (d.done_out) {  // a served request: the stop rule
            if ((int)tt >= d.discard && isfinite(I) && isfinite(V)) {
                if (V > 0.0) {
                    st->cw += 1.0 / V;
                    st->cwi += I / V;
                } else {
                    st->n_zero += 1u;
                    st->zsum += I;
                }
            }
            uint32_t done = 0u;
            const int meas = (int)tt + 1 - d.discard;
            if (meas >= d.min_meas && meas >= 1) {
                if (st->n_zero > 0u) {
                    done = kDoneStop | kDoneConverged;  // an exact iteration
                } else if (st->cw > 0.0) {
                    const double mean = st->cwi / st->cw, sdev = sqrt(1.0 / st->cw);
                    if (sdev <= d.rtol * fabs(mean)) done = kDoneStop | kDoneConverged;
                }
            }
            if ((int)tt + 1 >= d.stop_it || (st->status & kStatusNonFinite)) done |= kDoneStop;
            st->done = done;
            *d.done_out = done;
        }
    }
}

// ---------------------------------------------------------------------------
// Floor of a double 0 <= q < 2^52 from its bits (no FP64 instructions: they
// are scarce on this part), with two tests on the distance to the integers:
// near -- q is within 2^-40 q of an integer (the reciprocal product below is
// within a few ulp of the IEEE quotient, so only such q need the division);
// tie  -- q lies within 2^-50 q below an integer, i.e. exactly
//         (floor(q) + 1) - q <= q 2^-50, the test of the allocation reading.
// With q = M 2^(e - 52), M in [2^52, 2^53): distances are counted in units
// of 2^(e - 52) and q itself is M units, so "within c q" is "<= floor(c M)".
// ---------------------------------------------------------------------------
struct FloorBits {
    uint64_t iq;
    bool near, tie;
};

__device__ __forceinline__ FloorBits floor_bits(double q) {
    FloorBits r = {0ull, false, false};
    const uint64_t b = (uint64_t)__double_as_longlong(q);
    if (b == 0ull) return r;
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    const uint64_t M = (b & ((1ull << 52) - 1ull)) | (1ull << 52);
    if (e >= 52) {  // an integer (not reached: q < 2^32 here)
        r.iq = M << (e - 52);
        return r;
    }
    uint64_t up;  // distance to the next integer, in units
    if (e >= 0) {
        const int sh = 52 - e;
        r.iq = M >> sh;
        const uint64_t frac = M & ((1ull << sh) - 1ull);
        up = (1ull << sh) - frac;
        r.near = frac <= (M >> 40);
    } else if (e == -1) {  // q in [1/2, 1): the next integer is 1 = 2^53 units
        up = (1ull << 53) - M;
    } else {
        return r;  // q < 1/2: floor 0, far from both integers
    }
    r.near = r.near || up <= (M >> 40);
    r.tie = up <= (M >> 50);
    return r;
}

__device__ __forceinline__ bool finite_bits(double x) {
    return ((uint64_t)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// n_h of one hypercube (§3 Eq. nh with the library's reading): max(2,
// floor(N_ev d_h / sum d)), or floor(.) + 2; the equal split when sum d = 0 or
// on the first allocation.  The quotient is the IEEE one, (N_ev d_h) then
// / sum d.  One FP64 product decides almost every hypercube: q ~ d_h c with
// c = N_ev / sum d (within a few ulp of the IEEE quotient), and only a q within
// 2^-40 q of an integer takes the exact quotient; where N_ev d_h would not be
// a normal number, or c is unavailable (st.alloc_c = 0), the exact quotient
// is taken directly.
struct AllocK {
    double n_ev_d, sum_d, c, dmin;
};

__device__ __forceinline__ uint32_t alloc_one(const Desc &d, double dh, const AllocK &K,
                                              int initial) {
    uint64_t iq;
    if (__double_as_longlong(K.sum_d) > 0ll) {  // sum d > 0 (sum_d is finite here)
        if ((uint64_t)__double_as_longlong(dh) == 0ull) {
            iq = 0ull;  // (a zero numerator is exact)
        } else if ((uint64_t)__double_as_longlong(dh) >= (uint64_t)__double_as_longlong(K.dmin) &&
                   (uint64_t)__double_as_longlong(K.c) != 0ull) {  // (integer compares: d_h, c >= 0)
            const double q = dh * K.c;
            FloorBits f = floor_bits(q);
            iq = f.iq;
            // (below 2 - tol the max(2, .) decides)
            const bool above = (uint64_t)__double_as_longlong(q) > 0x3FF8000000000000ull;  // q > 1.5
            if ((d.plus2 || above) && f.near) {
                f = floor_bits(__ddiv_rn(__dmul_rn(K.n_ev_d, dh), K.sum_d));
                iq = f.iq + (f.tie ? 1ull : 0ull);
            }
        } else {
            const FloorBits f = floor_bits(__ddiv_rn(__dmul_rn(K.n_ev_d, dh), K.sum_d));
            iq = f.iq + (f.tie ? 1ull : 0ull);
        }
    } else {
        const FloorBits f = floor_bits(__ddiv_rn(K.n_ev_d, (double)d.n_hc));
        iq = f.iq + (f.tie ? 1ull : 0ull);
    }
    if (d.plus2 && !initial) return (uint32_t)iq + 2u;
    return iq > 2ull ? (uint32_t)iq : 2u;
}

__device__ __forceinline__ AllocK alloc_consts(const Desc &d) {
    AllocK K;
    K.n_ev_d = d.n_ev_d;
    K.sum_d = d.st->sum_d;
    K.c = d.st->alloc_c;
    K.dmin = d.st->alloc_dmin;
    return K;
}

// Exclusive scan of one value per thread over a CTA of 256 threads, in 32-bit
// arithmetic (sums of n_h: an iteration's samples number below 2^32); returns
// the exclusive prefix and (in *total) the CTA's sum.
__device__ __forceinline__ uint32_t cta_exclusive_scan32(uint32_t v, uint32_t *s_w,
                                                         uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    uint32_t base = 0u, all = 0u;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t x = s_w[w];
        if (w < warp) base += x;
        all += x;
    }
    __syncthreads();  // s_w may be reused
    *total = all;
    return base + inc - v;
}

// Sum of one 32-bit value per thread over a CTA of 256 threads (every thread
// gets it).
__device__ __forceinline__ uint32_t cta_sum32(uint32_t v, uint32_t *s_w) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t all = 0u;
#pragma unroll
    for (int w = 0; w < 8; ++w) all += s_w[w];
    __syncthreads();
    return all;
}

// ---------------------------------------------------------------------------
// k_alloc: n_h, one hypercube per thread, kSub CTAs of kSubH hypercubes per
// block of kTreeBlock (so the FP64 work spreads over the whole GPU); each CTA
// stores its sum of n_h and the last CTA of each integral turns those sums
// into offsets (integers: any order is exact) and records the total.
// Skipped (allocation kept) when sum_d is not finite; the status flag records it.
// ---------------------------------------------------------------------------
// (eight CTAs per SM: the batched loads of the last CTA's scan must not cost
// the other CTAs their occupancy)
template <uint32_t kScanV>
__device__ __forceinline__ void alloc_scan_tail(const Desc &d, uint32_t n_sub, uint32_t *s_w,
                                                uint32_t *s_carry);

__global__ void __launch_bounds__(kSubH, 8) k_alloc(const Desc *desc, const uint32_t *tree_base,
                                                    int n_int, int initial) {
    __shared__ uint32_t s_w[8];
    __shared__ bool s_last;
    __shared__ uint32_t s_carry;
    pdl_wait();
    pdl_trigger();
    const uint32_t tb = blockIdx.x / kSub;
    const int b = owner_of(tree_base, n_int, tb);
    const Desc &d = desc[b];
    const uint32_t sub = (tb - tree_base[b]) * kSub + blockIdx.x % kSub;
    const uint64_t h = (uint64_t)sub * kSubH + threadIdx.x;
    const AllocK K = alloc_consts(d);
    if (!finite_bits(K.sum_d)) {
        if (threadIdx.x == 0 && sub == 0) d.st->status |= kStatusNonFinite;
        return;
    }
    uint32_t n = 0;
    if (h < d.n_hc) {
        n = alloc_one(d, d.dh[h], K, initial);
        d.n_h[h] = n;
    }
    const uint32_t tot = cta_sum32(n, s_w);
    const uint32_t n_sub = d.n_tree * kSub;
    if (threadIdx.x == 0) {
        d.bsum[sub] = tot;
        __threadfence();
        const uint32_t ticket = atomicAdd(&d.st->done_alloc, 1u);
        s_last = (ticket == n_sub - 1);
        s_carry = 0u;
    }
    __syncthreads();
    if (!s_last) return;
    alloc_scan_tail<4>(d, n_sub, s_w, &s_carry);
}

// The last CTA of an integral's allocation: the exclusive scan of its n_sub
// partial sums of n_h in place (bsum[q] becomes the offset of part q),
// off[N_h] and the iteration's sample count.  kScanV consecutive sums per
// thread per pass, their loads issued together; 32-bit sums (an iteration's
// samples number below 2^32).
template <uint32_t kScanV>
__device__ __forceinline__ void alloc_scan_tail(const Desc &d, uint32_t n_sub, uint32_t *s_w,
                                                uint32_t *s_carry) {
    __threadfence();
    for (uint32_t q0 = 0; q0 < n_sub; q0 += kSubH * kScanV) {
        const uint32_t q = q0 + threadIdx.x * kScanV;
        uint32_t v[kScanV];
#pragma unroll
        for (uint32_t k = 0; k < kScanV; ++k)
            v[k] = q + k < n_sub ? (uint32_t)__ldcg(d.bsum + q + k) : 0u;
        uint32_t own = 0u;
#pragma unroll
        for (uint32_t k = 0; k < kScanV; ++k) {  // exclusive within the thread's run
            const uint32_t x = v[k];
            v[k] = own;
            own += x;
        }
        uint32_t all;
        const uint32_t ex = cta_exclusive_scan32(own, s_w, &all);
        const uint32_t base = *s_carry + ex;
#pragma unroll
        for (uint32_t k = 0; k < kScanV; ++k)
            if (q + k < n_sub) d.bsum[q + k] = (unsigned long long)(base + v[k]);
        __syncthreads();
        if (threadIdx.x == 0) *s_carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned long long run = *s_carry;
        d.off[d.n_hc] = run;
        d.st->n_samples = run;
        d.st->done_alloc = 0u;
    }
}

// k_offsets: off[h] = offset of the sub-block + exclusive scan of n_h within it.
__global__ void __launch_bounds__(kSubH) k_offsets(const Desc *desc, const uint32_t *tree_base,
                                                   int n_int) {
    __shared__ uint32_t s_w[8];
    pdl_wait();
    const uint32_t tb = blockIdx.x / kSub;
    const int b = owner_of(tree_base, n_int, tb);
    const Desc &d = desc[b];
    if (!finite_bits(d.st->sum_d)) return;
    const uint32_t sub = (tb - tree_base[b]) * kSub + blockIdx.x % kSub;
    const uint64_t h = (uint64_t)sub * kSubH + threadIdx.x;
    const uint32_t n = h < d.n_hc ? d.n_h[h] : 0u;
    uint32_t tot;
    const uint32_t ex = cta_exclusive_scan32(n, s_w, &tot);
    if (h < d.n_hc) d.off[h] = d.bsum[sub] + ex;
}

// k_alloc and k_offsets for many blocks (large N_h): one CTA of kSubH threads
// per block of kTreeBlock hypercubes, thread t holding hypercubes 4t .. 4t + 3
// of the block (vector loads and stores), one sum of n_h per block; the last
// CTA scans the n_tree block sums (16 per thread per pass).
__device__ __forceinline__ void load4_dh(const Desc &d, uint64_t h0, bool full, double (&dh)[4]) {
    if (full) {
        const double2 a = __ldcs((const double2 *)(d.dh + h0));
        const double2 b = __ldcs((const double2 *)(d.dh + h0 + 2));
        dh[0] = a.x; dh[1] = a.y; dh[2] = b.x; dh[3] = b.y;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) dh[q] = h0 + q < d.n_hc ? d.dh[h0 + q] : 0.0;
    }
}

__global__ void __launch_bounds__(kSubH, 4) k_alloc_wide(const Desc *desc,
                                                         const uint32_t *tree_base, int n_int,
                                                         int initial, int group) {
    __shared__ uint32_t s_w[8];
    __shared__ bool s_last;
    __shared__ uint32_t s_carry;
    pdl_wait();
    pdl_trigger();
    // blocks k0 .. k0 + group - 1 of one integral (group > 1 only for one integral)
    const uint32_t tb = blockIdx.x;
    const int b = group > 1 ? 0 : owner_of(tree_base, n_int, tb);
    const Desc &d = desc[b];
    const uint32_t k0 = group > 1 ? tb * (uint32_t)group : tb - tree_base[b];
    const uint32_t k1 = min(k0 + (uint32_t)group, d.n_tree);
    const AllocK K = alloc_consts(d);
    if (!finite_bits(K.sum_d)) {
        if (threadIdx.x == 0 && k0 == 0) d.st->status |= kStatusNonFinite;
        return;
    }
    for (uint32_t k = k0; k < k1; ++k) {
        const uint64_t h0 = (uint64_t)k * kTreeBlock + 4u * threadIdx.x;
        const bool full = h0 + 4 <= d.n_hc;
        double dh[4];
        load4_dh(d, h0, full, dh);
        uint32_t n[4], own = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            n[q] = h0 + q < d.n_hc ? alloc_one(d, dh[q], K, initial) : 0u;
            own += n[q];
        }
        if (full) {
            *(uint4 *)(d.n_h + h0) = make_uint4(n[0], n[1], n[2], n[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (h0 + q < d.n_hc) d.n_h[h0 + q] = n[q];
        }
        const uint32_t tot = cta_sum32(own, s_w);
        if (threadIdx.x == 0) d.bsum[k] = tot;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t ticket = atomicAdd(&d.st->done_alloc, 1u);
        const uint32_t n_cta = (d.n_tree + (uint32_t)group - 1u) / (uint32_t)group;
        s_last = (ticket == n_cta - 1);
        s_carry = 0u;
    }
    __syncthreads();
    if (!s_last) return;
    alloc_scan_tail<16>(d, d.n_tree, s_w, &s_carry);
}

__global__ void __launch_bounds__(kSubH, 4) k_offsets_wide(const Desc *desc,
                                                           const uint32_t *tree_base, int n_int,
                                                           int group) {
    __shared__ uint32_t s_w[8];
    pdl_wait();
    const uint32_t tb = blockIdx.x;
    const int b = group > 1 ? 0 : owner_of(tree_base, n_int, tb);
    const Desc &d = desc[b];
    if (!finite_bits(d.st->sum_d)) return;
    const uint32_t k0 = group > 1 ? tb * (uint32_t)group : tb - tree_base[b];
    const uint32_t k1 = min(k0 + (uint32_t)group, d.n_tree);
    for (uint32_t k = k0; k < k1; ++k) {
        const uint64_t h0 = (uint64_t)k * kTreeBlock + 4u * threadIdx.x;
        const bool full = h0 + 4 <= d.n_hc;
        uint32_t n[4];
        if (full) {
            const uint4 v = __ldcs((const uint4 *)(d.n_h + h0));
            n[0] = v.x; n[1] = v.y; n[2] = v.z; n[3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) n[q] = h0 + q < d.n_hc ? d.n_h[h0 + q] : 0u;
        }
        const unsigned long long blk = d.bsum[k];
        uint32_t e[4], own = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            e[q] = own;
            own += n[q];
        }
        uint32_t tot;
        const uint32_t ex = cta_exclusive_scan32(own, s_w, &tot);
        const unsigned long long base = blk + ex;
        if (full) {
            ulonglong2 *o = (ulonglong2 *)(d.off + h0);
            o[0] = make_ulonglong2(base + e[0], base + e[1]);
            o[1] = make_ulonglong2(base + e[2], base + e[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (h0 + q < d.n_hc) d.off[h0 + q] = base + e[q];
        }
    }
}

// ---------------------------------------------------------------------------
// k_refine: a8 for one (integral, axis) on a cluster of kRefineCtas CTAs.
// CTA r of the cluster owns increments [r S, (r + 1) S), S = ceil(N_g / 8);
// the FP64 work (d_i, smoothing, log and root of the compression) is spread
// over the cluster, and the CTAs exchange the partial sums they need through
// distributed shared memory:
//   1. d_i for the owned range plus one halo increment each side; partial sum
//   2. sum_i d_i = the 8 partials in rank order (identical in every CTA)
//   3. smoothing, normalisation, compression; local inclusive scan
//   4. cumulative base of every CTA = the totals of lower ranks
//   5. new edge k (for k in the owned range) where the cumulative reaches
//      k sum(c)/N_g: the owning rank is found from the totals, then a binary
//      search in that rank's local scan, read remotely
//   6. edges and the FP32 table {x_i, dx_i} written back.
// ---------------------------------------------------------------------------
constexpr int kRefineCtas = 8;
constexpr int kRefineThreads = 128;
constexpr int kRefineSlice = kMaxNg / kRefineCtas;  // 512

struct RefineShared {
    double x[kRefineSlice + 1];   // old edges x_{i0} .. x_{i0 + S}
    double d[kRefineSlice + 2];   // raw d_{i0 - 1} .. d_{i0 + S}
    double c[kRefineSlice];       // compressed d of the owned increments
    double C[kRefineSlice];       // local inclusive scan of c
    double xn[kRefineSlice + 1];  // new edges of the owned range (and one more)
    double red[kRefineThreads / 32];
    double part;                  // sum of own raw d
    double tot;                   // sum of own c
    int n_own;
};

__global__ void __cluster_dims__(kRefineCtas, 1, 1) __launch_bounds__(kRefineThreads)
    k_refine(const Desc *desc, const uint32_t *axis_base, int n_int) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ RefineShared sm;
    pdl_wait();
    const int rank = (int)cl.block_rank();
    const uint32_t axis_id = blockIdx.x / kRefineCtas;
    const int b = owner_of(axis_base, n_int, axis_id);
    const Desc &d = desc[b];
    const int mu = (int)(axis_id - axis_base[b]);
    const int n_g = d.n_g;
    if (d.alpha == 0.0 || n_g < 2) return;  // uniform over the cluster
    const int S = (n_g + kRefineCtas - 1) / kRefineCtas;
    const int i0 = min(rank * S, n_g), i1 = min(i0 + S, n_g);
    const int t = threadIdx.x, nt = blockDim.x;
    double *edges = d.edges + (size_t)mu * (size_t)(n_g + 1);
    // histograms of the latest sampling pass (double-buffered by iteration
    // parity; the sampling kernel records which, so that this kernel may run
    // beside the estimate that advances t)
    const uint32_t hpar = d.st->hist_par;
    const bool weighted = (hpar & 2u) != 0u;  // sums already weighted by 1/n_h: d_i = sum
    const size_t hb = (size_t)(hpar & 1u) * (size_t)d.dim * n_g;
    const double *hs = d.hsum + hb + (size_t)mu * n_g;
    const uint32_t *hc = d.hcnt + hb + (size_t)mu * n_g;

    // 1. old edges and raw d (with halo)
    for (int i = i0 + t; i <= i1; i += nt) sm.x[i - i0] = edges[i];
    double part = 0.0;
    for (int i = i0 - 1 + t; i <= i1; i += nt) {
        double v = 0.0;
        if (i >= 0 && i < n_g) {
            const uint32_t c = hc[i];
            v = c ? (weighted ? hs[i] : hs[i] / (double)c) : 0.0;
        }
        sm.d[i - (i0 - 1)] = v;
        if (i >= i0 && i < i1) part += v;
    }
    for (int o = 16; o >= 1; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((t & 31) == 0) sm.red[t >> 5] = part;
    __syncthreads();
    if (t == 0) {
        double p = 0.0;
        for (int w = 0; w < nt / 32; ++w) p += sm.red[w];
        sm.part = p;
        sm.n_own = i1 - i0;
    }
    cl.sync();
    // 2. the axis total, in rank order
    double sum_d = 0.0;
    for (int q = 0; q < kRefineCtas; ++q) sum_d += *cl.map_shared_rank(&sm.part, q);
    if (!(sum_d > 0.0) || !isfinite(sum_d)) {  // nothing to refine (reading); uniform
        cl.sync();
        return;
    }
    const double inv_sum = 1.0 / sum_d;
    // 3. smoothing, normalisation, compression; contiguous quarter-slices per thread
    const int n_own = i1 - i0;
    const int per = (n_own + nt - 1) / nt;
    const int a0 = min(t * per, n_own), a1 = min(a0 + per, n_own);
    double local = 0.0;
    for (int a = a0; a < a1; ++a) {
        const int i = i0 + a;
        const double dm = sm.d[a], d0 = sm.d[a + 1], dp = sm.d[a + 2];
        double s;
        if (i == 0) s = (7.0 * d0 + dp) * 0.125;
        else if (i == n_g - 1) s = (dm + 7.0 * d0) * 0.125;
        else s = (dm + 6.0 * d0 + dp) * 0.125;
        s = s * inv_sum;
        // reading: an unsampled increment keeps the weight of the smallest
        // normal double (the alpha -> 0 limit stays "no refinement")
        if (s <= 0.0) s = 2.2250738585072014e-308;
        double cv;
        if (s == 1.0) cv = 1.0;
        else {
            const double r = (1.0 - s) / -log(s);
            cv = d.alpha == 1.0 ? r : (d.alpha == 0.5 ? sqrt(r) : pow(r, d.alpha));
        }
        sm.c[a] = cv;
        local += cv;
        sm.C[a] = local;  // thread-local inclusive prefix, fixed below
    }
    // exclusive prefix of the thread totals (warp shuffles, then warps)
    double inc = local;
    const int lane = t & 31, w = t >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    __syncthreads();
    if (lane == 31) sm.red[w] = inc;
    __syncthreads();
    double wbase = 0.0;
    for (int q = 0; q < w; ++q) wbase += sm.red[q];
    const double tbase = wbase + inc - local;
    for (int a = a0; a < a1; ++a) sm.C[a] += tbase;
    __syncthreads();
    if (t == 0) sm.tot = n_own > 0 ? sm.C[n_own - 1] : 0.0;
    cl.sync();
    // 4. bases of every rank and the axis total of c
    double base[kRefineCtas];
    double total = 0.0;
    for (int q = 0; q < kRefineCtas; ++q) {
        base[q] = total;
        total += *cl.map_shared_rank(&sm.tot, q);
    }
    const double delta_d = total / (double)n_g;
    // 5. new edges k in [max(i0, 1), min(i1, n_g - 1)]
    for (int k = max(i0, 1) + t; k < min(i1, n_g); k += nt) {
        const double target = (double)k * delta_d;
        int q = 0;
        while (q < kRefineCtas - 1 && base[q + 1] < target) ++q;
        // rank q holds the crossing: smallest m with base[q] + C_q[m] >= target
        const RefineShared *rs = cl.map_shared_rank(&sm, q);
        const int nq = rs->n_own;
        int lo = -1, hi = nq - 1;  // base + C[hi] >= target (the last one is, up to rounding)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (base[q] + rs->C[mid] < target) lo = mid;
            else hi = mid;
        }
        // cumulative at the right end of increment j - 1 = q S + hi
        const double Cj = base[q] + rs->C[hi];
        const double cj = rs->c[hi];
        const double xr = rs->x[hi + 1], xl = rs->x[hi];
        sm.xn[k - i0] = cj > 0.0 ? xr - ((Cj - target) / cj) * (xr - xl) : xr;
    }
    if (t == 0) {
        if (i0 == 0) sm.xn[0] = sm.x[0];
        if (i1 == n_g && n_own > 0) sm.xn[n_own] = sm.x[n_own];
    }
    cl.sync();
    // 6. write back edges and the FP32 table; x'_{i1} comes from rank + 1
    for (int i = i0 + t; i < i1; i += nt) {
        const double xi = sm.xn[i - i0];
        const double xe = (i + 1 < i1 || i1 == n_g) ? sm.xn[i + 1 - i0]
                                                      : cl.map_shared_rank(&sm, rank + 1)->xn[0];
        if (i > 0) edges[i] = xi;
        d.tab[(size_t)mu * n_g + i] = make_float2((float)xi, (float)(xe - xi));
    }
    cl.sync();  // keep this CTA's shared memory alive until every remote read is done
}

// ---------------------------------------------------------------------------
// Host-side launchers: programmatic dependent launches (each kernel waits for
// its predecessor in pdl_wait), so that a kernel's launch overlaps the end of
// the one before it.
// ---------------------------------------------------------------------------
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// ---------------------------------------------------------------------------
// Several integrals from the same samples (App. B): the iteration's estimates of
// every output and their covariance, summed over hypercubes (§2.1 Eq. sigest
// in several variables, §3 Eq. sumI):
//   I[k]    = sum_h Omega X1_h[k] / n_h
//   C[k][l] = sum_h Omega^2 (X2_h[k,l]/n_h - (X1_h[k]/n_h)(X1_h[l]/n_h)) / (n_h - 1)
// (diagonal terms clamped at zero), every sum in the fixed order of the
// one-integral sums: blocks of kTreeBlock hypercubes by pairwise halving, then
// an adjacent pairwise tree over the blocks.  One CTA per block; the last CTA
// to finish combines the blocks and writes the iteration's row of the
// history.  Launched between the sampling kernel and k_estimate (which
// advances the iteration counter); it clears the other buffer of X1, X2 for
// the next iteration.  It does not release its dependents early.
// ---------------------------------------------------------------------------
constexpr int kMultiThreads = 256;
constexpr int kMultiMaxBlocks = (int)(kMultiMaxHc / kTreeBlock);  // 4096

__device__ __forceinline__ double multi_term(const Desc &d, const double *X1, const double *X2,
                                             int M, int s, uint64_t h) {
    if (h >= d.n_hc) return 0.0;
    const double n = (double)d.n_h[h];
    const double om = d.omega;
    if (s < M) return __dmul_rn(om, __ddiv_rn(X1[h * M + s], n));
    int k = 0, q = s - M;  // (k, l) of triangle entry q
    while (q >= M - k) {
        q -= M - k;
        ++k;
    }
    const int l = k + q;
    const uint64_t T = (uint64_t)M * (M + 1) / 2;
    const double mk = __ddiv_rn(X1[h * M + k], n), ml = __ddiv_rn(X1[h * M + l], n);
    double c = __dsub_rn(__ddiv_rn(X2[h * T + (s - M)], n), __dmul_rn(mk, ml));
    if (k == l && c < 0.0) c = 0.0;
    return __ddiv_rn(__dmul_rn(__dmul_rn(om, om), c), __dsub_rn(n, 1.0));
}

__global__ void __launch_bounds__(kMultiThreads) k_estimate_multi(const Desc *desc) {
    __shared__ double sh[kMultiThreads];
    __shared__ double tree[kMultiMaxBlocks];
    __shared__ bool s_last;
    pdl_wait();
    const Desc &d = *desc;
    const int M = d.n_out, T = M * (M + 1) / 2, NS = M + T;
    const uint32_t t_it = __ldcg(&d.st->t);  // the iteration being estimated
    const uint64_t par = t_it & 1u;
    const double *X1 = d.x1 + par * d.n_hc * M, *X2 = d.x2 + par * d.n_hc * T;
    const uint32_t blk = blockIdx.x, t = threadIdx.x;
    const uint64_t h0 = (uint64_t)blk * kTreeBlock;
    for (int s = 0; s < NS; ++s) {
        // halving over the block's 1024 terms: i += i + 512, then i += i + 256
        // (thread t holds terms t, t + 256, t + 512, t + 768), then in shared
        // memory down to 32 terms, then by shuffles
        const double v0 = multi_term(d, X1, X2, M, s, h0 + t);
        const double v1 = multi_term(d, X1, X2, M, s, h0 + t + 256);
        const double v2 = multi_term(d, X1, X2, M, s, h0 + t + 512);
        const double v3 = multi_term(d, X1, X2, M, s, h0 + t + 768);
        sh[t] = __dadd_rn(__dadd_rn(v0, v2), __dadd_rn(v1, v3));
        __syncthreads();
        for (int w = 128; w >= 32; w >>= 1) {
            if (t < (uint32_t)w) sh[t] = __dadd_rn(sh[t], sh[t + w]);
            __syncthreads();
        }
        if (t < 32) {
            double a = sh[t];
            for (int o = 16; o >= 1; o >>= 1) a = __dadd_rn(a, __shfl_down_sync(0xffffffffu, a, o));
            if (t == 0) d.mpart[(size_t)blk * NS + s] = a;
        }
        __syncthreads();
    }
    {  // the other buffer, zero for the next iteration (this block's hypercubes)
        const uint64_t hb = min((uint64_t)kTreeBlock, d.n_hc - h0);
        double *Y1 = d.x1 + (par ^ 1u) * d.n_hc * M + h0 * M;
        double *Y2 = d.x2 + (par ^ 1u) * d.n_hc * T + h0 * T;
        for (uint64_t i = t; i < hb * M; i += kMultiThreads) Y1[i] = 0.0;
        for (uint64_t i = t; i < hb * T; i += kMultiThreads) Y2[i] = 0.0;
    }
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(&d.st->done_multi, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    uint32_t P = 1;
    while (P < gridDim.x) P <<= 1;
    for (int s = 0; s < NS; ++s) {
        for (uint32_t i = t; i < P; i += kMultiThreads)
            tree[i] = i < gridDim.x ? __ldcg(d.mpart + (size_t)i * NS + s) : 0.0;
        __syncthreads();
        for (uint32_t w = 1; w < P; w <<= 1) {
            for (uint32_t i = t * 2 * w; i < P; i += kMultiThreads * 2 * w)
                tree[i] = __dadd_rn(tree[i], tree[i + w]);
            __syncthreads();
        }
        if (t == 0 && t_it < (uint32_t)d.hist_cap) {
            if (s < M) d.hist_im[(size_t)t_it * M + s] = tree[0];
            else d.hist_cm[(size_t)t_it * T + (s - M)] = tree[0];
        }
        __syncthreads();
    }
    if (t == 0) d.st->done_multi = 0u;
}

// ---------------------------------------------------------------------------
// k_partials: one integral sampled in parts (several devices, each a range of
// the iteration's samples) -- the partial sums of the current iteration
// (buffer t & 1): S1_h, S2_h [N_h] (§3 step 2), hsum, hcnt [D][N_g] (§2.3
// d_i), packed into (dir 0) or unpacked from (dir 1) one flat FP64 vector
// [S1 | S2 | hsum | hcnt], the counts as doubles (exact: below 2^32).  The sum
// of every part's vector is the vector of the whole iteration, so the
// exchange is one FP64 sum over the devices.
// ---------------------------------------------------------------------------
__global__ void k_partials(const Desc *desc, double *buf, int dir) {
    pdl_wait();
    pdl_trigger();
    const Desc &d = desc[0];
    const uint64_t par = __ldcg(&d.st->t) & 1u;
    const uint64_t nh = d.n_hc, bins = (uint64_t)d.dim * (uint64_t)d.n_g;
    double *s1 = d.s1 + par * nh, *s2 = d.s2 + par * nh, *hs = d.hsum + par * bins;
    uint32_t *hc = d.hcnt + par * bins;
    const uint64_t total = 2 * nh + 2 * bins;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        double *p = nullptr;
        uint32_t *pc = nullptr;
        if (i < nh) p = s1 + i;
        else if (i < 2 * nh) p = s2 + (i - nh);
        else if (i < 2 * nh + bins) p = hs + (i - 2 * nh);
        else pc = hc + (i - 2 * nh - bins);
        if (dir == 0) buf[i] = p ? *p : (double)*pc;
        else if (p) *p = buf[i];
        else *pc = (uint32_t)buf[i];
    }
}

cudaError_t launch_partials(const Desc *desc, double *buf, uint64_t n, int dir, cudaStream_t s) {
    const uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 152ull * 8);
    return launch_pdl(k_partials, dim3((unsigned)std::max<uint64_t>(blocks, 1)), dim3(256), s,
                      desc, buf, dir);
}

cudaError_t launch_estimate_multi(const Desc *desc, uint32_t n_blocks, cudaStream_t s) {
    // (programmatic serialisation: waits for the sampling kernel in pdl_wait;
    // it never triggers early, so k_estimate after it sees its whole result)
    return launch_pdl(k_estimate_multi, dim3(n_blocks), dim3(kMultiThreads), s, desc);
}

cudaError_t launch_chunks(const Desc *desc, const uint32_t *members, int n_group,
                          uint64_t *chunk_base, uint32_t *head, uint32_t C, cudaStream_t s) {
    return launch_pdl(k_chunks, dim3(1), dim3(1024), s, desc, members, n_group, chunk_base, head,
                      C);
}

// Blocks of kTreeBlock hypercubes from which the per-hypercube kernels take
// one CTA per block, four hypercubes per thread, instead of several CTAs per
// block: with fewer blocks the one-CTA form leaves SMs (and their FP64 units)
// idle, with more it keeps more loads in flight per thread.
constexpr uint32_t kWideBlocks = 512, kGroupBlocks = 4096;

cudaError_t launch_estimate(const Desc *desc, const uint32_t *tree_base, int n_int,
                            uint32_t n_blocks, int mode, cudaStream_t s, int prec) {
    if (n_blocks >= kWideBlocks) {
        // one integral of many blocks: four blocks per CTA (the per-CTA fence
        // and ticket amortised over 4096 hypercubes)
        const int group = (n_int == 1 && n_blocks >= kGroupBlocks) ? 4 : 1;
        const uint32_t n_cta = (n_blocks + (uint32_t)group - 1u) / (uint32_t)group;
        if (prec == VP_FP32)
            return launch_pdl(k_estimate_wide<VP_FP32>, dim3(n_cta), dim3(256), s, desc,
                              tree_base, n_int, mode, group);
        if (prec == VP_FP64)
            return launch_pdl(k_estimate_wide<VP_FP64>, dim3(n_cta), dim3(256), s, desc,
                              tree_base, n_int, mode, group);
        return launch_pdl(k_estimate_wide<-1>, dim3(n_cta), dim3(256), s, desc, tree_base, n_int,
                          mode, group);
    }
    return launch_pdl(k_estimate, dim3(n_blocks * kEstCtas), dim3(256), s, desc, tree_base, n_int,
                      mode);
}

cudaError_t launch_alloc(const Desc *desc, const uint32_t *tree_base, int n_int,
                         uint32_t n_blocks, cudaStream_t s, int initial) {
    if (n_blocks >= kWideBlocks) {
        // one integral of many blocks: four blocks per CTA (the per-CTA sum,
        // fence and ticket amortised over 4096 hypercubes)
        const int group = (n_int == 1 && n_blocks >= kGroupBlocks) ? 4 : 1;
        const uint32_t n_cta = (n_blocks + (uint32_t)group - 1u) / (uint32_t)group;
        cudaError_t e = launch_pdl(k_alloc_wide, dim3(n_cta), dim3(kSubH), s, desc, tree_base,
                                   n_int, initial, group);
        if (e != cudaSuccess) return e;
        return launch_pdl(k_offsets_wide, dim3(n_cta), dim3(kSubH), s, desc, tree_base, n_int,
                          group);
    }
    cudaError_t e = launch_pdl(k_alloc, dim3(n_blocks * kSub), dim3(kSubH), s, desc, tree_base,
                               n_int, initial);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_offsets, dim3(n_blocks * kSub), dim3(kSubH), s, desc, tree_base, n_int);
}

cudaError_t launch_refine(const Desc *desc, const uint32_t *axis_base, int n_int,
                          uint32_t n_axes, int max_ng, cudaStream_t s) {
    (void)max_ng;
    return launch_pdl(k_refine, dim3(n_axes * kRefineCtas), dim3(kRefineThreads), s, desc,
                      axis_base, n_int);
}

}  // namespace vp
