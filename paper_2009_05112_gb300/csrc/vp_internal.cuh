// vp_internal.cuh -- device-side data layout and shared device helpers of
// libvegasp (vegas+ hot path, arXiv:2009.05112).
//
// A "problem set" is a list of independent integrals iterated together.  The
// single-integral context is a set of one.  Every integral's state lives in
// device memory (HBM) for its whole life; the kernels read it through a
// descriptor array, so one launch can serve many integrals.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "vegasp.h"

namespace vp {

constexpr int kMaxDim = 24;        // D limit (largest bucket of the sampling kernel)
constexpr int kMaxNg = 4096;       // N_g limit (refinement keeps a whole axis in shared memory)
constexpr int kTreeBlock = 1024;   // hypercubes per block of the fixed-order sum
constexpr int kSub = 4;            // CTAs of the allocation kernels per block of kTreeBlock
constexpr int kSubH = kTreeBlock / kSub;
constexpr int kMaxPeaks = 64;
constexpr int kMaxPoints = 256;
constexpr int kInvTab = 4096;      // table of 1/n, 1/(n(n-1)) and log2 n for small integers n
constexpr int kInvTabWords = 4 * kInvTab;  // 32 bytes per n: 1/n, 1/(n(n-1)), log2 n (2 floats), pad
// several integrals from the same samples (App. B): at most kMaxOut outputs, the
// upper triangle of their covariance kMaxTri entries, at most 2^22 hypercubes
constexpr int kMaxOut = 8;
constexpr int kMaxTri = kMaxOut * (kMaxOut + 1) / 2;
constexpr uint64_t kMultiMaxHc = 1ull << 22;

// Status bits (State::status).
constexpr uint32_t kStatusNonFinite = 1u;


// Mutable per-integral scalars, device resident.
struct State {
    uint32_t t;           // iterations done = Philox counter word 2 of the next one
    int32_t scale_exp;    // the sampling kernel accumulates v = J f 2^scale_exp
    uint32_t done_est;    // last-block counter of the estimate kernel
    uint32_t done_alloc;  // last-block counter of the allocation kernel
    uint32_t done_multi;  // last-block counter of the several-outputs estimate (App. B)
    uint32_t status;      // kStatus* bits
    uint32_t hist_par;    // histogram buffer of the latest sampling pass (bit 0, read by the
                          // refinement) and its kind (bit 1: sums weighted by 1/n_h, d_i = sum)
    double sum_d;         // sum_h d_h in the fixed order (set by the estimate kernel)
    double inv_sum_d;     // 1 / sum_d
    uint64_t n_samples;   // sum_h n_h of the current allocation
    uint64_t n_eval_total;// integrand evaluations over all iterations
    double last_i, last_var;
    // served requests: running §2.5 sums over the iterations j >= discard
    double cw, cwi;       // sum 1/var_j, sum I_j/var_j
    double zsum;          // sum of I_j over iterations with var_j = 0 (exact)
    uint32_t n_zero;      // number of those
    uint32_t done;        // kDone* bits once the stop rule has fired
    // the allocation's fast quotient q ~ d_h alloc_c (alloc_c = N_ev / sum d;
    // 0 where 1 / sum d or the product leaves the normal range), taken for
    // d_h >= alloc_dmin (then N_ev d_h is a normal number)
    double alloc_c, alloc_dmin;
};

// Bits of State::done and of the server's per-slot flag.
constexpr uint32_t kDoneStop = 1u;       // the request is finished
constexpr uint32_t kDoneConverged = 2u;  // ... because sdev <= rtol |mean|

// Strata per axis (§3 uses the same N_st on every axis; §3.2 lets them
// differ) and the constants the sampling loop derives from them.  Hypercube h
// is the mixed-radix number with digit k_mu in [0, n[mu]) on axis mu, axis 0
// least significant; entries mu >= D hold 1.
struct Strata {
    uint32_t n[kMaxDim];       // strata on axis mu
    uint32_t magic[kMaxDim];   // h / n[mu] = ((t + ((h - t) >> 1)) >> (shift[mu] - 1)),
    int32_t shift[kMaxDim];    //   t = umulhi(magic[mu], h); shift 0: n[mu] = 1
    float c32[kMaxDim];        // N_g / n[mu] (FP32 path)
    double nd[kMaxDim];        // n[mu] (FP64 path)
};

// Read-only (per iteration) description of one integral.
struct Desc {
    int32_t dim, n_g, kind, prec;
    int32_t plus2, n_peaks;    // n_peaks: K for peak families, n points for POSTERIOR
    int32_t n_par;             // POSTERIOR: P (dim = P + G)
    int32_t hist_cap;          // capacity of the iteration history
    uint32_t n_st, integral_id;  // n_st: strata on axis 0 (every axis unless mixed)
    uint32_t key0, key1;       // Philox key (seed lo, hi)
    uint32_t n_tree;           // ceil(n_hc / kTreeBlock)
    uint32_t uniform;          // 1: the same strata on every axis (the task kernel's case)
    int64_t n_ev;
    uint64_t n_hc;             // N_h = prod_mu strata[mu] (N_st^D when uniform)
    double omega;              // y-volume of a hypercube, 1 / N_h
    double omega2;             // omega * omega (IEEE product, as the kernels would form it)
    double n_ev_d;             // (double) n_ev (exact below 2^53)
    double alpha, beta;
    int32_t lob_i;             // beta log2(Omega) = lob_i + lob_f, lob_f in [0, 1)
    float lob_f;               //   (FP32 path: d_h = 2^(beta/2 log2 var + beta log2 Omega))
    float half_beta_hi, half_beta_lo;  // beta/2 = hi + lo (FP32 path)
    float ng_over_nst;         // N_g / N_st (FP32 path)
    float inv_ng;              // 1 / N_g (FP32 path)
    float ngD_m;               // N_g^D = ngD_m 2^ngD_e (FP32 path: J = N_g^D prod dx_i)
    int32_t ngD_e;
    uint32_t nst_magic;        // h / N_st = ((t + ((h - t) >> 1)) >> (nst_shift - 1)),
    int32_t nst_shift;         //   t = umulhi(nst_magic, h) (Granlund-Montgomery); shift 0: N_st = 1
    // device buffers (all owned by the set)
    double *edges;     // [dim][n_g + 1] FP64 grid
    float2 *tab;       // [dim][n_g] {x_i, dx_i}, FP32 mirror of the grid
    const double *prm;  // integrand blob as given (FP64 path)
    const float *prm32; // FP32 constants derived from the blob (FP32 path)
    uint32_t *n_h;     // [n_hc]
    uint64_t *off;     // [n_hc + 1] exclusive offsets; off[n_hc] = samples this iteration
    const double *inv_tab; // [kInvTab][4]: 1/n, 1/(n (n-1)) (IEEE), log2 n as a float pair
                           // hi + lo, padding (one 32-byte sector per n); shared by the set
    double *s1, *s2;   // [2][n_hc] per-hypercube sums of v, v^2 (unscaled); iteration t
                       // accumulates into buffer t & 1 while the estimate of t clears the other
    double *dh;        // [n_hc] d_h of the latest estimate
    double *hsum;      // [2][dim][n_g] sum v^2 per increment (unscaled), same double buffering
    uint32_t *hcnt;    // [2][dim][n_g] samples per increment
    double *part;      // [n_tree][3] block partial sums (I, var, d), then [n_tree][4][3]
                       // the four residue classes' sums of each block (k_estimate)
    uint64_t *bsum;    // [n_tree kSub] sums of n_h over kSubH hypercubes, then their offsets
    double *hist_i, *hist_var;  // [hist_cap] iteration history
    State *st;
    // served requests (done_out == nullptr elsewhere): stop when the §2.5
    // combination of iterations j >= discard has sdev <= rtol |mean| after at
    // least min_meas of them, or after stop_it iterations in all
    double rtol;
    int32_t discard, min_meas, stop_it, pad1;
    uint32_t *done_out;        // the server's flag for this request's slot
    Strata strata;
    // several integrals from the same samples (App. B), n_out = M >= 2 outputs
    // (1: the integrand alone).  Output k is J f g_k(x), g_k = x^a x^b for
    // (a, b) = mono[2k], mono[2k+1] (< 0: that factor is 1); output 0 is f.
    int32_t n_out;
    int32_t d_weighted;        // 1: the grid's d_i from samples weighted by 1/n_h (else the mean)
    int32_t mono[2 * kMaxOut];
    double *x1;        // [2][n_hc][M] per-hypercube sums of the outputs (double-buffered)
    double *x2;        // [2][n_hc][M (M+1)/2] sums of their products, upper triangle by rows
    double *mpart;     // [n_tree][M + M (M+1)/2] block partial sums
    double *hist_im;   // [hist_cap][M] I_j of every output
    double *hist_cm;   // [hist_cap][M (M+1)/2] covariance of the I_j, upper triangle
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32
// S-P network, key bumped by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct U4 { uint32_t a, b, c, d; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = __umulhi(m0, c.a), lo0 = m0 * c.a;
        uint32_t hi1 = __umulhi(m1, c.c), lo1 = m1 * c.c;
        U4 n;
        n.a = hi1 ^ c.b ^ k0;
        n.b = lo1;
        n.c = hi0 ^ c.d ^ k1;
        n.d = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t lane_of(const U4 &r, int l) {
    return l == 0 ? r.a : (l == 1 ? r.b : (l == 2 ? r.c : r.d));
}

// Uniforms strictly inside (0,1): FP64 (r + 1/2) 2^-32 (exact); FP32
// ((r >> 9) + 1/2) 2^-23 (exact, 24 significant bits).
__device__ __forceinline__ double u01_f64(uint32_t r) {
    return __dmul_rn(__dadd_rn((double)r, 0.5), 2.3283064365386962890625e-10);
}
__device__ __forceinline__ float u01_f32(uint32_t r) {
    return ((float)(r >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

// PTX MUFU forms (documented instructions; ~2^-22 relative error).
// 2^e as a double, |e| <= 1022, from its bits.
__device__ __forceinline__ double pow2d(int e) {
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// (double)n of a 32-bit unsigned integer from its bits with integer
// operations only (exact; a conversion instruction would run on the FP64
// pipe, a few operations per SM per clock on this part).
__device__ __forceinline__ double u32_to_f64(uint32_t n) {
    if (n == 0u) return 0.0;
    const int e = 31 - __clz((int)n);
    const uint64_t man = ((uint64_t)n << (52 - e)) & ((1ull << 52) - 1ull);
    return __longlong_as_double((long long)(((uint64_t)(e + 1023) << 52) | man));
}

// (double)x 2^e built from the bits of x with integer operations only (FP64
// instructions are scarce on this part, a few per SM per clock, so the FP32
// path's values leave the kernels without them): exact whenever the result is
// a normal double; below that range the result is a signed zero, above it an
// infinity; infinities and NaNs pass through.
__device__ __forceinline__ double f2d_pow2(float x, int e) {
    const uint32_t b = __float_as_uint(x);
    const uint64_t sign = (uint64_t)(b >> 31) << 63;
    int ex = (int)((b >> 23) & 0xffu);
    uint32_t man = b & 0x7fffffu;
    if (ex == 0xff)  // inf, nan
        return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull | ((uint64_t)man << 29)));
    if (ex == 0) {
        if (man == 0u) return __longlong_as_double((long long)sign);  // +-0
        const int sh = __clz((int)man) - 8;  // subnormal: normalise the mantissa
        man = (man << sh) & 0x7fffffu;
        ex = 1 - sh;
    }
    const int E = ex - 127 + e + 1023;
    if (E <= 0) return __longlong_as_double((long long)sign);
    if (E >= 2047) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull));
    return __longlong_as_double((long long)(sign | ((uint64_t)E << 52) | ((uint64_t)man << 29)));
}

// The library's fixed order for combining the block sums (each the sum of a
// block of kTreeBlock hypercubes): an adjacent pairwise tree over P leaves, P
// the least power of two >= n, leaves past n zero, level by level (leaf 2i +
// leaf 2i+1, then 4i + 4i+2, ...); its depth is log2 P, where adding the block
// sums left to right would chain n dependent FP64 additions (slow on this
// part).  One CTA (blockDim.x a power of two) evaluates it: thread t takes the
// aligned run of Q = P / T leaves [t Q, (t + 1) Q) (T = min(P, blockDim.x))
// and reduces it with a binary counter, which builds exactly the tree
// restricted to the run; the T run sums are then combined level by level in
// shared memory.  NS series at once, leaf i of series c at part[NS i + c]
// (read through L2: written by other CTAs); sh holds NS x blockDim.x doubles.
// Every thread calls it; the sums are returned in thread 0.
template <int NS>
__device__ void block_tree_sum(const double *part, uint32_t n, double *sh, double (&out)[NS]) {
    uint32_t P = 1;
    while (P < n) P <<= 1;
    const uint32_t nt = blockDim.x, t = threadIdx.x;
    if (P <= 64 && (uint32_t)NS * 32u <= nt) {
        // at most 64 leaves: one warp per series, lane l adds leaves 2l and
        // 2l + 1 (level 1), then level k adds lane 2^(k-2) further down, the
        // left node first: the same tree, with no barrier between levels
        const uint32_t w = t >> 5, l = t & 31u;
        if (w < (uint32_t)NS) {
            double x = 0.0;
            if (P == 1) {
                x = (n > 0) ? __ldcg(part + w) : 0.0;
            } else if (2u * l < P) {
                const double a = 2u * l < n ? __ldcg(part + (size_t)NS * (2u * l) + w) : 0.0;
                const double b = 2u * l + 1u < n ? __ldcg(part + (size_t)NS * (2u * l + 1u) + w) : 0.0;
                x = __dadd_rn(a, b);
            }
            for (uint32_t o = 1; 4u * o <= P; o <<= 1) x = __dadd_rn(x, __shfl_down_sync(0xffffffffu, x, o));
            if (l == 0) sh[w] = x;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < NS; ++c) out[c] = sh[c];
        return;
    }
    const uint32_t T = P < nt ? P : nt;
    const uint32_t Q = P / T;
    double run[NS];
#pragma unroll
    for (int c = 0; c < NS; ++c) run[c] = 0.0;
    if (t < T) {
        double st[NS][24];  // one partial sum per tree level (Q <= 2^23)
        uint32_t full = 0u;  // bit l: st[.][l] holds a complete subtree of 2^l leaves
        // leaves in groups of up to 4 whose loads are issued together, then
        // folded into the stack one by one (the same order of additions)
        constexpr uint32_t G = 4;
        for (uint32_t j0 = 0; j0 < Q; j0 += G) {
            double buf[G][NS];
#pragma unroll
            for (uint32_t g = 0; g < G; ++g) {
                const uint32_t i = t * Q + j0 + g;
#pragma unroll
                for (int c = 0; c < NS; ++c)
                    buf[g][c] = (j0 + g < Q && i < n) ? __ldcg(part + (size_t)NS * i + c) : 0.0;
            }
#pragma unroll
            for (uint32_t g = 0; g < G; ++g) {
                if (j0 + g >= Q) break;
                double carry[NS];
#pragma unroll
                for (int c = 0; c < NS; ++c) carry[c] = buf[g][c];
                int l = 0;
                while (full & (1u << l)) {
#pragma unroll
                    for (int c = 0; c < NS; ++c) carry[c] = __dadd_rn(st[c][l], carry[c]);
                    full &= ~(1u << l);
                    ++l;
                }
#pragma unroll
                for (int c = 0; c < NS; ++c) st[c][l] = carry[c];
                full |= 1u << l;
            }
        }
        const int top = __ffs((int)full) - 1;  // Q is a power of two: one subtree is left
#pragma unroll
        for (int c = 0; c < NS; ++c) run[c] = st[c][top];
    }
#pragma unroll
    for (int c = 0; c < NS; ++c) sh[c * nt + t] = run[c];
    __syncthreads();
    if (NS > 1 && NS * T <= nt) {  // one thread group per series, the series in parallel
        const uint32_t c = t / T, u = t - c * T;
        for (uint32_t w = 1; w < T; w <<= 1) {
            if (c < (uint32_t)NS && (u & (2 * w - 1)) == 0)
                sh[c * nt + u] = __dadd_rn(sh[c * nt + u], sh[c * nt + u + w]);
            __syncthreads();
        }
    } else {
        for (uint32_t w = 1; w < T; w <<= 1) {
            if (t < T && (t & (2 * w - 1)) == 0) {
#pragma unroll
                for (int c = 0; c < NS; ++c) sh[c * nt + t] = __dadd_rn(sh[c * nt + t], sh[c * nt + t + w]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int c = 0; c < NS; ++c) out[c] = sh[c * nt];
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialisation may be scheduled while its predecessor in
// the stream is still finishing; pdl_wait() blocks until that predecessor grid
// has completed and its memory operations are visible (a no-op for a normal
// launch), so every kernel calls it before reading what earlier kernels wrote.
// pdl_trigger() lets the successor be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace vp
