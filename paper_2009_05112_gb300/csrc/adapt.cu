// adapt.cu -- the per-hypercube and per-axis kernels of one vegas+ iteration:
//
//   k_zero      clears the accumulators of the coming iteration;
//   k_chunks    prefix of sample chunks over the integrals of a launch group
//               (the sampling kernel's work queue);
//   k_estimate  step a6 and the first half of a7: per hypercube
//               dI_h = Omega S1_h / n_h, var_h = Omega^2 (S2_h/n_h - (S1_h/n_h)^2)/(n_h - 1)
//               (§3 Eq. sumI with §2.1 Eqs. MCIy, sigest inside each hypercube),
//               sigma_h = Omega sqrt(S2_h/n_h - (S1_h/n_h)^2) (§3 step 2) and
//               d_h = sigma_h^beta (§3 Eq. dh); sums over h in the library's
//               fixed order (blocks of 1024 hypercubes, pairwise halving inside
//               a block, block sums left to right), so sum_h d_h -- and with it
//               every integer n_h -- is reproducible bit for bit;
//   k_alloc     a7: n_h = max(2, floor(N_ev d_h / sum d)) (§3 Eq. nh; or + 2;
//               the first allocation is always the equal split max(2, .)),
//               block sums of n_h, then (last block) the block offsets;
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
// k_zero: S1, S2 (per hypercube) and the histograms of every integral.
// grid: tree blocks of all integrals (tree_base); 256 threads.
// ---------------------------------------------------------------------------
__global__ void k_zero(const Desc *desc, const uint32_t *tree_base, int n_int) {
    const int b = owner_of(tree_base, n_int, blockIdx.x);
    const Desc &d = desc[b];
    const uint32_t k = blockIdx.x - tree_base[b];
    const uint64_t h0 = (uint64_t)k * kTreeBlock;
    for (int i = threadIdx.x; i < kTreeBlock; i += blockDim.x) {
        const uint64_t h = h0 + i;
        if (h < d.n_hc) {
            d.s1[h] = 0.0;
            d.s2[h] = 0.0;
        }
    }
    // histograms: spread over the integral's blocks
    const int bins = d.dim * d.n_g;
    for (int i = k * blockDim.x + threadIdx.x; i < bins; i += d.n_tree * blockDim.x) {
        d.hsum[i] = 0.0;
        d.hcnt[i] = 0u;
    }
}

// ---------------------------------------------------------------------------
// k_chunks: chunk_base[g + 1] = chunk_base[g] + ceil(N_b / C) over the group
// members; resets the queue head.  One CTA.
// ---------------------------------------------------------------------------
__global__ void k_chunks(const Desc *desc, const uint32_t *members, int n_group,
                         uint64_t *chunk_base, uint32_t *head, uint32_t C) {
    __shared__ uint64_t s_cnt[1024];
    __shared__ uint64_t s_carry;
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
            cnt = (n + C - 1) / C;
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

// ---------------------------------------------------------------------------
// Fixed-order block reduction of three doubles over kTreeBlock = 1024 terms
// with 512 threads: thread i first adds terms i and i + 512 (halving step
// s = 512), then s = 256 ... 32 through shared memory, then s = 16 ... 1 with
// shuffles (lane i receives lane i + s: the same pairing).  Result valid in
// thread 0.
// ---------------------------------------------------------------------------
struct D3 { double a, b, c; };

__device__ __forceinline__ D3 tree_reduce3(D3 v, double (*sh)[512]) {
    const int t = threadIdx.x;
    sh[0][t] = v.a;
    sh[1][t] = v.b;
    sh[2][t] = v.c;
    __syncthreads();
    for (int s = 256; s >= 32; s >>= 1) {
        if (t < s) {
            sh[0][t] = __dadd_rn(sh[0][t], sh[0][t + s]);
            sh[1][t] = __dadd_rn(sh[1][t], sh[1][t + s]);
            sh[2][t] = __dadd_rn(sh[2][t], sh[2][t + s]);
        }
        __syncthreads();
    }
    D3 r = {0.0, 0.0, 0.0};
    if (t < 32) {
        r.a = sh[0][t];
        r.b = sh[1][t];
        r.c = sh[2][t];
        for (int s = 16; s >= 1; s >>= 1) {
            const double oa = __shfl_down_sync(0xffffffffu, r.a, s);
            const double ob = __shfl_down_sync(0xffffffffu, r.b, s);
            const double oc = __shfl_down_sync(0xffffffffu, r.c, s);
            r.a = __dadd_rn(r.a, oa);
            r.b = __dadd_rn(r.b, ob);
            r.c = __dadd_rn(r.c, oc);
        }
    }
    return r;
}

// d_h = sigma_h^beta; beta = 0 and 1 exactly.
__device__ __forceinline__ double damp(double sigma, double beta) {
    if (beta == 0.0) return 1.0;
    if (beta == 1.0) return sigma;
    return pow(sigma, beta);
}

// ---------------------------------------------------------------------------
// k_estimate.  mode 0: from the moments (a6 + sigma_h + d_h), records the
// iteration; mode 1: dh[] holds sigma_h, turn it into d_h and sum; mode 2:
// dh[] holds d_h, sum only.  grid: tree blocks of all integrals; 512 threads.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_estimate(const Desc *desc, const uint32_t *tree_base,
                                                  int n_int, int mode) {
    __shared__ double sh[3][512];
    __shared__ bool s_last;
    const int b = owner_of(tree_base, n_int, blockIdx.x);
    const Desc &d = desc[b];
    const uint32_t k = blockIdx.x - tree_base[b];
    const uint64_t h0 = (uint64_t)k * kTreeBlock;
    const double om = d.omega, om2 = __dmul_rn(d.omega, d.omega);

    D3 acc = {0.0, 0.0, 0.0};
    for (int half = 0; half < 2; ++half) {
        const uint64_t h = h0 + threadIdx.x + half * 512;
        D3 v = {0.0, 0.0, 0.0};
        if (h < d.n_hc) {
            if (mode == 0) {
                const double n = (double)d.n_h[h];
                const double s1 = d.s1[h], s2 = d.s2[h];
                v.a = __dmul_rn(om, __ddiv_rn(s1, n));
                const double m1 = __ddiv_rn(s1, n), m2 = __ddiv_rn(s2, n);
                double var = __dsub_rn(m2, __dmul_rn(m1, m1));
                var = var < 0.0 ? 0.0 : var;
                v.b = __ddiv_rn(__dmul_rn(om2, var), __dsub_rn(n, 1.0));
                const double sa = __dmul_rn(__ddiv_rn(om2, n), s2);
                const double sb = __dmul_rn(__ddiv_rn(om, n), s1);
                const double sv = __dsub_rn(sa, __dmul_rn(sb, sb));
                const double sigma = sv > 0.0 ? sqrt(sv) : 0.0;
                v.c = damp(sigma, d.beta);
                d.dh[h] = v.c;
            } else if (mode == 1) {
                v.c = damp(d.dh[h], d.beta);
                d.dh[h] = v.c;
            } else {
                v.c = d.dh[h];
            }
        }
        if (half == 0) acc = v;
        else {
            acc.a = __dadd_rn(acc.a, v.a);  // the s = 512 halving step
            acc.b = __dadd_rn(acc.b, v.b);
            acc.c = __dadd_rn(acc.c, v.c);
        }
    }
    const D3 r = tree_reduce3(acc, sh);
    if (threadIdx.x == 0) {
        d.part[3 * k + 0] = r.a;
        d.part[3 * k + 1] = r.b;
        d.part[3 * k + 2] = r.c;
        __threadfence();
        const uint32_t ticket = atomicAdd(&d.st->done_est, 1u);
        s_last = (ticket == d.n_tree - 1);
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    // last block of this integral: block sums left to right
    __threadfence();
    double I = 0.0, V = 0.0, Sd = 0.0;
    for (uint32_t q = 0; q < d.n_tree; ++q) {
        I = __dadd_rn(I, __ldcg(d.part + 3 * q + 0));
        V = __dadd_rn(V, __ldcg(d.part + 3 * q + 1));
        Sd = __dadd_rn(Sd, __ldcg(d.part + 3 * q + 2));
    }
    State *st = d.st;
    st->done_est = 0u;
    st->sum_d = Sd;
    if (mode == 0) {
        const uint32_t t = st->t;
        if (t < (uint32_t)d.hist_cap) {
            d.hist_i[t] = I;
            d.hist_var[t] = V;
        }
        st->last_i = I;
        st->last_var = V;
        st->n_eval_total += st->n_samples;
        if (!isfinite(I) || !isfinite(V)) st->status |= kStatusNonFinite;
        // keep J f 2^scale_exp near one in the next iteration: the mean of J f
        // over y-space is the integral (an exact power-of-two rescaling).
        if (isfinite(I) && I != 0.0) {
            int e = ilogb(fabs(I));
            e = e > 120 ? 120 : (e < -120 ? -120 : e);
            st->scale_exp = -e;
        }
        st->t = t + 1;
    }
}

// ---------------------------------------------------------------------------
// k_alloc: n_h for 1024 hypercubes per block (256 threads x 4), block sum of
// n_h; the last block of each integral turns the block sums into block
// offsets and records the total.  Skipped (allocation kept) when sum_d is not
// finite; the status flag records it.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_alloc(const Desc *desc, const uint32_t *tree_base,
                                               int n_int, int initial) {
    __shared__ unsigned long long s_sum;
    __shared__ bool s_last;
    const int b = owner_of(tree_base, n_int, blockIdx.x);
    const Desc &d = desc[b];
    const uint32_t k = blockIdx.x - tree_base[b];
    const uint64_t h0 = (uint64_t)k * kTreeBlock;
    const double sum_d = d.st->sum_d;
    if (!isfinite(sum_d)) {
        if (threadIdx.x == 0 && k == 0) d.st->status |= kStatusNonFinite;
        return;
    }
    if (threadIdx.x == 0) s_sum = 0ull;
    __syncthreads();
    unsigned long long mine = 0;
    for (int i = threadIdx.x; i < kTreeBlock; i += blockDim.x) {
        const uint64_t h = h0 + i;
        if (h >= d.n_hc) break;
        double q;
        if (sum_d > 0.0) q = __ddiv_rn(__dmul_rn((double)d.n_ev, d.dh[h]), sum_d);
        else q = __ddiv_rn((double)d.n_ev, (double)d.n_hc);
        const double fl = floor(q);
        uint32_t n;
        if (d.plus2 && !initial) n = (uint32_t)fl + 2u;
        else n = fl > 2.0 ? (uint32_t)fl : 2u;
        d.n_h[h] = n;
        mine += n;
    }
    for (int s = 16; s >= 1; s >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, s);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_sum, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
        d.bsum[k] = s_sum;
        __threadfence();
        const uint32_t ticket = atomicAdd(&d.st->done_alloc, 1u);
        s_last = (ticket == d.n_tree - 1);
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    uint64_t run = 0;
    for (uint32_t q = 0; q < d.n_tree; ++q) {
        const uint64_t v = __ldcg(d.bsum + q);
        d.bsum[q] = run;
        run += v;
    }
    d.off[d.n_hc] = run;
    d.st->n_samples = run;
    d.st->done_alloc = 0u;
}

// k_offsets: off[h] = bsum[block] + exclusive scan of n_h within the block.
__global__ void __launch_bounds__(256) k_offsets(const Desc *desc, const uint32_t *tree_base,
                                                 int n_int) {
    __shared__ unsigned long long s_warp[8];
    const int b = owner_of(tree_base, n_int, blockIdx.x);
    const Desc &d = desc[b];
    if (!isfinite(d.st->sum_d)) return;
    const uint32_t k = blockIdx.x - tree_base[b];
    const uint64_t h0 = (uint64_t)k * kTreeBlock + (uint64_t)threadIdx.x * 4;
    // 4 consecutive hypercubes per thread
    uint32_t n[4];
    unsigned long long tot = 0;
    for (int i = 0; i < 4; ++i) {
        const uint64_t h = h0 + i;
        n[i] = h < d.n_hc ? d.n_h[h] : 0u;
        tot += n[i];
    }
    // exclusive scan of tot over the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = tot;
    for (int s = 1; s < 32; s <<= 1) {
        const unsigned long long o = __shfl_up_sync(0xffffffffu, inc, s);
        if (lane >= s) inc += o;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    unsigned long long wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += s_warp[w];
    unsigned long long run = d.bsum[k] + wbase + inc - tot;
    for (int i = 0; i < 4; ++i) {
        const uint64_t h = h0 + i;
        if (h < d.n_hc) d.off[h] = run;
        run += n[i];
    }
}

// ---------------------------------------------------------------------------
// k_refine: a8 for one (integral, axis); 256 threads; N_g <= 4096.
// Shared: x[N_g + 1], dd[N_g] (raw d, then compressed), C[N_g + 1].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_refine(const Desc *desc, const uint32_t *axis_base,
                                                int n_int) {
    extern __shared__ double rsm[];
    __shared__ double s_red[256];
    __shared__ double s_scan[256];
    const int b = owner_of(axis_base, n_int, blockIdx.x);
    const Desc &d = desc[b];
    const int mu = blockIdx.x - axis_base[b];
    const int n_g = d.n_g;
    if (d.alpha == 0.0 || n_g < 2) return;
    double *x = rsm;
    double *dd = rsm + (n_g + 1);
    double *C = dd + n_g;
    double *edges = d.edges + (size_t)mu * (size_t)(n_g + 1);
    const double *hs = d.hsum + (size_t)mu * n_g;
    const uint32_t *hc = d.hcnt + (size_t)mu * n_g;
    const int t = threadIdx.x, nt = blockDim.x;

    double part = 0.0;
    for (int i = t; i <= n_g; i += nt) x[i] = edges[i];
    for (int i = t; i < n_g; i += nt) {
        const uint32_t c = hc[i];
        const double v = c ? __ddiv_rn(hs[i], (double)c) : 0.0;
        dd[i] = v;
        part += v;
    }
    s_red[t] = part;
    __syncthreads();
    for (int s = nt / 2; s >= 1; s >>= 1) {
        if (t < s) s_red[t] += s_red[t + s];
        __syncthreads();
    }
    const double sum_d = s_red[0];
    if (!(sum_d > 0.0) || !isfinite(sum_d)) return;  // nothing to refine (reading)
    // smoothing, normalisation, compression; each thread owns a contiguous segment
    const int seg = (n_g + nt - 1) / nt;
    const int i0 = t * seg, i1 = min(i0 + seg, n_g);
    double cval[16];
    double local = 0.0;
    for (int i = i0; i < i1; ++i) {
        double s;
        if (i == 0) s = (7.0 * dd[0] + dd[1]) / 8.0;
        else if (i == n_g - 1) s = (dd[n_g - 2] + 7.0 * dd[n_g - 1]) / 8.0;
        else s = (dd[i - 1] + 6.0 * dd[i] + dd[i + 1]) / 8.0;
        s = s / sum_d;
        // reading: an unsampled increment keeps the weight of the smallest
        // normal double (the alpha -> 0 limit stays "no refinement")
        if (s <= 0.0) s = 2.2250738585072014e-308;
        double c;
        if (s == 1.0) c = 1.0;
        else c = pow((1.0 - s) / log(1.0 / s), d.alpha);
        cval[i - i0] = c;
        local += c;
    }
    __syncthreads();  // every read of the raw d is done
    for (int i = i0; i < i1; ++i) dd[i] = cval[i - i0];
    // inclusive scan of the thread totals (Hillis-Steele over 256 values)
    s_scan[t] = local;
    __syncthreads();
    for (int s = 1; s < nt; s <<= 1) {
        const double o = t >= s ? s_scan[t - s] : 0.0;
        __syncthreads();
        s_scan[t] += o;
        __syncthreads();
    }
    double run = s_scan[t] - local;  // exclusive prefix of this segment
    if (t == 0) C[0] = 0.0;
    for (int i = i0; i < i1; ++i) {
        run += dd[i];
        C[i + 1] = run;
    }
    __syncthreads();
    const double total = C[n_g];
    const double delta_d = total / (double)n_g;
    for (int k = 1 + t; k < n_g; k += nt) {
        const double target = (double)k * delta_d;
        int lo = 0, hi = n_g;  // C[lo] < target <= C[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (C[mid] < target) lo = mid;
            else hi = mid;
        }
        const int j = hi;
        const double dj = dd[j - 1];
        const double xn = dj > 0.0 ? x[j] - ((C[j] - target) / dj) * (x[j] - x[j - 1]) : x[j];
        edges[k] = xn;
    }
    __syncthreads();
    // FP32 mirror {x_i, dx_i}
    float2 *tab = d.tab + (size_t)mu * n_g;
    for (int i = t; i < n_g; i += nt) {
        const double e0 = __ldcg(edges + i), e1 = __ldcg(edges + i + 1);
        tab[i] = make_float2((float)e0, (float)(e1 - e0));
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers.
// ---------------------------------------------------------------------------
cudaError_t launch_zero(const Desc *desc, const uint32_t *tree_base, int n_int,
                        uint32_t n_blocks, cudaStream_t s) {
    k_zero<<<n_blocks, 256, 0, s>>>(desc, tree_base, n_int);
    return cudaGetLastError();
}

cudaError_t launch_chunks(const Desc *desc, const uint32_t *members, int n_group,
                          uint64_t *chunk_base, uint32_t *head, uint32_t C, cudaStream_t s) {
    k_chunks<<<1, 1024, 0, s>>>(desc, members, n_group, chunk_base, head, C);
    return cudaGetLastError();
}

cudaError_t launch_estimate(const Desc *desc, const uint32_t *tree_base, int n_int,
                            uint32_t n_blocks, int mode, cudaStream_t s) {
    k_estimate<<<n_blocks, 512, 0, s>>>(desc, tree_base, n_int, mode);
    return cudaGetLastError();
}

cudaError_t launch_alloc(const Desc *desc, const uint32_t *tree_base, int n_int,
                         uint32_t n_blocks, cudaStream_t s, int initial) {
    k_alloc<<<n_blocks, 256, 0, s>>>(desc, tree_base, n_int, initial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_offsets<<<n_blocks, 256, 0, s>>>(desc, tree_base, n_int);
    return cudaGetLastError();
}

cudaError_t launch_refine(const Desc *desc, const uint32_t *axis_base, int n_int,
                          uint32_t n_blocks, int max_ng, cudaStream_t s) {
    const size_t smem = (size_t)(3 * max_ng + 2) * sizeof(double);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)((3 * kMaxNg + 2) * sizeof(double)));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_refine<<<n_blocks, 256, smem, s>>>(desc, axis_base, n_int);
    return cudaGetLastError();
}

}  // namespace vp
