// noalloc.cu -- vp_alloc_static: the reallocation step without any device
// allocation.
//
// Some callers cannot allocate device memory while they work: a serving
// process that reserved all device memory up front for a pool it manages
// itself, or code that must not call cudaMalloc in the middle of a step
// because cudaMalloc may synchronise the whole device.  For them this file
// offers the reallocation step (the same arithmetic as vp_adapt's: the
// fixed-order sum of d_h, n_h = max(2, floor(N_ev d_h / sum d)) or the "+2"
// form, exclusive offsets) on buffers the caller provides, with its scratch in
// a static device array instead of memory it allocates.
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>

#include "vp_internal.cuh"

namespace vp {
const char *set_error_message(vp_status s, const char *msg);  // api.cu
}

namespace {

constexpr uint64_t kStaticMaxHc = 1ull << 22;          // 4,194,304 hypercubes
constexpr int kStaticMaxBlocks = (int)(kStaticMaxHc / 1024);

// Scratch of vp_alloc_static: 4096 x 16 bytes + counters, ~64 KB per device.
struct StaticScratch {
    double part[kStaticMaxBlocks];               // fixed-order block sums of d_h
    unsigned long long bsum[kStaticMaxBlocks];   // block sums of n_h -> block offsets
    double sum_d;
    unsigned int done_sum, done_alloc;
};

static __device__ __align__(256) StaticScratch g_alloc_scratch;

// Block sum of 1024 terms with 512 threads in the library's fixed order:
// i + 512 first, then halving through shared memory, then shuffles.
__device__ double tree_sum_1024(double v, double *sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = 256; s >= 32; s >>= 1) {
        if (t < s) sh[t] = __dadd_rn(sh[t], sh[t + s]);
        __syncthreads();
    }
    double r = 0.0;
    if (t < 32) {
        r = sh[t];
        for (int s = 16; s >= 1; s >>= 1) r = __dadd_rn(r, __shfl_down_sync(0xffffffffu, r, s));
    }
    return r;
}

__global__ void __launch_bounds__(512) ks_sum(const double *d_h, uint64_t n_hc,
                                              StaticScratch *sc) {
    __shared__ double sh[512];
    __shared__ bool s_last;
    const uint64_t h0 = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
    const double a = h0 < n_hc ? d_h[h0] : 0.0;
    const double b = h0 + 512 < n_hc ? d_h[h0 + 512] : 0.0;
    const double r = tree_sum_1024(__dadd_rn(a, b), sh);
    if (threadIdx.x == 0) {
        sc->part[blockIdx.x] = r;
        __threadfence();
        s_last = atomicAdd(&sc->done_sum, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    __syncthreads();
    double S[1];  // the block sums in the library's fixed tree order
    vp::block_tree_sum<1>(sc->part, gridDim.x, sh, S);
    if (threadIdx.x != 0) return;
    sc->sum_d = S[0];
    sc->done_sum = 0u;
}

__global__ void __launch_bounds__(256) ks_alloc(const double *d_h, uint64_t n_hc, int64_t n_ev,
                                                int plus2, uint32_t *n_h, uint64_t *off,
                                                StaticScratch *sc) {
    __shared__ unsigned long long s_sum;
    __shared__ bool s_last;
    const double sum_d = __ldcg(&sc->sum_d);
    if (!isfinite(sum_d)) return;  // allocation left unchanged
    if (threadIdx.x == 0) s_sum = 0ull;
    __syncthreads();
    unsigned long long mine = 0;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
        const uint64_t h = (uint64_t)blockIdx.x * 1024 + i;
        if (h >= n_hc) break;
        double q;
        if (sum_d > 0.0) q = __ddiv_rn(__dmul_rn((double)n_ev, d_h[h]), sum_d);
        else q = __ddiv_rn((double)n_ev, (double)n_hc);
        double fl = floor(q);
        // a quotient within 2^-50 q below an integer counts as that integer
        if (__dsub_rn(__dadd_rn(fl, 1.0), q) <= __dmul_rn(q, 8.8817841970012523e-16)) fl += 1.0;
        uint32_t n;
        if (plus2) n = (uint32_t)fl + 2u;
        else n = fl > 2.0 ? (uint32_t)fl : 2u;
        n_h[h] = n;
        mine += n;
    }
    for (int s = 16; s >= 1; s >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, s);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_sum, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
        sc->bsum[blockIdx.x] = s_sum;
        __threadfence();
        s_last = atomicAdd(&sc->done_alloc, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    unsigned long long run = 0;
    for (unsigned q = 0; q < gridDim.x; ++q) {
        const unsigned long long v = __ldcg(sc->bsum + q);
        sc->bsum[q] = run;
        run += v;
    }
    off[n_hc] = run;
    sc->done_alloc = 0u;
}

__global__ void __launch_bounds__(256) ks_offsets(const uint32_t *n_h, uint64_t n_hc,
                                                  uint64_t *off, const StaticScratch *sc) {
    __shared__ unsigned long long s_warp[8];
    if (!isfinite(__ldcg(&sc->sum_d))) return;
    const uint64_t h0 = (uint64_t)blockIdx.x * 1024 + (uint64_t)threadIdx.x * 4;
    uint32_t n[4];
    unsigned long long tot = 0;
    for (int i = 0; i < 4; ++i) {
        n[i] = h0 + i < n_hc ? n_h[h0 + i] : 0u;
        tot += n[i];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = tot;
    for (int s = 1; s < 32; s <<= 1) {
        const unsigned long long o = __shfl_up_sync(0xffffffffu, inc, s);
        if (lane >= s) inc += o;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    unsigned long long base = __ldcg(sc->bsum + blockIdx.x);
    for (int w = 0; w < warp; ++w) base += s_warp[w];
    unsigned long long run = base + inc - tot;
    for (int i = 0; i < 4; ++i) {
        if (h0 + i < n_hc) off[h0 + i] = run;
        run += n[i];
    }
}

// Device address of the scratch, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
StaticScratch *g_scratch_ptr[kMaxDevices] = {};

vp_status scratch_for_current_device(StaticScratch **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        vp::set_error_message(VP_ECUDA, cudaGetErrorString(e));
        return VP_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        vp::set_error_message(VP_EINVAL, "vp_alloc_static: device index beyond 64");
        return VP_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_alloc_scratch);
        if (e != cudaSuccess || !p) {
            vp::set_error_message(VP_ECUDA, "vp_alloc_static: cudaGetSymbolAddress of the scratch failed");
            return VP_ECUDA;
        }
        g_scratch_ptr[dev] = (StaticScratch *)p;
    }
    *out = g_scratch_ptr[dev];
    return VP_OK;
}

}  // namespace

extern "C" vp_status vp_alloc_static(const double *d_h, int64_t n_hc, int64_t n_ev, int plus2,
                                     uint32_t *n_h, uint64_t *offsets, void *stream) {
    if (!d_h || !n_h || !offsets)
        return vp::set_error_message(VP_EINVAL, "vp_alloc_static: NULL buffer"), VP_EINVAL;
    if (n_hc < 1 || (uint64_t)n_hc > kStaticMaxHc)
        return vp::set_error_message(
                   VP_EINVAL, "vp_alloc_static: n_hc must be 1..4194304 (the static scratch holds "
                              "4096 blocks of 1024 hypercubes)"),
               VP_EINVAL;
    // every n_h is at most floor(N_ev) (+ 2 with plus2) and is stored as a
    // 32-bit integer: larger N_ev would not fit (the contexts bound N_ev more
    // tightly still, through the Philox counter)
    if (n_ev < 2 || n_ev > (int64_t)0xFFFFFFFFll - 2)
        return vp::set_error_message(VP_EINVAL, "vp_alloc_static: n_ev must be 2 .. 4294967293"),
               VP_EINVAL;
    StaticScratch *sc = nullptr;
    vp_status st = scratch_for_current_device(&sc);
    if (st != VP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)(((uint64_t)n_hc + 1023) / 1024);
    // the two last-block counters must start at zero
    cudaError_t e = cudaMemsetAsync(&sc->done_sum, 0, 2 * sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        ks_sum<<<blocks, 512, 0, s>>>(d_h, (uint64_t)n_hc, sc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ks_alloc<<<blocks, 256, 0, s>>>(d_h, (uint64_t)n_hc, n_ev, plus2 ? 1 : 0, n_h, offsets, sc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ks_offsets<<<blocks, 256, 0, s>>>(n_h, (uint64_t)n_hc, offsets, sc);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        vp::set_error_message(VP_ECUDA, cudaGetErrorString(e));
        return VP_ECUDA;
    }
    return VP_OK;
}
