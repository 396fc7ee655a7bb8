// probe.cu -- throughput of shared-memory atomic adds in the sampling kernel's
// access pattern, the bound of its histogram steps (a5: one count per axis per
// sample, and one FP32 sum per axis per sample with a nonzero integrand).
// Each thread holds one random increment per axis (D = 20 axes of 1000
// increments, as on the 20-D ball with N_g = 1000) and adds to them in turn,
// so the adds meet the bank conflicts and collisions of random increments and
// no other instruction stands between them.
#include "host.h"

namespace vp {

constexpr int kProbeAxes = 20, kProbeNg = 1000, kProbeThreads = 768, kProbeIters = 256;

template <bool F32>
__global__ void __launch_bounds__(kProbeThreads, 1) k_probe_atomics(uint32_t *sink) {
    extern __shared__ __align__(16) uint32_t ps[];
    for (int b = threadIdx.x; b < kProbeAxes * kProbeNg; b += blockDim.x) ps[b] = 0u;
    __syncthreads();
    uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    int bin[kProbeAxes];
#pragma unroll
    for (int mu = 0; mu < kProbeAxes; ++mu) {
        s ^= s << 13;
        s ^= s >> 17;
        s ^= s << 5;
        bin[mu] = mu * kProbeNg + (int)(s % (uint32_t)kProbeNg);
    }
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int mu = 0; mu < kProbeAxes; ++mu) {
            if (F32) atomicAdd((float *)ps + bin[mu], 1.0f);
            else atomicAdd(ps + bin[mu], 1u);
        }
    }
    __syncthreads();
    uint32_t acc = 0u;
    for (int b = threadIdx.x; b < kProbeAxes * kProbeNg; b += blockDim.x) acc ^= ps[b];
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1u);  // (keeps the adds; practically never taken)
}

}  // namespace vp

using namespace vp;

extern "C" vp_status vp_shared_atomic_rate(int f32, double *per_s) {
    if (!per_s) return fail(VP_EINVAL, "NULL out");
    *per_s = 0.0;
    int dev = 0, n_sm = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    void (*k)(uint32_t *) = f32 ? k_probe_atomics<true> : k_probe_atomics<false>;
    const int smem = kProbeAxes * kProbeNg * 4;
    CU(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    uint32_t *sink = nullptr;
    CU(cudaMalloc(&sink, 4));
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
        e = cudaEventRecord(a, 0);
        if (e == cudaSuccess) {
            k<<<n_sm, kProbeThreads, smem, 0>>>(sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(sink);
    if (e != cudaSuccess) return fail(VP_ECUDA, "vp_shared_atomic_rate: %s", cudaGetErrorString(e));
    const double n = (double)n_sm * kProbeThreads * kProbeIters * kProbeAxes;
    *per_s = best > 0.0f ? n / (best * 1e-3) : 0.0;
    return VP_OK;
}
