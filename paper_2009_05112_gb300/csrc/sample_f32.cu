// sample_f32.cu -- instantiations of the fused sampling kernel and its
// inspection twin for the FP32 path (one translation unit per precision
// so the two compile in parallel).
#include "sample_impl.cuh"

namespace vp {


template <int DMAX, int KIND>
static cudaError_t launch_one(dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              const SampleArgs &a) {
    k_sample<DMAX, false, KIND><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <int DMAX>
static cudaError_t launch_kind(int kind, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                               const SampleArgs &a) {
    switch (kind) {
        case VP_GAUSS: return launch_one<DMAX, VP_GAUSS>(grid, block, smem, s, a);
        case VP_BALL: return launch_one<DMAX, VP_BALL>(grid, block, smem, s, a);
        case VP_EXPNORM: return launch_one<DMAX, VP_EXPNORM>(grid, block, smem, s, a);
        case VP_POSTERIOR: return launch_one<DMAX, VP_POSTERIOR>(grid, block, smem, s, a);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sample_f32(int bucket, int kind, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, const SampleArgs &a) {
    switch (bucket) {
        case 0: return launch_kind<4>(kind, grid, block, smem, s, a);
        case 1: return launch_kind<8>(kind, grid, block, smem, s, a);
        case 2: return launch_kind<12>(kind, grid, block, smem, s, a);
        case 3: return launch_kind<16>(kind, grid, block, smem, s, a);
        case 4: return launch_kind<24>(kind, grid, block, smem, s, a);
    }
    return cudaErrorInvalidValue;
}

template <int DMAX, int KIND>
static const void *kernel_ptr() { return (const void *)k_sample<DMAX, false, KIND>; }

template <int DMAX>
static const void *kernel_kind(int kind) {
    switch (kind) {
        case VP_GAUSS: return kernel_ptr<DMAX, VP_GAUSS>();
        case VP_BALL: return kernel_ptr<DMAX, VP_BALL>();
        case VP_EXPNORM: return kernel_ptr<DMAX, VP_EXPNORM>();
        case VP_POSTERIOR: return kernel_ptr<DMAX, VP_POSTERIOR>();
    }
    return nullptr;
}

static const void *kernel_of(int bucket, int kind) {
    switch (bucket) {
        case 0: return kernel_kind<4>(kind);
        case 1: return kernel_kind<8>(kind);
        case 2: return kernel_kind<12>(kind);
        case 3: return kernel_kind<16>(kind);
        case 4: return kernel_kind<24>(kind);
    }
    return nullptr;
}

cudaError_t sample_smem_config_f32(int bucket, int kind, int max_smem) {
    const void *k = kernel_of(bucket, kind);
    if (!k) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

int sample_occupancy_f32(int bucket, int kind, int threads, size_t smem) {
    const void *k = kernel_of(bucket, kind);
    int n = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess)
        return 0;
    return n;
}

template <int DMAX, int KIND>
static cudaError_t eval_one(cudaStream_t s, const Desc *desc, int member, int64_t n,
                            const uint64_t *h, const uint32_t *j, uint32_t t, double *x,
                            int32_t *idx, double *jac, double *f, int pw) {
    int blocks = (int)((n + 127) / 128);
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    k_eval<DMAX, false, KIND><<<blocks, 128, (size_t)pw * 4, s>>>(desc, member, n, h, j, t, x, idx, jac, f, pw);
    return cudaGetLastError();
}

template <int DMAX>
static cudaError_t eval_kind(int kind, cudaStream_t s, const Desc *desc, int member, int64_t n,
                             const uint64_t *h, const uint32_t *j, uint32_t t, double *x,
                             int32_t *idx, double *jac, double *f, int pw) {
    switch (kind) {
        case VP_GAUSS: return eval_one<DMAX, VP_GAUSS>(s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case VP_BALL: return eval_one<DMAX, VP_BALL>(s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case VP_EXPNORM: return eval_one<DMAX, VP_EXPNORM>(s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case VP_POSTERIOR: return eval_one<DMAX, VP_POSTERIOR>(s, desc, member, n, h, j, t, x, idx, jac, f, pw);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_eval_f32(int bucket, int kind, cudaStream_t s, const Desc *desc, int member,
                            int64_t n, const uint64_t *h, const uint32_t *j, uint32_t t,
                            double *x, int32_t *idx, double *jac, double *f, int pw) {
    switch (bucket) {
        case 0: return eval_kind<4>(kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case 1: return eval_kind<8>(kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case 2: return eval_kind<12>(kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case 3: return eval_kind<16>(kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case 4: return eval_kind<24>(kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
    }
    return cudaErrorInvalidValue;
}

}  // namespace vp
