// sample_f32.cu -- instantiations of the fused sampling kernel and its inspection
// twin for the FP32 path, dimension-guarded buckets (separate translation units compile in parallel).
#include "sample_impl.cuh"

namespace vp {

template <int DMAX, int KIND>
static const void *kptr_f32_g() { return (const void *)k_sample<DMAX, false, false, KIND>; }

template <int DMAX>
static const void *kkind_f32_g(int kind) {
    switch (kind) {
        case VP_GAUSS: return kptr_f32_g<DMAX, VP_GAUSS>();
        case VP_BALL: return kptr_f32_g<DMAX, VP_BALL>();
        case VP_EXPNORM: return kptr_f32_g<DMAX, VP_EXPNORM>();
        case VP_POSTERIOR: return kptr_f32_g<DMAX, VP_POSTERIOR>();
    }
    return nullptr;
}

const void *sample_kernel_f32_g(int bucket, int kind) {
    switch (bucket) {
        case 0: return kkind_f32_g<4>(kind);
        case 1: return kkind_f32_g<8>(kind);
        case 2: return kkind_f32_g<12>(kind);
        case 3: return kkind_f32_g<16>(kind);
        case 4: return kkind_f32_g<20>(kind);
        case 5: return kkind_f32_g<24>(kind);
    }
    return nullptr;
}

template <int DMAX, int KIND>
static cudaError_t eval_one_f32_g(cudaStream_t s, const Desc *desc, int member, int64_t n,
                                const uint64_t *h, const uint32_t *j, uint32_t t, double *x,
                                int32_t *idx, double *jac, double *f, int pw) {
    int blocks = (int)((n + 127) / 128);
    blocks = blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks);
    k_eval<DMAX, false, false, KIND><<<blocks, 128, (size_t)pw * 4, s>>>(desc, member, n, h, j, t, x,
                                                                   idx, jac, f, pw);
    return cudaGetLastError();
}

template <int DMAX>
static cudaError_t eval_kind_f32_g(int kind, cudaStream_t s, const Desc *desc, int member,
                                 int64_t n, const uint64_t *h, const uint32_t *j, uint32_t t,
                                 double *x, int32_t *idx, double *jac, double *f, int pw) {
    switch (kind) {
        case VP_GAUSS: return eval_one_f32_g<DMAX, VP_GAUSS>(s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case VP_BALL: return eval_one_f32_g<DMAX, VP_BALL>(s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case VP_EXPNORM: return eval_one_f32_g<DMAX, VP_EXPNORM>(s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case VP_POSTERIOR: return eval_one_f32_g<DMAX, VP_POSTERIOR>(s, desc, member, n, h, j, t, x, idx, jac, f, pw);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_eval_f32_g(int bucket, int kind, cudaStream_t s, const Desc *desc, int member,
                             int64_t n, const uint64_t *h, const uint32_t *j, uint32_t t,
                             double *x, int32_t *idx, double *jac, double *f, int pw) {
    switch (bucket) {
        case 0: return eval_kind_f32_g<4>(kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case 1: return eval_kind_f32_g<8>(kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case 2: return eval_kind_f32_g<12>(kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case 3: return eval_kind_f32_g<16>(kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case 4: return eval_kind_f32_g<20>(kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
        case 5: return eval_kind_f32_g<24>(kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
    }
    return cudaErrorInvalidValue;
}

const void *sample_kernel_f32_x(int bucket, int kind);
cudaError_t launch_eval_f32_x(int bucket, int kind, cudaStream_t s, const Desc *desc, int member,
                              int64_t n, const uint64_t *h, const uint32_t *j, uint32_t t,
                              double *x, int32_t *idx, double *jac, double *f, int pw);

static const void *pick_f32(int bucket, bool exact, int kind) {
    (void)exact;
    return exact ? sample_kernel_f32_x(bucket, kind) : sample_kernel_f32_g(bucket, kind);
}

cudaError_t launch_sample_f32(int bucket, bool exact, int kind, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, const SampleArgs &a) {
    const void *k = pick_f32(bucket, exact, kind);
    if (!k) return cudaErrorInvalidValue;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(k, grid, block, args, smem, s);
}

cudaError_t sample_smem_config_f32(int bucket, bool exact, int kind, int max_smem) {
    const void *k = pick_f32(bucket, exact, kind);
    if (!k) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

int sample_occupancy_f32(int bucket, bool exact, int kind, int threads, size_t smem) {
    const void *k = pick_f32(bucket, exact, kind);
    int n = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_eval_f32(int bucket, bool exact, int kind, cudaStream_t s, const Desc *desc,
                            int member, int64_t n, const uint64_t *h, const uint32_t *j,
                            uint32_t t, double *x, int32_t *idx, double *jac, double *f, int pw) {
    (void)exact;
    return exact ? launch_eval_f32_x(bucket, kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw)
                 : launch_eval_f32_g(bucket, kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
}

}  // namespace vp
