// sample_dispatch.cu -- host-side choice among the sampling kernel instantiations.
#include <mutex>
#include <vector>

#include "sample_impl.cuh"

namespace vp {

const void *kptr_one_f32_g(int bucket, int kind);
const void *kptr_many_f32_g(int bucket, int kind);
cudaError_t launch_eval_f32_g(int bucket, int kind, cudaStream_t s, const Desc *desc, int member, int64_t n, const uint64_t *h, const uint32_t *j, uint32_t t, double *x, int32_t *idx, double *jac, double *f, int pw);
const void *kptr_one_f32_x(int bucket, int kind);
const void *kptr_one_f32_p1(int bucket, int kind);
const void *kptr_many_f32_x(int bucket, int kind);
cudaError_t launch_eval_f32_x(int bucket, int kind, cudaStream_t s, const Desc *desc, int member, int64_t n, const uint64_t *h, const uint32_t *j, uint32_t t, double *x, int32_t *idx, double *jac, double *f, int pw);
const void *kptr_one_f64_g(int bucket, int kind);
const void *kptr_one_f64_mo(int bucket, int kind);
const void *kptr_many_f32_ax(int bucket, int kind);
const void *kptr_many_f64_ax(int bucket, int kind);
const void *kptr_many_f64_g(int bucket, int kind);
cudaError_t launch_eval_f64_g(int bucket, int kind, cudaStream_t s, const Desc *desc, int member, int64_t n, const uint64_t *h, const uint32_t *j, uint32_t t, double *x, int32_t *idx, double *jac, double *f, int pw);

// (p1: the one-integral FP32 kernel's single-peak form, dimension-exact buckets)
static const void *pick(bool f64, int bucket, bool exact, int kind, bool one, bool mo = false,
                        bool ax = false, bool p1 = false) {
    if (f64 && one && mo) return kptr_one_f64_mo(bucket, kind);
    if (!f64 && one && exact && p1 && kind != VP_POSTERIOR) return kptr_one_f32_p1(bucket, kind);
    if (!one && ax) return f64 ? kptr_many_f64_ax(bucket, kind) : kptr_many_f32_ax(bucket, kind);
    if (f64) return one ? kptr_one_f64_g(bucket, kind) : kptr_many_f64_g(bucket, kind);
    if (exact) return one ? kptr_one_f32_x(bucket, kind) : kptr_many_f32_x(bucket, kind);
    return one ? kptr_one_f32_g(bucket, kind) : kptr_many_f32_g(bucket, kind);
}

static cudaError_t launch_many(bool f64, int bucket, bool exact, int kind, dim3 grid, dim3 block,
                               size_t smem, cudaStream_t s, const SampleArgs &a, bool ax) {
    const void *k = pick(f64, bucket, exact, kind, false, false, ax);
    if (!k) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];  // programmatic dependent launch (the kernel waits first)
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {(void *)&a};
    return cudaLaunchKernelExC(&cfg, k, args);
}

static cudaError_t launch_one(bool f64, int bucket, bool exact, int kind, dim3 grid, dim3 block,
                              size_t smem, int cs, cudaStream_t s, const SampleOne &a) {
    const void *k = pick(f64, bucket, exact, kind, true, f64 && a.n_out > 1, false,
                         !f64 && a.kp_peaks == 1);
    if (!k) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // (the kernel waits first)
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    void *args[] = {(void *)&a};
    return cudaLaunchKernelExC(&cfg, k, args);
}

cudaError_t launch_sample_f32(int bucket, bool exact, int kind, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, const SampleArgs &a, bool ax) {
    return launch_many(false, bucket, exact, kind, grid, block, smem, s, a, ax);
}
cudaError_t launch_sample_f64(int bucket, bool exact, int kind, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, const SampleArgs &a, bool ax) {
    return launch_many(true, bucket, false, kind, grid, block, smem, s, a, ax);
}
cudaError_t launch_sample_one_f32(int bucket, bool exact, int kind, dim3 grid, dim3 block,
                                  size_t smem, int cs, cudaStream_t s, const SampleOne &a) {
    return launch_one(false, bucket, exact, kind, grid, block, smem, cs, s, a);
}
cudaError_t launch_sample_one_f64(int bucket, bool exact, int kind, dim3 grid, dim3 block,
                                  size_t smem, int cs, cudaStream_t s, const SampleOne &a) {
    return launch_one(true, bucket, false, kind, grid, block, smem, cs, s, a);
}

// The limit is a property of the kernel for the whole process, shared by every
// context, batch and server that launches it: it only ever grows, so that
// configuring a kernel for small launches cannot break another user's larger ones.
static std::mutex g_smem_mu;
struct SmemLimit {
    const void *kernel;
    int device, bytes;
};
static std::vector<SmemLimit> g_smem_limit;

static cudaError_t smem_config(bool f64, int bucket, bool exact, int kind, bool one, int max_smem,
                               bool mo = false, bool ax = false, bool p1 = false) {
    const void *k = pick(f64, bucket, exact, kind, one, mo, ax, p1);
    if (!k) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_smem_mu);
    int *cur = nullptr;  // the attribute is per device
    for (auto &l : g_smem_limit)
        if (l.kernel == k && l.device == dev) cur = &l.bytes;
    if (cur && *cur >= max_smem) return cudaSuccess;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess && one)  // clusters of up to 16 CTAs
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    if (cur) *cur = max_smem;
    else g_smem_limit.push_back({k, dev, max_smem});
    return cudaSuccess;
}
cudaError_t sample_smem_config_f32(int bucket, bool exact, int kind, bool one, int max_smem,
                                   bool ax, bool p1) {
    return smem_config(false, bucket, exact, kind, one, max_smem, false, ax, p1);
}
cudaError_t sample_smem_config_f64(int bucket, bool exact, int kind, bool one, int max_smem,
                                   bool mo, bool ax) {
    return smem_config(true, bucket, false, kind, one, max_smem, mo, ax);
}

static int occupancy(bool f64, int bucket, bool exact, int kind, bool one, int threads, size_t smem,
                     bool mo = false, bool ax = false, bool p1 = false) {
    const void *k = pick(f64, bucket, exact, kind, one, mo, ax, p1);
    int n = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess)
        return 0;
    return n;
}
int sample_occupancy_f32(int bucket, bool exact, int kind, bool one, int threads, size_t smem,
                         bool ax, bool p1) {
    return occupancy(false, bucket, exact, kind, one, threads, smem, false, ax, p1);
}
int sample_occupancy_f64(int bucket, bool exact, int kind, bool one, int threads, size_t smem,
                         bool mo, bool ax) {
    return occupancy(true, bucket, false, kind, one, threads, smem, mo, ax);
}

static int cluster_ctas(bool f64, int bucket, bool exact, int kind, int cs, int grid, int threads,
                        size_t smem, bool mo = false, bool p1 = false) {
    const void *k = pick(f64, bucket, exact, kind, true, mo, false, p1);
    if (!k) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n * cs;
}
int sample_cluster_ctas_f32(int bucket, bool exact, int kind, int cs, int grid, int threads,
                            size_t smem, bool p1) {
    return cluster_ctas(false, bucket, exact, kind, cs, grid, threads, smem, false, p1);
}
int sample_cluster_ctas_f64(int bucket, bool exact, int kind, int cs, int grid, int threads,
                            size_t smem, bool mo) {
    return cluster_ctas(true, bucket, false, kind, cs, grid, threads, smem, mo);
}

cudaError_t launch_eval_f32(int bucket, bool exact, int kind, cudaStream_t s, const Desc *desc,
                            int member, int64_t n, const uint64_t *h, const uint32_t *j,
                            uint32_t t, double *x, int32_t *idx, double *jac, double *f, int pw) {
    return exact ? launch_eval_f32_x(bucket, kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw)
                 : launch_eval_f32_g(bucket, kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
}
cudaError_t launch_eval_f64(int bucket, bool exact, int kind, cudaStream_t s, const Desc *desc,
                            int member, int64_t n, const uint64_t *h, const uint32_t *j,
                            uint32_t t, double *x, int32_t *idx, double *jac, double *f, int pw) {
    (void)exact;
    return launch_eval_f64_g(bucket, kind, s, desc, member, n, h, j, t, x, idx, jac, f, pw);
}

}  // namespace vp
