// precond.cu -- instantiations of the data-histogram kernel of the map's
// training on sample data (§4.2, preconditioned integrators).
#include <algorithm>

#include "sample_impl.cuh"

namespace vp {

template <int DMAX> static const void *kptr_precond_d(int kind) {
    switch (kind) {
        case VP_GAUSS: return (const void *)k_precondition<DMAX, VP_GAUSS>;
        case VP_BALL: return (const void *)k_precondition<DMAX, VP_BALL>;
        case VP_EXPNORM: return (const void *)k_precondition<DMAX, VP_EXPNORM>;
        case VP_POSTERIOR: return (const void *)k_precondition<DMAX, VP_POSTERIOR>;
    }
    return nullptr;
}

static const void *kptr_precond(int bucket, int kind) {
    switch (bucket) {
        case 0: return kptr_precond_d<4>(kind);
        case 1: return kptr_precond_d<8>(kind);
        case 2: return kptr_precond_d<12>(kind);
        case 3: return kptr_precond_d<16>(kind);
        case 4: return kptr_precond_d<20>(kind);
        case 5: return kptr_precond_d<24>(kind);
    }
    return nullptr;
}

cudaError_t launch_precondition(int bucket, int kind, cudaStream_t s, const Desc *desc, int member,
                                int64_t n, const double *x, const double *f, uint32_t buf) {
    const void *k = kptr_precond(bucket, kind);
    if (!k) return cudaErrorInvalidValue;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    void *args[] = {(void *)&desc, (void *)&member, (void *)&n, (void *)&x, (void *)&f,
                    (void *)&buf};
    return cudaLaunchKernel(k, dim3((unsigned)std::max<int64_t>(blocks, 1)), dim3(256), args, 0, s);
}

}  // namespace vp
