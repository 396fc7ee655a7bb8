// sample_f32_gm.cu -- instantiations of the several-integral kernel and the per-sample inspection kernel, FP32 path.
// (Split into several translation units so that they compile in parallel.)
#include "sample_impl.cuh"

namespace vp {

template <int DMAX, int KIND> static const void *kptr_many_f32_g_k() { return (const void *)k_sample_many<DMAX, false, false, KIND>; }
template <int DMAX> static const void *kptr_many_f32_g_d(int kind) {
    switch (kind) {
        case VP_GAUSS: return kptr_many_f32_g_k<DMAX, VP_GAUSS>();
        case VP_BALL: return kptr_many_f32_g_k<DMAX, VP_BALL>();
        case VP_EXPNORM: return kptr_many_f32_g_k<DMAX, VP_EXPNORM>();
        case VP_POSTERIOR: return kptr_many_f32_g_k<DMAX, VP_POSTERIOR>();
    }
    return nullptr;
}
const void *kptr_many_f32_g(int bucket, int kind) {
    switch (bucket) {
        case 0: return kptr_many_f32_g_d<4>(kind);
        case 1: return kptr_many_f32_g_d<8>(kind);
        case 2: return kptr_many_f32_g_d<12>(kind);
        case 3: return kptr_many_f32_g_d<16>(kind);
        case 4: return kptr_many_f32_g_d<20>(kind);
        case 5: return kptr_many_f32_g_d<24>(kind);
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

}  // namespace vp
