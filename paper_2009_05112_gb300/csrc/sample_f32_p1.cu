// sample_f32_p1.cu -- instantiations of the one-integral kernel, FP32 path, dimension-exact
// buckets, for integrands of a single peak (the form that keeps fewer registers).
// (Split into several translation units so that they compile in parallel.)
#include "sample_impl.cuh"

namespace vp {

template <int DMAX, int KIND> static const void *kptr_one_f32_p1_k() { return (const void *)k_sample_one<DMAX, true, false, KIND, false, true>; }
template <int DMAX> static const void *kptr_one_f32_p1_d(int kind) {
    switch (kind) {
        case VP_GAUSS: return kptr_one_f32_p1_k<DMAX, VP_GAUSS>();
        case VP_BALL: return kptr_one_f32_p1_k<DMAX, VP_BALL>();
        case VP_EXPNORM: return kptr_one_f32_p1_k<DMAX, VP_EXPNORM>();
    }
    return nullptr;
}
const void *kptr_one_f32_p1(int bucket, int kind) {
    switch (bucket) {
        case 0: return kptr_one_f32_p1_d<4>(kind);
        case 1: return kptr_one_f32_p1_d<8>(kind);
        case 2: return kptr_one_f32_p1_d<12>(kind);
        case 3: return kptr_one_f32_p1_d<16>(kind);
        case 4: return kptr_one_f32_p1_d<20>(kind);
        case 5: return kptr_one_f32_p1_d<24>(kind);
    }
    return nullptr;
}

}  // namespace vp
