// sample_f32_ax.cu -- instantiations of the several-integral kernel, FP32 path,
// with the strata per axis read from each integral's descriptor (§3.2).
#include "sample_impl.cuh"

namespace vp {

template <int DMAX, int KIND> static const void *kptr_many_f32_ax_k() { return (const void *)k_sample_many<DMAX, false, false, KIND, true>; }
template <int DMAX> static const void *kptr_many_f32_ax_d(int kind) {
    switch (kind) {
        case VP_GAUSS: return kptr_many_f32_ax_k<DMAX, VP_GAUSS>();
        case VP_BALL: return kptr_many_f32_ax_k<DMAX, VP_BALL>();
        case VP_EXPNORM: return kptr_many_f32_ax_k<DMAX, VP_EXPNORM>();
        case VP_POSTERIOR: return kptr_many_f32_ax_k<DMAX, VP_POSTERIOR>();
    }
    return nullptr;
}
const void *kptr_many_f32_ax(int bucket, int kind) {
    switch (bucket) {
        case 0: return kptr_many_f32_ax_d<4>(kind);
        case 1: return kptr_many_f32_ax_d<8>(kind);
        case 2: return kptr_many_f32_ax_d<12>(kind);
        case 3: return kptr_many_f32_ax_d<16>(kind);
        case 4: return kptr_many_f32_ax_d<20>(kind);
        case 5: return kptr_many_f32_ax_d<24>(kind);
    }
    return nullptr;
}

}  // namespace vp
