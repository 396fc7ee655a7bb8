// sample_f64_mo.cu -- instantiations of the one-integral kernel, FP64 path,
// with several outputs summed per hypercube (App. B: several integrals from the
// same samples).
#include "sample_impl.cuh"

namespace vp {

template <int DMAX, int KIND> static const void *kptr_one_f64_mo_k() { return (const void *)k_sample_one<DMAX, false, true, KIND, true>; }
template <int DMAX> static const void *kptr_one_f64_mo_d(int kind) {
    switch (kind) {
        case VP_GAUSS: return kptr_one_f64_mo_k<DMAX, VP_GAUSS>();
        case VP_BALL: return kptr_one_f64_mo_k<DMAX, VP_BALL>();
        case VP_EXPNORM: return kptr_one_f64_mo_k<DMAX, VP_EXPNORM>();
        case VP_POSTERIOR: return kptr_one_f64_mo_k<DMAX, VP_POSTERIOR>();
    }
    return nullptr;
}
const void *kptr_one_f64_mo(int bucket, int kind) {
    switch (bucket) {
        case 0: return kptr_one_f64_mo_d<4>(kind);
        case 1: return kptr_one_f64_mo_d<8>(kind);
        case 2: return kptr_one_f64_mo_d<12>(kind);
        case 3: return kptr_one_f64_mo_d<16>(kind);
        case 4: return kptr_one_f64_mo_d<20>(kind);
        case 5: return kptr_one_f64_mo_d<24>(kind);
    }
    return nullptr;
}

}  // namespace vp
