// vg_pass_group.cu -- instantiations of the pass kernel for grouped conditioning (the
// isotropic and space-time families; 4 to 32 lanes per block, FP64 and mixed).
#include "vg_internal.h"
#include "vg_pass.cuh"

namespace vg {

template <int COV, typename T>
static const void* group_kernel_for_lanes(int L) {
    switch (L) {
    case 4: return reinterpret_cast<const void*>(&k_pass<COV, 4, T, true>);
    case 8: return reinterpret_cast<const void*>(&k_pass<COV, 8, T, true>);
    case 16: return reinterpret_cast<const void*>(&k_pass<COV, 16, T, true>);
    case 32: return reinterpret_cast<const void*>(&k_pass<COV, 32, T, true>);
    default: return nullptr;
    }
}

template <typename T>
static const void* group_kernel(int cov, int L) {
    switch (cov) {
    case COV_EXP: return group_kernel_for_lanes<COV_EXP, T>(L);
    case COV_MATERN: return group_kernel_for_lanes<COV_MATERN, T>(L);
    case COV_ST: return group_kernel_for_lanes<COV_ST, T>(L);
    default: return nullptr;
    }
}

const void* pass_group_kernel(int cov, int L, int prec) {
    return prec == 0 ? group_kernel<double>(cov, L) : group_kernel<float>(cov, L);
}

}  // namespace vg
