// vg_pass_f64.cu -- instantiations of the pass kernel with working type double.
#include "vg_internal.h"
#include "vg_pass.cuh"

namespace vg {

template <int COV>
static const void* kernel_for_lanes(int L) {
    switch (L) {
    case 1: return reinterpret_cast<const void*>(&k_pass<COV, 1, double>);
    case 2: return reinterpret_cast<const void*>(&k_pass<COV, 2, double>);
    case 4: return reinterpret_cast<const void*>(&k_pass<COV, 4, double>);
    case 8: return reinterpret_cast<const void*>(&k_pass<COV, 8, double>);
    case 16: return reinterpret_cast<const void*>(&k_pass<COV, 16, double>);
    case 32: return reinterpret_cast<const void*>(&k_pass<COV, 32, double>);
    default: return nullptr;
    }
}

// one range per coordinate: items spread over the lanes, at least 4 lanes per observation
static const void* aniso_kernel_for_lanes(int L) {
    switch (L) {
    case 4: return reinterpret_cast<const void*>(&k_pass<COV_ANISO, 4, double>);
    case 8: return reinterpret_cast<const void*>(&k_pass<COV_ANISO, 8, double>);
    case 16: return reinterpret_cast<const void*>(&k_pass<COV_ANISO, 16, double>);
    case 32: return reinterpret_cast<const void*>(&k_pass<COV_ANISO, 32, double>);
    default: return nullptr;
    }
}

static const void* aniso_batch_kernel_for_lanes(int L) {
    switch (L) {
    case 4: return reinterpret_cast<const void*>(&k_pass_batch<COV_ANISO, 4, double>);
    case 8: return reinterpret_cast<const void*>(&k_pass_batch<COV_ANISO, 8, double>);
    case 16: return reinterpret_cast<const void*>(&k_pass_batch<COV_ANISO, 16, double>);
    case 32: return reinterpret_cast<const void*>(&k_pass_batch<COV_ANISO, 32, double>);
    default: return nullptr;
    }
}

const void* pass_kernel_f64(int cov, int L) {
    switch (cov) {
    case COV_EXP: return kernel_for_lanes<COV_EXP>(L);
    case COV_MATERN: return kernel_for_lanes<COV_MATERN>(L);
    case COV_ST: return kernel_for_lanes<COV_ST>(L);
    case COV_ANISO: return aniso_kernel_for_lanes(L);
    default: return nullptr;
    }
}

template <int COV>
static const void* batch_kernel_for_lanes(int L) {
    switch (L) {
    case 1: return reinterpret_cast<const void*>(&k_pass_batch<COV, 1, double>);
    case 2: return reinterpret_cast<const void*>(&k_pass_batch<COV, 2, double>);
    case 4: return reinterpret_cast<const void*>(&k_pass_batch<COV, 4, double>);
    case 8: return reinterpret_cast<const void*>(&k_pass_batch<COV, 8, double>);
    case 16: return reinterpret_cast<const void*>(&k_pass_batch<COV, 16, double>);
    case 32: return reinterpret_cast<const void*>(&k_pass_batch<COV, 32, double>);
    default: return nullptr;
    }
}

const void* pass_batch_kernel_f64(int cov, int L) {
    switch (cov) {
    case COV_EXP: return batch_kernel_for_lanes<COV_EXP>(L);
    case COV_MATERN: return batch_kernel_for_lanes<COV_MATERN>(L);
    case COV_ST: return batch_kernel_for_lanes<COV_ST>(L);
    case COV_ANISO: return aniso_batch_kernel_for_lanes(L);
    default: return nullptr;
    }
}

}  // namespace vg
