// lbm_step_f32.cu -- fused step kernels with float storage and float arithmetic.
#include "lbm_aux.h"
#include "lbm_step.cuh"
#include "lbm_step_smem.cuh"

namespace lbm {

const void* step_kernel_f32(int lattice, int collision, int V) {
    if (V == 2) return pick_step_kernel<float, float, 2>(lattice, collision);
    if (V == 4) return pick_step_kernel<float, float, 4>(lattice, collision);
    return nullptr;
}

const void* step_kernel_smem_f32(int collision, int variant, size_t* smem_bytes) {
    if (variant == 2) return pick_step_kernel_smem<float, 2>(collision, smem_bytes);
    if (variant == 3) return pick_step_kernel_smem<float, 3>(collision, smem_bytes);
    return variant == 1 ? pick_step_kernel_smem<float, 1>(collision, smem_bytes)
                        : pick_step_kernel_smem<float, 0>(collision, smem_bytes);
}

}  // namespace lbm
