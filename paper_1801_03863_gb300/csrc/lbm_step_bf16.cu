// lbm_step_bf16.cu -- fused step kernels with __nv_bfloat16 storage and float arithmetic.
#include "lbm_aux.h"
#include "lbm_step.cuh"
#include "lbm_step_smem.cuh"

namespace lbm {

const void* step_kernel_bf16(int lattice, int collision, int V) {
    if (V == 4) return pick_step_kernel<__nv_bfloat16, float, 4>(lattice, collision);
    if (V == 8) return pick_step_kernel<__nv_bfloat16, float, 8>(lattice, collision);
    return nullptr;
}

const void* step_kernel_smem_bf16(int collision, int variant, size_t* smem_bytes) {
    if (variant == 2) return pick_step_kernel_smem<__nv_bfloat16, 2>(collision, smem_bytes);
    if (variant == 3) return pick_step_kernel_smem<__nv_bfloat16, 3>(collision, smem_bytes);
    return variant == 1 ? pick_step_kernel_smem<__nv_bfloat16, 1>(collision, smem_bytes)
                        : pick_step_kernel_smem<__nv_bfloat16, 0>(collision, smem_bytes);
}

}  // namespace lbm
