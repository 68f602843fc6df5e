// lbm_step_bf16.cu -- fused step kernels with __nv_bfloat16 storage and float arithmetic.
#include "lbm_aux.h"
#include "lbm_step.cuh"
#include "lbm_step_smem.cuh"

namespace lbm {

const void* step_kernel_bf16(int lattice, int collision, int V) {
    if (V == 4) {
        if (lattice == 2)
            return collision == COLL_SRT
                       ? (const void*)&step_kernel<D2Q9, __nv_bfloat16, float, 4, COLL_SRT>
                       : (const void*)&step_kernel<D2Q9, __nv_bfloat16, float, 4, COLL_MINXENT4>;
        return (const void*)&step_kernel<D1Q3, __nv_bfloat16, float, 4, COLL_MINXENT4>;
    }
    if (V == 8) {
        if (lattice == 2)
            return collision == COLL_SRT
                       ? (const void*)&step_kernel<D2Q9, __nv_bfloat16, float, 8, COLL_SRT>
                       : (const void*)&step_kernel<D2Q9, __nv_bfloat16, float, 8, COLL_MINXENT4>;
        return (const void*)&step_kernel<D1Q3, __nv_bfloat16, float, 8, COLL_MINXENT4>;
    }
    return nullptr;
}

const void* step_kernel_smem_bf16(int collision, int P, size_t* smem_bytes) {
    using TS = SmemTile<__nv_bfloat16>;
    *smem_bytes = TS::SMEM_BYTES;
    constexpr int TN = TS::TILE_NODES, NS = TS::STAGES;
    if (P == 1)
        return collision == COLL_SRT ? (const void*)&step_kernel_smem<__nv_bfloat16, COLL_SRT, TN, NS, 1>
                                     : (const void*)&step_kernel_smem<__nv_bfloat16, COLL_MINXENT4, TN, NS, 1>;
    return collision == COLL_SRT ? (const void*)&step_kernel_smem<__nv_bfloat16, COLL_SRT, TN, NS, 2>
                                 : (const void*)&step_kernel_smem<__nv_bfloat16, COLL_MINXENT4, TN, NS, 2>;
}

}  // namespace lbm
