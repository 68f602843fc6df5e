// lbm_step_f16.cu -- fused step kernels with __half storage and float arithmetic.
#include "lbm_aux.h"
#include "lbm_step.cuh"
#include "lbm_step_smem.cuh"

namespace lbm {

const void* step_kernel_f16(int lattice, int collision, int V) {
    if (V == 4) {
        if (lattice == 2)
            return collision == COLL_SRT
                       ? (const void*)&step_kernel<D2Q9, __half, float, 4, COLL_SRT>
                       : (const void*)&step_kernel<D2Q9, __half, float, 4, COLL_MINXENT4>;
        return (const void*)&step_kernel<D1Q3, __half, float, 4, COLL_MINXENT4>;
    }
    if (V == 8) {
        if (lattice == 2)
            return collision == COLL_SRT
                       ? (const void*)&step_kernel<D2Q9, __half, float, 8, COLL_SRT>
                       : (const void*)&step_kernel<D2Q9, __half, float, 8, COLL_MINXENT4>;
        return (const void*)&step_kernel<D1Q3, __half, float, 8, COLL_MINXENT4>;
    }
    return nullptr;
}

const void* step_kernel_smem_f16(int collision, int P, size_t* smem_bytes) {
    using TS = SmemTile<__half>;
    *smem_bytes = TS::SMEM_BYTES;
    constexpr int TN = TS::TILE_NODES, NS = TS::STAGES;
    if (P == 1)
        return collision == COLL_SRT ? (const void*)&step_kernel_smem<__half, COLL_SRT, TN, NS, 1>
                                     : (const void*)&step_kernel_smem<__half, COLL_MINXENT4, TN, NS, 1>;
    return collision == COLL_SRT ? (const void*)&step_kernel_smem<__half, COLL_SRT, TN, NS, 2>
                                 : (const void*)&step_kernel_smem<__half, COLL_MINXENT4, TN, NS, 2>;
}

}  // namespace lbm
