// lbm_step_f64.cu -- fused step kernels with double storage and double arithmetic.
#include "lbm_aux.h"
#include "lbm_step.cuh"

namespace lbm {

const void* step_kernel_f64(int lattice, int collision, int V) {
    if (V == 2) {
        if (lattice == 2)
            return collision == COLL_SRT
                       ? (const void*)&step_kernel<D2Q9, double, double, 2, COLL_SRT>
                       : (const void*)&step_kernel<D2Q9, double, double, 2, COLL_MINXENT4>;
        return (const void*)&step_kernel<D1Q3, double, double, 2, COLL_MINXENT4>;
    }
    return nullptr;
}

}  // namespace lbm
