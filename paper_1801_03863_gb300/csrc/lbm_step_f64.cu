// lbm_step_f64.cu -- fused step kernels with double storage and double arithmetic.
#include "lbm_aux.h"
#include "lbm_step.cuh"

namespace lbm {

const void* step_kernel_f64(int lattice, int collision, int V) {
    if (V == 2) return pick_step_kernel<double, double, 2>(lattice, collision);
    return nullptr;
}

}  // namespace lbm
