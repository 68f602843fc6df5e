// lbm_aux.h -- host-side entry points of the kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_common.cuh"

namespace lbm {

// Conservation reduction: instance i is split into P_i = min(CONS_PARTIALS,
// ny_i) partial sums, partial b over the rows y = b mod P_i, each summed by
// one block of CONS_THREADS threads; the split is a function of the instance
// alone, so the FP64 summation order never depends on the device.
constexpr int CONS_PARTIALS = 64;
constexpr int CONS_THREADS = 256;
constexpr int CONS_MIN_BLOCKS = 3;  // resident blocks per SM the register budget aims at
__host__ __device__ inline int cons_partials(int ny) { return ny < CONS_PARTIALS ? ny : CONS_PARTIALS; }

enum class AuxOp { Init, SetF, CollideInPlace, Moments, GatherF, Conservation };

struct AuxArgs {
    int lattice;   // 1 = D1Q3, 2 = D2Q9
    int storage;   // DT_*
    int compute;   // DT_F64 or DT_F32
    int collision; // COLL_*
    int count;     // instances
    int64_t max_nodes;
    const InstDesc* inst;  // device
    double rho0;
    bool pulled;           // stored field is post-collision (pull to read f(t_n))
    unsigned long long* status;
    cudaStream_t stream;
    const int2* cons_items;  // device: (instance, partial) of each conservation block
    int32_t cons_nitems;
    int64_t node_base = 0;   // host-array index of the first node the call covers (Init,
                             // Moments, stream_function): arrays start at that node
};

// Init:           dst <- f^eq(rho=p0, ux=p1, uy=p2) deviations
// SetF:           dst <- p0 (FP64 populations, [inst][a][y][x])
// CollideInPlace: dst <- collide(src) without streaming
// Moments:        o0, o1, o2 <- rho, ux, uy of f(t_n) read from src
// GatherF:        o0 <- FP64 populations of f(t_n)
// Conservation:   o0 <- per-instance totals (3 doubles each), o1 = partials scratch
//                 (count * CONS_PARTIALS * 3 doubles; partial b of instance i at
//                 (i * CONS_PARTIALS + b) * 3)
cudaError_t run_aux(AuxOp op, const AuxArgs& a, const void* src, void* dst, const double* p0,
                    const double* p1, const double* p2, double* o0, double* o1, double* o2);

// psi <- stream function of u_y (both [inst][y][x] FP64 device arrays in the
// concatenated node order); max_ny = largest instance height.
cudaError_t stream_function(const AuxArgs& a, int64_t max_ny, const double* uy, double* psi);

// Fused step kernels, one translation unit per storage type.  Each returns
// the __global__ function for (lattice, collision, V), or nullptr.
const void* step_kernel_f64(int lattice, int collision, int V);
const void* step_kernel_f32(int lattice, int collision, int V);
const void* step_kernel_f16(int lattice, int collision, int V);
const void* step_kernel_bf16(int lattice, int collision, int V);

// D2Q9 step kernels with shared-memory tile staging (FP32 arithmetic); also
// return the dynamic shared memory they need.
const void* step_kernel_smem_f32(int collision, int variant, size_t* smem_bytes);
const void* step_kernel_smem_f16(int collision, int variant, size_t* smem_bytes);
const void* step_kernel_smem_bf16(int collision, int variant, size_t* smem_bytes);
// Geometries of the TMA-staged kernel (variant = launch-shape kind - 1).
// Every CTA has one copy warp, which writes finished tiles out and issues
// the copies of the next ones, besides its colliding warps; a tile holds
// 64 nodes per unit x the units of each colliding warp:
//   0  large tiles: 8 warps, 7 colliding with 4 units each (2-byte storage;
//      2 for FP32): 1792 / 896 nodes, two-stage ring;
//   1  small tiles: 8 warps, 2 / 1 units each: 896 / 448 nodes, three-stage
//      ring (more copies in flight per node);
//   2  wide CTAs: 10 warps, 4 / 2 units each: 2304 / 1152 nodes, two stages;
//   3  deep ring: one CTA of 16 warps per SM, 2 / 1 units each: 1920 / 960
//      nodes on a five- / four-stage ring, so a stage is refilled four /
//      three tiles before it is needed.
// Two CTAs of the 8- and 10-warp geometries fit an SM (registers and
// shared memory); the 16-warp one keeps all 128 registers per thread.
#ifndef LBM_SMEM_STAGES_DEEP
#define LBM_SMEM_STAGES_DEEP 4   // FP32 storage
#endif
#ifndef LBM_SMEM_STAGES_DEEP2
#define LBM_SMEM_STAGES_DEEP2 5  // 2-byte storage
#endif
#ifndef LBM_DEEP_WARPS
#define LBM_DEEP_WARPS 15  // colliding warps of the deep-ring CTA
#endif
// colliding threads of a CTA (the copy warp comes on top)
constexpr int smem_threads(int variant) {
    return variant == 2 ? 288 : (variant == 3 ? 32 * LBM_DEEP_WARPS : 224);
}
constexpr int smem_block_threads(int variant) { return smem_threads(variant) + 32; }
// units of 32 node pairs per colliding warp and tile (storage 1: FP32)
#ifndef LBM_DEEP_UNITS
#define LBM_DEEP_UNITS 2  // units per colliding warp and tile of the deep ring (2-byte storage)
#endif
constexpr int smem_units(int storage, int variant) {
    return (variant == 0 || variant == 2 ? 4 : (variant == 3 ? LBM_DEEP_UNITS : 2)) /
           (storage == 1 ? 2 : 1);
}
constexpr int smem_tile_nodes(int storage, int variant) {
    return 64 * smem_units(storage, variant) * (smem_threads(variant) / 32);
}
// Tile width X of an nx x ny instance: 64, 128 or 256 nodes (at most nx
// unless 64), at most 32 tile_nodes / threads so that each warp's units
// (tile_nodes / (2 threads) units of 64 nodes) cover whole tile rows.  Of
// those, the widest (fewest halo columns and tile copies per node: what
// the bandwidth-bound rules want), or with least_padding the one whose
// tiles (X by tile_nodes / X rows) cover the instance with the fewest
// padding nodes (what arithmetic-bound rules want: a padding lane collides
// for nothing); ties go to the wider tile.
inline int smem_tile_width(int64_t nx, int64_t ny, int tile_nodes, int threads,
                           bool least_padding) {
    int best = 64;
    int64_t best_cells = -1;
    for (int w = 256; w >= 64; w /= 2) {
        if ((int64_t)w * threads > 32LL * tile_nodes) continue;
        if (w > 64 && nx < w) continue;
        if (!least_padding) return w;
        const int64_t R = tile_nodes / w;
        const int64_t cells = ((nx + w - 1) / w) * w * (((ny + R - 1) / R) * R);
        if (best_cells < 0 || cells < best_cells) {
            best_cells = cells;
            best = w;
        }
    }
    return best;
}
// The MinxEnt rules are arithmetic-bound on the TMA kernel, the others
// bandwidth-bound.
constexpr bool smem_least_padding(int collision) {
    return collision == COLL_MINXENT4 || collision == COLL_MINXENT2;
}

}  // namespace lbm
