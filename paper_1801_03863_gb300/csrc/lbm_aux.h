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
constexpr int CONS_THREADS = 1024;
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
// Tile geometry of those kernels: nodes per tile for a storage type, and
// the tile width for an instance of width nx.
#ifndef LBM_SMEM_TILE2
#define LBM_SMEM_TILE2 2048
#endif
#ifndef LBM_SMEM_TILE4
#define LBM_SMEM_TILE4 1024
#endif
#ifndef LBM_SMEM_TILE2_SMALL
#define LBM_SMEM_TILE2_SMALL 1024
#endif
#ifndef LBM_SMEM_TILE4_SMALL
#define LBM_SMEM_TILE4_SMALL 512
#endif
#ifndef LBM_SMEM_TILE2_WIDE
#define LBM_SMEM_TILE2_WIDE 2560
#endif
#ifndef LBM_SMEM_TILE4_WIDE
#define LBM_SMEM_TILE4_WIDE 1280
#endif
// Geometries of the TMA-staged kernel (variant = launch-shape kind - 1):
//   0  large tiles: 2048 nodes (2-byte storage) / 1024 (FP32), 256 threads,
//      two-stage ring (fewer per-tile costs, for arithmetic-bound rules);
//   1  small tiles: 1024 / 512 nodes, 256 threads, three-stage ring (more
//      copies in flight, for bandwidth-bound rules);
//   2  wide CTAs: 2560 / 1280 nodes, 320 threads (ten warps), two-stage
//      ring: two CTAs give 20 warps per SM instead of 16, at a register
//      budget of 102 per thread;
//   3  deep ring: one CTA per SM of 512 threads (16 warps) with 2048 /
//      1024-node tiles on a four-stage ring, so a stage is refilled three
//      tiles before it is needed.
#ifndef LBM_SMEM_STAGES_DEEP
#define LBM_SMEM_STAGES_DEEP 4
#endif
inline int smem_tile_nodes(int storage, int variant) {
    if (variant == 1) return storage == 1 ? LBM_SMEM_TILE4_SMALL : LBM_SMEM_TILE2_SMALL;
    if (variant == 2) return storage == 1 ? LBM_SMEM_TILE4_WIDE : LBM_SMEM_TILE2_WIDE;
    return storage == 1 ? LBM_SMEM_TILE4 : LBM_SMEM_TILE2;
}
inline int smem_threads(int variant) { return variant == 2 ? 320 : (variant == 3 ? 512 : 256); }
// Tile width: 64, 128 or 256 nodes by the instance width, at most
// 32 tile_nodes / threads, so that each warp's units (tile_nodes /
// (2 threads) units of 64 nodes) cover whole tile rows.
inline int smem_tile_width(int64_t nx, int tile_nodes, int threads) {
    int w = nx >= 256 ? 256 : (nx >= 128 ? 128 : 64);
    while (w > 64 && (int64_t)w * threads > 32LL * tile_nodes) w /= 2;
    return w;
}

}  // namespace lbm
