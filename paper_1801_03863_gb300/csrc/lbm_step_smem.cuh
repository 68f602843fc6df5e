// lbm_step_smem.cuh -- the D2Q9 step with TMA staging of halo tiles
// (FP32 collide arithmetic, FP32 / FP16 / BF16 storage).
//
// Same time step as step_kernel (pull-stream + collide + boundary rules of
// Sec. IV.F, Eq. 2), organised around the Tensor Memory Accelerator:
//
//  * A CTA (256 threads) walks the tile table of the context; a tile is X
//    nodes (64, 128 or 256, chosen per instance) by R = TILE_NODES / X rows.
//    Two geometries are compiled: large tiles (2048 nodes for 2-byte storage,
//    1024 for 4-byte) with a two-stage ring, which halve the per-tile costs
//    of arithmetic-bound rules, and small tiles (1024 / 512) with a
//    three-stage ring, which keep more copies in flight for bandwidth-bound
//    ones; the autotuner picks per context.
//  * Each instance's populations are described to TMA as a 4-D tensor
//    (element within a 16-byte chunk, chunk, row, plane).  For every plane
//    one elected thread issues a single tensor copy of the tile's rows
//    shifted by -v_y, one chunk wider on each side in x (the halo); copies
//    outside the lattice are zero-filled by the hardware, which is exactly
//    the cavity's "outside" value (deviation 0).
//  * A ring of STAGES shared-memory stages, each with a "full" mbarrier (the
//    copies landed) and an "empty" one (every warp is done with it): the
//    copies of the next tiles are in flight while one is collided.  Every
//    wait is bounded; on timeout the kernel records an error word and the
//    CTA leaves after a bounded wait for its own copies still in flight.
//  * Nodes whose pull crosses a periodic or zero-gradient edge, which a zero
//    fill cannot express, read their neighbours from global memory with the
//    boundary rule.
//  * Each thread collides one node pair (packed FP32x2 arithmetic) or one
//    node per unit, reading 4-byte words from shared memory (consecutive
//    threads, consecutive words: no bank conflicts) and storing each plane's
//    pair with one 4- or 8-byte store (a warp writes 128 or 256 contiguous
//    bytes).
#pragma once
#include "lbm_aux.h"
#include "lbm_collide.cuh"
#include "lbm_step.cuh"

namespace lbm {

#ifndef LBM_SMEM_STAGES
#define LBM_SMEM_STAGES 2        // ring depth, large tiles
#endif
#ifndef LBM_SMEM_STAGES_SMALL
#define LBM_SMEM_STAGES_SMALL 3  // ring depth, small tiles
#endif

template <typename S, int TILE = (sizeof(S) == 2 ? LBM_SMEM_TILE2 : LBM_SMEM_TILE4),
          int NST = LBM_SMEM_STAGES>
struct SmemTile {
    static constexpr int E = 16 / (int)sizeof(S);  // elements per 16-byte chunk
    static constexpr int TILE_NODES = TILE;        // X * R
    static constexpr int STAGES = NST;             // depth of the shared-memory ring
    static constexpr int THREADS = 256;
    static constexpr int WARPS = THREADS / 32;
    static constexpr int MAX_ROWS = TILE_NODES / 64;  // R at X = 64
    // elements of one plane at the largest smem footprint (X = 64); a
    // multiple of 64 elements, so every plane region is 128-byte aligned
    static constexpr int PLANE_ELEMS = TILE_NODES + 2 * E * MAX_ROWS;
    static constexpr int STAGE_ELEMS = 9 * PLANE_ELEMS;
    static constexpr size_t STAGES_BYTES = (size_t)STAGES * STAGE_ELEMS * sizeof(S);
    // + room to round the dynamic base up to 128 bytes, per-stage tile
    // parameters and two mbarriers per stage
    static constexpr size_t PARAMS_OFF = STAGES_BYTES;
    static constexpr size_t BARS_OFF = PARAMS_OFF + 128 * STAGES;
    static constexpr size_t SMEM_BYTES = 128 + BARS_OFF + 16 * STAGES;
    static_assert((PLANE_ELEMS * sizeof(S)) % 128 == 0, "plane regions must stay 128-byte aligned");
};

// Parameters of the tile held by one stage, written by the producing thread
// before it arms the stage's barrier (consumers read them after the wait).
struct StageParams {
    int64_t off, pitch, plane;
    int32_t inst, X, x0, y0, nx, ny, bc, R, xl2;  // xl2 = log2(X)
    float omega, omega2, s_e, s_eps;
    float lid[9];
};
static_assert(sizeof(StageParams) <= 128, "stage parameters must fit 128 bytes");

// Bounded spin limit of one mbarrier wait (each try_wait may itself suspend
// for a while); a copy that has not landed by then is treated as lost.
constexpr int MBAR_SPIN_LIMIT = 1 << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (int i = 0; i < MBAR_SPIN_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, int c0, int c1, int c2,
                                            int c3, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// Pair of nodes (2p, 2p+1) of one plane as FP32x2.  `row` points at the
// shared-memory row of the plane; `wb` is the index (in 32-bit words for
// 2-byte types, in elements for FP32) of the pair's own position, element
// E + 2p.  The pull shift -v_x is a compile-time offset from it.
template <typename S, int VX>
__device__ __forceinline__ float2 smem_pair(const S* row, int wb) {
    if constexpr (sizeof(S) == 2) {
        const uint32_t* w = reinterpret_cast<const uint32_t*>(row) + wb;
        uint32_t v;
        if constexpr (VX == 0) v = w[0];
        else if constexpr (VX == 1) v = __byte_perm(w[-1], w[0], 0x5432);  // elements 2p-1, 2p
        else v = __byte_perm(w[0], w[1], 0x5432);                           // elements 2p+1, 2p+2
        if constexpr (std::is_same<S, __half>::value) {
            return __half22float2(*reinterpret_cast<const __half2*>(&v));
        } else {
            return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v));
        }
    } else {
        const float* f = reinterpret_cast<const float*>(row) + wb - VX;
        return make_float2(f[0], f[1]);
    }
}

// Store one pair.
template <typename S>
__device__ __forceinline__ void store_pair(S* p, float a, float b) {
    if constexpr (std::is_same<S, __half>::value) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
    } else if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
    } else {
        *reinterpret_cast<float2*>(p) = make_float2(a, b);
    }
}

// The nine pulled values of one node pair from the stage rows of the
// current tile row.
template <typename S>
__device__ __forceinline__ void load_unit(const S* srow, int wb, int plane_elems, F2 (&d)[9]) {
    d[0] = F2(smem_pair<S, 0>(srow + 0 * plane_elems, wb));
    d[1] = F2(smem_pair<S, 1>(srow + 1 * plane_elems, wb));
    d[2] = F2(smem_pair<S, 0>(srow + 2 * plane_elems, wb));
    d[3] = F2(smem_pair<S, -1>(srow + 3 * plane_elems, wb));
    d[4] = F2(smem_pair<S, 0>(srow + 4 * plane_elems, wb));
    d[5] = F2(smem_pair<S, 1>(srow + 5 * plane_elems, wb));
    d[6] = F2(smem_pair<S, -1>(srow + 6 * plane_elems, wb));
    d[7] = F2(smem_pair<S, -1>(srow + 7 * plane_elems, wb));
    d[8] = F2(smem_pair<S, 1>(srow + 8 * plane_elems, wb));
}

__device__ __forceinline__ int wrap_index(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// Pair of nodes (x, x+1) of row y pulled straight from global memory with
// the periodic (wrap) or zero-gradient (x clamp, y wrap) rule: used by the
// nodes of periodic / zero-gradient lattices whose pull crosses an edge,
// where the zero-filled tile halo does not hold the boundary value.
template <typename S>
__device__ __forceinline__ float2 global_pair(const S* base, int64_t pitch, int nx, int ny, int bc,
                                              int x, int y, int vx, int vy) {
    const int sy = wrap_index(y - vy, ny);
    int xa = x - vx, xb = x + 1 - vx;
    if (bc == BC_PERIODIC) {
        xa = wrap_index(xa, nx);
        xb = wrap_index(xb, nx);
    } else {
        xa = min(max(xa, 0), nx - 1);
        xb = min(max(xb, 0), nx - 1);
    }
    const S* row = base + (int64_t)sy * pitch;
    return make_float2(to_compute<float, S>(row[xa]), to_compute<float, S>(row[xb]));
}

#ifndef LBM_SMEM_MINBLOCKS
#define LBM_SMEM_MINBLOCKS 2  // resident CTAs per SM the register budget aims at
#endif

// Every thread collides node pairs (P = 2 nodes per unit) in packed FP32x2
// arithmetic.  All step kernels run the same packed collision code, so their
// results agree bit for bit: the compiler may fuse a packed product into a
// following packed add, and it does so alike wherever the collision is
// inlined, which scalar code would not reproduce.
template <typename S, int COLL, int TILE, int NST>
__global__ void __launch_bounds__(256, LBM_SMEM_MINBLOCKS)
    step_kernel_smem(const StepArgs args) {
    using TS = SmemTile<S, TILE, NST>;
    constexpr int E = TS::E;
    constexpr int Q = 9;
    constexpr int NS = TS::STAGES;
    constexpr int P = 2;
    using CT = F2;
    using N = Num<CT>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations must be 16-byte (here: 128-byte) aligned: round the
    // dynamic base up explicitly.  Layout: stages | stage parameters |
    // full barriers | empty barriers.
    unsigned char* smem_al = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    S* stage_base = reinterpret_cast<S*>(smem_al);
    StageParams* params = reinterpret_cast<StageParams*>(smem_al + TS::PARAMS_OFF);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_al + TS::BARS_OFF);
    uint64_t* empty = full + NS;
    const S* __restrict__ src = static_cast<const S*>(args.src);
    S* __restrict__ dst = static_cast<S*>(args.dst);
    const CUtensorMapOpaque* tmaps = static_cast<const CUtensorMapOpaque*>(args.tmaps);
    const int tid = threadIdx.x, lane = tid & 31;
    const CT rho0v = CT((float)args.rho0);
    const int G = gridDim.x;
    // local tile j of this CTA is global tile blockIdx.x + j * G
    const int ntl = (args.ntiles > (int)blockIdx.x) ? (args.ntiles - 1 - (int)blockIdx.x) / G + 1 : 0;

    if (tid == 0) {
        for (int k = 0; k < NS; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], TS::WARPS);
        }
        mbar_init_fence();
    }
    __syncthreads();

    // Thread 0 fills stage j % NS with local tile j: parameters, then the
    // nine plane copies on the stage's full barrier.  Returns false if the
    // stage was not released in time.
    auto produce = [&](int j) -> bool {
        const int st = j % NS, fill = j / NS;
        if (fill > 0 && !mbar_wait_bounded(&empty[st], (uint32_t)((fill - 1) & 1))) return false;
        const TileDesc tile = args.tiles[blockIdx.x + j * G];
        const InstDesc& in = args.inst[tile.inst];
        StageParams& p = params[st];
        p.off = in.off; p.pitch = in.pitch; p.plane = in.plane;
        p.inst = tile.inst; p.X = tile.pad; p.x0 = tile.cx0; p.y0 = tile.y0;
        p.nx = in.nx; p.ny = in.ny; p.bc = in.bc; p.R = TS::TILE_NODES / tile.pad;
        p.xl2 = 31 - __clz(tile.pad);
        p.omega = (float)in.omega;
        p.omega2 = (float)in.omega2;
        p.s_e = (float)in.s_e;
        p.s_eps = (float)in.s_eps;
#pragma unroll
        for (int a = 0; a < Q; ++a) p.lid[a] = in.lid_dev_f[a];
        const uint32_t bytes = (uint32_t)(Q * p.R * (p.X + 2 * E) * sizeof(S));
        S* sbase = stage_base + (size_t)st * TS::STAGE_ELEMS;
        const void* map = &tmaps[tile.inst];
        fence_proxy_async_smem();  // consumers' reads of this stage come first
        mbar_arrive_expect_tx(&full[st], bytes);
#pragma unroll
        for (int a = 0; a < Q; ++a)
            tma_load_4d(sbase + a * TS::PLANE_ELEMS, map, 0, tile.cx0 / E - 1,
                        tile.y0 - D2Q9::vy(a), a, &full[st]);
        return true;
    };

    bool fail = false;
    int issued = 0;  // local tiles handed to TMA (thread 0's count)
    int jdone = -1;  // last local tile whose copies this thread saw land
    if (tid == 0) {
        for (; issued < min(NS - 1, ntl); ++issued)
            if (!produce(issued)) { fail = true; break; }
    }
    for (int j = 0; j < ntl && !fail; ++j) {
        const int st = j % NS;
        // keep NS - 1 tiles in flight: refill the stage released by tile j - 1
        if (tid == 0 && issued < ntl && issued == j + NS - 1) {
            if (produce(issued)) ++issued;
            else fail = true;
        }
        if (!mbar_wait_bounded(&full[st], (uint32_t)((j / NS) & 1))) fail = true;
        if (fail) break;
        jdone = j;

        const StageParams& p = params[st];
        const int X = p.X;
        const int SP = X + 2 * E;  // smem row length (elements)
        const int x0 = p.x0, y0 = p.y0, nx = p.nx, ny = p.ny, bc = p.bc;
        const int64_t pitch = p.pitch, plane = p.plane, off = p.off;
        S* sbase = stage_base + (size_t)st * TS::STAGE_ELEMS;

        const int cl2 = p.xl2 - 1;  // log2 of the thread columns per row
        const int px = tid & ((1 << cl2) - 1);
        const int rg = tid >> cl2;                  // first row of this thread
        const int rstep = TS::THREADS >> cl2;       // rows between this thread's units
        const int x = x0 + P * px;
        // own position in a shared row: element E + P px (in words for pairs
        // of 2-byte types)
        const int wb = (sizeof(S) == 2) ? (E / 2 + px) : (E + 2 * px);
        const Rates<CT> rates{CT(p.omega), CT(p.omega2), CT(p.s_e), CT(p.s_eps)};
        uint32_t n_skip = 0, n_unst = 0;
        const bool second = x + 1 < nx;
        const bool xedge = (x == 0) || (x + P - 1 >= nx - 1);
        const bool xin = x < nx;
        constexpr int MAXP = TS::TILE_NODES / (P * TS::THREADS);  // units per thread
        float lid[Q];
        if (bc == BC_CAVITY) {
#pragma unroll
            for (int a = 0; a < Q; ++a) lid[a] = p.lid[a];
        }
        const int inst = p.inst;
        // this thread's output position in its first row; advanced by rstep
        // rows per unit
        S* orow = dst + off + (int64_t)(y0 + rg) * pitch + x;
        const int64_t ostep = (int64_t)rstep * pitch;
        // one unit at a time (unrolling raises register pressure and measured slower)
#pragma unroll 1
        for (int k = 0; k < MAXP; ++k) {
            const int r = rg + k * rstep;
            const int y = y0 + r;
            S* op = orow;
            orow += ostep;
            CT d[Q];
            {
                const S* srow = sbase + r * SP;
                load_unit<S>(srow, wb, TS::PLANE_ELEMS, d);
            }
            if (y >= ny || !xin) continue;
            // node (pair) on the lattice's outer ring: boundary rules apply
            const bool edge = (y == 0) | (y == ny - 1) | xedge;
            if (edge && bc != BC_CAVITY) {
                const S* gb = src + off;
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    const float2 g = global_pair<S>(gb + a * plane, pitch, nx, ny, bc, x, y,
                                                    D2Q9::vx(a), D2Q9::vy(a));
                    d[a] = F2(g);
                }
            }
            CT o[Q];
            uint32_t sts = Collide<D2Q9, COLL, CT>::run(d, rho0v, rates, o);
            if (edge && bc == BC_CAVITY) {
#pragma unroll
                for (int l = 0; l < P; ++l) {
                    const int xl2 = x + l;
                    const bool wall = (xl2 == 0) || (xl2 == nx - 1) || (y == 0);
                    const bool lidn = !wall && (y == ny - 1);
                    if (wall) {
                        // full-way bounce-back of the pulled populations, re-read
                        // from the stage so they need not stay live through the
                        // collision (the stage is released after the tile)
                        const S* srow = sbase + r * SP;
                        CT v[Q];
                        load_unit<S>(srow, wb, TS::PLANE_ELEMS, v);
#pragma unroll
                        for (int a = 0; a < Q; ++a) N::set_lane(o[a], l, N::lane(v[D2Q9::opp(a)], l));
                        sts &= ~(3u << (2 * l));
                    } else if (lidn) {
#pragma unroll
                        for (int a = 0; a < Q; ++a) N::set_lane(o[a], l, lid[a]);
                        sts &= ~(3u << (2 * l));
                    }
                }
            }
            if (sts) {  // rare: some lane skipped its Newton step or is unstable
                if (!second) sts &= 3u;
                n_skip += __popc(sts & (ST_NEWTON_SKIPPED * 5u));
                n_unst += __popc(sts & (ST_UNSTABLE * 5u));
            }
            // the second node of a pair beyond the row (odd widths) is row
            // padding: keep it zero
            if (!second) {
#pragma unroll
                for (int a = 0; a < Q; ++a) o[a].v.y = 0.f;
            }
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                store_pair<S>(op, o[a].v.x, o[a].v.y);
                op += plane;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);  // this warp is done with the stage
        if (n_skip | n_unst) {
            atomicAdd(args.status + 2 * inst + 0, (unsigned long long)n_skip);
            atomicAdd(args.status + 2 * inst + 1, (unsigned long long)n_unst);
        }
    }
    if (fail) {
        // a copy or a stage release never came: report it and give this
        // CTA's copies still in flight a bounded chance to land before exit
        atomicOr(args.error, 1u);
        if (tid == 0) {
            for (int j = jdone + 1; j < issued; ++j)
                mbar_wait_bounded(&full[j % NS], (uint32_t)((j / NS) & 1));
        }
    }
}

// The TMA-staged D2Q9 kernel for a collision rule and tile geometry VARIANT
// (0: large tiles, 1: small tiles, see smem_tile_nodes); *smem_bytes
// receives its dynamic shared memory size.
template <typename S, int VARIANT>
const void* pick_step_kernel_smem(int collision, size_t* smem_bytes) {
    constexpr int TN = VARIANT == 0 ? (sizeof(S) == 2 ? LBM_SMEM_TILE2 : LBM_SMEM_TILE4)
                                    : (sizeof(S) == 2 ? LBM_SMEM_TILE2_SMALL : LBM_SMEM_TILE4_SMALL);
    constexpr int NS = VARIANT == 0 ? LBM_SMEM_STAGES : LBM_SMEM_STAGES_SMALL;
    using TS = SmemTile<S, TN, NS>;
    *smem_bytes = TS::SMEM_BYTES;
    switch (collision) {
        case COLL_MINXENT4: return (const void*)&step_kernel_smem<S, COLL_MINXENT4, TN, NS>;
        case COLL_SRT: return (const void*)&step_kernel_smem<S, COLL_SRT, TN, NS>;
        case COLL_MINXENT2: return (const void*)&step_kernel_smem<S, COLL_MINXENT2, TN, NS>;
        case COLL_MRT:
        case COLL_TRT: return (const void*)&step_kernel_smem<S, COLL_MRT, TN, NS>;
    }
    return nullptr;
}

}  // namespace lbm
