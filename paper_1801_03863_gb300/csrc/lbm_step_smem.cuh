// lbm_step_smem.cuh -- the D2Q9 step with TMA staging of tiles in and out
// (FP32 collide arithmetic, FP32 / FP16 / BF16 storage).
//
// Same time step as step_kernel (pull-stream + collide + boundary rules of
// Sec. IV.F, Eq. 2), organised around the Tensor Memory Accelerator:
//
//  * A CTA walks the tile table of the context; a tile is X nodes (64, 128
//    or 256, chosen per instance) by R = TILE_NODES / X rows.  Four
//    geometries are compiled (smem_tile_nodes): 8-warp CTAs with large or
//    small tiles on two- or three-stage rings, 10-warp CTAs, and one
//    16-warp CTA per SM on a five-stage ring (four for FP32 storage); the autotuner picks per
//    context.
//  * Each instance's populations are described to TMA as a 3-D tensor
//    (x < nx, row, plane).  Every copy starts at an x that is a multiple of
//    16 bytes (tiles start at multiples of 64 nodes, halo chunks 16 bytes
//    beside them), as tensor copies require.  For every plane
//    one elected thread issues a tensor copy of the tile's rows shifted by
//    -v_y into a dense R x X block of the stage, and for the six planes with
//    v_x != 0 one more copy of the 16-byte chunk beside the tile on the side
//    the pull comes from (the halo column).  Copies outside the lattice are
//    zero-filled by the hardware, which is exactly the cavity's "outside"
//    value (deviation 0).
//  * A ring of STAGES shared-memory stages, each with a "full" mbarrier (the
//    copies landed) and an "empty" one (every colliding warp is done with
//    it).  One warp of the CTA only moves data: it fills every stage at the
//    start, and whenever the colliding warps are done with a tile it writes
//    the stage's nine planes out with one tensor store each (rows and chunks
//    beyond the lattice are clipped by the hardware), waits for TMA to have
//    read them and refills the stage with the tile NS later.  Issuing those
//    26 copies takes a few thousand cycles per tile; a colliding warp that
//    did it (as the last one to finish a tile) fell behind every time and
//    held the whole CTA back.
//  * Each colliding warp owns whole rows of the tile and takes them in units
//    of 32 node pairs (one pair per lane, packed FP32x2 arithmetic), left to
//    right.  A unit writes its post-collision pairs back over its own
//    positions in the stage once every lane has read them; the one value a
//    later unit still needs from an overwritten position (the pair left of
//    the next unit's first node) is parked beforehand in the unused words of
//    the halo chunk.
//  * Every mbarrier wait is bounded; on timeout the kernel records an error
//    word and each warp leaves after a bounded wait for the CTA's copies
//    still in flight.
//  * Nodes whose pull crosses a periodic or zero-gradient edge, which a zero
//    fill cannot express, read their neighbours from global memory with the
//    boundary rule.
#pragma once
#include <cstddef>

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

// TILE nodes per tile, NST stages, NTHREADS colliding threads (the copy
// warp comes on top)
template <typename S, int TILE, int NST, int NTHREADS>
struct SmemTile {
    static constexpr int E = 16 / (int)sizeof(S);  // elements per 16-byte chunk
    static constexpr int TILE_NODES = TILE;        // X * R
    static constexpr int STAGES = NST;             // depth of the shared-memory ring
    static constexpr int THREADS = NTHREADS;
    static constexpr int WARPS = THREADS / 32;
    // units (32 node pairs = 64 nodes of one row) per warp; a warp's units
    // cover whole rows for X <= 64 * UNITS (smem_tile_width keeps to that)
    static constexpr int UNITS = TILE_NODES / (2 * THREADS);
    static constexpr int MAX_ROWS = TILE_NODES / 64;  // R at X = 64
    // one plane: the dense R x X tile, then its halo column (one 16-byte
    // chunk per row, room for MAX_ROWS rows)
    static constexpr int HALO_ELEMS =
        (MAX_ROWS * E + 128 / (int)sizeof(S) - 1) / (128 / (int)sizeof(S)) * (128 / (int)sizeof(S));
    static constexpr int PLANE_ELEMS = TILE_NODES + HALO_ELEMS;
    static constexpr int PLANE_BYTES = PLANE_ELEMS * (int)sizeof(S);
    static constexpr int HALO_OFF = TILE_NODES * (int)sizeof(S);  // bytes into a plane
    static constexpr int STAGE_ELEMS = 9 * PLANE_ELEMS;
    static constexpr size_t STAGES_BYTES = (size_t)STAGES * STAGE_ELEMS * sizeof(S);
    // + room to round the dynamic base up to 128 bytes, per-stage tile
    // parameters and two mbarriers per stage
    static constexpr size_t PARAMS_OFF = STAGES_BYTES;
    static constexpr size_t PARAMS_BYTES = 256;  // per stage
    static constexpr size_t BARS_OFF = PARAMS_OFF + PARAMS_BYTES * STAGES;
    // two mbarriers per stage, then the count of tiles whose copies were
    // issued
    static constexpr size_t COUNT_OFF = BARS_OFF + 16 * STAGES;
    static constexpr size_t SMEM_BYTES = 128 + COUNT_OFF + 16;
    static_assert(UNITS >= 1 && UNITS <= 4, "a unit's halo chunk parks at most 3 values");
    static_assert(TILE_NODES % (2 * THREADS) == 0, "whole units per warp");
    static_assert(HALO_OFF % 128 == 0 && PLANE_BYTES % 128 == 0,
                  "tile blocks and halo columns must stay 128-byte aligned");
};

// Parameters of the tile held by one stage: its instance's descriptor,
// copied in by TMA on the stage's full barrier, and the tile's place,
// written by the producing thread before it arms the barrier (consumers
// read both after the wait; the tensor stores read the place).
struct StageParams {
    InstDesc in;
    TileDesc next;  // descriptor of the tile this stage takes next (NS tiles later)
    int32_t inst, X, x0, y0;
};
static_assert(offsetof(StageParams, next) % 16 == 0 && sizeof(TileDesc) == 16,
              "the next-tile descriptor is a 16-byte bulk copy");
static_assert(sizeof(StageParams) <= 256, "stage parameters must fit 256 bytes");
static_assert(offsetof(StageParams, in) == 0, "the descriptor copy starts the slot");

// Bounded spin limit of one mbarrier wait (each try_wait may itself suspend
// for a while): StepArgs::spin_limit polls, 2^20 unless the context was
// created with a smaller LBM_SPIN_LIMIT (tests of the timeout path); a copy
// that has not landed by then is treated as lost.

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
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int limit) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const void* tmap, const void* src, int c0, int c1,
                                             int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group"
        " [%0, {%1, %2, %3}], [%4];\n" ::"l"(tmap),
        "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
        : "memory");
}
__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// the shared-memory sources of every committed store have been read
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
// every committed store has been performed
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

// Shared-memory byte offsets of one unit, relative to the stage's plane 0:
//   own  the lane's pair (elements 2p, 2p+1 of its tile row);
//   lft  the word whose last element is the one left of the pair (2p - 1):
//        the lane to the left's pair, or for lane 0 a word of the row's halo
//        chunk (the left halo, or the value parked by the previous unit);
//   rgt  the word whose first element is the one right of the pair
//        (2p + 2): the next lane's pair, or for the row's last lane word 0
//        of the right halo chunk.
struct UnitOffs {
    uint32_t own, lft, rgt;
};

// One unit's place: offsets, its row's halo chunk, index within the row,
// first node (x, y), and whether all its 64 nodes are interior nodes.
struct UnitGeom {
    UnitOffs uo;
    uint32_t hrow;
    int sg, x, y;
    bool interior;
};

// Pair of nodes (2p, 2p+1) of plane `pl` pulled with shift -VX in x, as
// FP32x2.
template <typename S, int VX>
__device__ __forceinline__ float2 smem_pair(const unsigned char* pl, const UnitOffs& u,
                                            uint32_t* own_word = nullptr) {
    if constexpr (sizeof(S) == 2) {
        using S2 = typename std::conditional<std::is_same<S, __half>::value, __half2,
                                             __nv_bfloat162>::type;
        const uint32_t w0 = *reinterpret_cast<const uint32_t*>(pl + u.own);
        if (own_word) *own_word = w0;
        // each half converted straight from the word that holds it (the
        // conversion picks either half of a register; no byte permute)
        auto lo = [](uint32_t w) { return __low2float(*reinterpret_cast<const S2*>(&w)); };
        auto hi = [](uint32_t w) { return __high2float(*reinterpret_cast<const S2*>(&w)); };
        if constexpr (VX == 0) return make_float2(lo(w0), hi(w0));
        else if constexpr (VX == 1)
            return make_float2(hi(*reinterpret_cast<const uint32_t*>(pl + u.lft)), lo(w0));
        else
            return make_float2(hi(w0), lo(*reinterpret_cast<const uint32_t*>(pl + u.rgt)));
    } else {
        if constexpr (VX == 0) return *reinterpret_cast<const float2*>(pl + u.own);
        else if constexpr (VX == 1)
            return make_float2(*reinterpret_cast<const float*>(pl + u.lft),
                               *reinterpret_cast<const float*>(pl + u.own));
        else
            return make_float2(*reinterpret_cast<const float*>(pl + u.own + 4),
                               *reinterpret_cast<const float*>(pl + u.rgt));
    }
}

// The nine pulled values of one node pair, and the words to park (see
// below): for 2-byte storage the pair's own words of planes 1, 5, 8, which
// the pulls from x - 1 read anyway.
template <typename S, int PB>
__device__ __forceinline__ void load_unit(const unsigned char* st, const UnitOffs& u, F2 (&d)[9],
                                          uint32_t (&pw)[3]) {
    d[0] = F2(smem_pair<S, 0>(st + 0 * PB, u));
    d[1] = F2(smem_pair<S, 1>(st + 1 * PB, u, &pw[0]));
    d[2] = F2(smem_pair<S, 0>(st + 2 * PB, u));
    d[3] = F2(smem_pair<S, -1>(st + 3 * PB, u));
    d[4] = F2(smem_pair<S, 0>(st + 4 * PB, u));
    d[5] = F2(smem_pair<S, 1>(st + 5 * PB, u, &pw[1]));
    d[6] = F2(smem_pair<S, -1>(st + 6 * PB, u));
    d[7] = F2(smem_pair<S, -1>(st + 7 * PB, u));
    d[8] = F2(smem_pair<S, 1>(st + 8 * PB, u, &pw[2]));
    if constexpr (sizeof(S) != 2) {
        // 4-byte storage: the pair's second element is a word of its own
        pw[0] = *reinterpret_cast<const uint32_t*>(st + 1 * PB + u.own + 4u);
        pw[1] = *reinterpret_cast<const uint32_t*>(st + 5 * PB + u.own + 4u);
        pw[2] = *reinterpret_cast<const uint32_t*>(st + 8 * PB + u.own + 4u);
    }
}
template <typename S, int PB>
__device__ __forceinline__ void load_unit(const unsigned char* st, const UnitOffs& u, F2 (&d)[9]) {
    uint32_t pw[3];
    load_unit<S, PB>(st, u, d, pw);
}

// Post-collision pair into the stage, over the lane's own position.
template <typename S>
__device__ __forceinline__ void smem_store_pair(unsigned char* p, float a, float b) {
    if constexpr (std::is_same<S, __half>::value) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
    } else if constexpr (std::is_same<S, __nv_bfloat16>::value) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
    } else {
        *reinterpret_cast<float2*>(p) = make_float2(a, b);
    }
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

#ifndef LBM_UNIT_UNROLL
#define LBM_UNIT_UNROLL 1  // 0: a warp takes its units of a tile in a rolled loop
#endif
#ifndef LBM_SMEM_MINBLOCKS
#define LBM_SMEM_MINBLOCKS 2  // resident CTAs per SM the register budget aims at
#endif

// Every thread collides node pairs (P = 2 nodes per unit) in packed FP32x2
// arithmetic.  All step kernels run the same packed collision code, so their
// results agree bit for bit: the compiler may fuse a packed product into a
// following packed add, and it does so alike wherever the collision is
// inlined, which scalar code would not reproduce.
template <typename S, int COLL, int TILE, int NST, int NTHREADS>
__global__ void __launch_bounds__(NTHREADS + 32, NTHREADS + 32 >= 512 ? 1 : LBM_SMEM_MINBLOCKS)
    step_kernel_smem(const StepArgs args) {
    using TS = SmemTile<S, TILE, NST, NTHREADS>;
    constexpr int E = TS::E;
    constexpr int Q = 9;
    constexpr int NS = TS::STAGES;
    constexpr int P = 2;
    constexpr int PB = TS::PLANE_BYTES;
    constexpr int ES = (int)sizeof(S);
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
    const CUtensorMapOpaque* tmaps = static_cast<const CUtensorMapOpaque*>(args.tmaps);
    const CUtensorMapOpaque* hmaps = static_cast<const CUtensorMapOpaque*>(args.tmaps_halo);
    const CUtensorMapOpaque* omaps = static_cast<const CUtensorMapOpaque*>(args.tmaps_dst);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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

    // tiles whose copies the copy warp has issued (read on the failure path)
    volatile int* filled = reinterpret_cast<volatile int*>(smem_al + TS::COUNT_OFF);
    if (tid == 0) *filled = 0;

    // Local tile j out of its stage (every warp is done with it): one
    // tensor store per plane, then a commit.
    auto store_tile = [&](int j) {
        const StageParams& p = params[j % NS];
        const S* sbase = stage_base + (size_t)(j % NS) * TS::STAGE_ELEMS;
        const void* map = &omaps[p.inst];
#pragma unroll
        for (int a = 0; a < Q; ++a) tma_store_3d(map, sbase + a * TS::PLANE_ELEMS, p.x0, p.y0, a);
        bulk_commit();
    };

    // Fill stage j % NS with local tile j (descriptor `tile`): store the
    // tile's place, then issue the instance-descriptor, plane and halo
    // copies, and the copy of the descriptor of tile j + NS (which this
    // stage takes next), all on the stage's full barrier.
    auto fill = [&](int j, const TileDesc tile) {
        const int st = j % NS;
        *filled = j + 1;
        // test hook of the timeout path: the copies of one chosen tile are
        // never issued, so its full barrier never completes
        if ((int)blockIdx.x + j * G == args.lost_tile) return;
        StageParams& p = params[st];
        const int X = tile.pad, R = TS::TILE_NODES / X;
        p.inst = tile.inst; p.X = X; p.x0 = tile.cx0; p.y0 = tile.y0;
        const bool more = j + NS < ntl;
        const uint32_t bytes = (uint32_t)((Q * R * X + 6 * R * E) * sizeof(S) + sizeof(InstDesc) +
                                          (more ? sizeof(TileDesc) : 0));
        S* sbase = stage_base + (size_t)st * TS::STAGE_ELEMS;
        const void* map = &tmaps[tile.inst];
        const void* hmap = &hmaps[tile.inst];
        fence_proxy_async_smem();  // consumers' accesses to this stage come first
        mbar_arrive_expect_tx(&full[st], bytes);
        bulk_load(&p.in, &args.inst[tile.inst], (uint32_t)sizeof(InstDesc), &full[st]);
        if (more)
            bulk_load(&p.next, &args.tiles[blockIdx.x + (j + NS) * G], (uint32_t)sizeof(TileDesc),
                      &full[st]);
#pragma unroll
        for (int a = 0; a < Q; ++a)
            tma_load_3d(sbase + a * TS::PLANE_ELEMS, map, tile.cx0, tile.y0 - D2Q9::vy(a), a,
                        &full[st]);
        // halo columns: the chunk left of the tile for the planes pulled
        // from x - 1, the chunk right of it for those pulled from x + 1
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            if (D2Q9::vx(a) == 0) continue;
            const int hx = D2Q9::vx(a) == 1 ? tile.cx0 - E : tile.cx0 + X;
            tma_load_3d(sbase + a * TS::PLANE_ELEMS + TS::TILE_NODES, hmap, hx,
                        tile.y0 - D2Q9::vy(a), a, &full[st]);
        }
    };

    // The tile table and tensor maps are constant; the populations, counters
    // and error word are read and written only after this.
    wait_previous_grid();
    allow_next_grid();
    __syncthreads();  // counters initialised
    if (warp == TS::WARPS) {
        // The copy warp (its lane 0): fill every stage with the CTA's first
        // tiles; then, once every colliding warp is done with tile j, write
        // it out and refill its stage with tile j + NS.
        if (lane == 0) {
            for (int t = 0; t < min(NS, ntl); ++t) fill(t, args.tiles[blockIdx.x + t * G]);
            int jp = 0;
            bool pfail = false;
            for (; jp < ntl; ++jp) {
                const int st = jp % NS;
                if (!mbar_wait_bounded(&empty[st], (uint32_t)((jp / NS) & 1), args.spin_limit)) {
                    pfail = true;
                    break;
                }
                store_tile(jp);
                if (jp + NS < ntl) {
                    const TileDesc nt = params[st].next;
                    bulk_wait_read();  // the stores have read the stage
                    fill(jp + NS, nt);
                }
            }
            if (pfail) {
                // the colliding warps gave up on a tile: report it, and give
                // the copies still in flight a bounded chance to land
                atomicOr(args.error, 1u);
                const int nf = *filled;
                for (int t = jp; t < nf; ++t)
                    mbar_wait_bounded(&full[t % NS], (uint32_t)((t / NS) & 1), args.spin_limit);
            }
            bulk_wait_all();  // no shared-memory reads left behind
        }
        return;
    }

    // Each colliding warp collides its units of a tile, then its lane 0
    // arrives on the stage's empty barrier; the copy warp takes the tile
    // from there.
    bool fail = false;
    int j = 0;
    for (; j < ntl && !fail; ++j) {
        const int st = j % NS;
        // the warp leaves together if the copies did not land in time
        const bool landed = mbar_wait_bounded(&full[st], (uint32_t)((j / NS) & 1), args.spin_limit);
        if (!__all_sync(0xffffffffu, landed)) {
            fail = true;
            break;
        }

        // what every unit needs; the boundary data (bc, strides, lid) is read
        // by the edge units only
        const StageParams& p = params[st];
        const int x0 = p.x0, y0 = p.y0, nx = p.in.nx, ny = p.in.ny;
        unsigned char* sb = reinterpret_cast<unsigned char*>(stage_base + (size_t)st * TS::STAGE_ELEMS);
        const int lgX = 31 - __clz(p.X);   // log2 of the tile width X
        const int sl2 = lgX - 6;           // log2 of the units per tile row (X / 64)
        const int smask = (1 << sl2) - 1;  // last unit of a row
        const Rates<CT> rates{CT(p.in.rates_f[0]), CT(p.in.rates_f[1]), CT(p.in.rates_f[2]),
                              CT(p.in.rates_f[3])};
        uint32_t n_skip = 0, n_unst = 0;
        const int inst = p.inst;
        // geometry of unit k of this warp
        auto geom = [&](int k) {
            UnitGeom g;
            const int u = warp * TS::UNITS + k;
            const int r = u >> sl2;       // tile row
            g.sg = u & smask;             // unit within the row
            const int px = (g.sg << 5) + lane;  // pair within the row
            g.x = x0 + P * px;
            g.y = y0 + r;
            g.hrow = (uint32_t)(TS::HALO_OFF + (r << 4));  // this row's halo chunk
            g.uo.own = (uint32_t)(((r << lgX) + P * px) * ES);
            g.uo.lft = (lane == 0) ? g.hrow + 4u * (uint32_t)(3 - g.sg) : g.uo.own - 4u;
            g.uo.rgt = (lane == 31 && g.sg == smask) ? g.hrow : g.uo.own + (uint32_t)(P * ES);
            // all 64 nodes of the unit are interior nodes of the lattice (the
            // same for every lane): no boundary rule, no padding lane
            const int xs = x0 + (g.sg << 6);
            g.interior = (g.y >= 1) & (g.y <= ny - 2) & (xs >= 1) & (xs + 63 <= nx - 2);
            return g;
        };
        // A second copy of the unit without the edge logic pays for the
        // arithmetic-heavy MinxEnt rules only (measured: +2 % MinxEnt4, -2 % SRT).
        constexpr bool FAST = COLL == COLL_MINXENT4 || COLL == COLL_MINXENT2;
            auto unit = [&](auto interior_tag, const UnitGeom& g) {
                const UnitOffs& uo = g.uo;
                const uint32_t hrow = g.hrow;
                const int sg = g.sg, x = g.x, y = g.y;
                constexpr bool INTERIOR = decltype(interior_tag)::value;
                CT d[Q];
                uint32_t pw[3];
                load_unit<S, PB>(sb, uo, d, pw);
                // The next unit of the row pulls element x - 1 of its first
                // pair from this unit's last pair, which this unit overwrites:
                // park the word holding it (planes 1, 5, 8) in the row's halo
                // chunk, word 3 - (sg + 1) (word 3 holds the left halo itself).
                {
                    if (lane == 31 && sg < smask) {
                        const uint32_t to = hrow + 4u * (uint32_t)(2 - sg);
                        *reinterpret_cast<uint32_t*>(sb + 1 * PB + to) = pw[0];
                        *reinterpret_cast<uint32_t*>(sb + 5 * PB + to) = pw[1];
                        *reinterpret_cast<uint32_t*>(sb + 8 * PB + to) = pw[2];
                    }
                }
                CT o[Q];
                uint32_t sts;
                if constexpr (INTERIOR) {
                    sts = Collide<D2Q9, COLL, CT, ES>::run(d, rho0v, rates, o);
                    if (__builtin_expect(sts != 0u, 0)) {  // rare: a lane skipped its Newton step or is unstable
                        n_skip += __popc(sts & (ST_NEWTON_SKIPPED * 5u));
                        n_unst += __popc(sts & (ST_UNSTABLE * 5u));
                    }
                } else {
                    // Lanes beyond the lattice (x >= nx or y >= ny) collide the
                    // zero-filled or wrapped values they read: their stores are
                    // clipped by TMA and their status is not counted.  So is
                    // the second node of a pair that ends at an odd width.
                    const bool active = (y < ny) && (x < nx);
                    const bool second = x + 1 < nx;
                    // node (pair) on the lattice's outer ring: boundary rules apply
                    const bool edge = (y == 0) | (y == ny - 1) | (x == 0) | (x + P - 1 >= nx - 1);
                    const int bc = p.in.bc;
                    if (edge && bc != BC_CAVITY) {
                        const int64_t pitch = p.in.pitch, plane = p.in.plane;
                        const S* gb = src + p.in.off;
#pragma unroll
                        for (int a = 0; a < Q; ++a) {
                            const float2 g = global_pair<S>(gb + a * plane, pitch, nx, ny, bc, x,
                                                            y, D2Q9::vx(a), D2Q9::vy(a));
                            d[a] = F2(g);
                        }
                    }
                    sts = Collide<D2Q9, COLL, CT, ES>::run(d, rho0v, rates, o);
                    if (edge && bc == BC_CAVITY) {
#pragma unroll
                        for (int l = 0; l < P; ++l) {
                            const int xl = x + l;
                            const bool wall = (xl == 0) || (xl == nx - 1) || (y == 0);
                            const bool lidn = !wall && (y == ny - 1);
                            if (wall) {
                                // full-way bounce-back of the pulled populations,
                                // re-read from the stage (no lane has written
                                // this unit's positions yet) so they need not
                                // stay live through the collision
                                CT v[Q];
                                load_unit<S, PB>(sb, uo, v);
#pragma unroll
                                for (int a = 0; a < Q; ++a)
                                    N::set_lane(o[a], l, N::lane(v[D2Q9::opp(a)], l));
                                sts &= ~(3u << (2 * l));
                            } else if (lidn) {
#pragma unroll
                                for (int a = 0; a < Q; ++a) N::set_lane(o[a], l, p.in.lid_dev_f[a]);
                                sts &= ~(3u << (2 * l));
                            }
                        }
                    }
                    if (sts && active) {  // rare: some lane skipped its Newton step or is unstable
                        if (!second) sts &= 3u;
                        n_skip += __popc(sts & (ST_NEWTON_SKIPPED * 5u));
                        n_unst += __popc(sts & (ST_UNSTABLE * 5u));
                    }
                }
                __syncwarp();  // every lane has read this unit's positions
#pragma unroll
                for (int a = 0; a < Q; ++a)
                    smem_store_pair<S>(sb + a * PB + uo.own, o[a].v.x, o[a].v.y);
            };
        auto single = [&](const UnitGeom& g) {
            if constexpr (FAST) {
                if (g.interior) unit(std::true_type{}, g);
                else unit(std::false_type{}, g);
            } else {
                unit(std::false_type{}, g);
            }
        };
        // one unit at a time, the loop unrolled (two units collided together
        // measured slower: registers)
#if LBM_UNIT_UNROLL
#pragma unroll
#else
#pragma unroll 1
#endif
        for (int k = 0; k < TS::UNITS; ++k) single(geom(k));
        if (n_skip | n_unst) {
            atomicAdd(args.status + 2 * inst + 0, (unsigned long long)n_skip);
            atomicAdd(args.status + 2 * inst + 1, (unsigned long long)n_unst);
        }
        // this thread's stage writes come before the tensor stores that read them
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);  // the copy warp takes it from here
    }
    if (fail) {
        // a copy or a stage release never came: report it and give the
        // copies still in flight (tiles j .. filled - 1) a bounded chance to
        // land before this warp leaves
        atomicOr(args.error, 1u);
        if (lane == 0) {
            const int nf = *filled;
            for (int t = j; t < nf; ++t)
                mbar_wait_bounded(&full[t % NS], (uint32_t)((t / NS) & 1), args.spin_limit);
        }
    }
}

// The TMA-staged D2Q9 kernel for a collision rule and tile geometry VARIANT
// (0: large tiles, 1: small tiles, 2: wide CTAs, 3: deep ring, see
// smem_tile_nodes);
// *smem_bytes receives its dynamic shared memory size.
template <typename S, int VARIANT>
const void* pick_step_kernel_smem(int collision, size_t* smem_bytes) {
    constexpr int TN = smem_tile_nodes(sizeof(S) == 4 ? 1 : 2, VARIANT);  // 1: FP32 storage
    constexpr int NS = VARIANT == 1   ? LBM_SMEM_STAGES_SMALL
                     : VARIANT == 3 ? (sizeof(S) == 2 ? LBM_SMEM_STAGES_DEEP2 : LBM_SMEM_STAGES_DEEP)
                                    : LBM_SMEM_STAGES;
    constexpr int NT = smem_threads(VARIANT);
    using TS = SmemTile<S, TN, NS, NT>;
    *smem_bytes = TS::SMEM_BYTES;
    switch (collision) {
        case COLL_MINXENT4: return (const void*)&step_kernel_smem<S, COLL_MINXENT4, TN, NS, NT>;
        case COLL_SRT: return (const void*)&step_kernel_smem<S, COLL_SRT, TN, NS, NT>;
        case COLL_MINXENT2: return (const void*)&step_kernel_smem<S, COLL_MINXENT2, TN, NS, NT>;
        case COLL_MRT:
        case COLL_TRT: return (const void*)&step_kernel_smem<S, COLL_MRT, TN, NS, NT>;
    }
    return nullptr;
}

}  // namespace lbm
