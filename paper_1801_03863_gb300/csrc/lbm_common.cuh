// lbm_common.cuh -- lattice tables, storage types and launch descriptors
// shared by the CUDA kernels and the host side of liblbm.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

// ---------------------------------------------------------------------------
// Lattices.  D2Q9 velocities of Table I, ordered like the columns of the
// moment matrix T (Eq. Tmatrix): rest, +x, +y, -x, -y, (+x,+y), (-x,+y),
// (-x,-y), (+x,-y).  In this order rows 4 and 6 of T are v_x and v_y.
// D1Q3: rest, +x, -x with weights 2/3, 1/6, 1/6 (c_s^2 = 1/3).
// ---------------------------------------------------------------------------
struct D2Q9 {
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int vx(int a) {
        return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int vy(int a) {
        return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr int opp(int a) {
        return a == 0 ? 0 : (a < 5 ? ((a + 1) % 4) + 1 : ((a - 3) % 4) + 5);
    }
    // weights: rest 4/9, axis 1/9, diagonal 1/36
    __host__ __device__ static constexpr double w(int a) {
        return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

struct D1Q3 {
    static constexpr int Q = 3;
    __host__ __device__ static constexpr int vx(int a) { return a == 1 ? 1 : (a == 2 ? -1 : 0); }
    __host__ __device__ static constexpr int vy(int) { return 0; }
    __host__ __device__ static constexpr int opp(int a) { return a == 0 ? 0 : 3 - a; }
    __host__ __device__ static constexpr double w(int a) { return a == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
};

static_assert(D2Q9::opp(1) == 3 && D2Q9::opp(2) == 4 && D2Q9::opp(3) == 1 && D2Q9::opp(4) == 2,
              "axis opposites");
static_assert(D2Q9::opp(5) == 7 && D2Q9::opp(6) == 8 && D2Q9::opp(7) == 5 && D2Q9::opp(8) == 6,
              "diagonal opposites");

// Boundary and collision codes (values of the public enums).  TRT runs on
// the MRT kernel with its own rates, so the kernels know four rules.
enum : int { BC_PERIODIC = 0, BC_ZERO_GRADIENT = 1, BC_CAVITY = 2 };
enum : int { COLL_MINXENT4 = 0, COLL_SRT = 1, COLL_MINXENT2 = 2, COLL_MRT = 3, COLL_TRT = 4 };
enum : int { TAU2_PRINTED = 0, TAU2_MAGIC = 1 };
enum : int { DT_F64 = 0, DT_F32 = 1, DT_F16 = 2, DT_BF16 = 3 };

// Status bits of one node.
enum : uint32_t { ST_NEWTON_SKIPPED = 1u, ST_UNSTABLE = 2u };

// ---------------------------------------------------------------------------
// Storage conversions (round to nearest even on the way down).
// ---------------------------------------------------------------------------
template <typename S> struct Store;
template <> struct Store<double> {
    __device__ static double to_f64(double v) { return v; }
    __device__ static float to_f32(double v) { return (float)v; }
    __device__ static double from(double v) { return v; }
    __device__ static double from(float v) { return (double)v; }
};
template <> struct Store<float> {
    __device__ static double to_f64(float v) { return (double)v; }
    __device__ static float to_f32(float v) { return v; }
    __device__ static float from(double v) { return (float)v; }
    __device__ static float from(float v) { return v; }
};
template <> struct Store<__half> {
    __device__ static double to_f64(__half v) { return (double)__half2float(v); }
    __device__ static float to_f32(__half v) { return __half2float(v); }
    __device__ static __half from(double v) { return __double2half(v); }
    __device__ static __half from(float v) { return __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    __device__ static double to_f64(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
    __device__ static float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __nv_bfloat16 from(double v) { return __double2bfloat16(v); }
    __device__ static __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------------------
// Launch descriptors (plain data, copied to the device once at create).
// ---------------------------------------------------------------------------
// 16-byte aligned and sized: the TMA step kernel copies it into shared
// memory with one bulk copy per tile.
struct alignas(16) InstDesc {
    int64_t off;        // element offset of plane 0 of this instance
    int64_t plane;      // elements per population plane (pitch * ny)
    int64_t node0;      // index of this instance's first node in concatenated host arrays
    int32_t nx, ny, pitch, bc;
    double omega;       // 1 / tau: rate of the stress moments (M8, M9)
    double omega2;      // 1 / tau2: rate of the heat-flux moments (M5, M7; MinxEnt2, MRT, TRT)
    double s_e, s_eps;  // rates of the energy moments M2, M3 (MRT, TRT)
    double u_lid;       // lid speed (cavity only)
    double lid_dev[9];  // f^eq_a(rho0, (u_lid, 0)) - W_a rho0, FP64
    float lid_dev_f[9]; // the same rounded to FP32
    float rates_f[4];   // omega, omega2, s_e, s_eps rounded to FP32
    int32_t tile0, ntiles;  // this instance's tiles in the tile table
};
static_assert(sizeof(InstDesc) % 16 == 0, "bulk copies move multiples of 16 bytes");

struct TileDesc {
    int32_t inst;  // instance index
    int32_t cx0;   // first thread chunk (units of V nodes) in x
    int32_t y0;    // first row
    int32_t pad;
};

// Opaque 128-byte TMA tensor map as the kernels see it (the host fills it
// with cuTensorMapEncodeTiled).
struct alignas(128) CUtensorMapOpaque {
    uint64_t q[16];
};

struct StepArgs {
    const void* src;  // populations f^post(t-1) (deviations)
    void* dst;        // populations f^post(t)
    const InstDesc* inst;
    const TileDesc* tiles;
    int32_t ntiles;
    int32_t tw;       // tile width in chunks (power of two)
    int32_t tw_log2;
    int32_t th;       // tile height in rows
    double rho0;
    unsigned long long* status;  // [count][2]: newton skipped, unstable
    const void* tmaps;           // TMA kernel only, per instance: tensor maps of src with
    const void* tmaps_halo;      // the tile box and with the halo box,
    const void* tmaps_dst;       // and of dst with the tile box (the stores)
    unsigned int* error;         // device error word (bounded waits that ran out)
    int32_t spin_limit;          // polls of one bounded mbarrier wait (TMA kernel)
    int32_t lost_tile;           // test hook: tile whose copies are never issued (-1: none)
};

__host__ __device__ inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Programmatic dependent launch between consecutive step kernels: a step
// kernel may be scheduled while the previous one drains; it runs its
// prologue, then waits here until the previous kernel in the stream has
// completed and its writes are visible, before it touches the population
// buffers, counters or error word.  Without a programmatic launch both are
// no-ops.
__device__ __forceinline__ void wait_previous_grid() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void allow_next_grid() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace lbm
