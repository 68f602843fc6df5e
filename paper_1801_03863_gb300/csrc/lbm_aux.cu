// lbm_aux.cu -- the kernels around the time step: initial equilibrium,
// the first (in-place) collision after a state is loaded, moments and
// population read-out, population load, and the FP64 conservation
// reduction.  One thread per node, grid = (blocks, instance); none of these
// is on the per-step hot path.
#include <algorithm>

#include "lbm_aux.h"
#include "lbm_collide.cuh"

namespace lbm {
namespace {

constexpr int AUX_THREADS = 256;

template <class Lat, typename S>
__device__ __forceinline__ const S* elem_ptr(const S* base, const InstDesc& in, int a, int x, int y) {
    return base + in.off + (int64_t)a * in.plane + (int64_t)y * in.pitch + x;
}

// Deviations of f(x, t_n) at one node, FP64.  pulled = true: the stored field
// is post-collision and the node pulls f_a from x - v_a with the boundary
// rules of the step; pulled = false: the stored field is f(x, t_n) itself.
template <class Lat, typename S>
__device__ void node_state(const S* base, const InstDesc& in, int x, int y, bool pulled,
                           double (&d)[Lat::Q]) {
#pragma unroll
    for (int a = 0; a < Lat::Q; ++a) {
        int sx = x, sy = y;
        bool inside = true;
        if (pulled) {
            sx = x - Lat::vx(a);
            sy = y - Lat::vy(a);
            if (in.bc == BC_CAVITY) {
                inside = sx >= 0 && sx < in.nx && sy >= 0 && sy < in.ny;
            } else {
                if (in.bc == BC_PERIODIC) sx = (sx + in.nx) % in.nx;
                else sx = sx < 0 ? 0 : (sx >= in.nx ? in.nx - 1 : sx);
                sy = (sy + in.ny) % in.ny;
            }
        }
        d[a] = inside ? Store<S>::to_f64(*elem_ptr<Lat, S>(base, in, a, sx, sy)) : 0.0;
    }
}

// f^eq(rho, u) - W rho0 in FP64 (Eq. numerical-plyeqm):
//   W_a (rho - rho0) + W_a rho (3 v.u + 9/2 (v.u)^2 - 3/2 u^2),
// with the even and odd parts in v shared by opposite velocities.
template <class Lat>
__device__ void eq_dev(double rho, double ux, double uy, double rho0, double (&d)[Lat::Q]) {
    const double dr = rho - rho0;
    const double b0 = -1.5 * (ux * ux + uy * uy);
#pragma unroll
    for (int a = 0; a < Lat::Q; ++a) {
        const int o = Lat::opp(a);
        if (o < a) continue;  // filled with its opposite
        const double w = Lat::w(a), wr = w * rho;
        const double vu = Lat::vx(a) * ux + Lat::vy(a) * uy;
        const double even = fma(4.5 * vu, vu, b0);
        const double odd = 3.0 * vu;
        const double base = fma(wr, even, w * dr);
        d[a] = fma(wr, odd, base);
        if (o != a) d[o] = fma(-wr, odd, base);
    }
}

// Node k of instance `in` (row-major, x fastest) as (x, y): 32-bit index
// arithmetic (nx * ny < 2^31 for every instance).
__device__ __forceinline__ void node_xy(uint32_t k, uint32_t nx, int& x, int& y) {
    const uint32_t yy = k / nx;
    y = (int)yy;
    x = (int)(k - yy * nx);
}

// Host arrays are indexed from the first node of the instances the launch
// covers: node0 - node_base (node_base = 0 for whole-context calls, the
// instance's node0 for single-instance calls).
template <class Lat, typename S>
__global__ void init_kernel(S* dst, const InstDesc* insts, const double* rho, const double* ux,
                            const double* uy, double rho0, int64_t node_base) {
    const InstDesc in = insts[blockIdx.y];
    const uint32_t n = (uint32_t)in.nx * (uint32_t)in.ny;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int x, y;
        node_xy(k, (uint32_t)in.nx, x, y);
        const int64_t g = in.node0 - node_base + k;
        double d[Lat::Q];
        eq_dev<Lat>(rho[g], ux ? ux[g] : 0.0, (uy && Lat::Q == 9) ? uy[g] : 0.0, rho0, d);
#pragma unroll
        for (int a = 0; a < Lat::Q; ++a)
            dst[in.off + (int64_t)a * in.plane + (int64_t)y * in.pitch + x] = Store<S>::from(d[a]);
    }
}

template <class Lat, typename S>
__global__ void set_f_kernel(S* dst, const InstDesc* insts, const double* f, double rho0) {
    const InstDesc in = insts[blockIdx.y];
    const uint32_t n = (uint32_t)in.nx * (uint32_t)in.ny;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int x, y;
        node_xy(k, (uint32_t)in.nx, x, y);
#pragma unroll
        for (int a = 0; a < Lat::Q; ++a) {
            const double fa = f[in.node0 * Lat::Q + (int64_t)a * n + k];
            dst[in.off + (int64_t)a * in.plane + (int64_t)y * in.pitch + x] =
                Store<S>::from(fa - Lat::w(a) * rho0);
        }
    }
}

// First step after a state was loaded: collide in place, no streaming
// (the loaded field is f(x, t_n) itself, Eq. 2's collision input).  The
// arithmetic is that of the step kernels -- FP64, or node pairs in packed
// FP32x2 for FP32 -- with the same rates and boundary rules, so this step
// rounds exactly like a step kernel colliding the same pulled values: a
// state saved from a running context and loaded into a new one continues
// bit for bit.  One thread per node pair (x, x + 1) of a row; at an odd
// width the second lane repeats the last node and is discarded.
template <class Lat, typename S, typename T, int COLL>
__global__ void collide_inplace_kernel(const S* src, S* dst, const InstDesc* insts, double rho0,
                                       unsigned long long* status) {
    using CT = typename std::conditional<std::is_same<T, float>::value, F2, T>::type;
    using N = Num<CT>;
    using LT = typename LaneOf<CT>::type;
    constexpr int P = N::LANES;
    const int inst = blockIdx.y;
    const InstDesc& in = insts[inst];
    const uint32_t groups = ((uint32_t)in.nx + P - 1) / P;  // node groups per row
    const uint32_t n = groups * (uint32_t)in.ny;
    const Rates<CT> rates{CT((LT)in.omega), CT((LT)in.omega2), CT((LT)in.s_e), CT((LT)in.s_eps)};
    const CT rho0v = CT((LT)rho0);
    unsigned long long n_skip = 0, n_unst = 0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int g, y;
        node_xy(k, groups, g, y);
        const int x0 = g * P;
        CT d[Lat::Q], o[Lat::Q];
#pragma unroll
        for (int a = 0; a < Lat::Q; ++a) {
#pragma unroll
            for (int l = 0; l < P; ++l) {
                const int x = min(x0 + l, in.nx - 1);
                const S v = *elem_ptr<Lat, S>(src, in, a, x, y);
                if constexpr (std::is_same<T, double>::value) d[a] = Store<S>::to_f64(v);
                else N::set_lane(d[a], l, Store<S>::to_f32(v));
            }
        }
        uint32_t st = Collide<Lat, COLL, CT, (int)sizeof(S)>::run(d, rho0v, rates, o);
        if (in.bc == BC_CAVITY) {
#pragma unroll
            for (int l = 0; l < P; ++l) {
                const int x = x0 + l;
                const bool wall = (x == 0) || (x == in.nx - 1) || (y == 0);
                const bool lid = !wall && (y == in.ny - 1);
                if (wall) {
#pragma unroll
                    for (int a = 0; a < Lat::Q; ++a) N::set_lane(o[a], l, N::lane(d[Lat::opp(a)], l));
                    st &= ~(3u << (2 * l));
                } else if (lid) {
#pragma unroll
                    for (int a = 0; a < Lat::Q; ++a) {
                        if constexpr (std::is_same<T, double>::value) N::set_lane(o[a], l, in.lid_dev[a]);
                        else N::set_lane(o[a], l, in.lid_dev_f[a]);
                    }
                    st &= ~(3u << (2 * l));
                }
            }
        }
#pragma unroll
        for (int l = 0; l < P; ++l) {
            if (x0 + l >= in.nx) continue;
            n_skip += (st >> (2 * l)) & ST_NEWTON_SKIPPED;
            n_unst += ((st >> (2 * l)) & ST_UNSTABLE) >> 1;
#pragma unroll
            for (int a = 0; a < Lat::Q; ++a)
                dst[in.off + (int64_t)a * in.plane + (int64_t)y * in.pitch + x0 + l] =
                    Store<S>::from(N::lane(o[a], l));
        }
    }
    if (n_skip) atomicAdd(status + 2 * inst + 0, n_skip);
    if (n_unst) atomicAdd(status + 2 * inst + 1, n_unst);
}

template <class Lat, typename S>
__global__ void moments_kernel(const S* src, const InstDesc* insts, bool pulled, double rho0,
                               double* rho, double* ux, double* uy, int64_t node_base) {
    const InstDesc in = insts[blockIdx.y];
    const uint32_t n = (uint32_t)in.nx * (uint32_t)in.ny;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int x, y;
        node_xy(k, (uint32_t)in.nx, x, y);
        double d[Lat::Q];
        node_state<Lat, S>(src, in, x, y, pulled, d);
        double dr = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int a = 0; a < Lat::Q; ++a) {
            dr += d[a];
            jx += Lat::vx(a) * d[a];
            jy += Lat::vy(a) * d[a];
        }
        const double r = rho0 + dr;
        const double ir = 1.0 / r;
        const int64_t g = in.node0 - node_base + k;
        rho[g] = r;
        if (ux) ux[g] = jx * ir;
        if (uy) uy[g] = jy * ir;
    }
}

template <class Lat, typename S>
__global__ void gather_f_kernel(const S* src, const InstDesc* insts, bool pulled, double rho0,
                                double* f) {
    const InstDesc in = insts[blockIdx.y];
    const uint32_t n = (uint32_t)in.nx * (uint32_t)in.ny;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int x, y;
        node_xy(k, (uint32_t)in.nx, x, y);
        double d[Lat::Q];
        node_state<Lat, S>(src, in, x, y, pulled, d);
#pragma unroll
        for (int a = 0; a < Lat::Q; ++a)
            f[in.node0 * Lat::Q + (int64_t)a * n + k] = Lat::w(a) * rho0 + d[a];
    }
}

// Deviations of f(x, t_n) at one node in FP32 (2- and 4-byte storage):
// same pull rule as node_state.
template <class Lat, typename S>
__device__ void node_state_f32(const S* base, const InstDesc& in, int x, int y, bool pulled,
                               float (&d)[Lat::Q]) {
#pragma unroll
    for (int a = 0; a < Lat::Q; ++a) {
        int sx = x, sy = y;
        bool inside = true;
        if (pulled) {
            sx = x - Lat::vx(a);
            sy = y - Lat::vy(a);
            if (in.bc == BC_CAVITY) {
                inside = sx >= 0 && sx < in.nx && sy >= 0 && sy < in.ny;
            } else {
                if (in.bc == BC_PERIODIC) sx = (sx + in.nx) % in.nx;
                else sx = sx < 0 ? 0 : (sx >= in.nx ? in.nx - 1 : sx);
                sy = (sy + in.ny) % in.ny;
            }
        }
        d[a] = inside ? Store<S>::to_f32(*elem_ptr<Lat, S>(base, in, a, sx, sy)) : 0.f;
    }
}

// Conservation, pass 1: the block of work item (i, b) sums (sum d,
// sum d v_x, sum d v_y) of f(t_n) over the rows y = b mod P_i of instance i
// (P_i = cons_partials(ny_i)); thread t takes x = t, t + CONS_THREADS, ...
// of each of those rows, rows in increasing order (issuing the loads of a
// few of its nodes of a row together, adding them in order), and the block
// reduces
// its threads in a fixed tree into partials[(i*CONS_PARTIALS + b)*3 + c].
// The order is fixed by the instance alone.  FP64 storage sums in FP64.
// FP32 and BF16 storage sum in compensated FP32 pairs (Knuth's two-sum;
// about twice FP32's precision, converted to FP64 once per thread), which
// spares the slow FP64 pipe.  FP16 storage sums exactly in integers: every
// FP16 value is a multiple of 2^-24 below 2^16 in magnitude, so 2^24 d is an
// integer below 2^40, and a thread's nodes add exactly in 64-bit integers,
// converted to FP64 once; nodes whose values are all below 8 in magnitude,
// which is every node of a physical state, sum in 32-bit integers first,
// without 64-bit conversions.  A node with a non-finite value takes the
// FP64 path, so that it propagates.  Interior nodes pull with plain shifted
// loads; the outer ring applies the boundary rules.
template <class Lat, typename S>
__global__ void __launch_bounds__(CONS_THREADS, CONS_MIN_BLOCKS)
cons_partial_kernel(const S* src, const InstDesc* insts, const int2* items, bool pulled,
                    double* partials) {
    using V = typename std::conditional<sizeof(S) == 8, double, float>::type;
    // FP32 and BF16 values sum in FP32 pairs (compensated: each addition's
    // rounding error is kept, so a pair carries about twice FP32's precision)
    constexpr bool DF = std::is_same<S, float>::value || std::is_same<S, __nv_bfloat16>::value;
    // nodes x, x + T, ..., x + (K - 1) T of a row (T = CONS_THREADS) whose
    // loads a thread issues together before it adds them in order
    constexpr int K = sizeof(S) == 8 ? 2 : 4;
    __shared__ double sh[3][CONS_THREADS];
    const int2 it = items[blockIdx.x];
    const InstDesc in = insts[it.x];
    const int nx = in.nx, ny = in.ny, P = cons_partials(ny);
    const S* base = src + in.off;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    long long i0 = 0, i1 = 0, i2 = 0;  // FP16: exact sums in units of 2^-24
    float h0 = 0.f, c0 = 0.f, h1 = 0.f, c1 = 0.f, h2 = 0.f, c2 = 0.f;  // FP32 / BF16: (sum, error)
    // h + v = s + e exactly (Knuth's two-sum); the error joins the running c
    auto add2 = [](float& h, float& c, float v) {
        const float sum = __fadd_rn(h, v);
        const float bv = __fsub_rn(sum, h);
        const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(sum, bv)), __fsub_rn(v, bv));
        h = sum;
        c = __fadd_rn(c, e);
    };
    for (int y = it.y; y < ny; y += P) {
        const bool yint = Lat::Q == 3 || (y >= 1 && y <= ny - 2);
        for (int x0 = threadIdx.x; x0 < nx; x0 += K * CONS_THREADS) {
          S raw[K][Lat::Q];
          uint32_t plain = 0u;  // bit k: node k is read with plain shifted loads
#pragma unroll
          for (int k = 0; k < K; ++k) {
              const int x = x0 + k * CONS_THREADS;
              if (x < nx && (!pulled || (yint && x >= 1 && x <= nx - 2))) {
                  plain |= 1u << k;
#pragma unroll
                  for (int a = 0; a < Lat::Q; ++a) {
                      const int sx = pulled ? x - Lat::vx(a) : x, sy = pulled ? y - Lat::vy(a) : y;
                      raw[k][a] = base[(int64_t)a * in.plane + (int64_t)sy * in.pitch + sx];
                  }
              }
          }
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int x = x0 + k * CONS_THREADS;
            if (x >= nx) break;
            V d[Lat::Q];
            if ((plain >> k) & 1u) {
#pragma unroll
                for (int a = 0; a < Lat::Q; ++a) {
                    if constexpr (sizeof(S) != 8) d[a] = Store<S>::to_f32(raw[k][a]);
                    else d[a] = Store<S>::to_f64(raw[k][a]);
                }
            } else if constexpr (sizeof(S) != 8) {
                node_state_f32<Lat, S>(src, in, x, y, pulled, d);
            } else {
                node_state<Lat, S>(src, in, x, y, pulled, d);
            }
            bool exact = false;
            if constexpr (std::is_same<S, __half>::value) {
                // every |d| < 8: 2^24 d below 2^27, the node sums of nine
                // such terms below 2^31, in 32-bit integers
                bool small = true;
#pragma unroll
                for (int a = 0; a < Lat::Q; ++a) small = small && (fabsf(d[a]) < 8.f);
                if (small) {
                    int r0 = 0, r1 = 0, r2 = 0;
#pragma unroll
                    for (int a = 0; a < Lat::Q; ++a) {
                        const int v = __float2int_rn(d[a] * 16777216.f);  // 2^24 d, exact
                        r0 += v;
                        if (Lat::vx(a) != 0) r1 += Lat::vx(a) > 0 ? v : -v;
                        if (Lat::vy(a) != 0) r2 += Lat::vy(a) > 0 ? v : -v;
                    }
                    i0 += r0;
                    i1 += r1;
                    i2 += r2;
                    exact = true;
                } else {
                    long long r0 = 0, r1 = 0, r2 = 0;
                    bool finite = true;
#pragma unroll
                    for (int a = 0; a < Lat::Q; ++a) {
                        finite = finite && (fabsf(d[a]) <= 65504.f);
                        const long long v = __float2ll_rn(d[a] * 16777216.f);
                        r0 += v;
                        if (Lat::vx(a) != 0) r1 += Lat::vx(a) > 0 ? v : -v;
                        if (Lat::vy(a) != 0) r2 += Lat::vy(a) > 0 ? v : -v;
                    }
                    if (finite) {
                        i0 += r0;
                        i1 += r1;
                        i2 += r2;
                        exact = true;
                    }
                }
            }
            if constexpr (DF) {
                bool finite = true;
#pragma unroll
                for (int a = 0; a < Lat::Q; ++a) finite = finite && (fabsf(d[a]) <= 3.4028235e38f);
                if (finite) {
#pragma unroll
                    for (int a = 0; a < Lat::Q; ++a) {
                        add2(h0, c0, d[a]);
                        if (Lat::vx(a) != 0) add2(h1, c1, Lat::vx(a) > 0 ? d[a] : -d[a]);
                        if (Lat::vy(a) != 0) add2(h2, c2, Lat::vy(a) > 0 ? d[a] : -d[a]);
                    }
                    exact = true;
                }
            }
            if (!exact) {
#pragma unroll
                for (int a = 0; a < Lat::Q; ++a) {
                    const double v = (double)d[a];
                    s0 += v;
                    if (Lat::vx(a) != 0) s1 += Lat::vx(a) * v;
                    if (Lat::vy(a) != 0) s2 += Lat::vy(a) * v;
                }
            }
          }
        }
    }
    if constexpr (std::is_same<S, __half>::value) {
        // the thread's exact FP16 node sums, in units of 2^-24 (at most
        // 2^15 nodes of 9 values below 2^40 each: no overflow), to FP64 once
        constexpr double inv = 1.0 / 16777216.0;
        s0 += (double)i0 * inv;
        s1 += (double)i1 * inv;
        s2 += (double)i2 * inv;
    }
    if constexpr (DF) {
        s0 += (double)h0 + (double)c0;
        s1 += (double)h1 + (double)c1;
        s2 += (double)h2 + (double)c2;
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    sh[2][threadIdx.x] = s2;
    __syncthreads();
    for (int h = CONS_THREADS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
#pragma unroll
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x < 3)
        partials[((int64_t)it.x * CONS_PARTIALS + it.y) * 3 + threadIdx.x] = sh[threadIdx.x][0];
}

// Conservation, pass 2: one thread per instance adds its partials in order;
// total mass = N rho0 + sum d (sum_a W_a = 1).
__global__ void cons_final_kernel(const double* partials, const InstDesc* insts, int count,
                                  double rho0, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double s[3] = {0.0, 0.0, 0.0};
    const int P = cons_partials(insts[i].ny);
    for (int b = 0; b < P; ++b)
        for (int c = 0; c < 3; ++c) s[c] += partials[((int64_t)i * CONS_PARTIALS + b) * 3 + c];
    const double nodes = (double)insts[i].nx * (double)insts[i].ny;
    out[3 * i + 0] = nodes * rho0 + s[0];
    out[3 * i + 1] = s[1];
    out[3 * i + 2] = s[2];
}

dim3 aux_grid(int64_t max_nodes, int count) {
    int64_t b = (max_nodes + AUX_THREADS - 1) / AUX_THREADS;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return dim3((unsigned)b, (unsigned)count);
}

template <class Lat, typename S, typename T, int COLL>
cudaError_t collide_inplace_dispatch(const AuxArgs& a, const void* src, void* dst) {
    collide_inplace_kernel<Lat, S, T, COLL><<<aux_grid(a.max_nodes, a.count), AUX_THREADS, 0, a.stream>>>(
        static_cast<const S*>(src), static_cast<S*>(dst), a.inst, a.rho0, a.status);
    return cudaGetLastError();
}

// TRT shares the MRT kernel; on D1Q3 every rule is BGK.
template <class Lat, typename S, typename T>
cudaError_t collide_inplace_by_rule(const AuxArgs& a, const void* src, void* dst) {
    if constexpr (Lat::Q == 3) {
        return collide_inplace_dispatch<Lat, S, T, COLL_MINXENT4>(a, src, dst);
    } else {
        switch (a.collision) {
            case COLL_MINXENT4: return collide_inplace_dispatch<Lat, S, T, COLL_MINXENT4>(a, src, dst);
            case COLL_SRT: return collide_inplace_dispatch<Lat, S, T, COLL_SRT>(a, src, dst);
            case COLL_MINXENT2: return collide_inplace_dispatch<Lat, S, T, COLL_MINXENT2>(a, src, dst);
            case COLL_MRT:
            case COLL_TRT: return collide_inplace_dispatch<Lat, S, T, COLL_MRT>(a, src, dst);
        }
        return cudaErrorInvalidValue;
    }
}

template <class Lat, typename S>
cudaError_t aux_dispatch(AuxOp op, const AuxArgs& a, const void* src, void* dst, const double* p0,
                         const double* p1, const double* p2, double* o0, double* o1, double* o2) {
    const dim3 g = aux_grid(a.max_nodes, a.count);
    switch (op) {
        case AuxOp::Init:
            init_kernel<Lat, S><<<g, AUX_THREADS, 0, a.stream>>>(static_cast<S*>(dst), a.inst, p0, p1,
                                                                 p2, a.rho0, a.node_base);
            break;
        case AuxOp::SetF:
            set_f_kernel<Lat, S><<<g, AUX_THREADS, 0, a.stream>>>(static_cast<S*>(dst), a.inst, p0,
                                                                  a.rho0);
            break;
        case AuxOp::Moments:
            moments_kernel<Lat, S><<<g, AUX_THREADS, 0, a.stream>>>(static_cast<const S*>(src), a.inst,
                                                                    a.pulled, a.rho0, o0, o1, o2,
                                                                    a.node_base);
            break;
        case AuxOp::GatherF:
            gather_f_kernel<Lat, S><<<g, AUX_THREADS, 0, a.stream>>>(static_cast<const S*>(src),
                                                                     a.inst, a.pulled, a.rho0, o0);
            break;
        case AuxOp::Conservation: {
            if (a.cons_nitems < 1 || !a.cons_items) return cudaErrorInvalidValue;
            cons_partial_kernel<Lat, S><<<a.cons_nitems, CONS_THREADS, 0, a.stream>>>(
                static_cast<const S*>(src), a.inst, a.cons_items, a.pulled, o1);
            cons_final_kernel<<<(a.count + 127) / 128, 128, 0, a.stream>>>(o1, a.inst, a.count,
                                                                           a.rho0, o0);
            break;
        }
        case AuxOp::CollideInPlace: {
            if (a.compute == DT_F64) {
                if constexpr (std::is_same<S, double>::value)
                    return collide_inplace_by_rule<Lat, S, double>(a, src, dst);
                return cudaErrorInvalidValue;
            }
            return collide_inplace_by_rule<Lat, S, float>(a, src, dst);
        }
    }
    return cudaGetLastError();
}

template <class Lat>
cudaError_t aux_by_storage(AuxOp op, const AuxArgs& a, const void* src, void* dst, const double* p0,
                           const double* p1, const double* p2, double* o0, double* o1, double* o2) {
    switch (a.storage) {
        case DT_F64: return aux_dispatch<Lat, double>(op, a, src, dst, p0, p1, p2, o0, o1, o2);
        case DT_F32: return aux_dispatch<Lat, float>(op, a, src, dst, p0, p1, p2, o0, o1, o2);
        case DT_F16: return aux_dispatch<Lat, __half>(op, a, src, dst, p0, p1, p2, o0, o1, o2);
        case DT_BF16:
            return aux_dispatch<Lat, __nv_bfloat16>(op, a, src, dst, p0, p1, p2, o0, o1, o2);
    }
    return cudaErrorInvalidValue;
}

// Stream function of the LDAS post-processing (Sec. IV.I) along each row of
// each instance: psi(x, y) = - integral_0^x u_y dx in lattice units, with
// the composite Simpson rule over pairs of unit intervals from the left
// wall and the trapezoidal rule on the last interval when x is odd.  One
// thread per row (rows of instance blockIdx.y).
__global__ void stream_function_kernel(const double* __restrict__ uy,
                                       const InstDesc* __restrict__ insts, double* __restrict__ psi,
                                       int64_t node_base) {
    const InstDesc& in = insts[blockIdx.y];
    const int nx = in.nx;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < in.ny; y += gridDim.x * blockDim.x) {
        const double* u = uy + (in.node0 - node_base) + (int64_t)y * nx;
        double* p = psi + (in.node0 - node_base) + (int64_t)y * nx;
        double simpson = 0.0;  // integral over [0, x] at the last even x
        p[0] = 0.0;
        for (int x = 1; x < nx; ++x) {
            if (x & 1) {
                p[x] = -(simpson + 0.5 * (u[x - 1] + u[x]));
            } else {
                simpson += (u[x - 2] + 4.0 * u[x - 1] + u[x]) * (1.0 / 3.0);
                p[x] = -simpson;
            }
        }
    }
}

}  // namespace

cudaError_t run_aux(AuxOp op, const AuxArgs& a, const void* src, void* dst, const double* p0,
                    const double* p1, const double* p2, double* o0, double* o1, double* o2) {
    if (a.lattice == 2) return aux_by_storage<D2Q9>(op, a, src, dst, p0, p1, p2, o0, o1, o2);
    return aux_by_storage<D1Q3>(op, a, src, dst, p0, p1, p2, o0, o1, o2);
}

cudaError_t stream_function(const AuxArgs& a, int64_t max_ny, const double* uy, double* psi) {
    const int threads = 128;
    const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((max_ny + threads - 1) / threads, 1024)),
                    (unsigned)a.count);
    stream_function_kernel<<<grid, threads, 0, a.stream>>>(uy, a.inst, psi, a.node_base);
    return cudaGetLastError();
}

}  // namespace lbm
