// lbm_step.cuh -- the fused pull-stream + collide + boundary kernel.
//
// One launch performs one time step of Eq. (2) for every instance of a
// context.  Populations are stored SoA (one plane per velocity, rows of
// `pitch` elements, pitch a multiple of 8) as deviations from W_a rho0, and
// the stored state is the post-collision field of the previous step, so the
// step is a pull:
//     f~_a(x) = f^post_a(x - v_a)  (with the boundary rules),
//     f^post(x) = collide(f~(x))   (or the wall / lid rule),
// reading each plane once and writing each plane once, both aligned.
//
// Work decomposition: a thread owns a chunk of V consecutive nodes of one
// row; a CTA owns a tile of tw x th chunks of one instance (tile table
// built on the host, walked with a grid-stride loop: one persistent launch
// covers an ensemble of uneven instances).  Each plane's chunk is one
// 8/16/32-byte vector load from row y - v_y; the x-shift of +-1 is served by
// a warp shuffle of the neighbouring lane's edge element, or by one scalar
// load (with the boundary rule) at tile, warp and row edges.
#pragma once
#include "lbm_collide.cuh"

namespace lbm {

template <typename S> __device__ __forceinline__ S bits_to(uint32_t lo, uint32_t hi);
template <> __device__ __forceinline__ double bits_to<double>(uint32_t lo, uint32_t hi) {
    return __hiloint2double((int)hi, (int)lo);
}
template <> __device__ __forceinline__ float bits_to<float>(uint32_t lo, uint32_t) {
    return __uint_as_float(lo);
}
template <> __device__ __forceinline__ __half bits_to<__half>(uint32_t lo, uint32_t) {
    return __ushort_as_half((unsigned short)(lo & 0xffffu));
}
template <> __device__ __forceinline__ __nv_bfloat16 bits_to<__nv_bfloat16>(uint32_t lo, uint32_t) {
    return __ushort_as_bfloat16((unsigned short)(lo & 0xffffu));
}

template <typename S> __device__ __forceinline__ uint32_t lo_bits(S v);
template <typename S> __device__ __forceinline__ uint32_t hi_bits(S v) { return 0u; }
template <> __device__ __forceinline__ uint32_t lo_bits<double>(double v) {
    return (uint32_t)__double2loint(v);
}
template <> __device__ __forceinline__ uint32_t hi_bits<double>(double v) {
    return (uint32_t)__double2hiint(v);
}
template <> __device__ __forceinline__ uint32_t lo_bits<float>(float v) { return __float_as_uint(v); }
template <> __device__ __forceinline__ uint32_t lo_bits<__half>(__half v) {
    return (uint32_t)__half_as_ushort(v);
}
template <> __device__ __forceinline__ uint32_t lo_bits<__nv_bfloat16>(__nv_bfloat16 v) {
    return (uint32_t)__bfloat16_as_ushort(v);
}

// V consecutive elements of type S held as 32-bit words.
template <typename S, int V> struct Chunk {
    static constexpr int BYTES = V * (int)sizeof(S);
    static constexpr int WORDS = BYTES / 4;
    static_assert(BYTES == 8 || BYTES == 16 || BYTES == 32, "chunk must be 8, 16 or 32 bytes");
    uint32_t w[WORDS];

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < WORDS; ++k) w[k] = 0u;
    }
    __device__ __forceinline__ void load(const S* p) {
        if constexpr (BYTES == 8) {
            const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
            w[0] = v.x; w[1] = v.y;
        } else {
#pragma unroll
            for (int k = 0; k < BYTES / 16; ++k) {
                const uint4 v = __ldg(reinterpret_cast<const uint4*>(p) + k);
                w[4 * k + 0] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
            }
        }
    }
    __device__ __forceinline__ void store(S* p) const {
        if constexpr (BYTES == 8) {
            *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
        } else {
#pragma unroll
            for (int k = 0; k < BYTES / 16; ++k)
                reinterpret_cast<uint4*>(p)[k] =
                    make_uint4(w[4 * k + 0], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
        }
    }
    // i must be a compile-time constant after unrolling
    __device__ __forceinline__ S get(int i) const {
        if constexpr (sizeof(S) == 2) {
            const uint32_t x = w[i >> 1];
            return bits_to<S>((i & 1) ? (x >> 16) : (x & 0xffffu), 0u);
        } else if constexpr (sizeof(S) == 4) {
            return bits_to<S>(w[i], 0u);
        } else {
            return bits_to<S>(w[2 * i], w[2 * i + 1]);
        }
    }
    __device__ __forceinline__ void set(int i, S v) {
        if constexpr (sizeof(S) == 2) {
            const uint32_t b = lo_bits<S>(v);
            w[i >> 1] = (i & 1) ? ((w[i >> 1] & 0xffffu) | (b << 16)) : ((w[i >> 1] & 0xffff0000u) | b);
        } else if constexpr (sizeof(S) == 4) {
            w[i] = lo_bits<S>(v);
        } else {
            w[2 * i] = lo_bits<S>(v);
            w[2 * i + 1] = hi_bits<S>(v);
        }
    }
};

// Warp shuffles of one element.
template <typename S> __device__ __forceinline__ S shfl_up1(S v) {
    const uint32_t lo = __shfl_up_sync(0xffffffffu, lo_bits<S>(v), 1);
    uint32_t hi = 0u;
    if constexpr (sizeof(S) == 8) hi = __shfl_up_sync(0xffffffffu, hi_bits<S>(v), 1);
    return bits_to<S>(lo, hi);
}
template <typename S> __device__ __forceinline__ S shfl_down1(S v) {
    const uint32_t lo = __shfl_down_sync(0xffffffffu, lo_bits<S>(v), 1);
    uint32_t hi = 0u;
    if constexpr (sizeof(S) == 8) hi = __shfl_down_sync(0xffffffffu, hi_bits<S>(v), 1);
    return bits_to<S>(lo, hi);
}

template <typename S> __device__ __forceinline__ S ldg_elem(const S* p) {
    if constexpr (sizeof(S) == 2) {
        return bits_to<S>((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p)), 0u);
    } else {
        return __ldg(p);
    }
}
template <typename S> __device__ __forceinline__ S zero_elem() { return bits_to<S>(0u, 0u); }

// Element xs of a source row, with the x boundary rule for xs = -1 or nx.
// row_ok = false: the row lies outside a cavity (fill: deviation 0).
template <typename S>
__device__ __forceinline__ S edge_elem(const S* rowp, bool row_ok, int xs, int nx, int bc) {
    if (!row_ok) return zero_elem<S>();
    if (xs < 0 || xs >= nx) {
        if (bc == BC_PERIODIC) xs = (xs < 0) ? xs + nx : xs - nx;
        else if (bc == BC_ZERO_GRADIENT) xs = (xs < 0) ? 0 : nx - 1;
        else return zero_elem<S>();  // cavity: outside the lattice
    }
    return ldg_elem<S>(rowp + xs);
}

template <typename T, typename S> __device__ __forceinline__ T to_compute(S v) {
    if constexpr (std::is_same<T, double>::value) return Store<S>::to_f64(v);
    else return Store<S>::to_f32(v);
}

template <class Lat, typename S, typename T, int V, int COLL>
__global__ void __launch_bounds__(256) step_kernel(const StepArgs args) {
    constexpr int Q = Lat::Q;
    const S* __restrict__ src = static_cast<const S*>(args.src);
    S* __restrict__ dst = static_cast<S*>(args.dst);
    const int tid = threadIdx.x;
    const int cx = tid & (args.tw - 1);
    const int cy = tid >> args.tw_log2;
    const int lane = tid & 31;
    const T rho0 = (T)args.rho0;
    wait_previous_grid();
    allow_next_grid();

    for (int t = blockIdx.x; t < args.ntiles; t += gridDim.x) {
        const TileDesc tile = args.tiles[t];
        const InstDesc& in = args.inst[tile.inst];
        const int nx = in.nx, ny = in.ny, bc = in.bc;
        const int64_t pitch = in.pitch, plane = in.plane;
        const int x0 = (tile.cx0 + cx) * V;
        const int y = tile.y0 + cy;
        const bool active = (x0 < nx) && (y < ny);
        const S* base = src + in.off;

        Chunk<S, V> raw[Q];
        S left[Q], right[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int vxa = Lat::vx(a), vya = Lat::vy(a);
            int sy = y - vya;
            bool row_ok = true;
            if (vya != 0) {
                if (bc == BC_CAVITY) row_ok = (sy >= 0) && (sy < ny);
                else sy = (sy < 0) ? sy + ny : ((sy >= ny) ? sy - ny : sy);
            }
            const S* rowp = base + a * plane + (int64_t)(row_ok ? sy : 0) * pitch;
            if (active && row_ok) raw[a].load(rowp + x0);
            else raw[a].zero();
            if (vxa == 1) {
                // node x0 pulls from x0 - 1: last element of the left neighbour chunk
                S nb = shfl_up1<S>(raw[a].get(V - 1));
                const bool use_shfl = (x0 > 0) && (cx > 0) && (lane > 0);
                if (active && !use_shfl) nb = edge_elem<S>(rowp, row_ok, x0 - 1, nx, bc);
                left[a] = nb;
            } else if (vxa == -1) {
                // node x0+V-1 pulls from x0 + V: first element of the right chunk
                S nb = shfl_down1<S>(raw[a].get(0));
                const bool use_shfl = (x0 + V < nx) && (cx < args.tw - 1) && (lane < 31);
                if (active && !use_shfl) nb = edge_elem<S>(rowp, row_ok, min(x0 + V, nx), nx, bc);
                right[a] = nb;
            } else {
                left[a] = right[a] = zero_elem<S>();
            }
        }
        // Inactive threads fall through to the next tile without returning
        // early, so every lane reaches the shuffles of the next iteration.
        if (active) {
        // Ragged last chunk of a row: node nx-1 sits before the chunk's end and
        // must see the boundary value fetched into right[] instead of padding.
        const bool ragged = (x0 + V > nx);
        const int jr = nx - 1 - x0;  // last valid position in a ragged chunk
        if (ragged) {
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                if (Lat::vx(a) == -1) {
#pragma unroll
                    for (int k = 1; k < V; ++k) {
                        // unconditional set of a selected value keeps raw[] in registers
                        const S v = raw[a].get(k);
                        raw[a].set(k, (k == jr + 1) ? right[a] : v);
                    }
                }
            }
        }

        // Collide nodes one at a time (FP64) or two at a time (FP32, packed
        // FP32x2 arithmetic).
        using CT = typename std::conditional<
            std::is_same<T, float>::value, typename std::conditional<(V % 2 == 0), F2, F1>::type,
            T>::type;
        using N = Num<CT>;
        constexpr int P = N::LANES;
        using LT = typename LaneOf<CT>::type;
        const Rates<CT> rates{CT((LT)in.omega), CT((LT)in.omega2), CT((LT)in.s_e), CT((LT)in.s_eps)};
        const CT rho0v = CT((LT)rho0);
        const bool cavity_edge =
            (bc == BC_CAVITY) && (y == 0 || y == ny - 1 || x0 == 0 || x0 + V >= nx);
        Chunk<S, V> out[Q];
        uint32_t n_skip = 0, n_unst = 0;
#pragma unroll
        for (int i = 0; i < V; i += P) {
            CT d[Q], o[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const int vxa = Lat::vx(a);
#pragma unroll
                for (int l = 0; l < P; ++l) {
                    const int j = i + l;
                    S s;
                    if (vxa == 0) s = raw[a].get(j);
                    else if (vxa == 1) s = (j == 0) ? left[a] : raw[a].get(j - 1);
                    else s = (j == V - 1) ? right[a] : raw[a].get(j + 1);
                    if constexpr (std::is_same<CT, double>::value) d[a] = to_compute<T, S>(s);
                    else N::set_lane(d[a], l, to_compute<float, S>(s));
                }
            }
            uint32_t st = Collide<Lat, COLL, CT, (int)sizeof(S)>::run(d, rho0v, rates, o);
            if (cavity_edge) {
#pragma unroll
                for (int l = 0; l < P; ++l) {
                    const int x = x0 + i + l;
                    const bool wall = (x == 0) || (x == nx - 1) || (y == 0);
                    const bool lid = !wall && (y == ny - 1);
                    if (wall) {
                        // full-way bounce-back: reverse every population (W_opp = W_a)
#pragma unroll
                        for (int a = 0; a < Q; ++a)
                            N::set_lane(o[a], l, N::lane(d[Lat::opp(a)], l));
                        st &= ~(3u << (2 * l));
                    } else if (lid) {
#pragma unroll
                        for (int a = 0; a < Q; ++a) {
                            if constexpr (std::is_same<T, double>::value)
                                N::set_lane(o[a], l, in.lid_dev[a]);
                            else
                                N::set_lane(o[a], l, in.lid_dev_f[a]);
                        }
                        st &= ~(3u << (2 * l));
                    }
                }
            }
#pragma unroll
            for (int l = 0; l < P; ++l) {
                if (x0 + i + l < nx) {
                    n_skip += (st >> (2 * l)) & ST_NEWTON_SKIPPED;
                    n_unst += ((st >> (2 * l)) & ST_UNSTABLE) >> 1;
                }
            }
#pragma unroll
            for (int a = 0; a < Q; ++a)
#pragma unroll
                for (int l = 0; l < P; ++l) out[a].set(i + l, Store<S>::from(N::lane(o[a], l)));
        }
        if (ragged) {
            // keep the row padding at deviation 0
#pragma unroll
            for (int a = 0; a < Q; ++a)
#pragma unroll
                for (int k = 1; k < V; ++k) {
                    const S v = out[a].get(k);
                    out[a].set(k, (k > jr) ? zero_elem<S>() : v);
                }
        }
        S* obase = dst + in.off + (int64_t)y * pitch + x0;
#pragma unroll
        for (int a = 0; a < Q; ++a) out[a].store(obase + a * plane);

        if (n_skip | n_unst) {
            atomicAdd(args.status + 2 * tile.inst + 0, (unsigned long long)n_skip);
            atomicAdd(args.status + 2 * tile.inst + 1, (unsigned long long)n_unst);
        }
        }  // active
    }
}

// The __global__ function for (lattice, collision rule) with storage S,
// arithmetic T and V nodes per thread.  TRT shares the MRT kernel (its rates
// come from the instance table); on D1Q3 every rule is BGK.
template <typename S, typename T, int V>
const void* pick_step_kernel(int lattice, int collision) {
    if (lattice == 1) return (const void*)&step_kernel<D1Q3, S, T, V, COLL_MINXENT4>;
    switch (collision) {
        case COLL_MINXENT4: return (const void*)&step_kernel<D2Q9, S, T, V, COLL_MINXENT4>;
        case COLL_SRT: return (const void*)&step_kernel<D2Q9, S, T, V, COLL_SRT>;
        case COLL_MINXENT2: return (const void*)&step_kernel<D2Q9, S, T, V, COLL_MINXENT2>;
        case COLL_MRT:
        case COLL_TRT: return (const void*)&step_kernel<D2Q9, S, T, V, COLL_MRT>;
    }
    return nullptr;
}

}  // namespace lbm
