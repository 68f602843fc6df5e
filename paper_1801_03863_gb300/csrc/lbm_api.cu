// lbm_api.cu -- the C ABI of liblbm (declared in include/lbm.h): context
// lifetime, device memory layout, tile tables, the launch-shape autotuner,
// CUDA-graph replay of the step loop, and host I/O.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_aux.h"

using namespace lbm;

namespace {

constexpr int64_t ROW_ALIGN = 8;       // row pitch multiple (nodes)
constexpr int64_t PLANE_ALIGN = 128;   // plane / instance alignment (elements)
constexpr int GRAPH_STEPS = 16;        // steps per captured graph (even)

size_t dtype_bytes(int dt) { return dt == DT_F64 ? 8 : (dt == DT_F32 ? 4 : 2); }

// Launch shape.  kind 0: register-chunk kernel (V nodes per thread, tiles of
// tw x th chunks); kind 1 / 2 / 3 / 4: TMA-staged D2Q9 kernel with node
// pairs (V = 2) in the large-tile / small-tile / wide-CTA / deep-ring
// geometry (smem_tile_nodes variant kind - 1), tile width per instance.
struct Shape {
    int V, tw, th;
    int kind = 0;
};

Shape default_shape(int lattice, int storage) {
    if (lattice == 1) return {storage == DT_F64 ? 2 : 4, 128, 1};
    if (storage == DT_F64) return {2, 16, 8};
    if (storage == DT_F32) return {4, 16, 8};
    return {8, 8, 16};
}

// Launch-shape candidates of the autotuner.  D2Q9 with FP32 arithmetic: the
// TMA-staged kernel in its four geometries and the default register-chunk
// shape (which wins only on small, cache-resident lattices).  D1Q3 and the
// FP64 path: register-chunk shapes, V = the compiled widths of the storage
// type, tiles of 128 or 256 threads.
std::vector<Shape> candidate_shapes(int lattice, int storage, int64_t max_nx, int64_t max_ny) {
    std::vector<Shape> out;
    if (lattice == 2 && storage != DT_F64) {
        out.push_back({2, 0, 0, 1});  // TMA-staged kernel, node pairs, large tiles
        out.push_back({2, 0, 0, 2});  // TMA-staged kernel, node pairs, small tiles
        out.push_back({2, 0, 0, 3});  // TMA-staged kernel, node pairs, wide CTAs
        out.push_back({2, 0, 0, 4});  // TMA-staged kernel, node pairs, deep ring
        out.push_back(default_shape(lattice, storage));
        return out;
    }
    std::vector<int> vs;
    if (storage == DT_F64) vs = {2};
    else if (storage == DT_F32) vs = {2, 4};
    else vs = {4, 8};
    for (int V : vs) {
        for (int block : {128, 256}) {
            if (lattice == 1) {
                if ((int64_t)block * V > 2 * std::max<int64_t>(max_nx, 8) && block > 128) continue;
                out.push_back({V, block, 1});
                continue;
            }
            for (int tw : {8, 16, 32}) {
                const int th = block / tw;
                if (th > max_ny && tw < 32) continue;
                if ((int64_t)tw * V > 2 * std::max<int64_t>(max_nx, 8) && tw > 8) continue;
                out.push_back({V, tw, th});
            }
        }
    }
    return out;
}

int64_t count_tiles(const std::vector<std::pair<int64_t, int64_t>>& dims, const Shape& s,
                    int storage, bool least_padding) {
    int64_t n = 0;
    if (s.kind >= 1) {
        for (auto& d : dims) {
            const int tn = smem_tile_nodes(storage, s.kind - 1);
            const int64_t X = smem_tile_width(d.first, d.second, tn, smem_threads(s.kind - 1),
                                              least_padding);
            const int64_t R = tn / X;
            n += ((d.first + X - 1) / X) * ((d.second + R - 1) / R);
        }
        return n;
    }
    for (auto& d : dims) {
        const int64_t chunks = (d.first + s.V - 1) / s.V;
        n += ((chunks + s.tw - 1) / s.tw) * ((d.second + s.th - 1) / s.th);
    }
    return n;
}

struct Layout {
    std::vector<InstDesc> inst;
    int64_t elems = 0;       // elements per population buffer
    int64_t total_nodes = 0;
    int64_t max_nodes = 0, max_nx = 0, max_ny = 0;
    int64_t max_tiles = 0;
};

Layout make_layout(int lattice, int storage, const std::vector<std::pair<int64_t, int64_t>>& dims) {
    Layout L;
    const int Q = lattice == 2 ? 9 : 3;
    int64_t off = 0, node0 = 0;
    for (auto& d : dims) {
        InstDesc in;
        std::memset(&in, 0, sizeof in);
        in.nx = (int32_t)d.first;
        in.ny = (int32_t)d.second;
        in.pitch = (int32_t)round_up(d.first, ROW_ALIGN);
        in.plane = round_up((int64_t)in.pitch * in.ny, PLANE_ALIGN);
        in.off = off;
        in.node0 = node0;
        off += Q * in.plane;
        node0 += d.first * d.second;
        L.max_nodes = std::max(L.max_nodes, d.first * d.second);
        L.max_nx = std::max(L.max_nx, d.first);
        L.max_ny = std::max(L.max_ny, d.second);
        L.inst.push_back(in);
    }
    L.elems = off;
    L.total_nodes = node0;
    // Tile-table capacity: a bound that holds for every register-chunk shape
    // (V >= 2, tw >= 4, tw * th >= 128 threads) and the shared-memory kernel's
    // tiling, so any shape the autotuner or LBM_SHAPE selects fits.
    int64_t bound = 0;
    for (auto& d : dims) {
        const int64_t chunks = (d.first + 1) / 2;
        bound += chunks * d.second / 128 + chunks / 4 + d.second + 1;
    }
    L.max_tiles = bound;
    for (int kind = 1; kind <= 4; ++kind)
        for (bool lp : {false, true})
            L.max_tiles = std::max(L.max_tiles, count_tiles(dims, Shape{2, 0, 0, kind}, storage, lp));
    return L;
}

struct Carve {
    size_t buf_bytes, inst_off, tiles_off, status_off, partials_off, cons_off, stage_off, tmap_off,
        err_off, total;
};

Carve carve(const Layout& L, int lattice, int storage, int count) {
    const int Q = lattice == 2 ? 9 : 3;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    Carve c;
    c.buf_bytes = al((size_t)L.elems * dtype_bytes(storage));
    size_t p = 2 * c.buf_bytes;
    c.inst_off = p;
    p += al(sizeof(InstDesc) * count);
    c.tiles_off = p;
    p += al(sizeof(TileDesc) * (size_t)std::max<int64_t>(L.max_tiles, 1));
    c.status_off = p;
    p += al(sizeof(unsigned long long) * 2 * count);
    c.partials_off = p;
    p += al(sizeof(double) * 3 * (size_t)CONS_PARTIALS * count);
    c.cons_off = p;  // (instance, partial) work list of the conservation reduction
    p += al(sizeof(int2) * (size_t)CONS_PARTIALS * count);
    c.stage_off = p;
    p += al(sizeof(double) * std::max<int64_t>(3 * L.total_nodes, Q * L.total_nodes));
    c.tmap_off = p;  // four TMA tensor maps per instance: [buffer][tile | halo]
    p += al(4 * sizeof(CUtensorMapOpaque) * count);
    c.err_off = p;
    p += 256;
    c.total = p;
    return c;
}

}  // namespace

struct lbm_ctx {
    int lattice = 2, Q = 9, count = 0, bc = 0, compute = DT_F64, storage = DT_F64;
    int collision = COLL_MINXENT4;
    double rho0 = 1.0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    int num_sms = 0;
    bool own_mem = false;
    char* mem = nullptr;
    Layout layout;
    Carve cv{};
    char* buf[2] = {nullptr, nullptr};
    int cur = 0;  // buffer holding the current state
    InstDesc* d_inst = nullptr;
    TileDesc* d_tiles = nullptr;
    unsigned long long* d_status = nullptr;
    double* d_partials = nullptr;
    int2* d_cons = nullptr;  // conservation work list
    int n_cons = 0;
    double* d_stage = nullptr;
    CUtensorMapOpaque* d_tmaps = nullptr;  // [buffer][tile | halo][instance]
    unsigned int* d_error = nullptr;
    int tmaps_variant = -1;  // tile variant the TMA tensor maps were built for
    std::vector<TileDesc> tiles;
    bool initialized = false;
    std::vector<uint8_t> inst_init;  // per-instance initial fields set (lbm_init_batch)
    bool post = false;  // stored field is post-collision
    int64_t steps = 0;
    Shape shape{};
    const void* kern = nullptr;
    int grid = 0;
    size_t smem = 0;  // dynamic shared memory of the step kernel
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool failed = false;
    int spin_limit = 1 << 20;  // polls of one bounded mbarrier wait in the TMA kernel
    int lost_tile = -1;        // timeout-path test hook (LBM_TEST_LOST_TILE)
};

namespace {

#define LBM_CK(call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            if (getenv("LBM_DEBUG"))                                                   \
                fprintf(stderr, "liblbm: %s failed: %s (%s:%d)\n", #call,              \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                   \
            if (ctx) ctx->failed = true;                                               \
            return LBM_ERR_CUDA;                                                       \
        }                                                                              \
    } while (0)

const void* find_step_kernel(int lattice, int storage, int collision, int V) {
    switch (storage) {
        case DT_F64: return step_kernel_f64(lattice, collision, V);
        case DT_F32: return step_kernel_f32(lattice, collision, V);
        case DT_F16: return step_kernel_f16(lattice, collision, V);
        case DT_BF16: return step_kernel_bf16(lattice, collision, V);
    }
    return nullptr;
}

AuxArgs aux_args(const lbm_ctx* ctx) {
    AuxArgs a;
    a.lattice = ctx->lattice;
    a.storage = ctx->storage;
    a.compute = ctx->compute;
    a.collision = ctx->collision;
    a.count = ctx->count;
    a.max_nodes = ctx->layout.max_nodes;
    a.inst = ctx->d_inst;
    a.rho0 = ctx->rho0;
    a.pulled = ctx->post;
    a.status = ctx->d_status;
    a.stream = ctx->stream;
    a.cons_items = ctx->d_cons;
    a.cons_nitems = ctx->n_cons;
    return a;
}

std::vector<TileDesc> build_tiles(const lbm_ctx* ctx, const Shape& s) {
    std::vector<TileDesc> t;
    if (s.kind >= 1) {
        for (int i = 0; i < ctx->count; ++i) {
            const InstDesc& in = ctx->layout.inst[i];
            const int tn = smem_tile_nodes(ctx->storage, s.kind - 1);
            const int X = smem_tile_width(in.nx, in.ny, tn, smem_threads(s.kind - 1),
                                          smem_least_padding(ctx->collision));
            const int R = tn / X;
            for (int64_t y0 = 0; y0 < in.ny; y0 += R)
                for (int64_t x0 = 0; x0 < in.nx; x0 += X)
                    t.push_back({(int32_t)i, (int32_t)x0, (int32_t)y0, (int32_t)X});
        }
        return t;
    }
    for (int i = 0; i < ctx->count; ++i) {
        const InstDesc& in = ctx->layout.inst[i];
        const int64_t chunks = (in.nx + s.V - 1) / s.V;
        for (int64_t y0 = 0; y0 < in.ny; y0 += s.th)
            for (int64_t c0 = 0; c0 < chunks; c0 += s.tw)
                t.push_back({(int32_t)i, (int32_t)c0, (int32_t)y0, 0});
    }
    return t;
}

int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

int build_tensor_maps(lbm_ctx* ctx, int variant);

// Make shape s current: tile table to the device, kernel and grid size.
int apply_shape(lbm_ctx* ctx, const Shape& s) {
    const void* k = nullptr;
    size_t smem = 0;
    if (s.kind >= 1) {
        if (ctx->lattice != 2 || ctx->compute != DT_F32 || s.kind > 4) return LBM_ERR_ARG;
        const int var = s.kind - 1;
        if (ctx->storage == DT_F32) k = step_kernel_smem_f32(ctx->collision, var, &smem);
        else if (ctx->storage == DT_F16) k = step_kernel_smem_f16(ctx->collision, var, &smem);
        else if (ctx->storage == DT_BF16) k = step_kernel_smem_bf16(ctx->collision, var, &smem);
        if (!k) return LBM_ERR_ARG;
        LBM_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int rc = build_tensor_maps(ctx, var);
        if (rc != LBM_OK) return rc;
    } else {
        k = find_step_kernel(ctx->lattice, ctx->storage, ctx->collision, s.V);
    }
    if (!k) return LBM_ERR_ARG;
    std::vector<TileDesc> t = build_tiles(ctx, s);
    if ((int64_t)t.size() > ctx->layout.max_tiles) return LBM_ERR_ARG;
    // the instance table records each instance's tile range
    int32_t idx = 0;
    for (int i = 0; i < ctx->count; ++i) {
        ctx->layout.inst[i].tile0 = idx;
        int32_t n = 0;
        while (idx + n < (int32_t)t.size() && t[idx + n].inst == i) ++n;
        ctx->layout.inst[i].ntiles = n;
        idx += n;
    }
    LBM_CK(cudaMemcpyAsync(ctx->d_tiles, t.data(), sizeof(TileDesc) * t.size(),
                           cudaMemcpyHostToDevice, ctx->stream));
    LBM_CK(cudaMemcpyAsync(ctx->d_inst, ctx->layout.inst.data(), sizeof(InstDesc) * ctx->count,
                           cudaMemcpyHostToDevice, ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    const int block = s.kind >= 1 ? smem_block_threads(s.kind - 1) : s.tw * s.th;
    int per_sm = 0;
    LBM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem));
    per_sm = std::max(per_sm, 1);
    const int64_t g = std::min<int64_t>((int64_t)per_sm * ctx->num_sms, (int64_t)t.size());
    ctx->tiles.swap(t);
    ctx->shape = s;
    ctx->kern = k;
    ctx->smem = smem;
    ctx->grid = (int)std::max<int64_t>(g, 1);
    for (int p = 0; p < 2; ++p) {
        if (ctx->graph[p]) cudaGraphExecDestroy(ctx->graph[p]);
        ctx->graph[p] = nullptr;
    }
    return LBM_OK;
}

// TMA tensor maps of both population buffers: per instance a 3-D view
// (x < nx, row, plane) of the populations, once with the box of one plane
// of a tile of the staged kernel (loads and stores: x beyond nx reads as
// zero and is not written) and once with a 16-byte-wide box of the tile's
// rows (the x halo loads).
int build_tensor_maps(lbm_ctx* ctx, int variant) {
    if (ctx->tmaps_variant == variant) return LBM_OK;
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    LBM_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                            &q));
    if (!fn || q != cudaDriverEntryPointSuccess) return LBM_ERR_CUDA;
    EncodeFn encode = reinterpret_cast<EncodeFn>(fn);
    const size_t es = dtype_bytes(ctx->storage);
    const int E = (int)(16 / es);
    const int tile_nodes = smem_tile_nodes(ctx->storage, variant);
    std::vector<CUtensorMap> maps(4 * (size_t)ctx->count);
    for (int m = 0; m < 4; ++m) {
        const int b = m >> 1;
        const bool halo = (m & 1) != 0;
        for (int i = 0; i < ctx->count; ++i) {
            const InstDesc& in = ctx->layout.inst[i];
            const int X = smem_tile_width(in.nx, in.ny, tile_nodes, smem_threads(variant),
                                          smem_least_padding(ctx->collision));
            const int R = tile_nodes / X;
            void* base = ctx->buf[b] + (size_t)in.off * es;
            cuuint64_t dims[3] = {(cuuint64_t)in.nx, (cuuint64_t)in.ny, 9};
            cuuint64_t strides[2] = {(cuuint64_t)in.pitch * es, (cuuint64_t)in.plane * es};
            cuuint32_t box[3] = {(cuuint32_t)(halo ? E : X), (cuuint32_t)R, 1};
            cuuint32_t estr[3] = {1, 1, 1};
            CUresult r = encode(&maps[(size_t)m * ctx->count + i],
                                es == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                if (getenv("LBM_DEBUG")) fprintf(stderr, "liblbm: tensor map encode failed (%d)\n", (int)r);
                return LBM_ERR_CUDA;
            }
        }
    }
    static_assert(sizeof(CUtensorMap) == sizeof(CUtensorMapOpaque), "tensor map size");
    LBM_CK(cudaMemcpyAsync(ctx->d_tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                           cudaMemcpyHostToDevice, ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    ctx->tmaps_variant = variant;
    return LBM_OK;
}

StepArgs step_args(const lbm_ctx* ctx, int src) {
    StepArgs a;
    a.src = ctx->buf[src];
    a.dst = ctx->buf[1 - src];
    a.inst = ctx->d_inst;
    a.tiles = ctx->d_tiles;
    a.ntiles = (int32_t)ctx->tiles.size();
    a.tw = ctx->shape.tw;
    a.tw_log2 = ctx->shape.tw > 0 ? ilog2(ctx->shape.tw) : 0;
    a.th = ctx->shape.th;
    a.rho0 = ctx->rho0;
    a.status = ctx->d_status;
    a.tmaps = ctx->d_tmaps + (size_t)src * 2 * ctx->count;
    a.tmaps_halo = ctx->d_tmaps + (size_t)(src * 2 + 1) * ctx->count;
    a.tmaps_dst = ctx->d_tmaps + (size_t)(1 - src) * 2 * ctx->count;
    a.error = ctx->d_error;
    a.spin_limit = ctx->spin_limit;
    a.lost_tile = ctx->lost_tile;
    return a;
}

// One step launch.  It is a programmatic dependent launch: the kernel may be
// scheduled while the previous kernel in the stream drains, and waits for its
// completion (griddepcontrol.wait) before touching device state.
cudaError_t launch_step(lbm_ctx* ctx, int src, cudaStream_t s) {
    StepArgs a = step_args(ctx, src);
    void* params[] = {&a};
    const int block = ctx->shape.kind >= 1 ? smem_block_threads(ctx->shape.kind - 1)
                                           : ctx->shape.tw * ctx->shape.th;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctx->grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = ctx->smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, ctx->kern, params);
}

// Median of three timed launches of the current shape (after one untimed
// launch) on the rest-state buffers, in milliseconds; < 0 on a CUDA error.
float time_current_shape(lbm_ctx* ctx, cudaEvent_t* ev) {
    // one warm-up launch, then twice three back-to-back launches (as the
    // step loop runs them: a launch's tail overlaps the next one's start);
    // the faster of the two, per launch
    if (launch_step(ctx, 0, ctx->stream) != cudaSuccess) return -1.f;
    int src = 1;
    float t[2];
    for (int r = 0; r < 2; ++r) {
        if (cudaEventRecord(ev[2 * r], ctx->stream) != cudaSuccess) return -1.f;
        for (int k = 0; k < 3; ++k, src ^= 1)
            if (launch_step(ctx, src, ctx->stream) != cudaSuccess) return -1.f;
        if (cudaEventRecord(ev[2 * r + 1], ctx->stream) != cudaSuccess) return -1.f;
    }
    if (cudaEventSynchronize(ev[3]) != cudaSuccess) return -1.f;
    for (int r = 0; r < 2; ++r)
        if (cudaEventElapsedTime(&t[r], ev[2 * r], ev[2 * r + 1]) != cudaSuccess) return -1.f;
    return std::min(t[0], t[1]) / 3.f;
}

// The same timing through a captured graph of four launches, as the step
// loop replays them: one warm-up replay, then the faster of two, per launch.
// The deep ring with FP32 storage ran 5 % slower in graphs than as single
// launches (the 10-warp CTAs did not), so close calls are decided here.
float time_current_shape_graph(lbm_ctx* ctx, cudaEvent_t* ev) {
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return -1.f;
    bool ok = true;
    for (int k = 0; k < 4; ++k) ok = ok && launch_step(ctx, k & 1, ctx->capture_stream) == cudaSuccess;
    if (cudaStreamEndCapture(ctx->capture_stream, &graph) != cudaSuccess || !ok) return -1.f;
    cudaGraphExec_t g = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&g, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return -1.f;
    float t[2] = {-1.f, -1.f};
    ok = cudaGraphLaunch(g, ctx->stream) == cudaSuccess;
    for (int r = 0; r < 2 && ok; ++r)
        ok = cudaEventRecord(ev[2 * r], ctx->stream) == cudaSuccess &&
             cudaGraphLaunch(g, ctx->stream) == cudaSuccess &&
             cudaEventRecord(ev[2 * r + 1], ctx->stream) == cudaSuccess;
    ok = ok && cudaEventSynchronize(ev[3]) == cudaSuccess;
    for (int r = 0; r < 2 && ok; ++r)
        ok = cudaEventElapsedTime(&t[r], ev[2 * r], ev[2 * r + 1]) == cudaSuccess;
    cudaGraphExecDestroy(g);
    return ok ? std::min(t[0], t[1]) / 4.f : -1.f;
}

// Autotuner cache: the chosen shape per (device, lattice, types, rule,
// boundary, instance sizes).  Kept for the life of the process, and in the
// text file named by LBM_AUTOTUNE_CACHE when that variable is set (one line
// per key: "<key> V tw th kind"), so that a later process -- a profiler run,
// for instance -- takes the same shape without timing anything.
std::mutex g_tune_mu;
std::map<std::string, Shape>& tune_cache() {
    static std::map<std::string, Shape> m;
    return m;
}

std::string tune_key(const lbm_ctx* ctx) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    std::string name = "?";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char& c : name)
        if (c == ' ') c = '_';
    // sizes as a sorted histogram, hashed (FNV-1a)
    std::vector<std::pair<int64_t, int64_t>> d;
    for (const InstDesc& in : ctx->layout.inst) d.push_back({in.nx, in.ny});
    std::sort(d.begin(), d.end());
    uint64_t h = 1469598103934665603ull;
    for (auto& p : d)
        for (int64_t v : {p.first, p.second}) {
            h ^= (uint64_t)v;
            h *= 1099511628211ull;
        }
    char buf[256];
    snprintf(buf, sizeof buf, "%s/sm%d/lat%d/st%d/cp%d/co%d/bc%d/n%d/%016llx", name.c_str(),
             ctx->num_sms, ctx->lattice, ctx->storage, ctx->compute, ctx->collision, ctx->bc,
             ctx->count, (unsigned long long)h);
    return buf;
}

bool tune_lookup(const std::string& key, Shape* s) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) {
        *s = it->second;
        return true;
    }
    const char* path = getenv("LBM_AUTOTUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char k[256];
    Shape t{};
    bool found = false;
    while (fscanf(f, "%255s %d %d %d %d", k, &t.V, &t.tw, &t.th, &t.kind) == 5) {
        if (key == k) {
            *s = t;
            found = true;  // the last entry for a key wins
        }
    }
    fclose(f);
    if (found) tune_cache()[key] = *s;
    return found;
}

void tune_store(const std::string& key, const Shape& s) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache()[key] = s;
    const char* path = getenv("LBM_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d\n", key.c_str(), s.V, s.tw, s.th, s.kind);
    fclose(f);
}

// Keep the fastest candidate shape: each is timed over back-to-back
// launches on the rest-state buffers (the collision's instruction stream
// does not depend on the data); the ones within 5 % of the fastest are
// timed again in a captured graph, which decides.  Then the buffers and
// counters are cleared.  A shape found in the cache is applied without
// timing.
int autotune(lbm_ctx* ctx) {
    const std::string key = tune_key(ctx);
    Shape cached;
    if (tune_lookup(key, &cached) && apply_shape(ctx, cached) == LBM_OK) return LBM_OK;
    std::vector<Shape> cands = candidate_shapes(ctx->lattice, ctx->storage, ctx->layout.max_nx,
                                                ctx->layout.max_ny);
    cudaEvent_t ev[6];
    for (int i = 0; i < 6; ++i) LBM_CK(cudaEventCreate(&ev[i]));
    float best = 1e30f;
    Shape best_s = default_shape(ctx->lattice, ctx->storage);
    int rc = LBM_OK;
    std::vector<float> t(cands.size(), -1.f);
    for (size_t c = 0; c < cands.size(); ++c) {
        if (apply_shape(ctx, cands[c]) != LBM_OK) continue;
        const float ms = time_current_shape(ctx, ev);
        if (ms < 0.f) {
            rc = LBM_ERR_CUDA;
            break;
        }
        t[c] = ms;
        best = std::min(best, ms);
    }
    // The candidates within 5 % of the fastest are timed once more, after
    // the others, through a captured graph as the step loop runs them, and
    // that time decides between them.
    std::vector<float> tg(cands.size(), -1.f);
    for (size_t c = 0; c < cands.size() && rc == LBM_OK; ++c) {
        if (t[c] < 0.f || t[c] > 1.05f * best) continue;
        if (apply_shape(ctx, cands[c]) != LBM_OK) continue;
        const float ms = time_current_shape_graph(ctx, ev);
        if (ms < 0.f) {
            rc = LBM_ERR_CUDA;
            break;
        }
        tg[c] = ms;
    }
    best = 1e30f;
    for (size_t c = 0; c < cands.size(); ++c) {
        if (getenv("LBM_DEBUG"))
            fprintf(stderr, "liblbm: autotune kind %d V %d tw %d th %d: %.4f ms per launch, %.4f in a graph\n",
                    cands[c].kind, cands[c].V, cands[c].tw, cands[c].th, t[c], tg[c]);
        if (tg[c] >= 0.f && tg[c] < best) {  // only the close call's graph times compete
            best = tg[c];
            best_s = cands[c];
        }
    }
    for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
    if (rc != LBM_OK) {
        ctx->failed = true;
        return rc;
    }
    // undo the tuning steps: back to the rest state, counters cleared
    LBM_CK(cudaMemsetAsync(ctx->buf[0], 0, 2 * ctx->cv.buf_bytes, ctx->stream));
    LBM_CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned long long) * 2 * ctx->count,
                           ctx->stream));
    rc = apply_shape(ctx, best_s);
    if (rc == LBM_OK) tune_store(key, best_s);
    return rc;
}

// Capture the step loop of GRAPH_STEPS launches for both buffer parities and
// upload the executable graphs, so that no capture or first-launch upload
// happens inside a later lbm_step.
int capture_graphs(lbm_ctx* ctx) {
    for (int p = 0; p < 2; ++p) {
        cudaGraphExec_t& g = ctx->graph[p];
        if (g) continue;
        cudaGraph_t graph;
        LBM_CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        int src = p;
        for (int k = 0; k < GRAPH_STEPS; ++k) {
            cudaError_t e = launch_step(ctx, src, ctx->capture_stream);
            if (e != cudaSuccess) {
                cudaStreamEndCapture(ctx->capture_stream, &graph);
                LBM_CK(e);
            }
            src = 1 - src;
        }
        LBM_CK(cudaStreamEndCapture(ctx->capture_stream, &graph));
        cudaError_t e = cudaGraphInstantiate(&g, graph, 0);
        cudaGraphDestroy(graph);
        LBM_CK(e);
        LBM_CK(cudaGraphUpload(g, ctx->stream));
    }
    return LBM_OK;
}

bool parse_shape_env(Shape* s) {
    const char* e = getenv("LBM_SHAPE");
    if (!e) return false;
    if (strcmp(e, "smem") == 0 || strcmp(e, "smem2") == 0) {
        *s = {2, 0, 0, 1};
        return true;
    }
    if (strcmp(e, "smems") == 0) {
        *s = {2, 0, 0, 2};
        return true;
    }
    if (strcmp(e, "smemw") == 0) {
        *s = {2, 0, 0, 3};
        return true;
    }
    if (strcmp(e, "smemd") == 0) {
        *s = {2, 0, 0, 4};
        return true;
    }

    int v, tw, th;
    if (sscanf(e, "%d,%d,%d", &v, &tw, &th) != 3) return false;
    *s = {v, tw, th};
    return true;
}

void lid_deviation(double rho0, double u, double* dev) {
    // f^eq_a(rho0, (u, 0)) - W_a rho0, Eq. (numerical-plyeqm); D2Q9 in T's column order.
    static const int vx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    for (int a = 0; a < 9; ++a) {
        const double w = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        const double vu = vx[a] * u;
        dev[a] = w * rho0 * (3.0 * vu + 4.5 * vu * vu - 1.5 * u * u);
    }
}

int validate_opts(const lbm_opts* o) {
    if (o->compute != DT_F64 && o->compute != DT_F32) return LBM_ERR_ARG;
    if (o->storage < DT_F64 || o->storage > DT_BF16) return LBM_ERR_ARG;
    if (o->compute == DT_F64 && o->storage != DT_F64) return LBM_ERR_ARG;
    if (o->compute == DT_F32 && o->storage == DT_F64) return LBM_ERR_ARG;
    if (o->collision < COLL_MINXENT4 || o->collision > COLL_TRT) return LBM_ERR_ARG;
    if (o->tau2_reading != TAU2_PRINTED && o->tau2_reading != TAU2_MAGIC) return LBM_ERR_ARG;
    if (o->reserved != 0) return LBM_ERR_ARG;
    if (!(o->rho0 > 0.0) || !std::isfinite(o->rho0)) return LBM_ERR_ARG;
    return LBM_OK;
}

int validate_dims(int lat, int32_t count, const int64_t* dims,
                  std::vector<std::pair<int64_t, int64_t>>* out) {
    if (lat != 1 && lat != 2) return LBM_ERR_ARG;
    if (count < 1 || count > 65535 || !dims) return LBM_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        const int64_t nx = dims[2 * i], ny = dims[2 * i + 1];
        if (nx < 1 || ny < 1 || nx > (1 << 26) || ny > (1 << 26)) return LBM_ERR_ARG;
        if (lat == 1 && ny != 1) return LBM_ERR_ARG;
        if (nx * ny > ((int64_t)1 << 31)) return LBM_ERR_ARG;
        out->push_back({nx, ny});
    }
    return LBM_OK;
}

// Device address of a host array the GPU can read and write in place
// (page-locked memory registered with CUDA: cudaHostAlloc, cudaHostRegister,
// torch's pin_memory), or nullptr.  A null array counts as addressable.
// Host I/O with such arrays runs its kernels straight on them, without
// staging copies: on a GB300 the kernel streams them over the CPU-GPU link.
template <typename P> bool device_view(P* host, P** dev) {
    if (!host) {
        *dev = nullptr;
        return true;
    }
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return false;
    *dev = static_cast<P*>(at.devicePointer);
    return true;
}

// Auxiliary-kernel arguments that cover instance i alone, with host arrays
// indexed from its first node.
AuxArgs aux_args_instance(const lbm_ctx* ctx, int i) {
    AuxArgs a = aux_args(ctx);
    const InstDesc& in = ctx->layout.inst[i];
    a.inst = ctx->d_inst + i;
    a.count = 1;
    a.max_nodes = (int64_t)in.nx * in.ny;
    a.node_base = in.node0;
    return a;
}

// Header of a saved state (lbm_save_state): the layout it fits and the
// context's position in its run, followed by the status counters and the
// raw population buffer.
struct StateHeader {
    char magic[8];
    uint32_t version;
    int32_t lattice, storage, count;
    int32_t post, reserved;
    int64_t steps;
    uint64_t layout_hash, buf_bytes, status_bytes;
    uint64_t pad[8];
};
static_assert(sizeof(StateHeader) == 128, "state header is 128 bytes");
constexpr char STATE_MAGIC[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', 'E'};

uint64_t layout_hash(const lbm_ctx* ctx) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        h ^= v;
        h *= 1099511628211ull;
    };
    mix((uint64_t)ctx->lattice);
    mix((uint64_t)ctx->storage);
    for (const InstDesc& in : ctx->layout.inst) {
        mix((uint64_t)in.nx);
        mix((uint64_t)in.ny);
        mix((uint64_t)in.pitch);
        mix((uint64_t)in.plane);
        mix((uint64_t)in.off);
    }
    return h;
}

// LBM_ERR_UNSTABLE when instance i has flagged an unstable node (sticky
// error word first); syncs.
int instance_status(lbm_ctx* ctx, int32_t instance) {
    int64_t c[3];
    int rc = lbm_status_instance(ctx, instance, c);
    if (rc != LBM_OK) return rc;
    unsigned int err = 0;
    LBM_CK(cudaMemcpyAsync(&err, ctx->d_error, sizeof err, cudaMemcpyDeviceToHost, ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    if (err) return LBM_ERR_TIMEOUT;
    return c[1] ? LBM_ERR_UNSTABLE : LBM_OK;
}

uint64_t state_bytes(const lbm_ctx* ctx) {
    return sizeof(StateHeader) + sizeof(unsigned long long) * 2 * (uint64_t)ctx->count +
           (uint64_t)ctx->cv.buf_bytes;
}

}  // namespace

namespace lbm {
// Inputs of the conservation reduction of a context, for entry points that
// live in other translation units.  Returns LBM_OK, or the code the public
// conservation call would return for this context.
int ctx_conservation_inputs(const lbm_ctx* ctx, AuxArgs* args, const void** src, int* count) {
    if (!ctx) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    if (!ctx->initialized) return LBM_ERR_STATE;
    *args = aux_args(ctx);
    *src = ctx->buf[ctx->cur];
    *count = ctx->count;
    return LBM_OK;
}
}  // namespace lbm

extern "C" {

void lbm_default_opts(lbm_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->compute = DT_F64;
    o->storage = DT_F64;
    o->collision = COLL_MINXENT4;
    o->autotune = 1;
    o->rho0 = 1.0;
}

int lbm_required_bytes(lbm_lattice lat, int32_t count, const int64_t* dims, const lbm_opts* opts,
                       uint64_t* bytes) {
    if (!bytes) return LBM_ERR_ARG;
    lbm_opts o;
    if (opts) o = *opts;
    else lbm_default_opts(&o);
    if (validate_opts(&o) != LBM_OK) return LBM_ERR_ARG;
    std::vector<std::pair<int64_t, int64_t>> d;
    if (validate_dims(lat, count, dims, &d) != LBM_OK) return LBM_ERR_ARG;
    Layout L = make_layout(lat, o.storage, d);
    *bytes = carve(L, lat, o.storage, count).total;
    return LBM_OK;
}

int lbm_create_batch(lbm_ctx** out, lbm_lattice lat, int32_t count, const int64_t* dims,
                     const double* nu, const double* u_lid, lbm_bc bc, const lbm_opts* opts) {
    lbm_ctx* ctx = nullptr;
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    lbm_opts o;
    if (opts) o = *opts;
    else lbm_default_opts(&o);
    if (validate_opts(&o) != LBM_OK) return LBM_ERR_ARG;
    std::vector<std::pair<int64_t, int64_t>> d;
    if (validate_dims(lat, count, dims, &d) != LBM_OK || !nu) return LBM_ERR_ARG;
    if (bc != LBM_BC_PERIODIC && bc != LBM_BC_ZERO_GRADIENT && bc != LBM_BC_CAVITY)
        return LBM_ERR_ARG;
    if (bc == LBM_BC_CAVITY) {
        if (lat != LBM_D2Q9) return LBM_ERR_ARG;
        for (auto& p : d)
            if (p.first < 3 || p.second < 3) return LBM_ERR_ARG;
    }
    for (int i = 0; i < count; ++i) {
        // Eq. (visco-tau): tau = 3 nu + 1/2 must exceed 1/2
        if (!(nu[i] > 0.0) || !std::isfinite(nu[i])) return LBM_ERR_ARG;
        if (u_lid && !std::isfinite(u_lid[i])) return LBM_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_NODEV;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return LBM_ERR_NODEV;
    if (prop.major != 10 || prop.minor != 3) return LBM_ERR_NODEV;

    ctx = new lbm_ctx();
    ctx->lattice = lat;
    ctx->Q = lat == LBM_D2Q9 ? 9 : 3;
    ctx->count = count;
    ctx->bc = bc;
    ctx->compute = o.compute;
    ctx->storage = o.storage;
    ctx->collision = o.collision;
    ctx->rho0 = o.rho0;
    ctx->stream = static_cast<cudaStream_t>(o.stream);
    ctx->num_sms = prop.multiProcessorCount;
    // Test hooks of the bounded-wait timeout path (TMA kernel): a smaller
    // spin limit, and one tile whose copies are never issued.
    if (const char* e = getenv("LBM_SPIN_LIMIT")) {
        const long v = strtol(e, nullptr, 10);
        if (v >= 1 && v <= (1 << 20)) ctx->spin_limit = (int)v;
    }
    if (const char* e = getenv("LBM_TEST_LOST_TILE")) ctx->lost_tile = (int)strtol(e, nullptr, 10);
    ctx->layout = make_layout(lat, o.storage, d);
    ctx->cv = carve(ctx->layout, lat, o.storage, count);
    for (int i = 0; i < count; ++i) {
        InstDesc& in = ctx->layout.inst[i];
        const double tau = 3.0 * nu[i] + 0.5;
        in.bc = bc;
        in.omega = 1.0 / tau;
        // Eq. (tau2), as printed or in the magic-parameter reading
        const double tau2 = (8.0 * tau - 1.0) /
                            ((o.tau2_reading == TAU2_MAGIC ? 8.0 : 1.0) * (2.0 * tau - 1.0));
        in.omega2 = 1.0 / tau2;
        // Table III: MRT fixes the energy rates, TRT uses 1/tau for them
        in.s_e = o.collision == COLL_MRT ? 1.64 : in.omega;
        in.s_eps = o.collision == COLL_MRT ? 1.54 : in.omega;
        in.u_lid = u_lid ? u_lid[i] : 0.0;
        in.rates_f[0] = (float)in.omega;
        in.rates_f[1] = (float)in.omega2;
        in.rates_f[2] = (float)in.s_e;
        in.rates_f[3] = (float)in.s_eps;
        if (bc == LBM_BC_CAVITY) {
            lid_deviation(o.rho0, in.u_lid, in.lid_dev);
            for (int a = 0; a < 9; ++a) in.lid_dev_f[a] = (float)in.lid_dev[a];
        }
    }
    int rc = LBM_OK;
    if (o.device_mem) {
        if (o.device_mem_bytes < ctx->cv.total || ((uintptr_t)o.device_mem & 255u)) {
            delete ctx;
            return LBM_ERR_ARG;
        }
        ctx->mem = static_cast<char*>(o.device_mem);
    } else {
        void* p = nullptr;
        if (cudaMalloc(&p, ctx->cv.total) != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return LBM_ERR_ALLOC;
        }
        ctx->mem = static_cast<char*>(p);
        ctx->own_mem = true;
    }
    ctx->buf[0] = ctx->mem;
    ctx->buf[1] = ctx->mem + ctx->cv.buf_bytes;
    ctx->d_inst = reinterpret_cast<InstDesc*>(ctx->mem + ctx->cv.inst_off);
    ctx->d_tiles = reinterpret_cast<TileDesc*>(ctx->mem + ctx->cv.tiles_off);
    ctx->d_status = reinterpret_cast<unsigned long long*>(ctx->mem + ctx->cv.status_off);
    ctx->d_partials = reinterpret_cast<double*>(ctx->mem + ctx->cv.partials_off);
    ctx->d_cons = reinterpret_cast<int2*>(ctx->mem + ctx->cv.cons_off);
    ctx->d_stage = reinterpret_cast<double*>(ctx->mem + ctx->cv.stage_off);
    ctx->d_tmaps = reinterpret_cast<CUtensorMapOpaque*>(ctx->mem + ctx->cv.tmap_off);
    ctx->d_error = reinterpret_cast<unsigned int*>(ctx->mem + ctx->cv.err_off);
    auto fail = [&](int code) {
        lbm_destroy(ctx);
        return code;
    };
    if (cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(LBM_ERR_CUDA);
    if (cudaMemsetAsync(ctx->mem, 0, ctx->cv.total, ctx->stream) != cudaSuccess)
        return fail(LBM_ERR_CUDA);
    {
        std::vector<int2> items;
        for (int i = 0; i < count; ++i)
            for (int b = 0; b < cons_partials(ctx->layout.inst[i].ny); ++b) items.push_back({i, b});
        ctx->n_cons = (int)items.size();
        if (cudaMemcpyAsync(ctx->d_cons, items.data(), sizeof(int2) * items.size(),
                            cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            return fail(LBM_ERR_CUDA);
    }
    Shape s;
    if (parse_shape_env(&s)) rc = apply_shape(ctx, s);
    else if (o.autotune && !getenv("LBM_NO_AUTOTUNE")) rc = autotune(ctx);
    else rc = apply_shape(ctx, default_shape(lat, o.storage));
    if (rc != LBM_OK) return fail(rc);
    rc = capture_graphs(ctx);
    if (rc != LBM_OK) return fail(rc);
    *out = ctx;
    return LBM_OK;
}

int lbm_create(lbm_ctx** out, lbm_lattice lat, const int64_t* dims, double nu, lbm_bc bc,
               double u_lid, const lbm_opts* opts) {
    return lbm_create_batch(out, lat, 1, dims, &nu, &u_lid, bc, opts);
}

int lbm_destroy(lbm_ctx* ctx) {
    if (!ctx) return LBM_OK;
    for (int p = 0; p < 2; ++p)
        if (ctx->graph[p]) cudaGraphExecDestroy(ctx->graph[p]);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->own_mem && ctx->mem) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->mem);
    }
    delete ctx;
    return LBM_OK;
}

int lbm_init_device(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy) {
    if (!ctx || !rho) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    AuxArgs a = aux_args(ctx);
    LBM_CK(run_aux(AuxOp::Init, a, nullptr, ctx->buf[ctx->cur], rho, ux, uy, nullptr, nullptr,
                   nullptr));
    LBM_CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned long long) * 2 * ctx->count,
                           ctx->stream));
    LBM_CK(cudaMemsetAsync(ctx->d_error, 0, sizeof(unsigned int), ctx->stream));
    ctx->post = false;
    ctx->initialized = true;
    ctx->inst_init.assign(ctx->count, 1);
    ctx->steps = 0;
    return LBM_OK;
}

int lbm_init(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy) {
    if (!ctx || !rho) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    const double *dr, *dx, *dy;
    if (device_view(rho, &dr) && device_view(ux, &dx) && device_view(uy, &dy)) {
        // page-locked arrays: the init kernel reads them in place
        int rc = lbm_init_device(ctx, dr, dx, ctx->Q == 9 ? dy : nullptr);
        if (rc != LBM_OK) return rc;
        LBM_CK(cudaStreamSynchronize(ctx->stream));
        return LBM_OK;
    }
    const size_t n = (size_t)ctx->layout.total_nodes;
    double* r = ctx->d_stage;
    double* x = ux ? ctx->d_stage + n : nullptr;
    double* y = (uy && ctx->Q == 9) ? ctx->d_stage + 2 * n : nullptr;
    LBM_CK(cudaMemcpyAsync(r, rho, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (x) LBM_CK(cudaMemcpyAsync(x, ux, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (y) LBM_CK(cudaMemcpyAsync(y, uy, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    int rc = lbm_init_device(ctx, r, x, y);
    if (rc != LBM_OK) return rc;
    // the caller may reuse its arrays once we return
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

int lbm_step(lbm_ctx* ctx, int64_t n) {
    if (!ctx || n < 0) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    if (!ctx->initialized) return LBM_ERR_STATE;
    if (n == 0) return LBM_OK;
    if (!ctx->post) {
        AuxArgs a = aux_args(ctx);
        LBM_CK(run_aux(AuxOp::CollideInPlace, a, ctx->buf[ctx->cur], ctx->buf[1 - ctx->cur],
                       nullptr, nullptr, nullptr, nullptr, nullptr, nullptr));
        ctx->cur = 1 - ctx->cur;
        ctx->post = true;
        ctx->steps += 1;
        --n;
    }
    while (n >= GRAPH_STEPS) {
        cudaGraphExec_t& g = ctx->graph[ctx->cur];
        if (!g) {
            const int rc = capture_graphs(ctx);
            if (rc != LBM_OK) return rc;
        }
        LBM_CK(cudaGraphLaunch(g, ctx->stream));
        n -= GRAPH_STEPS;
        ctx->steps += GRAPH_STEPS;
    }
    for (; n > 0; --n) {
        LBM_CK(launch_step(ctx, ctx->cur, ctx->stream));
        ctx->cur = 1 - ctx->cur;
        ctx->steps += 1;
    }
    return LBM_OK;
}

int lbm_moments_device(lbm_ctx* ctx, double* rho, double* ux, double* uy) {
    if (!ctx || !rho) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    if (!ctx->initialized) return LBM_ERR_STATE;
    AuxArgs a = aux_args(ctx);
    LBM_CK(run_aux(AuxOp::Moments, a, ctx->buf[ctx->cur], nullptr, nullptr, nullptr, nullptr, rho,
                   ux, ctx->Q == 9 ? uy : nullptr));
    return LBM_OK;
}

int lbm_stream_function_device(lbm_ctx* ctx, double* psi) {
    if (!ctx || !psi) return LBM_ERR_ARG;
    if (ctx->Q != 9) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    if (!ctx->initialized) return LBM_ERR_STATE;
    const size_t n = (size_t)ctx->layout.total_nodes;
    AuxArgs a = aux_args(ctx);
    // u_y of f(t_n) into the staging area (rho and u_x beside it), then the
    // row integrals
    LBM_CK(run_aux(AuxOp::Moments, a, ctx->buf[ctx->cur], nullptr, nullptr, nullptr, nullptr,
                   ctx->d_stage, ctx->d_stage + n, ctx->d_stage + 2 * n));
    LBM_CK(stream_function(a, ctx->layout.max_ny, ctx->d_stage + 2 * n, psi));
    return LBM_OK;
}

int lbm_stream_function(lbm_ctx* ctx, double* psi) {
    if (!ctx || !psi) return LBM_ERR_ARG;
    const size_t n = (size_t)ctx->layout.total_nodes;
    double* dpsi = ctx->d_stage + 3 * n;
    int rc = lbm_stream_function_device(ctx, dpsi);
    if (rc != LBM_OK) return rc;
    LBM_CK(cudaMemcpyAsync(psi, dpsi, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    int64_t c[3];
    rc = lbm_status(ctx, c);
    if (rc != LBM_OK) return rc;
    return c[1] ? LBM_ERR_UNSTABLE : LBM_OK;
}

int lbm_status_instance(lbm_ctx* ctx, int32_t instance, int64_t* counters) {
    if (!ctx || !counters || instance < 0 || instance >= ctx->count) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    unsigned long long h[2];
    LBM_CK(cudaMemcpyAsync(h, ctx->d_status + 2 * instance, sizeof h, cudaMemcpyDeviceToHost,
                           ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    counters[0] = (int64_t)h[0];
    counters[1] = (int64_t)h[1];
    counters[2] = ctx->steps;
    return LBM_OK;
}

int lbm_status(lbm_ctx* ctx, int64_t* counters) {
    if (!ctx || !counters) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    std::vector<unsigned long long> h(2 * (size_t)ctx->count);
    LBM_CK(cudaMemcpyAsync(h.data(), ctx->d_status, sizeof(unsigned long long) * h.size(),
                           cudaMemcpyDeviceToHost, ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    counters[0] = counters[1] = 0;
    for (int i = 0; i < ctx->count; ++i) {
        counters[0] += (int64_t)h[2 * i];
        counters[1] += (int64_t)h[2 * i + 1];
    }
    counters[2] = ctx->steps;
    unsigned int err = 0;
    LBM_CK(cudaMemcpyAsync(&err, ctx->d_error, sizeof err, cudaMemcpyDeviceToHost, ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    return err ? LBM_ERR_TIMEOUT : LBM_OK;
}

int lbm_moments(lbm_ctx* ctx, double* rho, double* ux, double* uy) {
    if (!ctx || !rho) return LBM_ERR_ARG;
    double *hr, *hx, *hy;
    if (device_view(rho, &hr) && device_view(ux, &hx) && device_view(uy, &hy)) {
        // page-locked arrays: the moments kernel writes them in place
        int rc = lbm_moments_device(ctx, hr, hx, hy);
        if (rc != LBM_OK) return rc;
    } else {
        const size_t n = (size_t)ctx->layout.total_nodes;
        double* r = ctx->d_stage;
        double* x = ctx->d_stage + n;
        double* y = ctx->d_stage + 2 * n;
        int rc = lbm_moments_device(ctx, r, x, y);
        if (rc != LBM_OK) return rc;
        LBM_CK(cudaMemcpyAsync(rho, r, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        if (ux)
            LBM_CK(cudaMemcpyAsync(ux, x, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        if (uy && ctx->Q == 9)
            LBM_CK(cudaMemcpyAsync(uy, y, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    int rc;
    int64_t c[3];
    rc = lbm_status(ctx, c);
    if (rc != LBM_OK) return rc;
    return c[1] ? LBM_ERR_UNSTABLE : LBM_OK;
}

int lbm_get_populations(lbm_ctx* ctx, double* f) {
    if (!ctx || !f) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    if (!ctx->initialized) return LBM_ERR_STATE;
    const size_t n = (size_t)ctx->layout.total_nodes * ctx->Q;
    AuxArgs a = aux_args(ctx);
    LBM_CK(run_aux(AuxOp::GatherF, a, ctx->buf[ctx->cur], nullptr, nullptr, nullptr, nullptr,
                   ctx->d_stage, nullptr, nullptr));
    LBM_CK(cudaMemcpyAsync(f, ctx->d_stage, n * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

int lbm_set_populations(lbm_ctx* ctx, const double* f) {
    if (!ctx || !f) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    const size_t n = (size_t)ctx->layout.total_nodes * ctx->Q;
    LBM_CK(cudaMemcpyAsync(ctx->d_stage, f, n * sizeof(double), cudaMemcpyHostToDevice,
                           ctx->stream));
    AuxArgs a = aux_args(ctx);
    LBM_CK(run_aux(AuxOp::SetF, a, nullptr, ctx->buf[ctx->cur], ctx->d_stage, nullptr, nullptr,
                   nullptr, nullptr, nullptr));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    ctx->post = false;
    ctx->initialized = true;
    ctx->inst_init.assign(ctx->count, 1);
    return LBM_OK;
}

int lbm_conservation(lbm_ctx* ctx, double* out) {
    if (!ctx || !out) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    if (!ctx->initialized) return LBM_ERR_STATE;
    AuxArgs a = aux_args(ctx);
    LBM_CK(run_aux(AuxOp::Conservation, a, ctx->buf[ctx->cur], nullptr, nullptr, nullptr, nullptr,
                   ctx->d_stage, ctx->d_partials, nullptr));
    LBM_CK(cudaMemcpyAsync(out, ctx->d_stage, sizeof(double) * 3 * ctx->count,
                           cudaMemcpyDeviceToHost, ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

int lbm_conservation_device(lbm_ctx* ctx, double* out) {
    if (!ctx || !out) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    if (!ctx->initialized) return LBM_ERR_STATE;
    AuxArgs a = aux_args(ctx);
    LBM_CK(run_aux(AuxOp::Conservation, a, ctx->buf[ctx->cur], nullptr, nullptr, nullptr, nullptr,
                   out, ctx->d_partials, nullptr));
    return LBM_OK;
}

int lbm_init_batch(lbm_ctx* ctx, int32_t instance, const double* rho, const double* ux,
                   const double* uy) {
    if (!ctx || !rho || instance < 0 || instance >= ctx->count) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    if (ctx->post) return LBM_ERR_STATE;  // mid-run: the stored field is post-collision
    const InstDesc& in = ctx->layout.inst[instance];
    const size_t n = (size_t)in.nx * in.ny;
    double* r = ctx->d_stage;
    double* x = ux ? ctx->d_stage + n : nullptr;
    double* y = (uy && ctx->Q == 9) ? ctx->d_stage + 2 * n : nullptr;
    LBM_CK(cudaMemcpyAsync(r, rho, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (x) LBM_CK(cudaMemcpyAsync(x, ux, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (y) LBM_CK(cudaMemcpyAsync(y, uy, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    AuxArgs a = aux_args_instance(ctx, instance);
    LBM_CK(run_aux(AuxOp::Init, a, nullptr, ctx->buf[ctx->cur], r, x, y, nullptr, nullptr,
                   nullptr));
    LBM_CK(cudaMemsetAsync(ctx->d_status + 2 * instance, 0, 2 * sizeof(unsigned long long),
                           ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->inst_init.size() != (size_t)ctx->count) ctx->inst_init.assign(ctx->count, 0);
    ctx->inst_init[instance] = 1;
    if (!ctx->initialized &&
        std::all_of(ctx->inst_init.begin(), ctx->inst_init.end(), [](uint8_t v) { return v; })) {
        LBM_CK(cudaMemsetAsync(ctx->d_error, 0, sizeof(unsigned int), ctx->stream));
        LBM_CK(cudaStreamSynchronize(ctx->stream));
        ctx->initialized = true;
        ctx->steps = 0;
    }
    return LBM_OK;
}

int lbm_moments_batch_device(lbm_ctx* ctx, int32_t instance, double* rho, double* ux, double* uy) {
    if (!ctx || !rho || instance < 0 || instance >= ctx->count) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    if (!ctx->initialized) return LBM_ERR_STATE;
    AuxArgs a = aux_args_instance(ctx, instance);
    LBM_CK(run_aux(AuxOp::Moments, a, ctx->buf[ctx->cur], nullptr, nullptr, nullptr, nullptr, rho,
                   ux, ctx->Q == 9 ? uy : nullptr));
    return LBM_OK;
}

int lbm_moments_batch(lbm_ctx* ctx, int32_t instance, double* rho, double* ux, double* uy) {
    if (!ctx || !rho || instance < 0 || instance >= ctx->count) return LBM_ERR_ARG;
    const InstDesc& in = ctx->layout.inst[instance];
    const size_t n = (size_t)in.nx * in.ny;
    double* r = ctx->d_stage;
    double* x = ctx->d_stage + n;
    double* y = ctx->d_stage + 2 * n;
    int rc = lbm_moments_batch_device(ctx, instance, r, x, y);
    if (rc != LBM_OK) return rc;
    LBM_CK(cudaMemcpyAsync(rho, r, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (ux) LBM_CK(cudaMemcpyAsync(ux, x, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (uy && ctx->Q == 9)
        LBM_CK(cudaMemcpyAsync(uy, y, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    return instance_status(ctx, instance);
}

int lbm_stream_function_batch(lbm_ctx* ctx, int32_t instance, double* psi) {
    if (!ctx || !psi || instance < 0 || instance >= ctx->count) return LBM_ERR_ARG;
    if (ctx->Q != 9) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    if (!ctx->initialized) return LBM_ERR_STATE;
    const InstDesc& in = ctx->layout.inst[instance];
    const size_t n = (size_t)in.nx * in.ny;
    AuxArgs a = aux_args_instance(ctx, instance);
    LBM_CK(run_aux(AuxOp::Moments, a, ctx->buf[ctx->cur], nullptr, nullptr, nullptr, nullptr,
                   ctx->d_stage, ctx->d_stage + n, ctx->d_stage + 2 * n));
    LBM_CK(stream_function(a, in.ny, ctx->d_stage + 2 * n, ctx->d_stage + 3 * n));
    LBM_CK(cudaMemcpyAsync(psi, ctx->d_stage + 3 * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    return instance_status(ctx, instance);
}

int lbm_state_bytes(lbm_ctx* ctx, uint64_t* bytes) {
    if (!ctx || !bytes) return LBM_ERR_ARG;
    *bytes = state_bytes(ctx);
    return LBM_OK;
}

int lbm_save_state(lbm_ctx* ctx, void* host_buf) {
    if (!ctx || !host_buf) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    if (!ctx->initialized) return LBM_ERR_STATE;
    StateHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, STATE_MAGIC, sizeof h.magic);
    h.version = 1;
    h.lattice = ctx->lattice;
    h.storage = ctx->storage;
    h.count = ctx->count;
    h.post = ctx->post ? 1 : 0;
    h.steps = ctx->steps;
    h.layout_hash = layout_hash(ctx);
    h.status_bytes = sizeof(unsigned long long) * 2 * (uint64_t)ctx->count;
    h.buf_bytes = ctx->cv.buf_bytes;
    char* out = static_cast<char*>(host_buf);
    std::memcpy(out, &h, sizeof h);
    LBM_CK(cudaMemcpyAsync(out + sizeof h, ctx->d_status, h.status_bytes, cudaMemcpyDeviceToHost,
                           ctx->stream));
    LBM_CK(cudaMemcpyAsync(out + sizeof h + h.status_bytes, ctx->buf[ctx->cur], h.buf_bytes,
                           cudaMemcpyDeviceToHost, ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

int lbm_load_state(lbm_ctx* ctx, const void* host_buf) {
    if (!ctx || !host_buf) return LBM_ERR_ARG;
    if (ctx->failed) return LBM_ERR_CUDA;
    StateHeader h;
    std::memcpy(&h, host_buf, sizeof h);
    if (std::memcmp(h.magic, STATE_MAGIC, sizeof h.magic) != 0 || h.version != 1 ||
        h.lattice != ctx->lattice || h.storage != ctx->storage || h.count != ctx->count ||
        h.layout_hash != layout_hash(ctx) || h.buf_bytes != ctx->cv.buf_bytes ||
        h.status_bytes != sizeof(unsigned long long) * 2 * (uint64_t)ctx->count)
        return LBM_ERR_ARG;
    const char* in = static_cast<const char*>(host_buf);
    LBM_CK(cudaMemcpyAsync(ctx->d_status, in + sizeof h, h.status_bytes, cudaMemcpyHostToDevice,
                           ctx->stream));
    LBM_CK(cudaMemcpyAsync(ctx->buf[0], in + sizeof h + h.status_bytes, h.buf_bytes,
                           cudaMemcpyHostToDevice, ctx->stream));
    LBM_CK(cudaMemsetAsync(ctx->d_error, 0, sizeof(unsigned int), ctx->stream));
    LBM_CK(cudaStreamSynchronize(ctx->stream));
    ctx->cur = 0;
    ctx->post = h.post != 0;
    ctx->steps = h.steps;
    ctx->initialized = true;
    ctx->inst_init.assign(ctx->count, 1);
    return LBM_OK;
}

int lbm_launch_shape(lbm_ctx* ctx, int32_t* out) {
    if (!ctx || !out) return LBM_ERR_ARG;
    out[0] = ctx->shape.V;
    out[1] = ctx->shape.tw;
    out[2] = ctx->shape.th;
    out[3] = ctx->grid;
    out[4] = ctx->shape.kind;
    return LBM_OK;
}

const char* lbm_status_string(int code) {
    switch (code) {
        case LBM_OK: return "ok";
        case LBM_ERR_ARG: return "invalid argument";
        case LBM_ERR_ALLOC: return "device memory allocation failed";
        case LBM_ERR_CUDA: return "CUDA runtime error";
        case LBM_ERR_UNSTABLE: return "unstable: negative or non-finite population";
        case LBM_ERR_STATE: return "call out of order (context not initialised)";
        case LBM_ERR_NODEV: return "no sm_103 CUDA device";
        case LBM_ERR_TIMEOUT: return "a bounded device-side wait ran out (data copy never completed)";
    }
    return "unknown status code";
}

}  // extern "C"
