// lbm_num.cuh -- arithmetic types of the collision kernels.
//
// The collision rules are written once over a number type T:
//   double  FP64 path: IEEE division, library log1p.
//   float   FP32 path, one node per value.
//   F2      FP32 path, two nodes per value: the packed FP32x2 instructions of
//           sm_100+ (__fadd2_rn, __fmul2_rn, __ffma2_rn) do both nodes in one
//           issue; reciprocals and logarithms run per lane on the MUFU unit.
//   F1      FP32, one node per value (the one-off in-place collision).
// The compiler may fuse a packed product whose only use is a following
// packed add into one packed FMA (it does so even for the _rn forms), which
// scalar __fmul_rn / __fadd_rn never are; so F1 and F2 agree to FP32
// rounding, not bit for bit.  All step kernels use F2 with the same
// collision code and agree bit for bit with each other.
//
// FP32 transcendental choice: ln(p/W) is needed as log(1 + delta) with
// |delta| < 1 typically; the FP32 path evaluates log2(1 + delta) with the
// hardware approximation (absolute error about 2^-22) and folds ln 2 into the
// final scale factor; reciprocals use the hardware approximation (about 1 ulp).
// Both errors stay at the FP32 rounding level of the populations (the tests
// bound the FP32 results against the FP64 oracle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct F2 {
    float2 v;
    F2() = default;
    __device__ __forceinline__ constexpr F2(float a) : v{a, a} {}
    __device__ __forceinline__ constexpr F2(float a, float b) : v{a, b} {}
    __device__ __forceinline__ F2(float2 a) : v(a) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
    return F2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y)));
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }

// Scalar FP32: every + - * rounds separately (__fadd_rn / __fmul_rn are
// never contracted into FMAs) and fused operations are explicit
// (Num<F1>::mad).
struct F1 {
    float v;
    F1() = default;
    __device__ __forceinline__ constexpr F1(float a) : v(a) {}
};
__device__ __forceinline__ F1 operator+(F1 a, F1 b) { return F1(__fadd_rn(a.v, b.v)); }
__device__ __forceinline__ F1 operator-(F1 a) { return F1(-a.v); }
__device__ __forceinline__ F1 operator-(F1 a, F1 b) { return F1(__fsub_rn(a.v, b.v)); }
__device__ __forceinline__ F1 operator*(F1 a, F1 b) { return F1(__fmul_rn(a.v, b.v)); }
__device__ __forceinline__ bool operator>=(F1 a, F1 b) { return a.v >= b.v; }
__device__ __forceinline__ bool operator<(F1 a, F1 b) { return a.v < b.v; }
__device__ __forceinline__ F1 fabs(F1 a) { return F1(fabsf(a.v)); }

// Per-lane predicate.
struct B2 {
    bool x, y;
};

template <typename T> struct Num;

template <> struct Num<double> {
    using Pred = bool;
    static constexpr int LANES = 1;
    static constexpr double LOG_SCALE = 1.0;  // log returns natural logs
    __device__ static __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
    __device__ static __forceinline__ double rcp(double x) { return 1.0 / x; }
    // ln(1 + delta), given delta and y = 1 + delta
    __device__ static __forceinline__ double lnp(double delta, double) { return log1p(delta); }
    __device__ static __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
    __device__ static __forceinline__ Pred gt(double a, double b) { return a > b; }
    __device__ static __forceinline__ double sel(Pred p, double a, double b) { return p ? a : b; }
    __device__ static __forceinline__ double lane(double v, int) { return v; }
    __device__ static __forceinline__ void set_lane(double& v, int, double x) { v = x; }
};

template <> struct Num<float> {
    using Pred = bool;
    static constexpr int LANES = 1;
    static constexpr float LOG_SCALE = 0.693147180559945309f;  // log returns log2
    __device__ static __forceinline__ float mad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    __device__ static __forceinline__ float rcp(float x) { return rcp_approx(x); }
    __device__ static __forceinline__ float lnp(float, float y) { return lg2_approx(y); }
    __device__ static __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
    __device__ static __forceinline__ Pred gt(float a, float b) { return a > b; }
    __device__ static __forceinline__ float sel(Pred p, float a, float b) { return p ? a : b; }
    __device__ static __forceinline__ float lane(float v, int) { return v; }
    __device__ static __forceinline__ void set_lane(float& v, int, float x) { v = x; }
};

template <> struct Num<F1> {
    using Pred = bool;
    static constexpr int LANES = 1;
    static constexpr float LOG_SCALE = 0.693147180559945309f;  // log returns log2
    __device__ static __forceinline__ F1 mad(F1 a, F1 b, F1 c) { return F1(__fmaf_rn(a.v, b.v, c.v)); }
    __device__ static __forceinline__ F1 rcp(F1 x) { return F1(rcp_approx(x.v)); }
    __device__ static __forceinline__ F1 lnp(F1, F1 y) { return F1(lg2_approx(y.v)); }
    __device__ static __forceinline__ F1 vmin(F1 a, F1 b) { return F1(fminf(a.v, b.v)); }
    __device__ static __forceinline__ Pred gt(F1 a, F1 b) { return a.v > b.v; }
    __device__ static __forceinline__ F1 sel(Pred p, F1 a, F1 b) { return p ? a : b; }
    __device__ static __forceinline__ float lane(F1 v, int) { return v.v; }
    __device__ static __forceinline__ void set_lane(F1& v, int, float x) { v.v = x; }
};

template <> struct Num<F2> {
    using Pred = B2;
    static constexpr int LANES = 2;
    static constexpr float LOG_SCALE = 0.693147180559945309f;
    __device__ static __forceinline__ F2 mad(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
    __device__ static __forceinline__ F2 rcp(F2 x) { return F2(rcp_approx(x.v.x), rcp_approx(x.v.y)); }
    __device__ static __forceinline__ F2 lnp(F2, F2 y) { return F2(lg2_approx(y.v.x), lg2_approx(y.v.y)); }
    __device__ static __forceinline__ F2 vmin(F2 a, F2 b) {
        return F2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y));
    }
    __device__ static __forceinline__ Pred gt(F2 a, F2 b) { return {a.v.x > b.v.x, a.v.y > b.v.y}; }
    __device__ static __forceinline__ F2 sel(Pred p, F2 a, F2 b) {
        return F2(p.x ? a.v.x : b.v.x, p.y ? a.v.y : b.v.y);
    }
    __device__ static __forceinline__ float lane(F2 v, int i) { return i ? v.v.y : v.v.x; }
    __device__ static __forceinline__ void set_lane(F2& v, int i, float x) {
        if (i) v.v.y = x;
        else v.v.x = x;
    }
};

// Scalar type of one lane.
template <typename T> struct LaneOf { using type = T; };
template <> struct LaneOf<F2> { using type = float; };
template <> struct LaneOf<F1> { using type = float; };

}  // namespace lbm
