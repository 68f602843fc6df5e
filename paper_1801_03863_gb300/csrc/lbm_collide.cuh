// lbm_collide.cuh -- per-node collision rules in deviation variables.
//
// Every population is carried as its deviation d_a = f_a - W_a rho0 from the
// rest state at the reference density.  Mass, momentum and stress moments
// of f and d coincide except for the mass (sum W_a = 1, sum W_a v_a = 0,
// sum W_a (v_x^2 - v_y^2) = sum W_a v_x v_y = 0), so no moment suffers the
// cancellation f - W rho0 would cause in low precision.
//
// MinxEnt4 (Sec. IV.C-E of Wilson, Pugh & Dawson, arXiv:1801.03863).  The
// paper's Newton step in the free moments m = (M2, M3, M5, M7),
//     g_k  = sum_a (T^-1)_{a k} [ln(p_a / W_a) + 1],
//     H_jk = sum_a (T^-1)_{a j} (T^-1)_{a k} / p_a,
//     m^1  = m^0 - H^-1 g,   p^post = T^-1 M^post,
// is evaluated here through the orthogonality of T's rows (T T^T = diag(d),
// d = 9, 36, 36, 6, 12, 6, 12, 4, 4), which gives (T^-1)_{a k} = T_{k a}/d_k.
// With s~_k = s_k / d_k the system H s = g becomes
//     A s~ = b,  A_jk = sum_a T_ja T_ka / p_a,  b_j = sum_a T_ja ln(p_a/W_a)
// (the "+1" drops out because sum_a T_ka = 0 for every free row k), and
//     p^post_a = p^start_a - sum_k T_ka s~_k.
// A and b have small integer coefficients, so the 4x4 system is assembled in
// about 40 additions.  The start point p^start = T^-1 M^start (constraints
// imposed, free moments at their equilibrium values) equals the polynomial
// equilibrium plus the BGK-relaxed non-equilibrium stress:
//     p^start_a = W_a [1 + delta_a],
//     delta_a = 3 v.u + 9/2 (v.u)^2 - 3/2 u^2
//             + (1 - omega)/(4 W_a) [(v_x^2 - v_y^2)_a s8 + (v_x v_y)_a s9],
//     s8 = P_xx/rho - (u_x^2 - u_y^2),  s9 = P_xy/rho - u_x u_y,
// so ln(p_a/W_a) = log1p(delta_a) is formed without cancellation.
#pragma once
#include "lbm_common.cuh"

namespace lbm {

// Math used by the collisions.  FP64: IEEE division and the library log1p.
// FP32: the library log1pf and a correctly rounded reciprocal.
template <typename T> struct Math;
template <> struct Math<double> {
    __device__ static __forceinline__ double log1p_(double x) { return log1p(x); }
    __device__ static __forceinline__ double rcp(double x) { return 1.0 / x; }
};
template <> struct Math<float> {
    __device__ static __forceinline__ float log1p_(float x) { return log1pf(x); }
    __device__ static __forceinline__ float rcp(float x) { return __frcp_rn(x); }
};

// 4x4 symmetric positive definite solve by LDL^T (no square roots).
// A given as its 10 unique entries; returns x.
template <typename T>
__device__ __forceinline__ void spd4_solve(T a11, T a21, T a22, T a31, T a32, T a33, T a41, T a42,
                                           T a43, T a44, T b1, T b2, T b3, T b4, T& x1, T& x2,
                                           T& x3, T& x4) {
    const T d1 = a11;
    const T i1 = Math<T>::rcp(d1);
    const T l21 = a21 * i1, l31 = a31 * i1, l41 = a41 * i1;
    const T d2 = a22 - l21 * a21;
    const T i2 = Math<T>::rcp(d2);
    const T e32 = a32 - l31 * a21;  // (A32 - L31 D1 L21)
    const T e42 = a42 - l41 * a21;
    const T l32 = e32 * i2, l42 = e42 * i2;
    const T d3 = a33 - l31 * a31 - l32 * e32;
    const T i3 = Math<T>::rcp(d3);
    const T e43 = a43 - l41 * a31 - l42 * e32;
    const T l43 = e43 * i3;
    const T d4 = a44 - l41 * a41 - l42 * e42 - l43 * e43;
    const T i4 = Math<T>::rcp(d4);
    // forward (unit lower), diagonal, backward
    const T z1 = b1;
    const T z2 = b2 - l21 * z1;
    const T z3 = b3 - l31 * z1 - l32 * z2;
    const T z4 = b4 - l41 * z1 - l42 * z2 - l43 * z3;
    x4 = z4 * i4;
    x3 = z3 * i3 - l43 * x4;
    x2 = z2 * i2 - l32 * x3 - l42 * x4;
    x1 = z1 * i1 - l21 * x2 - l31 * x3 - l41 * x4;
}

// ---------------------------------------------------------------------------
// D2Q9 MinxEnt4 collision of one fluid node.
//   d      pulled pre-collision deviations f_a - W_a rho0
//   rho0   reference density; omega = 1/tau
//   out    post-collision deviations
// Returns ST_* bits: ST_NEWTON_SKIPPED when some p^start_a <= 0 (the node
// keeps p^start, which meets every constraint), ST_UNSTABLE when some
// post-collision population is negative or not finite.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ uint32_t minxent4_d2q9(const T (&d)[9], T rho0, T omega, T (&out)[9]) {
    const T W0 = T(4.0 / 9.0), WA = T(1.0 / 9.0), WD = T(1.0 / 36.0);
    // Moments of the pulled state (Sec. II.A) and the stress moments
    // M8 = sum f (v_x^2 - v_y^2), M9 = sum f v_x v_y (rows 8, 9 of T).
    const T drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    const T a57 = d[5] - d[7], a86 = d[8] - d[6];
    const T jx = (d[1] - d[3]) + a57 + a86;
    const T jy = (d[2] - d[4]) + a57 - a86;
    const T pxx = (d[1] + d[3]) - (d[2] + d[4]);
    const T pxy = (d[5] + d[7]) - (d[6] + d[8]);
    const T rho = rho0 + drho;
    const T ir = Math<T>::rcp(rho);
    const T ux = jx * ir, uy = jy * ir;
    const T uxx = ux * ux, uyy = uy * uy;
    // Non-equilibrium stress relaxed at 1/tau (Eqs. discreteviscoconst/isoconst):
    // c8 - M8eq = (1 - omega)(M8pre - M8eq), and likewise for M9.
    const T k = (T(1) - omega) * T(0.25);
    const T a8 = k * (pxx * ir - (uxx - uyy));
    const T a9 = k * (pxy * ir - ux * uy);
    // delta_a = p^start_a / W_a - 1.
    const T b0 = T(-1.5) * (uxx + uyy);
    const T sx = T(4.5) * uxx + b0 + T(9) * a8;
    const T sy = T(4.5) * uyy + b0 - T(9) * a8;
    const T sp_ = ux + uy, dm_ = uy - ux;
    const T sp = T(4.5) * sp_ * sp_ + b0 + T(36) * a9;
    const T sm = T(4.5) * dm_ * dm_ + b0 - T(36) * a9;
    T del[9];
    del[0] = b0;
    del[1] = sx + T(3) * ux;
    del[3] = sx - T(3) * ux;
    del[2] = sy + T(3) * uy;
    del[4] = sy - T(3) * uy;
    del[5] = sp + T(3) * sp_;
    del[7] = sp - T(3) * sp_;
    del[6] = sm + T(3) * dm_;
    del[8] = sm - T(3) * dm_;

    T mn = del[0];
#pragma unroll
    for (int a = 1; a < 9; ++a) mn = fmin(mn, del[a]);

    uint32_t st = 0;
    T t[9];
    if (mn > T(-1)) {
        // ln(p/W) and 1/p (scaled by W: q_a = 1/(1 + delta_a) = W_a / p_a).
        T L[9], q[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            L[a] = Math<T>::log1p_(del[a]);
            q[a] = Math<T>::rcp(T(1) + del[a]);
        }
        // 1/p_a = q_a / W_a: rest 9/4 q, axis 9 q, diagonal 36 q.  A is formed
        // divided by 9 (coefficients 1/4, 1, 4); the solution is rescaled below.
        const T Q0 = T(0.25) * q[0];
        const T Qa = (q[1] + q[2]) + (q[3] + q[4]);
        const T Qd = T(4) * ((q[5] + q[6]) + (q[7] + q[8]));
        const T d13 = q[1] - q[3], d24 = q[2] - q[4];
        const T t57 = T(4) * (q[5] - q[7]), t68 = T(4) * (q[6] - q[8]);
        const T Dx = t57 - t68;  // 4(q5 - q6 - q7 + q8)
        const T Dy = t57 + t68;  // 4(q5 + q6 - q7 - q8)
        const T Dxy = T(4) * ((q[5] + q[7]) - (q[6] + q[8]));
        // rows of T used: e (M2), eps (M3), q_x (M5), q_y (M7)
        const T A_ee = T(16) * Q0 + Qa + T(4) * Qd;
        const T A_ep = T(-16) * Q0 + T(2) * Qa + T(2) * Qd;
        const T A_pp = T(16) * Q0 + T(4) * Qa + Qd;
        const T A_ex = T(2) * d13 + T(2) * Dx;
        const T A_px = T(4) * d13 + Dx;
        const T A_xx = T(4) * (q[1] + q[3]) + Qd;
        const T A_ey = T(2) * d24 + T(2) * Dy;
        const T A_py = T(4) * d24 + Dy;
        const T A_yy = T(4) * (q[2] + q[4]) + Qd;
        const T A_xy = Dxy;
        const T La = (L[1] + L[2]) + (L[3] + L[4]);
        const T Ld = (L[5] + L[6]) + (L[7] + L[8]);
        const T l57 = L[5] - L[7], l68 = L[6] - L[8];
        const T b_e = T(-4) * L[0] - La + T(2) * Ld;
        const T b_p = T(4) * L[0] - T(2) * La + Ld;
        const T b_x = T(2) * (L[3] - L[1]) + (l57 - l68);
        const T b_y = T(2) * (L[4] - L[2]) + (l57 + l68);
        T se, sps, sx_, sy_;
        spd4_solve<T>(A_ee, A_ep, A_pp, A_ex, A_px, A_xx, A_ey, A_py, A_xy, A_yy, b_e, b_p, b_x,
                      b_y, se, sps, sx_, sy_);
        // (T^T s~)_a; the 1/9 from A's scaling goes into rho below.
        const T ce = -se - T(2) * sps;
        const T cd = T(2) * se + sps;
        const T pxy_ = sx_ + sy_, mxy_ = sx_ - sy_;
        t[0] = T(4) * (sps - se);
        t[1] = ce - T(2) * sx_;
        t[3] = ce + T(2) * sx_;
        t[2] = ce - T(2) * sy_;
        t[4] = ce + T(2) * sy_;
        t[5] = cd + pxy_;
        t[7] = cd - pxy_;
        t[6] = cd - mxy_;
        t[8] = cd + mxy_;
    } else {
        st |= ST_NEWTON_SKIPPED;
#pragma unroll
        for (int a = 0; a < 9; ++a) t[a] = T(0);
    }
    // d^post_a = W_a (drho + rho delta_a) - rho (T^T s~)_a
    const T rs = rho * T(1.0 / 9.0);
    const T w0r = W0 * rho, war = WA * rho, wdr = WD * rho;
    out[0] = W0 * drho + w0r * del[0] - rs * t[0];
#pragma unroll
    for (int a = 1; a < 5; ++a) out[a] = WA * drho + war * del[a] - rs * t[a];
#pragma unroll
    for (int a = 5; a < 9; ++a) out[a] = WD * drho + wdr * del[a] - rs * t[a];
    // Stability criterion of Sec. IV.H: f^post = W rho0 + d^post finite, >= 0.
    T fmn = (out[0] + W0 * rho0) * T(9.0 / 4.0);
#pragma unroll
    for (int a = 1; a < 5; ++a) fmn = fmin(fmn, (out[a] + WA * rho0) * T(9));
#pragma unroll
    for (int a = 5; a < 9; ++a) fmn = fmin(fmn, (out[a] + WD * rho0) * T(36));
    T fsum = out[0];
#pragma unroll
    for (int a = 1; a < 9; ++a) fsum += out[a];
    if (!(fmn >= T(0)) || !isfinite(fsum)) st |= ST_UNSTABLE;
    return st;
}

// ---------------------------------------------------------------------------
// D2Q9 SRT/BGK collision, Eq. (bgkcollision): f + omega (f^eq - f).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ uint32_t srt_d2q9(const T (&d)[9], T rho0, T omega, T (&out)[9]) {
    const T W0 = T(4.0 / 9.0), WA = T(1.0 / 9.0), WD = T(1.0 / 36.0);
    const T drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    const T a57 = d[5] - d[7], a86 = d[8] - d[6];
    const T jx = (d[1] - d[3]) + a57 + a86;
    const T jy = (d[2] - d[4]) + a57 - a86;
    const T rho = rho0 + drho;
    const T ir = Math<T>::rcp(rho);
    const T ux = jx * ir, uy = jy * ir;
    const T b0 = T(-1.5) * (ux * ux + uy * uy);
    const T sx = T(4.5) * ux * ux + b0, sy = T(4.5) * uy * uy + b0;
    const T sp_ = ux + uy, dm_ = uy - ux;
    const T sp = T(4.5) * sp_ * sp_ + b0, sm = T(4.5) * dm_ * dm_ + b0;
    T xi[9];
    xi[0] = b0;
    xi[1] = sx + T(3) * ux;
    xi[3] = sx - T(3) * ux;
    xi[2] = sy + T(3) * uy;
    xi[4] = sy - T(3) * uy;
    xi[5] = sp + T(3) * sp_;
    xi[7] = sp - T(3) * sp_;
    xi[6] = sm + T(3) * dm_;
    xi[8] = sm - T(3) * dm_;
    const T w0r = W0 * rho, war = WA * rho, wdr = WD * rho;
    T deq;
    deq = W0 * drho + w0r * xi[0];
    out[0] = d[0] + omega * (deq - d[0]);
#pragma unroll
    for (int a = 1; a < 5; ++a) {
        deq = WA * drho + war * xi[a];
        out[a] = d[a] + omega * (deq - d[a]);
    }
#pragma unroll
    for (int a = 5; a < 9; ++a) {
        deq = WD * drho + wdr * xi[a];
        out[a] = d[a] + omega * (deq - d[a]);
    }
    T fmn = (out[0] + W0 * rho0) * T(9.0 / 4.0);
#pragma unroll
    for (int a = 1; a < 5; ++a) fmn = fmin(fmn, (out[a] + WA * rho0) * T(9));
#pragma unroll
    for (int a = 5; a < 9; ++a) fmn = fmin(fmn, (out[a] + WD * rho0) * T(36));
    T fsum = out[0];
#pragma unroll
    for (int a = 1; a < 9; ++a) fsum += out[a];
    return (!(fmn >= T(0)) || !isfinite(fsum)) ? ST_UNSTABLE : 0u;
}

// ---------------------------------------------------------------------------
// D1Q3 collision.  MinxEnt on D1Q3: mass, momentum and the relaxed second
// moment fix all three populations, and BGK relaxation meets the same three
// constraints, so both rules reduce to f + omega (f^eq - f).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ uint32_t bgk_d1q3(const T (&d)[3], T rho0, T omega, T (&out)[3]) {
    const T W0 = T(2.0 / 3.0), W1 = T(1.0 / 6.0);
    const T drho = d[0] + d[1] + d[2];
    const T rho = rho0 + drho;
    const T u = (d[1] - d[2]) * Math<T>::rcp(rho);
    const T b0 = T(-1.5) * u * u;
    const T s = T(3) * u * u;  // 9/2 u^2 - 3/2 u^2
    const T deq0 = W0 * drho + W0 * rho * b0;
    const T deq1 = W1 * drho + W1 * rho * (s + T(3) * u);
    const T deq2 = W1 * drho + W1 * rho * (s - T(3) * u);
    out[0] = d[0] + omega * (deq0 - d[0]);
    out[1] = d[1] + omega * (deq1 - d[1]);
    out[2] = d[2] + omega * (deq2 - d[2]);
    const T fmn = fmin((out[0] + W0 * rho0) * T(1.5),
                       fmin((out[1] + W1 * rho0) * T(6), (out[2] + W1 * rho0) * T(6)));
    return (!(fmn >= T(0)) || !isfinite(out[0] + out[1] + out[2])) ? ST_UNSTABLE : 0u;
}

// Dispatch by lattice and rule.
template <class Lat, int COLL, typename T> struct Collide;
template <typename T> struct Collide<D2Q9, COLL_MINXENT4, T> {
    __device__ static __forceinline__ uint32_t run(const T (&d)[9], T rho0, T omega, T (&o)[9]) {
        return minxent4_d2q9<T>(d, rho0, omega, o);
    }
};
template <typename T> struct Collide<D2Q9, COLL_SRT, T> {
    __device__ static __forceinline__ uint32_t run(const T (&d)[9], T rho0, T omega, T (&o)[9]) {
        return srt_d2q9<T>(d, rho0, omega, o);
    }
};
template <int C, typename T> struct Collide<D1Q3, C, T> {
    __device__ static __forceinline__ uint32_t run(const T (&d)[3], T rho0, T omega, T (&o)[3]) {
        return bgk_d1q3<T>(d, rho0, omega, o);
    }
};

}  // namespace lbm
