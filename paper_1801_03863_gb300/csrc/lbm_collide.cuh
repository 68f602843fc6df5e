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
// about 30 additions; it is solved for D s~ with D = diag(1, 2, 2, 2), whose
// matrix D^-1 A D^-1 drops the common factors of the eps, q_x, q_y rows.  The start point p^start = T^-1 M^start (constraints
// imposed, free moments at their equilibrium values) equals the polynomial
// equilibrium plus the BGK-relaxed non-equilibrium stress:
//     p^start_a = W_a [1 + delta_a],
//     delta_a = 3 v.u + 9/2 (v.u)^2 - 3/2 u^2
//             + (1 - omega)/(4 W_a) [(v_x^2 - v_y^2)_a s8 + (v_x v_y)_a s9],
//     s8 = P_xx/rho - (u_x^2 - u_y^2),  s9 = P_xy/rho - u_x u_y,
// so ln(p_a/W_a) = ln(1 + delta_a) is formed without cancellation.
//
// MinxEnt2 (same sections) frees only the energy moments m = (M2, M3) and
// adds the heat-flux constraints c5, c7 (Eqs. extraconstraint1/2): M5 and M7
// relax at rate 1/tau2 (Eq. tau2).  Its start point adds to delta_a the
// relaxed heat-flux term
//     (T_5a g_x + T_7a g_y) / (12 W_a),  g = (1 - omega2)(q^pre - q^eq)/rho,
// and the Newton system shrinks to the 2x2 block of A for (M2, M3).
//
// MRT and TRT (Eq. mrtcollision with the diagonal rates of Table III) relax
// each non-conserved moment k of f toward f^eq at its own rate B_k:
//     f^post_a = f_a + sum_k T_ka B_k (m^eq_k - m_k) / d_k.
//
// The rules are templates over the number type T of lbm_num.cuh (double,
// float, or F2 = two nodes at once); a[b] below always means a * b + c with
// one rounding (Num<T>::mad).
#pragma once
#include "lbm_common.cuh"
#include "lbm_num.cuh"

namespace lbm {

// Relaxation rates of one instance, in the collision's number type.
template <typename T> struct Rates {
    T omega;   // 1 / tau     (M8, M9; SRT: every moment)
    T omega2;  // 1 / tau2    (M5, M7: MinxEnt2, MRT, TRT)
    T s_e;     // M2 rate     (MRT, TRT)
    T s_eps;   // M3 rate     (MRT, TRT)
};

// Status bits of lane l are (ST_* << 2 l).
template <typename T>
__device__ __forceinline__ uint32_t lane_status(typename Num<T>::Pred skipped_ok,
                                                typename Num<T>::Pred finite_nonneg) {
    if constexpr (Num<T>::LANES == 1) {
        return (skipped_ok ? 0u : ST_NEWTON_SKIPPED) | (finite_nonneg ? 0u : ST_UNSTABLE);
    } else {
        return (skipped_ok.x ? 0u : ST_NEWTON_SKIPPED) | (finite_nonneg.x ? 0u : ST_UNSTABLE) |
               ((skipped_ok.y ? 0u : ST_NEWTON_SKIPPED) << 2) |
               ((finite_nonneg.y ? 0u : ST_UNSTABLE) << 2);
    }
}

// Stability criterion of Sec. IV.H on f^post_a = W_a rho0 + out_a: every
// population finite and >= 0.  Returns a per-lane "all good" predicate.
template <typename T, int Q>
__device__ __forceinline__ typename Num<T>::Pred finite_nonneg(const T (&out)[Q],
                                                               const double (&w)[Q], T rho0) {
    using N = Num<T>;
    typename N::Pred ok;
    if constexpr (N::LANES == 1) {
        ok = true;
#pragma unroll
        for (int a = 0; a < Q; ++a) ok = ok && (out[a] >= -T(w[a]) * rho0);
        // out >= c is false for NaN; a +inf population needs a non-finite input
        // and then the mass sum is not finite
        T s = out[0];
#pragma unroll
        for (int a = 1; a < Q; ++a) s = s + out[a];
        ok = ok && (fabs(s) < T(1e30));
    } else {
        bool okx = true, oky = true;
        float sx = 0.f, sy = 0.f;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const float lo = -(float)w[a] * rho0.v.x;
            okx = okx && (out[a].v.x >= lo);
            oky = oky && (out[a].v.y >= lo);
        }
        T s = out[0];
#pragma unroll
        for (int a = 1; a < Q; ++a) s = s + out[a];
        sx = s.v.x;
        sy = s.v.y;
        ok = {okx && (fabsf(sx) < 1e30f), oky && (fabsf(sy) < 1e30f)};
    }
    return ok;
}

// Stability criterion for finite FP32 outputs: ST_UNSTABLE per lane when
// some f^post_a = W_a rho0 + out_a has its sign bit set.
template <typename T, int Q>
__device__ __forceinline__ uint32_t sign_status(const T (&out)[Q], const double (&w)[Q], T rho0) {
    using N = Num<T>;
    uint32_t bits[N::LANES];
#pragma unroll
    for (int l = 0; l < N::LANES; ++l) bits[l] = 0u;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const T f = N::mad(T((float)w[a]), rho0, out[a]);  // f^post_a, packed
#pragma unroll
        for (int l = 0; l < N::LANES; ++l) bits[l] |= __float_as_uint(N::lane(f, l));
    }
    uint32_t st = 0;
#pragma unroll
    for (int l = 0; l < N::LANES; ++l) st |= (bits[l] >> 31) ? (ST_UNSTABLE << (2 * l)) : 0u;
    return st;
}

// The stability criterion (finite, non-negative populations) for rules
// without a Newton step: the FP64 path compares every population, the FP32
// paths test the sign bits of f^post and that the sum of the deviations is
// finite (a NaN or infinite population makes it so).
template <typename T, int Q>
__device__ __forceinline__ uint32_t plain_status(const T (&out)[Q], const double (&w)[Q], T rho0) {
    using N = Num<T>;
    if constexpr (std::is_same<T, double>::value) {
        return lane_status<T>(true, finite_nonneg<T, Q>(out, w, rho0));
    } else {
        uint32_t st = sign_status<T, Q>(out, w, rho0);
        T s = out[0];
#pragma unroll
        for (int a = 1; a < Q; ++a) s = s + out[a];
#pragma unroll
        for (int l = 0; l < N::LANES; ++l)
            if (!(fabsf(N::lane(s, l)) < 1e30f)) st |= ST_UNSTABLE << (2 * l);
        return st;
    }
}

// 4x4 symmetric positive definite solve A x = b by an LDL^T factorisation:
// A = L D L^T with unit lower-triangular L, then L z = b, x = L^-T D^-1 z.
// Four reciprocals (of the pivots) and 32 multiply-adds; A is given as its
// 10 unique entries, unknown order (1, 2, 3, 4).
template <typename T>
__device__ __forceinline__ void spd4_solve(T a11, T a21, T a22, T a31, T a32, T a33, T a41, T a42,
                                           T a43, T a44, T b1, T b2, T b3, T b4, T& x1, T& x2,
                                           T& x3, T& x4) {
    using N = Num<T>;
    const T r1 = N::rcp(a11);
    const T l21 = a21 * r1, l31 = a31 * r1, l41 = a41 * r1;
    const T r2 = N::rcp(N::mad(-l21, a21, a22));
    const T t32 = N::mad(-l31, a21, a32), t42 = N::mad(-l41, a21, a42);
    const T l32 = t32 * r2, l42 = t42 * r2;
    const T r3 = N::rcp(N::mad(-l32, t32, N::mad(-l31, a31, a33)));
    const T t43 = N::mad(-l42, t32, N::mad(-l41, a31, a43));
    const T l43 = t43 * r3;
    const T r4 = N::rcp(N::mad(-l43, t43, N::mad(-l42, t42, N::mad(-l41, a41, a44))));
    const T z2 = N::mad(-l21, b1, b2);
    const T z3 = N::mad(-l32, z2, N::mad(-l31, b1, b3));
    const T z4 = N::mad(-l43, z3, N::mad(-l42, z2, N::mad(-l41, b1, b4)));
    x4 = z4 * r4;
    x3 = N::mad(-l43, x4, z3 * r3);
    x2 = N::mad(-l42, x4, N::mad(-l32, x3, z2 * r2));
    x1 = N::mad(-l41, x4, N::mad(-l31, x3, N::mad(-l21, x2, b1 * r1)));
}

#ifndef LBM_MX4_LOGP
#define LBM_MX4_LOGP 1  // FP32 MinxEnt4: logarithms of pair products / quotients (7 instead of 9)
#endif
#ifndef LBM_SHARED_RCP
#define LBM_SHARED_RCP 0  // FP32: one reciprocal for y_0 and the four opposite-pair products
#endif
#ifndef LBM_YFORM
#define LBM_YFORM 1  // 2-byte storage: start point and result as full populations (see below)
#endif

// Sign bits of f_a per lane -> ST_UNSTABLE bits (f finite).
template <typename T, int Q>
__device__ __forceinline__ uint32_t negative_status(const T (&f)[Q]) {
    using N = Num<T>;
    uint32_t st = 0;
#pragma unroll
    for (int l = 0; l < N::LANES; ++l) {
        uint32_t bits = 0u;
#pragma unroll
        for (int a = 0; a < Q; ++a) bits |= __float_as_uint(N::lane(f[a], l));
        st |= (bits >> 31) ? (ST_UNSTABLE << (2 * l)) : 0u;
    }
    return st;
}

// ---------------------------------------------------------------------------
// D2Q9 MinxEnt collision of one fluid node (or two, T = F2).
//   NFREE  4 (MinxEnt4: free M2, M3, M5, M7) or 2 (MinxEnt2: free M2, M3)
//   YFORM  FP32 with 2-byte storage: the start point is formed as
//          y_a = p^start_a / W_a directly and the result as the full
//          population f_a, whose deviation f_a - W_a rho0 is taken last.
//          That subtraction loses the low bits of small deviations (about
//          2^-24 W_a rho0 absolute), far below the FP16 / BF16 rounding of
//          the stored deviation, and saves the separate deviation variables.
//   d      pulled pre-collision deviations f_a - W_a rho0
//   rho0   reference density; r.omega = 1/tau, r.omega2 = 1/tau2
//   out    post-collision deviations
// Returns ST_* bits per lane: ST_NEWTON_SKIPPED when some p^start_a <= 0
// (the node keeps p^start, which meets every constraint), ST_UNSTABLE when
// some post-collision population is negative or not finite.
// ---------------------------------------------------------------------------
template <typename T, int NFREE, bool YFORM = false>
__device__ __forceinline__ uint32_t minxent_d2q9(const T (&d)[9], T rho0, const Rates<T>& r,
                                                 T (&out)[9]) {
    static_assert(NFREE == 4 || NFREE == 2, "MinxEnt4 or MinxEnt2");
    using N = Num<T>;
    constexpr bool FP64 = std::is_same<T, double>::value;
    static_assert(!(YFORM && FP64), "the direct form is for 2-byte storage with FP32 arithmetic");
    const T omega = r.omega;
    constexpr double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    // Moments of the pulled state (Sec. II.A) and the stress moments
    // M8 = sum f (v_x^2 - v_y^2), M9 = sum f v_x v_y (rows 8, 9 of T), from
    // the sums of opposite populations.
    const T n13 = d[1] + d[3], n24 = d[2] + d[4], n57 = d[5] + d[7], n68 = d[6] + d[8];
    const T drho = (d[0] + (n13 + n24)) + (n57 + n68);
    const T a57 = d[5] - d[7], a86 = d[8] - d[6];
    const T jx = (d[1] - d[3]) + a57 + a86;
    const T jy = (d[2] - d[4]) + a57 - a86;
    const T pxx = n13 - n24;
    const T pxy = n57 - n68;
    const T rho = rho0 + drho;
    const T ir = N::rcp(rho);
    const T ux = jx * ir, uy = jy * ir;
    const T uyy = uy * uy, uxy = ux * uy;
    const T U2 = N::mad(ux, ux, uyy), D2 = N::mad(ux, ux, -uyy);  // |u|^2, u_x^2 - u_y^2
    // Non-equilibrium stress relaxed at 1/tau (Eqs. discreteviscoconst/isoconst):
    // c8 - M8eq = (1 - omega)(M8pre - M8eq), likewise for M9; scaled by 1/(4 W).
    const T k = (T(1.0) - omega) * T(0.25);
    const T c8 = (T(9.0) * k) * N::mad(pxx, ir, -D2);
    const T c9 = (T(36.0) * k) * N::mad(pxy, ir, -uxy);
    // delta_a = p^start_a / W_a - 1 = (even part s) +- 3 (odd part h), the
    // even parts written with U2 = |u|^2:
    //   s_0 = -3/2 U2,  s_x,y = 3/4 U2 +- G,  s_+,- = 3 U2 +- P,
    //   G = 9/4 (u_x^2 - u_y^2) + c8,  P = 9 u_x u_y + c9.
    const T G = N::mad(T(2.25), D2, c8);
    const T P = N::mad(T(9.0), uxy, c9);
    const T C1 = T(1.0), C3 = T(3.0);
    // coefficients of the terms odd in v: 3 v.u, plus for MinxEnt2 the
    // relaxed heat flux, T_5a g_x / (12 W_a) = (-3/2 on +x, +3 on (+,+) ...)
    const T sp_ = ux + uy, dm_ = uy - ux;
    T hx = ux, hy = uy, lp = sp_, lm = dm_;
    if constexpr (NFREE == 2) {
        // q^pre - q^eq = -Q with Q_x = (d1 - d3) - 2 (a57 + a86) (deviation
        // form of m^eq_5 - m_5 = -rho u_x - M5), likewise Q_y
        const T Qx = N::mad(T(-2.0), a57 + a86, d[1] - d[3]);
        const T Qy = N::mad(T(-2.0), a57 - a86, d[2] - d[4]);
        const T k2 = (r.omega2 - T(1.0)) * ir;  // g = (omega2 - 1) Q / rho
        const T gx = k2 * Qx, gy = k2 * Qy;
        hx = N::mad(T(-0.5), gx, ux);
        hy = N::mad(T(-0.5), gy, uy);
        lp = sp_ + (gx + gy);
        lm = dm_ + (gy - gx);
    }
    // y_a = p^start_a / W_a = 1 + delta_a; all positive <=> the logarithms
    // exist (reading C-NEG).  cx .. cm: the even parts 1 + s of the opposite
    // pairs (the mean of y_a and y_opp(a)).
    T del[9], y[9];
    T cx, cy, cp, cm;
    if constexpr (YFORM) {
        const T F = N::mad(T(0.75), U2, C1), E = N::mad(C3, U2, C1);
        cx = F + G;
        cy = F - G;
        cp = E + P;
        cm = E - P;
        y[0] = N::mad(T(-1.5), U2, C1);
        y[1] = N::mad(C3, hx, cx);
        y[3] = N::mad(-C3, hx, cx);
        y[2] = N::mad(C3, hy, cy);
        y[4] = N::mad(-C3, hy, cy);
        y[5] = N::mad(C3, lp, cp);
        y[7] = N::mad(-C3, lp, cp);
        y[6] = N::mad(C3, lm, cm);
        y[8] = N::mad(-C3, lm, cm);
    } else {
        const T F0 = T(0.75) * U2, E0 = C3 * U2;
        const T sx = F0 + G, sy = F0 - G, sp = E0 + P, sm = E0 - P;
        del[0] = T(-1.5) * U2;
        del[1] = N::mad(C3, hx, sx);
        del[3] = N::mad(-C3, hx, sx);
        del[2] = N::mad(C3, hy, sy);
        del[4] = N::mad(-C3, hy, sy);
        del[5] = N::mad(C3, lp, sp);
        del[7] = N::mad(-C3, lp, sp);
        del[6] = N::mad(C3, lm, sm);
        del[8] = N::mad(-C3, lm, sm);
#pragma unroll
        for (int a = 0; a < 9; ++a) y[a] = C1 + del[a];
        cx = C1 + sx;
        cy = C1 + sy;
        cp = C1 + sp;
        cm = C1 + sm;
    }
    // FP64: the exact test of reading C-NEG.  FP32: see the Newton-step test below.
    typename N::Pred ok{};
    if constexpr (FP64) {
        const T mn = N::vmin(N::vmin(N::vmin(y[0], y[1]), N::vmin(y[2], y[3])),
                             N::vmin(N::vmin(y[4], y[5]), N::vmin(N::vmin(y[6], y[7]), y[8])));
        ok = N::gt(mn, T(0.0));
    }

    // q_a = W_a / p_a = 1 / y_a.  FP32: opposite populations share one
    // reciprocal of their product (each result within ~2 ulp); with
    // LBM_SHARED_RCP the four products and y_0 share a single one.
    T q[9];
    T p13 = T(0.0), p24 = T(0.0), p57 = T(0.0), p68 = T(0.0), pa = T(0.0), pd = T(0.0);
    if constexpr (!FP64) {
        p13 = y[1] * y[3]; p24 = y[2] * y[4]; p57 = y[5] * y[7]; p68 = y[6] * y[8];
        T r13, r24, r57, r68;
        if constexpr (LBM_SHARED_RCP) {
            pa = p13 * p24;
            pd = p57 * p68;
            const T pad = pa * pd;
            const T R = N::rcp(y[0] * pad);  // 1 / (y0 pa pd)
            q[0] = R * pad;
            const T Rad = R * y[0];          // 1 / (pa pd)
            const T ra = Rad * pd, rd = Rad * pa;
            r13 = ra * p24; r24 = ra * p13; r57 = rd * p68; r68 = rd * p57;
        } else {
            r13 = N::rcp(p13); r24 = N::rcp(p24); r57 = N::rcp(p57); r68 = N::rcp(p68);
            q[0] = N::rcp(y[0]);
        }
        q[1] = y[3] * r13; q[3] = y[1] * r13;
        q[2] = y[4] * r24; q[4] = y[2] * r24;
        q[5] = y[7] * r57; q[7] = y[5] * r57;
        q[6] = y[8] * r68; q[8] = y[6] * r68;
    } else {
#pragma unroll
        for (int a = 0; a < 9; ++a) q[a] = N::rcp(y[a]);
    }

    // Gradient terms ln(p/W) (natural or base-2 logs, see Num::LOG_SCALE):
    // L0 of the rest population, La / Ld the sums over the axis / diagonal
    // populations, D31 = L3 - L1, D42 = L4 - L2, l57 = L5 - L7, l68 = L6 - L8.
    // FP32 MinxEnt2 needs only L0, La, Ld: logarithms of y_0 and of the axis
    // and diagonal products (3 instead of 9).  FP32 MinxEnt4 with
    // LBM_MX4_LOGP takes the differences as logarithms of the quotients
    // y_a q_opp(a) as well (7 instead of 9).
    constexpr bool LOGP = !FP64 && (NFREE == 2 || LBM_MX4_LOGP);
    T L0, La, Ld, D31 = T(0.0), D42 = T(0.0), l57 = T(0.0), l68 = T(0.0);
    if constexpr (LOGP) {
        if constexpr (!LBM_SHARED_RCP) {
            pa = p13 * p24;
            pd = p57 * p68;
        }
        L0 = N::lnp(T(0.0), y[0]);
        La = N::lnp(T(0.0), pa);
        Ld = N::lnp(T(0.0), pd);
        if constexpr (NFREE == 4) {
            D31 = N::lnp(T(0.0), y[3] * q[1]);
            D42 = N::lnp(T(0.0), y[4] * q[2]);
            l57 = N::lnp(T(0.0), y[5] * q[7]);
            l68 = N::lnp(T(0.0), y[6] * q[8]);
        }
    } else {
        T L[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) L[a] = N::lnp(YFORM ? T(0.0) : del[a], y[a]);
        L0 = L[0];
        La = (L[1] + L[2]) + (L[3] + L[4]);
        Ld = (L[5] + L[6]) + (L[7] + L[8]);
        D31 = L[3] - L[1];
        D42 = L[4] - L[2];
        l57 = L[5] - L[7];
        l68 = L[6] - L[8];
    }

    // A/9 with 1/p_a = q_a / W_a: rest 9/4 q, axis 9 q, diagonal 36 q.
    const T e13 = q[1] + q[3], e24 = q[2] + q[4];
    const T d13 = q[1] - q[3], d24 = q[2] - q[4];
    const T s57 = q[5] + q[7], s68 = q[6] + q[8];
    const T d57 = q[5] - q[7], d68 = q[6] - q[8];
    const T Qa = e13 + e24;
    const T qd = s57 + s68;
    const T dx = d57 - d68, dy = d57 + d68;
    // rows of T used: e (M2), eps (M3), q_x (M5), q_y (M7).  The system is
    // solved in the scaled unknowns (s~_e, 2 s~_eps, 2 s~_x, 2 s~_y), i.e.
    // for D A D and D b with D = diag(1, 1/2, 1/2, 1/2): this removes the
    // common factors 2 and 4 of the eps, q_x and q_y rows of A/9.
    const T A_ee = N::mad(T(16.0), qd, N::mad(T(4.0), q[0], Qa));
    const T A_ep = N::mad(T(4.0), qd, N::mad(T(-2.0), q[0], Qa));
    const T A_pp = (q[0] + Qa) + qd;
    const T b_e = N::mad(T(-4.0), L0, N::mad(T(2.0), Ld, -La));
    const T b_p = N::mad(T(2.0), L0, N::mad(T(0.5), Ld, -La));
    T se, sps, sx_ = T(0.0), sy_ = T(0.0);
    if constexpr (NFREE == 4) {
        const T A_ex = N::mad(T(4.0), dx, d13);
        const T A_px = d13 + dx;
        const T A_xx = e13 + qd;
        const T A_ey = N::mad(T(4.0), dy, d24);
        const T A_py = d24 + dy;
        const T A_yy = e24 + qd;
        const T A_xy = s57 - s68;
        const T b_x = N::mad(T(0.5), l57 - l68, D31);
        const T b_y = N::mad(T(0.5), l57 + l68, D42);
        spd4_solve<T>(A_ee, A_ep, A_pp, A_ex, A_px, A_xx, A_ey, A_py, A_xy, A_yy, b_e, b_p, b_x,
                      b_y, se, sps, sx_, sy_);
    } else {
        // 2x2 SPD solve by Cramer's rule
        const T idet = N::rcp(N::mad(A_ee, A_pp, -(A_ep * A_ep)));
        se = N::mad(A_pp, b_e, -(A_ep * b_p)) * idet;
        sps = N::mad(A_ee, b_p, -(A_ep * b_e)) * idet;
    }
    // a node whose start point is not positive keeps p^start (reading C-NEG)
    bool rare = false;  // some lane skipped its Newton step (FP32 paths)
    if constexpr (FP64) {
        se = N::sel(ok, se, T(0.0));
        sps = N::sel(ok, sps, T(0.0));
        if constexpr (NFREE == 4) {
            sx_ = N::sel(ok, sx_, T(0.0));
            sy_ = N::sel(ok, sy_, T(0.0));
        }
    } else {
        // FP32: a start probability <= 0 gives log2 = NaN or -inf, which the
        // solve carries into every component of the step; a step that is not
        // finite (this, or an overflowing solve) is skipped.  chk = c - c is
        // +0 for finite c and NaN otherwise.
        T chk = (NFREE == 4) ? (se + sps) + (sx_ + sy_) : se + sps;
        chk = chk - chk;
        // logarithms of products and quotients: two negative y can cancel.
        // MinxEnt2 tests the sign bits of every y; MinxEnt4 (whose quotients
        // catch a single negative population of a pair) tests y_0 and the
        // pair means c, which are negative when both of a pair are.
        // One integer word decides the common case: chk is +0 for a finite
        // step (its bits are 0) and NaN otherwise, and the sign bits of the
        // tested values are 0 when none is negative.
        uint32_t neg[N::LANES], any = 0u;
#pragma unroll
        for (int l = 0; l < N::LANES; ++l) {
            uint32_t sgn = 0u;
            if constexpr (LOGP && NFREE == 2) {
#pragma unroll
                for (int a = 0; a < 9; ++a) sgn |= __float_as_uint(N::lane(y[a], l));
            } else if constexpr (LOGP) {
                sgn = __float_as_uint(N::lane(cx, l)) | __float_as_uint(N::lane(cy, l)) |
                      __float_as_uint(N::lane(cp, l)) | __float_as_uint(N::lane(cm, l));
            }
            neg[l] = sgn >> 31;
            any |= (sgn & 0x80000000u) | __float_as_uint(N::lane(chk, l));
        }
        rare = any != 0u;
        if (rare) {
            if constexpr (N::LANES == 1) {
                ok = N::lane(chk, 0) == 0.f && !neg[0];
            } else {
                ok = {N::lane(chk, 0) == 0.f && !neg[0], N::lane(chk, 1) == 0.f && !neg[1]};
            }
            se = N::sel(ok, se, T(0.0));
            sps = N::sel(ok, sps, T(0.0));
            if constexpr (NFREE == 4) {
                sx_ = N::sel(ok, sx_, T(0.0));
                sy_ = N::sel(ok, sy_, T(0.0));
            }
        }
    }
    // f^post_a = rho W_a (y_a - (T^T s~)_a), with the 1/9 of A's scaling and
    // the log base L (Num::LOG_SCALE) in the factor of T^T s~; sps, sx_, sy_
    // hold twice s~_eps, s~_x, s~_y.
    if constexpr (YFORM) {
        // g_a = f^post_a / W_a = rho y_a - u_a, u_a = rho L (T^T s~)_a / (9 W_a):
        // the solution is scaled by kappa = rho L once, and the class factors
        // 1 / (9 W_a) = 1/4, 1, 4 (rest, axis, diagonal) go into constants.
        const T kap = rho * T(N::LOG_SCALE);
        const T Se = kap * se, Sp = kap * sps;
        T u[9], g[9];
        u[0] = N::mad(T(0.5), Sp, -Se);
        const T CE = -(Se + Sp);
        const T CD4 = N::mad(T(8.0), Se, Sp + Sp);
        if constexpr (NFREE == 4) {
            const T Sx = kap * sx_, Sy = kap * sy_;
            const T pxy_ = Sx + Sy, mxy_ = Sx - Sy;
            u[1] = CE - Sx;
            u[3] = CE + Sx;
            u[2] = CE - Sy;
            u[4] = CE + Sy;
            u[5] = N::mad(T(2.0), pxy_, CD4);
            u[7] = N::mad(T(-2.0), pxy_, CD4);
            u[6] = N::mad(T(-2.0), mxy_, CD4);
            u[8] = N::mad(T(2.0), mxy_, CD4);
        } else {
            u[1] = u[2] = u[3] = u[4] = CE;
            u[5] = u[6] = u[7] = u[8] = CD4;
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            g[a] = N::mad(rho, y[a], -u[a]);
            out[a] = N::mad(T(W[a]), g[a], -(T(W[a]) * rho0));
        }
        if (rare) return lane_status<T>(ok, finite_nonneg<T, 9>(out, W, rho0));
        return negative_status<T, 9>(g);  // g_a has the sign of f^post_a
    } else {
        T t[9];
        const T ce = -(se + sps);
        const T cd = N::mad(T(0.5), sps, se + se);
        t[0] = N::mad(T(-4.0), se, sps + sps);
        if constexpr (NFREE == 4) {
            const T pxy_ = sx_ + sy_, mxy_ = sx_ - sy_;
            t[1] = ce - sx_;
            t[3] = ce + sx_;
            t[2] = ce - sy_;
            t[4] = ce + sy_;
            t[5] = N::mad(T(0.5), pxy_, cd);
            t[7] = N::mad(T(-0.5), pxy_, cd);
            t[6] = N::mad(T(-0.5), mxy_, cd);
            t[8] = N::mad(T(0.5), mxy_, cd);
        } else {
            t[1] = t[2] = t[3] = t[4] = ce;
            t[5] = t[6] = t[7] = t[8] = cd;
        }
        const T rs = rho * T(N::LOG_SCALE / 9.0);
        // d^post_a = W_a (drho + rho delta_a) - rho (T^T s~)_a
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const T wa = T(W[a]);
            out[a] = N::mad(-rs, t[a], N::mad(wa * rho, del[a], wa * drho));
        }
        if constexpr (FP64) {
            return lane_status<T>(ok, finite_nonneg<T, 9>(out, W, rho0));
        } else {
            if (rare) return lane_status<T>(ok, finite_nonneg<T, 9>(out, W, rho0));
            // every step was finite, and so are the populations: only the sign of
            // f^post = W rho0 + out remains to test (OR of the sign bits)
            return sign_status<T, 9>(out, W, rho0);
        }
    }
}

// ---------------------------------------------------------------------------
// D2Q9 SRT/BGK collision, Eq. (bgkcollision): f + omega (f^eq - f).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ uint32_t srt_d2q9(const T (&d)[9], T rho0, const Rates<T>& r,
                                             T (&out)[9]) {
    using N = Num<T>;
    const T omega = r.omega;
    constexpr double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    const T drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    const T a57 = d[5] - d[7], a86 = d[8] - d[6];
    const T jx = (d[1] - d[3]) + a57 + a86;
    const T jy = (d[2] - d[4]) + a57 - a86;
    const T rho = rho0 + drho;
    const T ir = N::rcp(rho);
    const T ux = jx * ir, uy = jy * ir;
    const T uxx = ux * ux, uyy = uy * uy;
    const T b0 = T(-1.5) * (uxx + uyy);
    const T sx = N::mad(T(4.5), uxx, b0), sy = N::mad(T(4.5), uyy, b0);
    const T sp_ = ux + uy, dm_ = uy - ux;
    const T sp = N::mad(T(4.5) * sp_, sp_, b0), sm = N::mad(T(4.5) * dm_, dm_, b0);
    T xi[9];
    xi[0] = b0;
    xi[1] = N::mad(T(3.0), ux, sx);
    xi[3] = N::mad(T(-3.0), ux, sx);
    xi[2] = N::mad(T(3.0), uy, sy);
    xi[4] = N::mad(T(-3.0), uy, sy);
    xi[5] = N::mad(T(3.0), sp_, sp);
    xi[7] = N::mad(T(-3.0), sp_, sp);
    xi[6] = N::mad(T(3.0), dm_, sm);
    xi[8] = N::mad(T(-3.0), dm_, sm);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const T wa = T(W[a]);
        const T deq = N::mad(wa * rho, xi[a], wa * drho);
        out[a] = N::mad(omega, deq - d[a], d[a]);
    }
    return plain_status<T, 9>(out, W, rho0);
}

// ---------------------------------------------------------------------------
// D2Q9 MRT / TRT collision, Eq. (mrtcollision): the moments of T relax
// toward those of the polynomial equilibrium at the rates of Table III,
//   B = diag(0, s_e, s_eps, 0, omega2, 0, omega2, omega, omega),
// MRT: s_e = 1.64, s_eps = 1.54; TRT: s_e = s_eps = omega.  In deviation
// variables (m_k(W) = (1, -2, 1, 0, ...)) the moment differences are
//   m^eq_2 - m_2 = 2 d0 - S_a - 4 S_d + 3 rho u^2,
//   m^eq_3 - m_3 = 3 (S_a - d0 - rho u^2),
//   m^eq_5 - m_5 = (d1 - d3) - 2 (a57 + a86),  m^eq_7 - m_7 likewise,
//   m^eq_8 - m_8 = rho (u_x^2 - u_y^2) - P_xx,  m^eq_9 - m_9 = rho u_x u_y - P_xy,
// with S_a, S_d the axis and diagonal sums; each is scaled by B_k / d_k and
// mapped back with the columns of T.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ uint32_t mrt_d2q9(const T (&d)[9], T rho0, const Rates<T>& r,
                                             T (&out)[9]) {
    using N = Num<T>;
    constexpr double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    const T Sa = (d[1] + d[2]) + (d[3] + d[4]);
    const T Sd = (d[5] + d[6]) + (d[7] + d[8]);
    const T drho = d[0] + Sa + Sd;
    const T a57 = d[5] - d[7], a86 = d[8] - d[6];
    const T d13 = d[1] - d[3], d24 = d[2] - d[4];
    const T jx = d13 + a57 + a86;
    const T jy = d24 + a57 - a86;
    const T pxx = (d[1] + d[3]) - (d[2] + d[4]);
    const T pxy = (d[5] + d[7]) - (d[6] + d[8]);
    const T rho = rho0 + drho;
    const T ir = N::rcp(rho);
    const T ux = jx * ir, uy = jy * ir;
    const T ru2 = N::mad(jx, ux, jy * uy);  // rho u^2
    const T Ee = N::mad(T(3.0), ru2, N::mad(T(2.0), d[0], N::mad(T(-4.0), Sd, -Sa)));
    const T Ep = T(3.0) * ((Sa - d[0]) - ru2);
    const T Qx = N::mad(T(-2.0), a57 + a86, d13);
    const T Qy = N::mad(T(-2.0), a57 - a86, d24);
    const T P8 = N::mad(jx, ux, -N::mad(jy, uy, pxx));
    const T P9 = N::mad(jx, uy, -pxy);
    const T re = (r.s_e * T(1.0 / 36.0)) * Ee;
    const T rp = (r.s_eps * T(1.0 / 36.0)) * Ep;
    const T rx = (r.omega2 * T(1.0 / 12.0)) * Qx;
    const T ry = (r.omega2 * T(1.0 / 12.0)) * Qy;
    const T r8 = (r.omega * T(0.25)) * P8;
    const T r9 = (r.omega * T(0.25)) * P9;
    const T c = N::mad(T(-2.0), rp, -re);  // axis columns of rows 2, 3
    const T g = N::mad(T(2.0), re, rp);    // diagonal columns of rows 2, 3
    const T cp = c + r8, cm = c - r8;
    const T xp = rx + ry, xm = rx - ry;
    const T gp = g + r9, gm = g - r9;
    out[0] = N::mad(T(4.0), rp - re, d[0]);
    out[1] = d[1] + N::mad(T(-2.0), rx, cp);
    out[3] = d[3] + N::mad(T(2.0), rx, cp);
    out[2] = d[2] + N::mad(T(-2.0), ry, cm);
    out[4] = d[4] + N::mad(T(2.0), ry, cm);
    out[5] = d[5] + (gp + xp);
    out[7] = d[7] + (gp - xp);
    out[6] = d[6] + (gm - xm);
    out[8] = d[8] + (gm + xm);
    return plain_status<T, 9>(out, W, rho0);
}

// ---------------------------------------------------------------------------
// D1Q3 collision.  MinxEnt on D1Q3: mass, momentum and the relaxed second
// moment fix all three populations, and BGK relaxation meets the same three
// constraints, so both rules reduce to f + omega (f^eq - f).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ uint32_t bgk_d1q3(const T (&d)[3], T rho0, const Rates<T>& r,
                                             T (&out)[3]) {
    using N = Num<T>;
    const T omega = r.omega;
    constexpr double W[3] = {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0};
    const T drho = d[0] + d[1] + d[2];
    const T rho = rho0 + drho;
    const T u = (d[1] - d[2]) * N::rcp(rho);
    const T b0 = T(-1.5) * (u * u);
    const T s = T(3.0) * (u * u);  // 9/2 u^2 - 3/2 u^2
    const T w0 = T(W[0]), w1 = T(W[1]);
    const T deq0 = N::mad(w0 * rho, b0, w0 * drho);
    const T deq1 = N::mad(w1 * rho, N::mad(T(3.0), u, s), w1 * drho);
    const T deq2 = N::mad(w1 * rho, N::mad(T(-3.0), u, s), w1 * drho);
    out[0] = N::mad(omega, deq0 - d[0], d[0]);
    out[1] = N::mad(omega, deq1 - d[1], d[1]);
    out[2] = N::mad(omega, deq2 - d[2], d[2]);
    // per-population compares (measured faster than the sign-bit test in
    // the bandwidth-bound D1Q3 kernel)
    typename N::Pred all;
    if constexpr (N::LANES == 1) all = true;
    else all = {true, true};
    return lane_status<T>(all, finite_nonneg<T, 3>(out, W, rho0));
}

// Dispatch by lattice, rule, number type and storage bytes SB (the MinxEnt
// rules take the direct start-point form for 2-byte storage, see
// minxent_d2q9).  Every kernel passes its own storage size, so all kernels
// of one context run the same arithmetic.
template <class Lat, int COLL, typename T, int SB = 8> struct Collide;
template <typename T, int SB> struct Collide<D2Q9, COLL_MINXENT4, T, SB> {
    __device__ static __forceinline__ uint32_t run(const T (&d)[9], T rho0, const Rates<T>& r,
                                                   T (&o)[9]) {
        return minxent_d2q9<T, 4, LBM_YFORM && SB == 2 && !std::is_same<T, double>::value>(
            d, rho0, r, o);
    }
};
template <typename T, int SB> struct Collide<D2Q9, COLL_MINXENT2, T, SB> {
    __device__ static __forceinline__ uint32_t run(const T (&d)[9], T rho0, const Rates<T>& r,
                                                   T (&o)[9]) {
        return minxent_d2q9<T, 2, LBM_YFORM && SB == 2 && !std::is_same<T, double>::value>(
            d, rho0, r, o);
    }
};
template <typename T, int SB> struct Collide<D2Q9, COLL_SRT, T, SB> {
    __device__ static __forceinline__ uint32_t run(const T (&d)[9], T rho0, const Rates<T>& r,
                                                   T (&o)[9]) {
        return srt_d2q9<T>(d, rho0, r, o);
    }
};
template <typename T, int SB> struct Collide<D2Q9, COLL_MRT, T, SB> {
    __device__ static __forceinline__ uint32_t run(const T (&d)[9], T rho0, const Rates<T>& r,
                                                   T (&o)[9]) {
        return mrt_d2q9<T>(d, rho0, r, o);
    }
};
// D1Q3: every rule reduces to BGK (one non-conserved moment, relaxed at 1/tau)
template <int C, typename T, int SB> struct Collide<D1Q3, C, T, SB> {
    __device__ static __forceinline__ uint32_t run(const T (&d)[3], T rho0, const Rates<T>& r,
                                                   T (&o)[3]) {
        return bgk_d1q3<T>(d, rho0, r, o);
    }
};

}  // namespace lbm
