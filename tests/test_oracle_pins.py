"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks a closed
form, an invariant, a special case that reduces to a textbook result, a value
printed in the paper (tests/golden/), or an independent solution of the same
problem (the Lagrange-dual solution of the constrained KLD minimisation,
solved here with scipy).  All run on the CPU (not marked gpu).
"""
import math
import os

import numpy as np
import pytest
from scipy import optimize

from paper_1801_03863_gb300 import workloads as wl


# ----------------------------------------------------------------------------
# Tables: Table I and Eq. (Tmatrix).
# ----------------------------------------------------------------------------
def _load_table1(golden_dir):
    rows = np.loadtxt(os.path.join(golden_dir, "d2q9_table1.txt"))
    v = rows[:, 1:3].astype(int)
    w = rows[:, 3] / rows[:, 4]
    return v, w


def test_velocity_set_matches_table1(orc, golden_dir):
    v_paper, w_paper = _load_table1(golden_dir)
    v, w, _, _ = orc.d2q9_tables()
    # same (velocity, weight) pairs; the oracle uses T's column order (reading C-ORD)
    paper = sorted((tuple(a), b) for a, b in zip(v_paper.tolist(), w_paper.tolist()))
    mine = sorted((tuple(a), b) for a, b in zip(v.tolist(), w.tolist()))
    assert len(mine) == 9
    for (va, wa), (vb, wb) in zip(paper, mine):
        assert va == vb and wa == pytest.approx(wb, abs=1e-16)


def test_tmatrix_matches_print(orc, golden_dir):
    T_paper = np.loadtxt(os.path.join(golden_dir, "tmatrix.txt")).astype(int)
    _, _, T, _ = orc.d2q9_tables()
    assert np.array_equal(T, T_paper)


def test_T_rows_are_the_constraint_moments(orc):
    """Reading C-ORD: in T's column order, rows 4, 6, 8, 9 are v_x, v_y,
    v_x^2 - v_y^2, v_x v_y (the constraint functionals of Sec. IV.C), and
    rows 5, 7 are (-5 + 3|v|^2) v_x,y (Eqs. extraconstraint1/2)."""
    v, _, T, _ = orc.d2q9_tables()
    vx, vy = v[:, 0], v[:, 1]
    vv = vx * vx + vy * vy
    assert np.array_equal(T[0], np.ones(9, int))
    assert np.array_equal(T[3], vx)
    assert np.array_equal(T[5], vy)
    assert np.array_equal(T[7], vx * vx - vy * vy)
    assert np.array_equal(T[8], vx * vy)
    assert np.array_equal(T[4], (-5 + 3 * vv) * vx)
    assert np.array_equal(T[6], (-5 + 3 * vv) * vy)
    # energy and energy-square rows of Lallemand & Luo (2000)
    assert np.array_equal(T[1], -4 + 3 * vv)
    assert np.array_equal(2 * T[2], 8 - 21 * vv + 9 * vv * vv)


def test_T_orthogonal_and_inverse(orc):
    _, _, T, Ti = orc.d2q9_tables()
    G = T @ T.T
    d = np.array([9, 36, 36, 6, 12, 6, 12, 4, 4])
    assert np.array_equal(G, np.diag(d))
    assert np.max(np.abs(Ti @ T - np.eye(9))) < 1e-14
    # orthogonal rows => T^{-1} = T^T diag(1/d)
    assert np.max(np.abs(Ti - T.T / d[None, :])) < 1e-15
    # sum_a (T^{-1})_{a k} = delta_{k1}: the "+1" of grad S vanishes (reading C-GRAD1)
    assert np.max(np.abs(Ti.sum(axis=0) - np.eye(9)[0])) < 1e-15


def test_lattice_isotropy(orc):
    """Textbook D2Q9 quadrature: sum W = 1, sum W v = 0, sum W v v = I/3,
    fourth moment = (1/9)(d_ij d_kl + d_ik d_jl + d_il d_jk)."""
    v, w, _, _ = orc.d2q9_tables()
    assert w.sum() == pytest.approx(1.0, abs=1e-16)
    assert np.abs(w @ v).max() < 1e-17
    m2 = np.einsum("a,ai,aj->ij", w, v, v)
    assert np.allclose(m2, np.eye(2) / 3, atol=1e-16)
    m4 = np.einsum("a,ai,aj,ak,al->ijkl", w, v, v, v, v)
    d = np.eye(2)
    iso = (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
           + np.einsum("il,jk->ijkl", d, d)) / 9
    assert np.allclose(m4, iso, atol=1e-16)
    v3, w3 = orc.d1q3_tables()
    assert w3.sum() == pytest.approx(1.0) and abs(w3 @ v3) < 1e-17
    assert w3 @ (v3 * v3) == pytest.approx(1.0 / 3.0, abs=1e-16)
    assert w3 @ (v3 ** 4) == pytest.approx(1.0 / 3.0, abs=1e-16)


def test_tau_from_nu_and_tau2(orc):
    """Eq. (visco-tau): nu = (2 tau - 1)/6 ; Eq. (tau2) as printed."""
    for nu in (1e-3, 0.04096, 0.1):
        t = orc.tau_from_nu(nu)
        assert (2 * t - 1) / 6 == pytest.approx(nu, rel=1e-14)
    assert orc.tau2(1.0) == pytest.approx(7.0)
    assert orc.tau2(0.75) == pytest.approx(10.0)


# ----------------------------------------------------------------------------
# Equilibrium, Eq. (numerical-plyeqm).
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (0.7, 0.05, -0.02),
                                       (2.7, -0.1, 0.08), (1.3, 0.02, 0.11)])
def test_feq_moments_closed_form(orc, rho, ux, uy):
    v, _, T, _ = orc.d2q9_tables()
    feq = orc.d2q9_feq(rho, ux, uy)
    assert feq.sum() == pytest.approx(rho, rel=1e-15)
    assert feq @ v[:, 0] == pytest.approx(rho * ux, abs=1e-15)
    assert feq @ v[:, 1] == pytest.approx(rho * uy, abs=1e-15)
    P = np.einsum("a,ai,aj->ij", feq, v, v)
    assert np.allclose(P, rho * (np.outer([ux, uy], [ux, uy]) + np.eye(2) / 3), atol=1e-15)
    uu = ux * ux + uy * uy
    M = T @ (feq / rho)
    closed = [1, -2 + 3 * uu, 1 - 3 * uu, ux, -ux, uy, -uy, ux * ux - uy * uy, ux * uy]
    assert np.allclose(M, closed, atol=1e-15)


def test_d1q3_feq_moments(orc):
    v3, _ = orc.d1q3_tables()
    for rho, u in [(1.0, 0.0), (0.5, 0.1), (3.0, -0.07)]:
        f = orc.d1q3_feq(rho, u)
        assert f.sum() == pytest.approx(rho, rel=1e-15)
        assert f @ v3 == pytest.approx(rho * u, abs=1e-15)
        assert f @ (v3 * v3) == pytest.approx(rho * (1 / 3 + u * u), rel=1e-15)


# ----------------------------------------------------------------------------
# KLD, Eq. (discrete_KLD): Gibbs' inequality.
# ----------------------------------------------------------------------------
def test_kld_gibbs(orc):
    _, w, _, _ = orc.d2q9_tables()
    rng = np.random.default_rng(3)
    assert orc.kld(w, w) == 0.0
    for _ in range(200):
        p = rng.dirichlet(np.ones(9))
        assert orc.kld(p, w) >= 0.0
        # closed form: sum p ln p - sum p ln w
        assert orc.kld(p, w) == pytest.approx(float(p @ np.log(p) - p @ np.log(w)), rel=1e-12)


# ----------------------------------------------------------------------------
# MinxEnt collision (Sec. IV.C-E).
# ----------------------------------------------------------------------------
def _random_states(n, seed, eps=0.3):
    f = wl.random_populations(9, 1, n, eps=eps, seed=seed)
    return [f[:, 0, i] for i in range(n)]


def _constraints(orc, f, tau, tau2=None):
    """Constraint values of Sec. IV.C written from their definitions."""
    v, _, T, _ = orc.d2q9_tables()
    rho = f.sum()
    u = (f @ v) / rho
    ppre = f / rho
    peq = orc.d2q9_feq(rho, u[0], u[1]) / rho
    relax = ppre + (peq - ppre) / tau
    c = {1: 1.0, 4: u[0], 6: u[1], 8: relax @ T[7], 9: relax @ T[8]}
    if tau2 is not None:
        relax2 = ppre + (peq - ppre) / tau2
        c[5] = relax2 @ T[4]
        c[7] = relax2 @ T[6]
    return rho, c


@pytest.mark.parametrize("nfree", [4, 2])
def test_minxent_conserves_and_meets_constraints(orc, nfree):
    _, _, T, _ = orc.d2q9_tables()
    for tau in (0.503, 0.62288, 1.0, 1.7):
        t2 = orc.tau2(tau)
        for f in _random_states(40, seed=11):
            fp, st = orc.d2q9_minxent(f, tau, nfree=nfree)
            assert st == 0
            rho, c = _constraints(orc, f, tau, t2 if nfree == 2 else None)
            M = T @ (fp / rho)
            for k, val in c.items():
                assert M[k - 1] == pytest.approx(val, abs=2e-15), (k, tau)
            assert fp.sum() == pytest.approx(f.sum(), rel=1e-15)


def test_minxent_fixed_point_at_rest(orc):
    """At u = 0, p^eq = W, ln(p/W) = 0, grad S = 0: the collision is the identity."""
    for rho in (0.5, 1.0, 2.7):
        feq = orc.d2q9_feq(rho, 0.0, 0.0)
        for tau in (0.5 + 1e-9, 0.7, 1.3):
            fp, st = orc.d2q9_minxent(feq, tau)
            assert st == 0
            assert np.max(np.abs(fp - feq)) <= 4e-16 * rho


def test_minxent_equilibrium_defect_is_third_order(orc):
    """ln(p^eq/W) lies in span{1, v} only up to O(|u|^3), so the collision moves
    f^eq(u) by O(|u|^3): halving u divides the change by about 8."""
    d = []
    for s in (0.1, 0.05, 0.025, 0.0125):
        feq = orc.d2q9_feq(1.0, 0.8 * s, -0.6 * s)
        fp, _ = orc.d2q9_minxent(feq, 0.8)
        d.append(np.max(np.abs(fp - feq)))
    ratios = [d[i] / d[i + 1] for i in range(3)]
    assert all(6.5 < r < 9.0 for r in ratios), ratios


def test_start_modes_agree_when_tau_is_one(orc):
    """With tau = 1 the relaxed constraints equal the equilibrium moments, so
    M^start = M^0 and both readings of C-START give the same step."""
    for f in _random_states(20, seed=5):
        a, _ = orc.d2q9_minxent(f, 1.0, start=orc.START_HYBRID)
        b, _ = orc.d2q9_minxent(f, 1.0, start=orc.START_EQUILIBRIUM)
        assert np.max(np.abs(a - b)) < 1e-15


def _dual_minimiser(orc, f, tau, nfree):
    """Independent solution of Eq. (minxentLBM-collision): the minimiser of
    sum p ln(p/W) under linear constraints sum p phi_k = c_k is
    p = W exp(sum_k lam_k phi_k); solve for lam with scipy."""
    _, w, T, _ = orc.d2q9_tables()
    rows = [0, 3, 5, 7, 8] if nfree == 4 else [0, 3, 4, 5, 6, 7, 8]
    rho, c = _constraints(orc, f, tau, orc.tau2(tau) if nfree == 2 else None)
    phi = T[rows].astype(float)
    target = np.array([c[r + 1] for r in rows])

    def resid(lam):
        p = w * np.exp(lam @ phi)
        return phi @ p - target

    sol = optimize.root(resid, np.zeros(len(rows)), method="hybr", tol=1e-15)
    # hybr reports "no further improvement" once at machine precision: assess
    # convergence by the residual itself
    assert np.max(np.abs(resid(sol.x))) < 1e-14
    return rho * w * np.exp(sol.x @ phi)


@pytest.mark.parametrize("nfree", [4, 2])
def test_converged_minimiser_matches_lagrange_dual(orc, nfree):
    for tau in (0.51, 0.8):
        for f in _random_states(15, seed=21):
            fc, it, g = orc.d2q9_minxent_converged(f, tau, nfree=nfree)
            assert it >= 1 and g < 1e-13
            fd = _dual_minimiser(orc, f, tau, nfree)
            assert np.max(np.abs(fc - fd)) < 1e-12


def test_single_step_error_is_quadratic(orc):
    """Newton's quadratic convergence, Sec. IV.E.  Shrink a random state toward
    the rest equilibrium rho W by a factor s: velocity and non-equilibrium
    stress become O(s).  The start m^0 (equilibrium moments) misses the
    minimiser only at O(s^2) -- the W-weighted couplings between the free and
    the constrained moments vanish by lattice symmetry -- so halving s divides
    |p^start - p*| by ~4, and after one Newton step the error is the square of
    that: halving s divides it by ~16."""
    _, w, _, _ = orc.d2q9_tables()
    base = wl.random_populations(9, 1, 8, eps=1.0, seed=7)[:, 0, :]
    for i in range(8):
        f1 = base[:, i]
        rho = f1.sum()
        e0, e1 = [], []
        for s in (0.4, 0.2, 0.1, 0.05):
            f = rho * w + s * (f1 - rho * w)
            one, _ = orc.d2q9_minxent(f, 0.75)
            start, _, _ = orc.d2q9_minxent_converged(f, 0.75, maxit=0)
            conv, _, _ = orc.d2q9_minxent_converged(f, 0.75)
            e0.append(np.max(np.abs(start - conv)))
            e1.append(np.max(np.abs(one - conv)))
        r0 = [e0[k] / e0[k + 1] for k in range(3)]
        r1 = [e1[k] / e1[k + 1] for k in range(3)]
        assert all(3.3 < r < 4.7 for r in r0), (e0, r0)
        assert all(11.0 < r < 20.0 for r in r1[1:]), (e1, r1)
        assert all(e1[k] < 0.05 * e0[k] for k in range(4))


def test_newton_step_decreases_kld(orc):
    """H(p^post) <= H(p^start) on near-equilibrium states (the Newton step
    descends the convex S; p^start = zero Newton iterations)."""
    _, w, _, _ = orc.d2q9_tables()
    for tau in (0.51, 0.7, 1.2):
        for f in _random_states(50, seed=31, eps=0.2):
            rho = f.sum()
            start, it, _ = orc.d2q9_minxent_converged(f, tau, maxit=0)
            assert it == 0
            post, st = orc.d2q9_minxent(f, tau)
            assert st == 0
            assert orc.kld(post / rho, w) <= orc.kld(start / rho, w) + 1e-16


def test_negative_start_skips_newton(orc):
    """Reading C-NEG: a start point with p_a <= 0 keeps p^start and is flagged."""
    f = orc.d2q9_feq(1.0, 0.0, 0.0)
    f[7] += 0.3  # huge x-x stress, drives p^start of some axis population negative
    f[1] -= 0.15
    f[3] -= 0.15
    post, st = orc.d2q9_minxent(f, 0.5 + 1e-9)
    assert st & orc.NEWTON_SKIPPED
    assert post.sum() == pytest.approx(f.sum(), rel=1e-14)


# ----------------------------------------------------------------------------
# Other collision rules.
# ----------------------------------------------------------------------------
def test_d1q3_minxent_equals_bgk(orc):
    """Reading C-D1Q3: three constraints fix the three populations, and BGK
    relaxation meets the same three constraints, so the two coincide."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        f = np.array([2 / 3, 1 / 6, 1 / 6]) * rng.uniform(0.5, 1.5) * (1 + 0.3 * rng.uniform(-1, 1, 3))
        tau = rng.uniform(0.50001, 2.0)
        a, _ = orc.d1q3_minxent(f, tau)
        rho = f.sum()
        u = (f[1] - f[2]) / rho
        b = f + (orc.d1q3_feq(rho, u) - f) / tau  # Eq. (bgkcollision)
        assert np.max(np.abs(a - b)) < 2e-15 * rho


def test_trt_with_equal_rates_is_srt(orc):
    """Table III: with tau2 = tau every non-conserved rate of TRT is 1/tau and
    the conserved moments of f^eq - f vanish, so TRT = SRT."""
    for f in _random_states(20, seed=9):
        a, _ = orc.d2q9_mrt(f, 0.8, trt=True, tau2_=0.8)
        b, _ = orc.d2q9_srt(f, 0.8)
        assert np.max(np.abs(a - b)) < 1e-15


# ----------------------------------------------------------------------------
# Streaming and boundaries (Eq. 2, Sec. IV.F).
# ----------------------------------------------------------------------------
def test_periodic_streaming_is_a_shift(orc):
    nx, ny = 7, 5
    sim = orc.Sim(orc.D2Q9, nx, ny, 0.8, orc.BC_PERIODIC, collision=orc.NONE)
    f0 = wl.random_populations(9, ny, nx, seed=1)
    sim.set_f(f0)
    sim.step(1)
    v, _, _, _ = orc.d2q9_tables()
    f1 = sim.get_f()
    for a in range(9):
        assert np.array_equal(f1[a], np.roll(f0[a], shift=(v[a, 1], v[a, 0]), axis=(0, 1)))
    sim.step(nx * ny - 1)
    assert np.array_equal(sim.get_f(), f0)


def test_bounce_back_round_trip(orc):
    """Full-way bounce-back: a population sent into a wall returns reversed to
    the same node two steps later (identity collision isolates the walls)."""
    v, _, _, _ = orc.d2q9_tables()
    opp = [int(np.where((v == -v[a]).all(axis=1))[0][0]) for a in range(9)]
    n = 6
    for a, (x, y) in [(4, (3, 1)), (3, (1, 2)), (1, (n - 2, 3)), (7, (1, 1)), (8, (n - 2, 1))]:
        sim = orc.Sim(orc.D2Q9, n, n, 0.8, orc.BC_CAVITY, collision=orc.NONE, rho0=1.0, u_lid=0.0)
        f0 = np.zeros((9, n, n))
        f0[a, y, x] = 1.0
        sim.set_f(f0)
        sim.step(2)
        f2 = sim.get_f()
        assert f2[opp[a], y, x] == 1.0
        f2[opp[a], y, x] = 0.0
        # everything else is the out-of-lattice fill (rho0 W) or the lid, never the marker
        assert not np.any(f2 == 1.0)


def test_resting_cavity_stays_at_rest(orc):
    n = 12
    rho, ux, uy = wl.cavity(n, rho0=1.0)
    sim = orc.Sim(orc.D2Q9, n, n, 0.6, orc.BC_CAVITY, rho0=1.0, u_lid=0.0)
    sim.init(rho, ux, uy)
    sim.step(30)
    r, x, y = sim.moments()
    assert np.abs(r - 1.0).max() < 1e-15
    assert np.abs(x).max() < 1e-15 and np.abs(y).max() < 1e-15


def test_zero_gradient_ends(orc):
    n = 9
    sim = orc.Sim(orc.D1Q3, n, 1, 0.8, orc.BC_ZERO_GRADIENT, collision=orc.NONE)
    f0 = wl.random_populations(3, 1, n, seed=4)
    sim.set_f(f0)
    sim.step(1)
    f1 = sim.get_f()
    assert f1[1, 0, 0] == f0[1, 0, 0]        # +1 population at the left end: own copy
    assert f1[2, 0, n - 1] == f0[2, 0, n - 1]  # -1 population at the right end
    assert np.array_equal(f1[1, 0, 1:], f0[1, 0, :-1])
    assert np.array_equal(f1[2, 0, :-1], f0[2, 0, 1:])


def test_periodic_conservation(orc):
    n = 24
    rho, ux, uy = wl.taylor_green(n, u0=0.05)
    for col in (orc.MINXENT4, orc.MINXENT2, orc.SRT):
        sim = orc.Sim(orc.D2Q9, n, n, 0.52, orc.BC_PERIODIC, collision=col)
        sim.init(rho, ux, uy)
        c0 = sim.conservation()
        sim.step(100)
        c1 = sim.conservation()
        assert abs(c1[0] - c0[0]) < 1e-13 * c0[0]
        assert np.abs(c1[1:] - c0[1:]).max() < 1e-13 * c0[0]


# ----------------------------------------------------------------------------
# Physics: shear viscosity from Eq. (visco-tau) via Taylor-Green decay.
# ----------------------------------------------------------------------------
def _tg_rate(orc, n, nu, steps, collision, u0=0.02):
    rho, ux, uy = wl.taylor_green(n, u0=u0)
    sim = orc.Sim(orc.D2Q9, n, n, orc.tau_from_nu(nu), orc.BC_PERIODIC, collision=collision)
    sim.init(rho, ux, uy)
    ts, es = [], []
    chunk = steps // 10
    for k in range(11):
        r, x, y = sim.moments()
        ts.append(k * chunk)
        es.append(0.5 * float((r * (x * x + y * y)).sum()))
        if k < 10:
            sim.step(chunk)
    slope = -np.polyfit(ts, np.log(es), 1)[0]
    return slope, wl.taylor_green_energy_rate(nu, n)


@pytest.mark.parametrize("collision", [0, 1])  # MINXENT4, SRT
def test_taylor_green_decay_rate(orc, collision):
    rate, expect = _tg_rate(orc, 32, 0.02, 400, collision)
    assert rate == pytest.approx(expect, rel=1e-2)


def test_taylor_green_decay_low_viscosity(orc):
    """nu = 1e-3 as in the 512^2 run, on 64^2.  The equilibrium start launches
    acoustic waves that bias the fitted rate by ~2% for any collision rule, so
    the closed form is checked at 3%, and MinxEnt4 against SRT (same stress
    relaxation 1/tau via Eqs. discreteviscoconst/isoconst) at 0.2%."""
    rate, expect = _tg_rate(orc, 64, 1e-3, 2000, 0)
    rate_srt, _ = _tg_rate(orc, 64, 1e-3, 2000, 1)
    assert rate == pytest.approx(expect, rel=3e-2)
    assert rate == pytest.approx(rate_srt, rel=2e-3)


# ----------------------------------------------------------------------------
# Stream function of the LDAS post-processing (Sec. IV.I).
# ----------------------------------------------------------------------------
def test_stream_function_closed_forms(orc):
    """psi = -int_0^x u_y dx per row with composite Simpson over pairs of
    unit intervals and the trapezoid on a last odd interval:
      u = a + b x  -> exact:            -(a x + b x^2 / 2)
      u = x^2      -> Simpson exact at even x (-x^3/3); at odd x the
                      trapezoid over [x-1, x] adds 1/6:  -(x^3/3 + 1/6)
      u = x^3      -> Simpson exact at even x:          -x^4/4."""
    nx = 21
    x = np.arange(nx, dtype=float)
    uy = np.stack([0.3 - 0.05 * x, x ** 2, x ** 3])
    psi = orc.stream_function(uy)
    np.testing.assert_allclose(psi[0], -(0.3 * x - 0.025 * x ** 2), rtol=0, atol=1e-13)
    even, odd = x[0::2], x[1::2]
    np.testing.assert_allclose(psi[1, 0::2], -even ** 3 / 3, rtol=1e-14, atol=1e-12)
    np.testing.assert_allclose(psi[1, 1::2], -(odd ** 3 / 3 + 1 / 6), rtol=1e-14, atol=1e-12)
    np.testing.assert_allclose(psi[2, 0::2], -even ** 4 / 4, rtol=1e-14, atol=1e-12)


def test_stream_function_matches_library_simpson_and_converges(orc):
    """At even x the rule is the composite Simpson rule of scipy; for a
    smooth profile the error falls as h^4."""
    integrate = pytest.importorskip("scipy.integrate")
    rng = np.random.default_rng(4)
    uy = rng.standard_normal((3, 33))
    psi = orc.stream_function(uy)
    for k in range(2, 33, 2):
        ref = -integrate.simpson(uy[:, :k + 1], dx=1.0, axis=1)
        np.testing.assert_allclose(psi[:, k], ref, rtol=1e-12, atol=1e-12)
    errs = []
    for n in (17, 33, 65):
        L = n - 1
        x = np.arange(n, dtype=float)
        u = np.sin(np.pi * x / L)[None, :]
        exact = -(L / np.pi) * (1 - np.cos(np.pi * x / L))
        # error relative to the integral's scale L (spacing h = 1/L)
        errs.append(np.abs(orc.stream_function(u)[0, 0::2] - exact[0::2]).max() / L)
    assert errs[0] / errs[1] > 14 and errs[1] / errs[2] > 14, errs


def _table3(golden_dir):
    rows = {}
    for line in open(os.path.join(golden_dir, "table3_rates.txt")):
        line = line.split("#")[0].split()
        if line:
            rows[line[0]] = line[1:]
    return rows


def _rate(token: str, tau: float, tau2: float) -> float:
    return {"1/tau": 1.0 / tau, "1/tau2": 1.0 / tau2}.get(token) or float(token)


@pytest.mark.parametrize("rule", ["MRT", "TRT"])
@pytest.mark.parametrize("tau", [0.6, 0.7])
@pytest.mark.parametrize("reading", ["printed", "magic"])
def test_mrt_trt_rates_match_table3(orc, golden_dir, rule, tau, reading):
    """Table III, one moment at a time.  Start from f^eq(rho, u) and add
    eps rho (T^-1)_{:,k} for one non-conserved moment k (this leaves rho and u,
    hence f^eq, unchanged).  Eq. (mrtcollision) then moves only moment k,
    T (f^post - f^eq) = eps rho (1 - B_k) e_k, so B_k is read off and compared
    with the printed table; T^-1 here is numpy's inverse of the printed T.
    tau2 differs from tau under both readings of Eq. (tau2)."""
    T = np.loadtxt(os.path.join(golden_dir, "tmatrix.txt"))
    Tinv = np.linalg.inv(T)
    tau2 = (8 * tau - 1) / ((8.0 if reading == "magic" else 1.0) * (2 * tau - 1))
    assert abs(tau2 - tau) > 0.05
    table = _table3(golden_dir)[rule]
    rho, ux, uy, eps = 1.3, 0.04, -0.03, 1e-3
    feq = orc.d2q9_feq(rho, ux, uy)
    for k in range(9):
        if k in (0, 3, 5):  # mass and momentum: fixed by the conservation pins
            assert table[k] == "0"
            continue
        f = feq + eps * rho * Tinv[:, k]
        post, st = orc.d2q9_mrt(f, tau, trt=(rule == "TRT"), tau2_=tau2)
        assert st == 0
        m = T @ (post - feq) / (eps * rho)
        want = np.zeros(9)
        want[k] = 1.0 - _rate(table[k], tau, tau2)
        assert np.max(np.abs(m - want)) < 1e-10, (k, m, want)
