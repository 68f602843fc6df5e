/*
 * lbm_oracle.c -- plain, slow, FP64 CPU implementation of MinxEnt-LBM.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the oracle the CUDA path is checked
 * against.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark load it; the product library never does, and the two share no
 * code, header, table or helper.
 *
 * Source: T. L. Wilson, M. Pugh, F. Dawson, "Stabilization of the Lattice
 * Boltzmann Method Using Information Theory", arXiv:1801.03863.  Every
 * function names the section / equation / table it follows.  Readings of
 * points the paper leaves open are marked "reading:".
 *
 * Style: nested loops over nodes and populations, no blocking, no fusion, no
 * shortcuts from the structure of T (its inverse is obtained by Gauss-Jordan
 * elimination, moments by explicit matrix-vector products, linear systems by
 * Gaussian elimination with partial pivoting).  The only parallelism is an
 * OpenMP loop over lattice rows in the collision and streaming passes; every
 * node is independent there, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Codes used across the Python wrapper.                                      */
/* ------------------------------------------------------------------------ */
enum { ORC_D1Q3 = 1, ORC_D2Q9 = 2 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_ZERO_GRADIENT = 1, ORC_BC_CAVITY = 2 };
enum {
    ORC_MINXENT4 = 0, /* Sec. IV.C-E, four free moments                       */
    ORC_SRT = 1,      /* Eq. (bgkcollision)                                    */
    ORC_MINXENT2 = 2, /* Sec. IV.C-E, two free moments, extra constraints c5,c7 */
    ORC_MRT = 3,      /* Eq. (mrtcollision) with Table III "MRT-LBM"          */
    ORC_TRT = 4,      /* Eq. (mrtcollision) with Table III "TRT-LBM"          */
    ORC_NONE = 9      /* identity collision: isolates streaming and boundaries */
};
/* per-node status bits */
enum { ORC_NEWTON_SKIPPED = 1, ORC_UNSTABLE = 2 };
/* where the Newton gradient/Hessian is evaluated (reading C-START) */
enum { ORC_START_HYBRID = 0, ORC_START_EQUILIBRIUM = 1 };

/* ------------------------------------------------------------------------ */
/* D2Q9 lattice.                                                              */
/*                                                                            */
/* Velocities and weights: Table I.  Table I numbers the rest velocity 9th,   */
/* but the columns of T (Eq. Tmatrix) put it first: row 4 of T is v_x and     */
/* row 6 is v_y only in the order below.  Reading: T's column order is used   */
/* for everything.                                                            */
/* ------------------------------------------------------------------------ */
static const int V9[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                             {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* T as printed in Eq. (Tmatrix). */
static const int T9[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},        {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},     {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},     {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};
static double TINV9[9][9]; /* filled by orc_init_tables() */

/* D1Q3 (reading C-D1Q3: the paper does not list D1Q3; these are the standard
 * three-velocity quadrature with c_s^2 = 1/3, the 1D restriction of Table I). */
static const int V3[3] = {0, 1, -1};
static const double W3[3] = {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0};

/* Opposite direction index (full-way bounce-back, Sec. IV.F). */
static int opp9(int a) {
    for (int b = 0; b < 9; ++b)
        if (V9[b][0] == -V9[a][0] && V9[b][1] == -V9[a][1]) return b;
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Dense linear algebra (plain Gaussian elimination).                         */
/* ------------------------------------------------------------------------ */

/* Solve A x = b (n <= 9) by Gaussian elimination with partial pivoting.
 * A and b are copied.  Returns 0, or -1 for a singular matrix. */
static int gauss_solve(int n, const double* A_in, const double* b_in, double* x) {
    double A[9][10];
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) A[i][j] = A_in[i * n + j];
        A[i][n] = b_in[i];
    }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return -1;
        if (piv != c)
            for (int j = 0; j <= n; ++j) {
                double t = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = t;
            }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r][c] / A[c][c];
            for (int j = c; j <= n; ++j) A[r][j] -= f * A[c][j];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = A[i][n];
        for (int j = i + 1; j < n; ++j) s -= A[i][j] * x[j];
        x[i] = s / A[i][i];
    }
    return 0;
}

/* Inverse of T (Eq. Tmatrix) by Gauss-Jordan elimination with partial
 * pivoting -- deliberately not the transpose-over-norms shortcut. */
static void invert9(const int Tin[9][9], double out[9][9]) {
    double A[9][18];
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 18; ++j)
            A[i][j] = (j < 9) ? (double)Tin[i][j] : (j - 9 == i ? 1.0 : 0.0);
    for (int c = 0; c < 9; ++c) {
        int piv = c;
        for (int r = c + 1; r < 9; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        for (int j = 0; j < 18; ++j) {
            double t = A[c][j];
            A[c][j] = A[piv][j];
            A[piv][j] = t;
        }
        double d = A[c][c];
        for (int j = 0; j < 18; ++j) A[c][j] /= d;
        for (int r = 0; r < 9; ++r) {
            if (r == c) continue;
            double f = A[r][c];
            for (int j = 0; j < 18; ++j) A[r][j] -= f * A[c][j];
        }
    }
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) out[i][j] = A[i][9 + j];
}

__attribute__((constructor)) static void orc_init_tables(void) { invert9(T9, TINV9); }

/* ------------------------------------------------------------------------ */
/* Tables, exported for the pin tests.                                        */
/* ------------------------------------------------------------------------ */
ORC_EXPORT void orc_d2q9_tables(int32_t* v /*9x2*/, double* w /*9*/, int32_t* T /*9x9*/,
                                double* Tinv /*9x9*/) {
    for (int a = 0; a < 9; ++a) {
        v[2 * a] = V9[a][0];
        v[2 * a + 1] = V9[a][1];
        w[a] = W9[a];
    }
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            T[i * 9 + j] = T9[i][j];
            Tinv[i * 9 + j] = TINV9[i][j];
        }
}

ORC_EXPORT void orc_d1q3_tables(int32_t* v /*3*/, double* w /*3*/) {
    for (int a = 0; a < 3; ++a) {
        v[a] = V3[a];
        w[a] = W3[a];
    }
}

/* ------------------------------------------------------------------------ */
/* Equilibria.                                                                */
/* ------------------------------------------------------------------------ */

/* D2Q9 polynomial equilibrium, Eq. (numerical-plyeqm). */
ORC_EXPORT void orc_d2q9_feq(double rho, double ux, double uy, double* feq) {
    double uu = ux * ux + uy * uy;
    for (int a = 0; a < 9; ++a) {
        double vu = V9[a][0] * ux + V9[a][1] * uy;
        feq[a] = W9[a] * rho * (1.0 + 3.0 * vu + 4.5 * vu * vu - 1.5 * uu);
    }
}

/* D1Q3 polynomial equilibrium: Eq. (numerical-plyeqm) restricted to one
 * dimension (reading C-D1Q3). */
ORC_EXPORT void orc_d1q3_feq(double rho, double u, double* feq) {
    for (int a = 0; a < 3; ++a) {
        double vu = V3[a] * u;
        feq[a] = W3[a] * rho * (1.0 + 3.0 * vu + 4.5 * vu * vu - 1.5 * u * u);
    }
}

/* Discrete Kullback-Leibler divergence, Eq. (discrete_KLD):
 * H(p) = sum_a p_a ln(p_a / w_a). */
ORC_EXPORT double orc_kld(int q, const double* p, const double* w) {
    double h = 0.0;
    for (int a = 0; a < q; ++a) h += p[a] * log(p[a] / w[a]);
    return h;
}

/* ------------------------------------------------------------------------ */
/* Moment-space helpers (Sec. IV.E): M = T p and p = T^{-1} M.                */
/* ------------------------------------------------------------------------ */
static void mat_T_p(const double* p, double* M) {
    for (int k = 0; k < 9; ++k) {
        double s = 0.0;
        for (int a = 0; a < 9; ++a) s += T9[k][a] * p[a];
        M[k] = s;
    }
}
static void mat_Tinv_M(const double* M, double* p) {
    for (int a = 0; a < 9; ++a) {
        double s = 0.0;
        for (int k = 0; k < 9; ++k) s += TINV9[a][k] * M[k];
        p[a] = s;
    }
}

/* S(M) = H(T^{-1} M), Eq. (KL-moment).  Returns +inf if some p_a <= 0. */
static double entropy_of_M(const double* M) {
    double p[9];
    mat_Tinv_M(M, p);
    for (int a = 0; a < 9; ++a)
        if (!(p[a] > 0.0)) return INFINITY;
    return orc_kld(9, p, W9);
}

/* Gradient (with the "+1" term as printed) and Hessian of S with respect to
 * the free moments, Sec. IV.E.  Reading C-IDX: the free index k runs over the
 * positions of the free moments in M, i.e. columns free[k] of T^{-1}. */
static void grad_hess(const double* p, int nfree, const int* free, double* g, double* H) {
    for (int k = 0; k < nfree; ++k) {
        double s = 0.0;
        for (int a = 0; a < 9; ++a) s += TINV9[a][free[k]] * (log(p[a] / W9[a]) + 1.0);
        g[k] = s;
    }
    for (int j = 0; j < nfree; ++j)
        for (int k = 0; k < nfree; ++k) {
            double s = 0.0;
            for (int a = 0; a < 9; ++a) s += TINV9[a][free[k]] * TINV9[a][free[j]] / p[a];
            H[j * nfree + k] = s;
        }
}

/* Positions (0-based) of the free moments m in M, Sec. IV.E:
 * MinxEnt4: m = (M2, M3, M5, M7);  MinxEnt2: m = (M2, M3). */
static const int FREE4[4] = {1, 2, 4, 6};
static const int FREE2[2] = {1, 2};

/* tau_2 of Eq. (tau2), as printed. */
ORC_EXPORT double orc_tau2(double tau) { return (8.0 * tau - 1.0) / (2.0 * tau - 1.0); }

/*
 * Common set-up of the MinxEnt collision, step 1 of the algorithm in
 * Sec. IV.E: pre-collision and equilibrium moments, the constraint values
 * (Eqs. discreteprobconst .. discreteisoconst and, for MinxEnt2,
 * extraconstraint1/2), and the start vector M^start whose constrained entries
 * hold the constraint values and whose free entries hold m^0 = the free
 * entries of M^0 = T p^eq.
 *
 * Reading C-RHO: the collision acts on p = f / rho with the node's own
 * pre-collision density, which the constraints conserve (Eq. fandpdef).
 * Reading C-EQ: p^eq is the polynomial equilibrium (numerical-plyeqm).
 */
static void minxent_setup(const double* f, double tau, double tau2, int nfree, double* rho_out,
                          double* Mstart, double* M0) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < 9; ++a) {
        rho += f[a];
        jx += f[a] * V9[a][0];
        jy += f[a] * V9[a][1];
    }
    double ux = jx / rho, uy = jy / rho;
    double ppre[9], feq[9], peq[9];
    orc_d2q9_feq(rho, ux, uy, feq);
    for (int a = 0; a < 9; ++a) {
        ppre[a] = f[a] / rho;
        peq[a] = feq[a] / rho;
    }
    mat_T_p(peq, M0);
    /* c8, c9: Eqs. (discreteviscoconst), (discreteisoconst). */
    double c8 = 0.0, c9 = 0.0;
    for (int a = 0; a < 9; ++a) {
        double relaxed = ppre[a] + (peq[a] - ppre[a]) / tau;
        c8 += relaxed * (V9[a][0] * V9[a][0] - V9[a][1] * V9[a][1]);
        c9 += relaxed * (V9[a][0] * V9[a][1]);
    }
    Mstart[0] = 1.0; /* Eq. (discreteprobconst) */
    Mstart[3] = ux;  /* Eq. (discretexmomconst) */
    Mstart[5] = uy;
    Mstart[7] = c8;
    Mstart[8] = c9;
    if (nfree == 4) {
        for (int k = 0; k < 4; ++k) Mstart[FREE4[k]] = M0[FREE4[k]];
    } else {
        /* c5, c7: Eqs. (extraconstraint1/2), relaxed at rate 1/tau2.  The
         * stray comma in the printed equation is read as a product (C-C5). */
        double c5 = 0.0, c7 = 0.0;
        for (int a = 0; a < 9; ++a) {
            double relaxed = ppre[a] + (peq[a] - ppre[a]) / tau2;
            double vv = V9[a][0] * V9[a][0] + V9[a][1] * V9[a][1];
            c5 += relaxed * (-5.0 + 3.0 * vv) * V9[a][0];
            c7 += relaxed * (-5.0 + 3.0 * vv) * V9[a][1];
        }
        Mstart[1] = M0[1];
        Mstart[2] = M0[2];
        Mstart[4] = c5;
        Mstart[6] = c7;
    }
    *rho_out = rho;
}

/*
 * One MinxEnt collision at one node, the five-step algorithm of Sec. IV.E
 * with a single Newton-Raphson step ("terminate after a single step").
 *
 *   f      pre-collision populations (9, Table I in T's column order)
 *   tau    relaxation time; tau2 only used for MinxEnt2 (nfree == 2)
 *   nfree  4 (MinxEnt4) or 2 (MinxEnt2)
 *   start  ORC_START_HYBRID (reading C-START: gradient and Hessian at M^start,
 *          i.e. constraints already imposed) or ORC_START_EQUILIBRIUM
 *          (evaluate at M^0 = T p^eq itself; kept for comparison only)
 *   fpost  post-collision populations
 * Returns status bits: ORC_NEWTON_SKIPPED when some p^start_a <= 0 (reading
 * C-NEG: keep p^start, which satisfies every constraint), ORC_UNSTABLE when
 * some post-collision population is negative or not finite (Sec. IV.H's
 * stability criterion).
 */
ORC_EXPORT int orc_d2q9_minxent(const double* f, double tau, double tau2, int nfree, int start,
                                double* fpost) {
    const int* free = (nfree == 4) ? FREE4 : FREE2;
    double rho, Mstart[9], M0[9];
    minxent_setup(f, tau, tau2, nfree, &rho, Mstart, M0);
    int status = 0;

    /* Step 2: H and grad S at the evaluation point. */
    double Meval[9];
    for (int k = 0; k < 9; ++k) Meval[k] = (start == ORC_START_EQUILIBRIUM) ? M0[k] : Mstart[k];
    double p[9];
    mat_Tinv_M(Meval, p);
    int positive = 1;
    for (int a = 0; a < 9; ++a)
        if (!(p[a] > 0.0)) positive = 0;

    double Mpost[9];
    for (int k = 0; k < 9; ++k) Mpost[k] = Mstart[k];
    if (positive) {
        double g[4], H[16], s[4];
        grad_hess(p, nfree, free, g, H);
        /* Step 3: m^1 = m^0 - H^{-1} grad S. */
        if (gauss_solve(nfree, H, g, s) == 0) {
            /* Step 4: M^post = constraints + m^1. */
            for (int k = 0; k < nfree; ++k) Mpost[free[k]] = Mstart[free[k]] - s[k];
        } else {
            status |= ORC_NEWTON_SKIPPED;
        }
    } else {
        status |= ORC_NEWTON_SKIPPED;
    }
    /* Step 5: p^post = T^{-1} M^post, f^post = rho p^post. */
    double ppost[9];
    mat_Tinv_M(Mpost, ppost);
    for (int a = 0; a < 9; ++a) {
        fpost[a] = rho * ppost[a];
        if (!(fpost[a] >= 0.0) || !isfinite(fpost[a])) status |= ORC_UNSTABLE;
    }
    return status;
}

/*
 * The exact constrained minimiser of Eq. (minxentLBM-collision): Newton's
 * iteration of Sec. IV.E continued to convergence, with a backtracking line
 * search on S that keeps every p_a positive.  Stops when the largest gradient
 * entry is below gtol or after maxit iterations.  Returns the number of
 * iterations taken, or -1 if the start point is not positive.
 */
ORC_EXPORT int orc_d2q9_minxent_converged(const double* f, double tau, double tau2, int nfree,
                                          double gtol, int maxit, double* fpost,
                                          double* gnorm_out) {
    const int* free = (nfree == 4) ? FREE4 : FREE2;
    double rho, M[9], M0[9];
    minxent_setup(f, tau, tau2, nfree, &rho, M, M0);
    double p[9];
    mat_Tinv_M(M, p);
    for (int a = 0; a < 9; ++a)
        if (!(p[a] > 0.0)) return -1;
    int it = 0;
    double gnorm = 0.0;
    for (;;) {
        double g[4], H[16], s[4];
        mat_Tinv_M(M, p);
        grad_hess(p, nfree, free, g, H);
        gnorm = 0.0;
        for (int k = 0; k < nfree; ++k)
            if (fabs(g[k]) > gnorm) gnorm = fabs(g[k]);
        if (gnorm < gtol || it >= maxit) break;
        if (gauss_solve(nfree, H, g, s) != 0) break;
        double S0 = entropy_of_M(M), gs = 0.0;
        for (int k = 0; k < nfree; ++k) gs += g[k] * s[k];
        double t = 1.0, Mtry[9];
        for (int ls = 0; ls < 60; ++ls) {
            for (int k = 0; k < 9; ++k) Mtry[k] = M[k];
            for (int k = 0; k < nfree; ++k) Mtry[free[k]] = M[free[k]] - t * s[k];
            double St = entropy_of_M(Mtry);
            if (!isfinite(St)) { t *= 0.5; continue; } /* left the simplex */
            /* Armijo condition on S ... */
            if (St <= S0 - 1e-4 * t * gs) break;
            /* ... or, once S no longer resolves the decrease (near the
             * optimum), a smaller gradient at the trial point. */
            double ptry[9], gt[4], Ht[16], gtn = 0.0;
            mat_Tinv_M(Mtry, ptry);
            grad_hess(ptry, nfree, free, gt, Ht);
            for (int k = 0; k < nfree; ++k)
                if (fabs(gt[k]) > gtn) gtn = fabs(gt[k]);
            if (gtn < gnorm && St <= S0 + 1e-14) break;
            t *= 0.5;
        }
        for (int k = 0; k < 9; ++k) M[k] = Mtry[k];
        ++it;
    }
    mat_Tinv_M(M, p);
    for (int a = 0; a < 9; ++a) fpost[a] = rho * p[a];
    if (gnorm_out) *gnorm_out = gnorm;
    return it;
}

/* SRT-LBM collision, Eq. (bgkcollision), with the polynomial equilibrium. */
ORC_EXPORT int orc_d2q9_srt(const double* f, double tau, double* fpost) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < 9; ++a) {
        rho += f[a];
        jx += f[a] * V9[a][0];
        jy += f[a] * V9[a][1];
    }
    double feq[9];
    orc_d2q9_feq(rho, jx / rho, jy / rho, feq);
    int status = 0;
    for (int a = 0; a < 9; ++a) {
        fpost[a] = f[a] + (feq[a] - f[a]) / tau;
        if (!(fpost[a] >= 0.0) || !isfinite(fpost[a])) status |= ORC_UNSTABLE;
    }
    return status;
}

/* MRT-LBM collision, Eq. (mrtcollision): f + T^{-1} B T (f^eq - f), with
 * the diagonal B of Table III for MRT-LBM or TRT-LBM. */
ORC_EXPORT int orc_d2q9_mrt(const double* f, double tau, double tau2, int trt, double* fpost) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < 9; ++a) {
        rho += f[a];
        jx += f[a] * V9[a][0];
        jy += f[a] * V9[a][1];
    }
    double feq[9], d[9], Md[9], BMd[9], back[9];
    orc_d2q9_feq(rho, jx / rho, jy / rho, feq);
    for (int a = 0; a < 9; ++a) d[a] = feq[a] - f[a];
    double B[9];
    if (trt) {
        double b[9] = {0, 1 / tau, 1 / tau, 0, 1 / tau2, 0, 1 / tau2, 1 / tau, 1 / tau};
        memcpy(B, b, sizeof b);
    } else {
        double b[9] = {0, 1.64, 1.54, 0, 1 / tau2, 0, 1 / tau2, 1 / tau, 1 / tau};
        memcpy(B, b, sizeof b);
    }
    mat_T_p(d, Md);
    for (int k = 0; k < 9; ++k) BMd[k] = B[k] * Md[k];
    mat_Tinv_M(BMd, back);
    int status = 0;
    for (int a = 0; a < 9; ++a) {
        fpost[a] = f[a] + back[a];
        if (!(fpost[a] >= 0.0) || !isfinite(fpost[a])) status |= ORC_UNSTABLE;
    }
    return status;
}

/*
 * D1Q3 MinxEnt collision (reading C-D1Q3).  With three velocities the
 * constraints -- mass (Eq. discreteprobconst), momentum (Eq.
 * discretexmomconst) and the relaxed second moment (the 1D restatement of
 * Eq. discreteviscoconst) -- are three linear equations in the three p_a,
 * so the constraint set holds one point and the minimisation is trivial
 * (Sec. IV.G calls D1Q3 "over constrained").  The point is found by solving
 * the 3x3 system.
 */
ORC_EXPORT int orc_d1q3_minxent(const double* f, double tau, double* fpost) {
    double rho = 0.0, j = 0.0;
    for (int a = 0; a < 3; ++a) {
        rho += f[a];
        j += f[a] * V3[a];
    }
    double u = j / rho, feq[3];
    orc_d1q3_feq(rho, u, feq);
    double c2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double ppre = f[a] / rho, peq = feq[a] / rho;
        c2 += (ppre + (peq - ppre) / tau) * V3[a] * V3[a];
    }
    double A[9], b[3] = {1.0, u, c2}, p[3];
    for (int a = 0; a < 3; ++a) {
        A[0 * 3 + a] = 1.0;
        A[1 * 3 + a] = V3[a];
        A[2 * 3 + a] = V3[a] * V3[a];
    }
    gauss_solve(3, A, b, p);
    int status = 0;
    for (int a = 0; a < 3; ++a) {
        fpost[a] = rho * p[a];
        if (!(fpost[a] >= 0.0) || !isfinite(fpost[a])) status |= ORC_UNSTABLE;
    }
    return status;
}

/* D1Q3 SRT collision, Eq. (bgkcollision). */
ORC_EXPORT int orc_d1q3_srt(const double* f, double tau, double* fpost) {
    double rho = 0.0, j = 0.0;
    for (int a = 0; a < 3; ++a) {
        rho += f[a];
        j += f[a] * V3[a];
    }
    double feq[3];
    orc_d1q3_feq(rho, j / rho, feq);
    int status = 0;
    for (int a = 0; a < 3; ++a) {
        fpost[a] = f[a] + (feq[a] - f[a]) / tau;
        if (!(fpost[a] >= 0.0) || !isfinite(fpost[a])) status |= ORC_UNSTABLE;
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Lattice simulation: Eq. (2) collide-then-stream, boundaries of Sec. IV.F.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int lattice, q, nx, ny, bc, collision, start;
    double tau, tau2, rho0, u_lid;
    double* f; /* pre-collision populations f(x, t_n), [node][q] */
    double* g; /* post-collision scratch */
    long long n_skipped, n_unstable, steps;
    /* Slab of a taller lattice (orc_set_slab): local row y is global row
     * y + y_off of ny_global rows. */
    int y_off, ny_global;
} orc_sim;

ORC_EXPORT double orc_tau_from_nu(double nu) {
    /* Eq. (visco-tau) with delta_x = delta_t = 1: nu = (2 tau - 1) / 6. */
    return 3.0 * nu + 0.5;
}

ORC_EXPORT orc_sim* orc_create(int lattice, int nx, int ny, double tau, int bc, int collision,
                               double rho0, double u_lid) {
    if ((lattice != ORC_D1Q3 && lattice != ORC_D2Q9) || nx < 1 || ny < 1 || !(tau > 0.5))
        return NULL;
    if (lattice == ORC_D1Q3 && ny != 1) return NULL;
    if (bc == ORC_BC_CAVITY && (lattice != ORC_D2Q9 || nx < 3 || ny < 3)) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->lattice = lattice;
    s->q = (lattice == ORC_D2Q9) ? 9 : 3;
    s->nx = nx;
    s->ny = ny;
    s->bc = bc;
    s->collision = collision;
    s->start = ORC_START_HYBRID;
    s->tau = tau;
    s->tau2 = orc_tau2(tau);
    s->rho0 = rho0;
    s->u_lid = u_lid;
    s->y_off = 0;
    s->ny_global = ny;
    size_t n = (size_t)nx * ny * s->q;
    s->f = (double*)calloc(n, sizeof(double));
    s->g = (double*)calloc(n, sizeof(double));
    return s;
}

ORC_EXPORT void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->f);
    free(s->g);
    free(s);
}

ORC_EXPORT void orc_set_start(orc_sim* s, int start) { s->start = start; }
ORC_EXPORT void orc_set_tau2(orc_sim* s, double tau2) { s->tau2 = tau2; }

/* Initial populations at equilibrium (Sec. IV.F). rho, ux, uy: [y][x]. */
ORC_EXPORT void orc_init(orc_sim* s, const double* rho, const double* ux, const double* uy) {
    size_t nn = (size_t)s->nx * s->ny;
    for (size_t i = 0; i < nn; ++i) {
        double* fi = s->f + i * s->q;
        double vx = ux ? ux[i] : 0.0, vy = uy ? uy[i] : 0.0;
        if (s->lattice == ORC_D2Q9)
            orc_d2q9_feq(rho[i], vx, vy, fi);
        else
            orc_d1q3_feq(rho[i], vx, fi);
    }
    s->steps = 0;
}

/* Populations in and out, layout [a][y][x]. */
ORC_EXPORT void orc_set_f(orc_sim* s, const double* f) {
    size_t nn = (size_t)s->nx * s->ny;
    for (int a = 0; a < s->q; ++a)
        for (size_t i = 0; i < nn; ++i) s->f[i * s->q + a] = f[a * nn + i];
}
ORC_EXPORT void orc_get_f(const orc_sim* s, double* f) {
    size_t nn = (size_t)s->nx * s->ny;
    for (int a = 0; a < s->q; ++a)
        for (size_t i = 0; i < nn; ++i) f[a * nn + i] = s->f[i * s->q + a];
}

/* Node classes of the lid-driven cavity (readings C-WALL, C-LID): the outer
 * ring x = 0, x = nx-1, y = 0 (and the two top corners) are bounce-back
 * walls, the top row y = ny-1 strictly between the corners is the lid. */
enum { NODE_FLUID = 0, NODE_WALL = 1, NODE_LID = 2 };
static int node_class(const orc_sim* s, int x, int y) {
    if (s->bc != ORC_BC_CAVITY) return NODE_FLUID;
    const int yg = y + s->y_off; /* row in the whole lattice */
    if (x == 0 || x == s->nx - 1 || yg == 0) return NODE_WALL;
    if (yg == s->ny_global - 1) return NODE_LID;
    return NODE_FLUID;
}

static int collide_node(const orc_sim* s, const double* f, double* g) {
    if (s->lattice == ORC_D1Q3) {
        switch (s->collision) {
            case ORC_SRT: return orc_d1q3_srt(f, s->tau, g);
            case ORC_NONE: memcpy(g, f, 3 * sizeof(double)); return 0;
            default: return orc_d1q3_minxent(f, s->tau, g);
        }
    }
    switch (s->collision) {
        case ORC_SRT: return orc_d2q9_srt(f, s->tau, g);
        case ORC_MRT: return orc_d2q9_mrt(f, s->tau, s->tau2, 0, g);
        case ORC_TRT: return orc_d2q9_mrt(f, s->tau, s->tau2, 1, g);
        case ORC_MINXENT2: return orc_d2q9_minxent(f, s->tau, s->tau2, 2, s->start, g);
        case ORC_NONE: memcpy(g, f, 9 * sizeof(double)); return 0;
        default: return orc_d2q9_minxent(f, s->tau, s->tau2, 4, s->start, g);
    }
}

/*
 * One time step of Eq. (2), in its two halves: collide every node, then
 * stream.
 *
 * Collision (per node class, Sec. IV.F):
 *   fluid: the configured collision rule;
 *   wall:  full-way bounce-back, g_a = f_opp(a);
 *   lid:   g = f^eq(rho0, (u_lid, 0)) (reading C-LID: the lid density is the
 *          configured reference density rho0).
 * Streaming, f(x, t+1)_a = g_a(x - v_a)  (Eq. 2 with x_j = x - v_a):
 *   periodic: indices wrap;
 *   zero-gradient ends (reading C-ZG): the ghost node beyond each end holds a
 *     copy of the end node's post-collision populations;
 *   cavity: a source outside the lattice (only ring nodes have one) gives
 *     W_a rho0 (reading; such values never reach a fluid node).
 * A slab (orc_set_slab) streams across its lower / upper edge from the halo
 * rows lo / hi: the post-collision row below its first row and above its
 * last one, as the neighbouring slabs computed them ([a][x], q * nx values;
 * NULL = the boundary rule of the lattice applies at that edge).
 */
static void collide_pass(orc_sim* s) {
    const int q = s->q, nx = s->nx, ny = s->ny;
    long long skipped = 0, unstable = 0;
#pragma omp parallel for reduction(+ : skipped, unstable) schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            const double* f = s->f + i * q;
            double* g = s->g + i * q;
            int cls = node_class(s, x, y);
            if (cls == NODE_WALL) {
                for (int a = 0; a < 9; ++a) g[a] = f[opp9(a)];
            } else if (cls == NODE_LID) {
                orc_d2q9_feq(s->rho0, s->u_lid, 0.0, g);
            } else {
                int st = collide_node(s, f, g);
                if (st & ORC_NEWTON_SKIPPED) ++skipped;
                if (st & ORC_UNSTABLE) ++unstable;
            }
        }
    }
    s->n_skipped += skipped;
    s->n_unstable += unstable;
}

static void stream_pass(orc_sim* s, const double* lo, const double* hi) {
    const int q = s->q, nx = s->nx, ny = s->ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t i = (size_t)y * nx + x;
            for (int a = 0; a < q; ++a) {
                int vx = (q == 9) ? V9[a][0] : V3[a];
                int vy = (q == 9) ? V9[a][1] : 0;
                int sx = x - vx, sy = y - vy;
                const double* halo = (sy < 0) ? lo : ((sy >= ny) ? hi : NULL);
                double val;
                if (s->bc == ORC_BC_PERIODIC) {
                    sx = (sx % nx + nx) % nx;
                    sy = (sy % ny + ny) % ny;
                    val = halo ? halo[(size_t)a * nx + sx] : s->g[((size_t)sy * nx + sx) * q + a];
                } else if (s->bc == ORC_BC_ZERO_GRADIENT) {
                    /* ghost -1 copies node 0, ghost nx copies node nx-1 */
                    if (sx < 0) sx = 0;
                    if (sx > nx - 1) sx = nx - 1;
                    sy = (sy % ny + ny) % ny;
                    val = halo ? halo[(size_t)a * nx + sx] : s->g[((size_t)sy * nx + sx) * q + a];
                } else {
                    if (sx < 0 || sx >= nx)
                        val = W9[a] * s->rho0;
                    else if (halo)
                        val = halo[(size_t)a * nx + sx];
                    else if (sy < 0 || sy >= ny)
                        val = W9[a] * s->rho0;
                    else
                        val = s->g[((size_t)sy * nx + sx) * q + a];
                }
                s->f[i * q + a] = val;
            }
        }
    }
    s->steps += 1;
}

/* n time steps of Eq. (2) on the whole lattice. */
ORC_EXPORT void orc_step(orc_sim* s, int nsteps) {
    for (int it = 0; it < nsteps; ++it) {
        collide_pass(s);
        stream_pass(s, NULL, NULL);
    }
}

/* The slab form: this lattice is rows [y_off, y_off + ny) of one of
 * ny_global rows, for the node classes of the cavity (bottom wall at global
 * row 0, lid at global row ny_global - 1). */
ORC_EXPORT int orc_set_slab(orc_sim* s, int y_off, int ny_global) {
    if (y_off < 0 || ny_global < y_off + s->ny) return -1;
    s->y_off = y_off;
    s->ny_global = ny_global;
    return 0;
}

/* The two halves of one step, for a slab that exchanges its edge rows in
 * between: orc_collide, then orc_post_row of its first and last rows to the
 * neighbours, then orc_stream with the rows received from them. */
ORC_EXPORT void orc_collide(orc_sim* s) { collide_pass(s); }
ORC_EXPORT void orc_stream(orc_sim* s, const double* lo, const double* hi) {
    stream_pass(s, lo, hi);
}
/* Post-collision populations of local row y, [a][x]. */
ORC_EXPORT void orc_post_row(const orc_sim* s, int y, double* out) {
    for (int a = 0; a < s->q; ++a)
        for (int x = 0; x < s->nx; ++x) out[(size_t)a * s->nx + x] = s->g[((size_t)y * s->nx + x) * s->q + a];
}

/* Macroscopic fields of f(x, t_n) (Sec. II.A): rho = sum f, rho u = sum f v. */
ORC_EXPORT void orc_moments(const orc_sim* s, double* rho, double* ux, double* uy) {
    size_t nn = (size_t)s->nx * s->ny;
    for (size_t i = 0; i < nn; ++i) {
        const double* f = s->f + i * s->q;
        double r = 0.0, jx = 0.0, jy = 0.0;
        for (int a = 0; a < s->q; ++a) {
            r += f[a];
            if (s->q == 9) {
                jx += f[a] * V9[a][0];
                jy += f[a] * V9[a][1];
            } else {
                jx += f[a] * V3[a];
            }
        }
        rho[i] = r;
        if (ux) ux[i] = jx / r;
        if (uy) uy[i] = jy / r;
    }
}

/* Total mass and momentum of f(x, t_n): out = (sum rho, sum rho ux, sum rho uy). */
ORC_EXPORT void orc_conservation(const orc_sim* s, double* out) {
    size_t nn = (size_t)s->nx * s->ny;
    double m = 0.0, px = 0.0, py = 0.0;
    for (size_t i = 0; i < nn; ++i) {
        const double* f = s->f + i * s->q;
        for (int a = 0; a < s->q; ++a) {
            m += f[a];
            if (s->q == 9) {
                px += f[a] * V9[a][0];
                py += f[a] * V9[a][1];
            } else {
                px += f[a] * V3[a];
            }
        }
    }
    out[0] = m;
    out[1] = px;
    out[2] = py;
}

ORC_EXPORT void orc_counters(const orc_sim* s, long long* out) {
    out[0] = s->n_skipped;
    out[1] = s->n_unstable;
    out[2] = s->steps;
}

/*
 * Stream function of the LDAS post-processing (Sec. IV.I):
 *   psi(x, y) = - integral from the left wall (x = 0) to x of u_y dx,
 * evaluated along each row in lattice units (node spacing 1).  The integral
 * over [0, x] uses the composite Simpson rule on the pairs of intervals
 * [0, 2], [2, 4], ...; at odd x the last interval [x - 1, x] uses the
 * trapezoidal rule (the paper integrates with Simpson's rule where the
 * spacing allows it and with the trapezoid elsewhere).
 *   uy   [ny][nx] vertical velocity
 *   psi  [ny][nx] output
 */
ORC_EXPORT void orc_stream_function(int nx, int ny, const double* uy, double* psi) {
    for (int y = 0; y < ny; ++y) {
        const double* u = uy + (size_t)y * nx;
        double* p = psi + (size_t)y * nx;
        double simpson = 0.0; /* integral over [0, x] for the last even x */
        p[0] = 0.0;
        for (int x = 1; x < nx; ++x) {
            if (x % 2 == 0) {
                simpson += (u[x - 2] + 4.0 * u[x - 1] + u[x]) / 3.0;
                p[x] = -simpson;
            } else {
                p[x] = -(simpson + 0.5 * (u[x - 1] + u[x]));
            }
        }
    }
}

ORC_EXPORT int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
