/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle for the single-component
 * pseudo-potential D2Q9 lattice Boltzmann model of Hu, Li & Uddin,
 * "Force Method in a Pseudo-potential Lattice Boltzmann Model"
 * (arXiv:1412.5170): Kupershtokh's hybrid psi/psi^2 force, Guo / exact
 * difference / Shan-Chen forcing, BGK or MRT collision, periodic streaming;
 * and the comparison model of Li et al. (Sec. 4.3, Eqs. 31-32).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may include,
 * link or call this file; it is used by tests/, by __graft_entry__.smoke()
 * and by the CPU-baseline leg of bench.py.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * Every function follows the paper's equations in the paper's order, one
 * node at a time, with no blocking or fusion.  Compiled with
 * -O2 -ffp-contract=off (no FMA contraction), round to nearest.  The
 * lattice loops may run on several host threads (OpenMP over rows, see
 * orc_set_threads); nodes are independent, so results do not depend on it.
 *
 * Population layout: f[(a*ny + y)*nx + x], a = 0..8, double.
 * Velocity numbering (Sec. 2, text after Eq. 2):
 *   e0=(0,0); e1..e4 = (1,0),(0,1),(-1,0),(0,-1); e5..e8 = (1,1),(-1,1),(-1,-1),(1,-1)
 *   w0 = 4/9, w1..4 = 1/9, w5..8 = 1/36, c_s^2 = 1/3, dx = dt = 1.
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *   - G = -1 (the value Sec. 4.3 states), so U = G psi^2/2 = -psi^2/2 and,
 *     from Eq. 7, psi^2 = 2 (rho/3 - p).
 *   - The stencil weights omega of Eq. 6 are the force weights of Eq. 4:
 *     w(1) = 1/3 on the axes, w(2) = 1/12 on the diagonals.
 *   - A is used exactly as written in Eq. 6 (eps = -2A from Table 1).
 *   - Eq. 23's second index pair is read as (F_i v_j + v_i F_j).
 *   - Tc comes from the constants of Eq. 29: Tc = (0.18727/0.4963) a/(b R).
 *   - The macroscopic fields at time t are taken from the post-streaming
 *     populations before collision; v = u + F/(2 rho) (Sec. 3.2).
 *   - MRT (Eqs. 34-36): moment order rho, e, eps, j_x, q_x, j_y, q_y, p_xx,
 *     p_xy with the usual D2Q9 polynomial rows; Lambda =
 *     diag(s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, 1/tau, 1/tau) with
 *     s_rho = s_j = 1 (they drop out under Guo forcing).
 *   - Li et al.'s model (Eq. 31): BGK, the force of Eq. 4 (Eq. 6 with A = 0),
 *     Guo's source with v replaced by v' = v + sigma F / ((tau - 1/2) psi^2)
 *     in its second-order term; the paper's "upsilon" there is read as
 *     (tau - 1/2) dt, the form for which the pressure tensor gives Eq. 32's
 *     eps = -2 (alpha + 24 G sigma) / beta, i.e. eps = 16 sigma for the
 *     Eq. 4 force (alpha = 0, beta = 3, G = -1), matching the paper's
 *     sigma = 0.105 <-> eps = 1.68.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_E_EOS_DOMAIN 4   /* rho outside (0,1) or rho/3 - p < 0 */
#define ORC_E_NONFINITE 3
#define ORC_E_INVALID 1

enum { ORC_BGK = 0, ORC_MRT = 1 };
enum { ORC_GUO = 0, ORC_EDM = 1, ORC_SC = 2, ORC_LI = 3 };

typedef struct {
    int32_t nx, ny;
    int32_t collision;   /* ORC_BGK / ORC_MRT */
    int32_t forcing;     /* ORC_GUO / ORC_EDM / ORC_SC / ORC_LI */
    double T_over_Tc;    /* reduced temperature */
    double tau;          /* BGK relaxation time; MRT tau_nu */
    double A;            /* Eq. 6 weight */
    double K;            /* Eq. 30 EOS scale */
    double s_e, s_eps, s_q;  /* MRT rates (Eq. 35) */
    double sigma;        /* Li et al.'s sigma (Eq. 31), ORC_LI only */
} orc_params;

static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                            1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

static int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

/* Host threads of the lattice loops (OpenMP over rows when compiled with
 * it).  Every node is computed independently and written to its own place,
 * so the result is the same bit for bit for any thread count.  Default 1. */
static int orc_threads = 1;
void orc_set_threads(int n) { orc_threads = n > 0 ? n : 1; }
int orc_get_threads(void) { return orc_threads; }

/* ---------------- Sec. 4.1: Carnahan-Starling EOS ---------------- */

/* Tc implied by a = 0.4963 R^2 Tc^2/pc and b = 0.18727 R Tc/pc (Eq. 29),
 * with a = 1, b = 4, R = 1. */
double orc_Tc(void)
{
    const double a = 1.0, b = 4.0, R = 1.0;
    return (0.18727 / 0.4963) * a / (b * R);
}

/* Eq. 30: p = K [ rho R T (1 + eta + eta^2 - eta^3)/(1 - eta)^3 - a rho^2 ],
 * eta = b rho / 4. */
double orc_pressure(double rho, double T, double K)
{
    const double a = 1.0, b = 4.0, R = 1.0;
    double eta = b * rho / 4.0;
    double num = 1.0 + eta + eta * eta - eta * eta * eta;
    double den = (1.0 - eta) * (1.0 - eta) * (1.0 - eta);
    return K * (rho * R * T * num / den - a * rho * rho);
}

/* Eq. 7 with G = -1, c = 1: p = rho/3 + U, U = G psi^2/2  =>  psi^2 = 2(rho/3 - p). */
double orc_psi2(double rho, double T, double K)
{
    return 2.0 * (rho / 3.0 - orc_pressure(rho, T, K));
}

/* ---------------- Sec. 2: equilibrium, Eq. 2 ---------------- */

void orc_feq(double rho, double ux, double uy, double feq[9])
{
    const double cs2 = 1.0 / 3.0;
    double u2 = ux * ux + uy * uy;
    for (int a = 0; a < 9; ++a) {
        double eu = EX[a] * ux + EY[a] * uy;
        feq[a] = W[a] * rho * (1.0 + eu / cs2 + (eu * eu) / (2.0 * cs2 * cs2) - u2 / (2.0 * cs2));
    }
}

/* ---------------- Sec. 3.2: Guo source term, Eq. 23 ----------------
 * F_a = w_a (1 - 1/(2 tau)) [ F_i e_ai / cs^2 + (F_i v_j + v_i F_j)(e_ai e_aj - cs^2 d_ij)/(2 cs^4) ].
 * 'prefactor' is (1 - 1/(2 tau)) for BGK, 1 for the MRT source vector S of Eq. 34. */
void orc_guo_source(double prefactor, double Fx, double Fy, double vx, double vy, double S[9])
{
    const double cs2 = 1.0 / 3.0;
    double F[2] = {Fx, Fy}, v[2] = {vx, vy};
    for (int a = 0; a < 9; ++a) {
        double e[2] = {(double)EX[a], (double)EY[a]};
        double first = 0.0, second = 0.0;
        for (int i = 0; i < 2; ++i) first += F[i] * e[i] / cs2;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                double delta = (i == j) ? 1.0 : 0.0;
                second += (F[i] * v[j] + v[i] * F[j]) * (e[i] * e[j] - cs2 * delta) / (2.0 * cs2 * cs2);
            }
        S[a] = W[a] * prefactor * (first + second);
    }
}

/* ---------------- Sec. 2: interaction force, Eq. 6 ----------------
 * F3 = -A sum_a w_a U(x+e_a) e_a - (1-A) G psi(x) sum_a w_a psi(x+e_a) e_a,
 * U = G psi^2/2, G = -1, weights w(|e|^2): w(1) = 1/3, w(2) = 1/12 (Eq. 4). */
void orc_force(int nx, int ny, const double *psi, double A, double *Fx, double *Fy)
{
    const double G = -1.0;
    const double wforce[9] = {0.0, 1.0 / 3, 1.0 / 3, 1.0 / 3, 1.0 / 3,
                              1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12};
#pragma omp parallel for num_threads(orc_threads) schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double sumU[2] = {0.0, 0.0}, sumP[2] = {0.0, 0.0};
            for (int a = 1; a < 9; ++a) {
                int xn = wrap(x + EX[a], nx), yn = wrap(y + EY[a], ny);
                double pn = psi[yn * nx + xn];
                double Un = G * pn * pn / 2.0;
                sumU[0] += wforce[a] * Un * EX[a];
                sumU[1] += wforce[a] * Un * EY[a];
                sumP[0] += wforce[a] * pn * EX[a];
                sumP[1] += wforce[a] * pn * EY[a];
            }
            double p0 = psi[y * nx + x];
            Fx[y * nx + x] = -A * sumU[0] - (1.0 - A) * G * p0 * sumP[0];
            Fy[y * nx + x] = -A * sumU[1] - (1.0 - A) * G * p0 * sumP[1];
        }
}

/* ---------------- Sec. 4.4.2: MRT transform, Eqs. 34-35 ---------------- */

/* Rows of M as polynomials of e = (ex, ey), |e|^2 = ex^2 + ey^2, in the moment
 * order (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy). */
void orc_mrt_matrix(double M[81])
{
    for (int a = 0; a < 9; ++a) {
        double ex = EX[a], ey = EY[a], e2 = ex * ex + ey * ey;
        M[0 * 9 + a] = 1.0;
        M[1 * 9 + a] = -4.0 + 3.0 * e2;
        M[2 * 9 + a] = 4.0 - 21.0 / 2.0 * e2 + 9.0 / 2.0 * e2 * e2;
        M[3 * 9 + a] = ex;
        M[4 * 9 + a] = (-5.0 + 3.0 * e2) * ex;
        M[5 * 9 + a] = ey;
        M[6 * 9 + a] = (-5.0 + 3.0 * e2) * ey;
        M[7 * 9 + a] = ex * ex - ey * ey;
        M[8 * 9 + a] = ex * ey;
    }
}

/* Plain Gauss-Jordan inverse with partial pivoting (n = 9). Returns 0 on success. */
int orc_invert9(const double Min[81], double Minv[81])
{
    double a[9][18];
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 18; ++j)
            a[i][j] = (j < 9) ? Min[i * 9 + j] : ((j - 9 == i) ? 1.0 : 0.0);
    for (int c = 0; c < 9; ++c) {
        int piv = c;
        for (int r = c + 1; r < 9; ++r)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (a[piv][c] == 0.0) return -1;
        if (piv != c)
            for (int j = 0; j < 18; ++j) { double t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t; }
        double d = a[c][c];
        for (int j = 0; j < 18; ++j) a[c][j] /= d;
        for (int r = 0; r < 9; ++r)
            if (r != c) {
                double m = a[r][c];
                for (int j = 0; j < 18; ++j) a[r][j] -= m * a[c][j];
            }
    }
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) Minv[i * 9 + j] = a[i][j + 9];
    return 0;
}

static void matvec9(const double M[81], const double x[9], double y[9])
{
    for (int i = 0; i < 9; ++i) {
        double s = 0.0;
        for (int j = 0; j < 9; ++j) s += M[i * 9 + j] * x[j];
        y[i] = s;
    }
}

/* ---------------- one node: collision (Eqs. 1, 20-23, 31, 34) ----------------
 * f: post-streaming populations at the node; rho, ux, uy: Eq. 3 moments
 * (u = sum f e / rho); Fx, Fy: Eq. 6 force; psi: Eq. 7 effective density at
 * the node (used by Li et al.'s model only).  Writes the post-collision
 * populations to fstar. */
/* M and its inverse depend on nothing but the lattice: built once (before
 * any threaded loop, see orc_step). */
static double M[81], Minv[81];
static int tables_ready = 0;
static void mrt_tables(void)
{
    if (!tables_ready) {
        orc_mrt_matrix(M);
        orc_invert9(M, Minv);
        tables_ready = 1;
    }
}

void orc_collide_node(const orc_params *p, const double f[9], double rho, double ux, double uy,
                      double Fx, double Fy, double psi, double fstar[9])
{
    double tau = p->tau;
    double feq[9], S[9];
    if (p->collision == ORC_BGK) {
        if (p->forcing == ORC_LI) {
            /* Eq. 31: f^eq at v = u + F/(2 rho); Guo's source with v' in its
             * second-order term. */
            double vx = ux + Fx / (2.0 * rho), vy = uy + Fy / (2.0 * rho);
            double c = p->sigma / ((tau - 0.5) * psi * psi);
            orc_feq(rho, vx, vy, feq);
            orc_guo_source(1.0 - 1.0 / (2.0 * tau), Fx, Fy, vx + c * Fx, vy + c * Fy, S);
            for (int a = 0; a < 9; ++a) fstar[a] = f[a] - (f[a] - feq[a]) / tau + S[a];
        } else if (p->forcing == ORC_GUO) {
            /* Eqs. 1, 2, 23: f^eq evaluated at v = u + F/(2 rho). */
            double vx = ux + Fx / (2.0 * rho), vy = uy + Fy / (2.0 * rho);
            orc_feq(rho, vx, vy, feq);
            orc_guo_source(1.0 - 1.0 / (2.0 * tau), Fx, Fy, vx, vy, S);
            for (int a = 0; a < 9; ++a) fstar[a] = f[a] - (f[a] - feq[a]) / tau + S[a];
        } else if (p->forcing == ORC_EDM) {
            /* Eqs. 1, 22: F_a = f^eq(rho, u + du) - f^eq(rho, u), du = F/rho;
             * the BGK term relaxes toward f^eq(rho, u). */
            double feq_shift[9];
            orc_feq(rho, ux, uy, feq);
            orc_feq(rho, ux + Fx / rho, uy + Fy / rho, feq_shift);
            for (int a = 0; a < 9; ++a)
                fstar[a] = f[a] - (f[a] - feq[a]) / tau + (feq_shift[a] - feq[a]);
        } else {
            /* Eqs. 20, 21: no source; u^eq = u + tau F / rho. */
            orc_feq(rho, ux + tau * Fx / rho, uy + tau * Fy / rho, feq);
            for (int a = 0; a < 9; ++a) fstar[a] = f[a] - (f[a] - feq[a]) / tau;
        }
    } else {
        /* Eq. 34 with Guo's source in moment space: m = M f, m^eq = M f^eq(rho, v),
         * S = M F_a / (1 - 1/(2 tau)), m* = m - Lambda (m - m^eq) + (I - Lambda/2) S,
         * f* = M^-1 m*. */
        double m[9], meq[9], Sm[9], mstar[9];
        double vx = ux + Fx / (2.0 * rho), vy = uy + Fy / (2.0 * rho);
        mrt_tables();
        orc_feq(rho, vx, vy, feq);
        orc_guo_source(1.0, Fx, Fy, vx, vy, S);  /* F_a / (1 - 1/(2 tau)) */
        matvec9(M, f, m);
        matvec9(M, feq, meq);
        matvec9(M, S, Sm);
        double lam[9] = {1.0, p->s_e, p->s_eps, 1.0, p->s_q, 1.0, p->s_q, 1.0 / tau, 1.0 / tau};
        for (int k = 0; k < 9; ++k)
            mstar[k] = m[k] - lam[k] * (m[k] - meq[k]) + (1.0 - lam[k] / 2.0) * Sm[k];
        matvec9(Minv, mstar, fstar);
    }
}

/* ---------------- macroscopic fields at time t ----------------
 * From the post-streaming populations f: rho, u (Eq. 3), psi (Eq. 7),
 * F (Eq. 6), v = u + F/(2 rho).  Any output pointer may be NULL.
 * Returns ORC_E_EOS_DOMAIN if some node has rho outside (0,1) or psi^2 < 0. */
int orc_macro(const orc_params *p, const double *f, double *rho_o, double *ux_o, double *uy_o,
              double *psi_o, double *Fx_o, double *Fy_o, double *vx_o, double *vy_o)
{
    int nx = p->nx, ny = p->ny, n = nx * ny, status = ORC_OK;
    double T = p->T_over_Tc * orc_Tc();
    double *rho = malloc(sizeof(double) * n), *ux = malloc(sizeof(double) * n),
           *uy = malloc(sizeof(double) * n), *psi = malloc(sizeof(double) * n),
           *Fx = malloc(sizeof(double) * n), *Fy = malloc(sizeof(double) * n);
    int bad = 0;
#pragma omp parallel for num_threads(orc_threads) schedule(static) reduction(|: bad)
    for (int i = 0; i < n; ++i) {
        double r = 0.0, jx = 0.0, jy = 0.0;
        for (int a = 0; a < 9; ++a) {
            double fa = f[a * n + i];
            r += fa;
            jx += fa * EX[a];
            jy += fa * EY[a];
        }
        rho[i] = r;
        ux[i] = jx / r;
        uy[i] = jy / r;
        double s = orc_psi2(r, T, p->K);
        if (!(r > 0.0 && r < 1.0) || !(s >= 0.0)) { bad = 1; s = 0.0; }
        psi[i] = sqrt(s);
    }
    if (bad) status = ORC_E_EOS_DOMAIN;
    orc_force(nx, ny, psi, p->A, Fx, Fy);
#pragma omp parallel for num_threads(orc_threads) schedule(static)
    for (int i = 0; i < n; ++i) {
        if (rho_o) rho_o[i] = rho[i];
        if (ux_o) ux_o[i] = ux[i];
        if (uy_o) uy_o[i] = uy[i];
        if (psi_o) psi_o[i] = psi[i];
        if (Fx_o) Fx_o[i] = Fx[i];
        if (Fy_o) Fy_o[i] = Fy[i];
        if (vx_o) vx_o[i] = ux[i] + Fx[i] / (2.0 * rho[i]);
        if (vy_o) vy_o[i] = uy[i] + Fy[i] / (2.0 * rho[i]);
    }
    free(rho); free(ux); free(uy); free(psi); free(Fx); free(Fy);
    return status;
}

/* ---------------- one time step (Eq. 1 / Eq. 36) ----------------
 * f: post-streaming populations at t; fnext: at t+1 (distinct buffer).
 * Collision at every node, then streaming f_a(x + e_a, t+1) = f*_a(x, t). */
int orc_step(const orc_params *p, const double *f, double *fnext)
{
    int nx = p->nx, ny = p->ny, n = nx * ny;
    double *rho = malloc(sizeof(double) * n), *ux = malloc(sizeof(double) * n),
           *uy = malloc(sizeof(double) * n), *Fx = malloc(sizeof(double) * n),
           *Fy = malloc(sizeof(double) * n), *psi = malloc(sizeof(double) * n);
    int status = orc_macro(p, f, rho, ux, uy, psi, Fx, Fy, NULL, NULL), nonfinite = 0;
    if (p->collision == ORC_MRT) mrt_tables();
#pragma omp parallel for num_threads(orc_threads) schedule(static) reduction(|: nonfinite)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int i = y * nx + x;
            double fl[9], fs[9];
            for (int a = 0; a < 9; ++a) fl[a] = f[a * n + i];
            orc_collide_node(p, fl, rho[i], ux[i], uy[i], Fx[i], Fy[i], psi[i], fs);
            for (int a = 0; a < 9; ++a) {
                int xd = wrap(x + EX[a], nx), yd = wrap(y + EY[a], ny);
                if (!isfinite(fs[a])) nonfinite = 1;
                fnext[a * n + yd * nx + xd] = fs[a];
            }
        }
    if (nonfinite && !status) status = ORC_E_NONFINITE;
    free(rho); free(ux); free(uy); free(Fx); free(Fy); free(psi);
    return status;
}

/* nsteps steps in place on f (uses one scratch buffer).  Returns the first
 * non-zero step status, after which it stops. */
int orc_run(const orc_params *p, double *f, int64_t nsteps)
{
    int n = p->nx * p->ny;
    double *tmp = malloc(sizeof(double) * 9 * n);
    int status = ORC_OK;
    for (int64_t s = 0; s < nsteps; ++s) {
        status = orc_step(p, f, tmp);
        memcpy(f, tmp, sizeof(double) * 9 * n);
        if (status) break;
    }
    free(tmp);
    return status;
}

/* f_a = w_a rho0: the equilibrium at rest for a given density field. */
void orc_init_rest(int nx, int ny, const double *rho0, double *f)
{
    int n = nx * ny;
    for (int a = 0; a < 9; ++a)
        for (int i = 0; i < n; ++i) f[a * n + i] = W[a] * rho0[i];
}
