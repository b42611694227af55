/*
 * prc_oracle.c -- plain FP64 CPU oracle of the preconditioned rectangular
 * central-moment lattice Boltzmann method (PRC-LBM) on the D2Q9 lattice,
 * E. Yahia & K. N. Premnath, arXiv:2208.03562.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA path.  Only
 * the tests, the smoke check (__graft_entry__.smoke) and the CPU-baseline leg
 * of bench.py may load it.  It shares no code, header, table or constant with
 * the CUDA library, and the CUDA library never calls it.
 *
 * The collision follows the sub-steps of Appendix A in the paper's order and
 * notation:
 *   m = P f                      (App. A, pre-collision raw moments, Eq. 62)
 *   m <- S m                     (App. A, scaling, Eq. S-matrix)
 *   m^c = F m                    (App. A, central moments, Eq. 64)
 *   relax with B, Lambda         (App. A, extended equilibria, strain rates)
 *   m~ = F^-1 m~^c               (App. A, post-collision raw moments)
 *   m~ <- S^-1 m~                (App. A, inverse scaling)
 *   f~ = P^-1 m~                 (App. A, Eq. 72)
 *   f(x, t+1) = f~(x - e, t)     (App. A, streaming)
 *   rho, rho u                   (App. A, hydrodynamic fields)
 *
 * Readings taken where the paper is silent, garbled or inconsistent (each is
 * also listed in the design notes):
 *   A1  d(rho)/dx, d(rho)/dy: the paper asks for a second-order isotropic
 *       difference and gives no stencil (Sec. 3.5 and App. A).  Taken as
 *         d_x rho = [4(rE-rW) + (rNE-rNW) + (rSE-rSW)] / 12
 *         d_y rho = [4(rN-rS) + (rNE-rSE) + (rNW-rSW)] / (12 r)
 *       on the density of the same time level as the collision.  Outside the
 *       domain the density of the nearest fluid node is used per coordinate
 *       (zero normal gradient); periodic directions wrap.
 *   A2  App. A prints k~02 = (k~20 - k~02)/2; read as (k~2s - k~2d)/2, the
 *       inverse of the combination k2s = k20 + k02, k2d = k20 - k02.
 *   A3  The moving-wall bounce-back is deferred to another paper.  Taken as
 *       momentum-augmented half-way bounce-back in equilibrium-difference
 *       form, f_ibar(x, t+1) = f~_i(x, t) + f^eq_ibar(rho0, u_w) -
 *       f^eq_i(rho0, u_w), with this paper's equilibrium (Eq. 12 mapped
 *       through S^-1 and P^-1) and rho_w = rho0 = 1.  At r = 1 this is the
 *       textbook 2 w_i rho (e_i . u_w) / c_s^2 correction.  A link whose
 *       source lies above the top wall takes the top wall's velocity.
 *   A4  R_2s, R_2d: App. A drops the (1/gamma - 1) terms and flips the sign
 *       of e_s,rho relative to Eq. 45; Eq. 45 (which follows from Eqs. 41-42
 *       and the definition of the non-equilibrium moments) is used.  The
 *       parameter appendix_literal takes App. A's form instead, so that the
 *       effect of this reading can be measured.
 *   A5  The App. A list of F^-1 writes central moments on the left; read as
 *       raw = binomial expansion of the central moments.
 *   A6  lambda_3y printed twice in App. A is lambda_by and lambda_sy.
 *   A7  omega_xi = omega_1 = omega_21 = omega_12 = omega_22 = 1 by default
 *       (App. A); they are parameters here so that the matrix form of
 *       Eq. 10-equivalent-centralmoment can be cross-checked with any rates.
 *   A8  Residual ||u_x(t) - u_x(t-20)||_2 (Sec. 5.2), unnormalised, FP64.
 *   A12 PRNR-LBM (model = 1, Sec. 4.1 and Sec. 5.3): the raw-moment scheme of
 *       Eq. LBErawmomentrectangularlattice, m = S P f, relaxation of B m to
 *       the raw equilibria of Eq. 12 with the raw sources of Eq. 13, then
 *       B^-1, S^-1, P^-1.  The paper applies the Sec. 3.4 corrections to
 *       its second-order equilibria; they are the same expressions as in
 *       the central scheme, with the strain rates of
 *       Eq. 45, which is written for the central non-equilibrium moments.
 *
 * State layout: the post-collision populations f~ of the last completed
 * step, f~[i][y][x], i = 0..8, y = 0..ny-1, x = 0..nx-1 (x fastest).  One
 * step = stream (pull, with walls) -> hydrodynamic fields -> density
 * gradient -> collision; the fields kept are those of the paper's last
 * sub-step of the time step.
 *
 * Directions (Eq. 3): 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE with
 * e_x = (0,1,0,-1,0,1,-1,-1,1) and e_y = r * (0,0,1,0,-1,1,1,-1,-1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_BC_CAVITY 0   /* walls left/right/bottom, moving lid on top   */
#define ORC_BC_CHANNEL 1  /* periodic in x, wall at bottom, moving top    */
#define ORC_BC_PERIODIC 2 /* periodic in x and y                           */

typedef struct {
    int nx, ny;
    double r, gamma, nu, u_lid;
    double omega_xi, omega_1, omega_21, omega_12, omega_22;
    double fx, fy;
    int bc;
    int drho_off;    /* 1: density-gradient terms set to zero            */
    int corrections; /* 1: extended equilibria (Eq. 30-40); 0: Eq. 14    */
    int model;       /* 0: PRC-LBM (central moments, Sec. 4.2, App. A);
                        1: PRNR-LBM (raw moments, Sec. 4.1 and Sec. 5.3)   */
    int appendix_literal; /* 1: the strain-rate residuals exactly as App. A
                             prints them (reading A4 not applied); for
                             reporting the size of that reading only    */
} orc_params;

/* Per-run constants derived once from the parameters. */
typedef struct {
    orc_params p;
    double q;        /* Eq. 2: q = min(1, r)                      */
    double cs2;      /* q^2 c_s*^2 with c_s*^2 = 1/3 (Eq. 1-2)     */
    double omega_nu; /* from nu = gamma q^2 c_s*^2 (1/w - 1/2)     */
} orc_consts;

typedef struct {
    orc_consts c;
    double *ft;   /* post-collision populations, 9 * ny * nx */
    double *f;    /* scratch: streamed populations           */
    double *rho, *ux, *uy;
    double *ux_snap;
    long t;
} orc_state;

static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EYB[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1}; /* e_y / r */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

int orc_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static void make_consts(const orc_params *p, orc_consts *c)
{
    c->p = *p;
    c->q = p->r < 1.0 ? p->r : 1.0;
    c->cs2 = c->q * c->q / 3.0;
    /* Eq. transport-coefficients: nu = gamma q^2 cs*^2 (1/omega_nu - 1/2) */
    c->omega_nu = 1.0 / (p->nu / (p->gamma * c->cs2) + 0.5);
}

double orc_omega_nu(const orc_params *p)
{
    orc_consts c;
    make_consts(p, &c);
    return c.omega_nu;
}

/* ---------------------------------------------------------------------- */
/* Equilibrium populations f^eq(rho, u): the raw-moment equilibria of Eq. 12
 * (uncorrected), mapped to populations by S^-1 and P^-1 (Eq. S-matrix-inverse,
 * Eq. 72).  Used for the rest weights, field initialisation and the
 * equilibrium-difference bounce-back (reading A3). */
static void equilibrium(const orc_consts *c, double rho, double ux, double uy, double feq[9])
{
    const double g = c->p.gamma, cs2 = c->cs2, r = c->p.r;
    double k00 = rho, k10 = rho * ux, k01 = rho * uy;
    double k20 = cs2 * rho + rho * ux * ux / g;
    double k02 = cs2 * rho + rho * uy * uy / g;
    double k11 = rho * ux * uy / g;
    double k21 = rho * (cs2 + ux * ux / (g * g)) * uy;
    double k12 = rho * (cs2 + uy * uy / (g * g)) * ux;
    double k22 = rho * cs2 * cs2 + rho * cs2 * (ux * ux + uy * uy) + rho * ux * ux * uy * uy;
    /* S^-1: factor r^-n for k'_mn */
    k01 /= r;
    k02 /= r * r;
    k11 /= r;
    k21 /= r;
    k12 /= r * r;
    k22 /= r * r;
    /* P^-1 (Eq. 72) */
    feq[0] = k00 - k20 - k02 + k22;
    feq[1] = 0.5 * (k10 + k20 - k12 - k22);
    feq[2] = 0.5 * (k01 + k02 - k21 - k22);
    feq[3] = 0.5 * (-k10 + k20 + k12 - k22);
    feq[4] = 0.5 * (-k01 + k02 + k21 - k22);
    feq[5] = 0.25 * (k11 + k21 + k12 + k22);
    feq[6] = 0.25 * (-k11 + k21 - k12 + k22);
    feq[7] = 0.25 * (k11 - k21 - k12 + k22);
    feq[8] = 0.25 * (-k11 - k21 + k12 + k22);
}

/* Rest-state populations w_i(r) rho0 with rho0 = 1: f^eq(1, 0). */
void orc_rest_weights(const orc_params *p, double w[9])
{
    orc_consts c;
    make_consts(p, &c);
    equilibrium(&c, 1.0, 0.0, 0.0, w);
}

void orc_equilibrium(const orc_params *p, double rho, double ux, double uy, double feq[9])
{
    orc_consts c;
    make_consts(p, &c);
    equilibrium(&c, rho, ux, uy, feq);
}

/* ---------------------------------------------------------------------- */
/* One node's collision, App. A.  diag (if not NULL) receives
 * rho, u_x, u_y, d_x u_x, d_y u_y. */
static void collide(const orc_consts *c, const double f[9], double dxrho, double dyrho,
                    double ft[9], double *diag)
{
    const orc_params *p = &c->p;
    const double r = p->r, g = p->gamma, cs2 = c->cs2;
    const double wxi = p->omega_xi, wnu = c->omega_nu;

    /* -- pre-collision raw moments, square lattice (Eq. 62) -- */
    double k00 = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    double k10 = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    double k01 = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    double k20 = f[1] + f[3] + f[5] + f[6] + f[7] + f[8];
    double k02 = f[2] + f[4] + f[5] + f[6] + f[7] + f[8];
    double k11 = f[5] - f[6] + f[7] - f[8];
    double k21 = f[5] + f[6] - f[7] - f[8];
    double k12 = f[5] - f[6] - f[7] + f[8];
    double k22 = f[5] + f[6] + f[7] + f[8];

    /* -- scale for the rectangular lattice: factor r^n for k'_mn -- */
    k01 *= r;
    k02 *= r * r;
    k11 *= r;
    k21 *= r;
    k12 *= r * r;
    k22 *= r * r;

    /* -- hydrodynamic fields (Eq. hydrodynamicfields) -- */
    const double rho = k00;
    const double ux = (k10 + p->fx / (2.0 * g)) / rho;
    const double uy = (k01 + p->fy / (2.0 * g)) / rho;

    /* -- central moments m^c = F m (binomial transforms, App. A) -- */
    double c00 = k00;
    double c10 = k10 - ux * k00;
    double c01 = k01 - uy * k00;
    double c20 = k20 - 2 * ux * k10 + ux * ux * k00;
    double c02 = k02 - 2 * uy * k01 + uy * uy * k00;
    double c11 = k11 - uy * k10 - ux * k01 + ux * uy * k00;
    double c21 = k21 - 2 * ux * k11 + ux * ux * k01 - uy * k20 + 2 * ux * uy * k10 - ux * ux * uy * k00;
    double c12 = k12 - 2 * uy * k11 + uy * uy * k10 - ux * k02 + 2 * ux * uy * k01 - ux * uy * uy * k00;
    double c22 = k22 - 2 * ux * k12 + ux * ux * k02 - 2 * uy * k21 + 4 * ux * uy * k11
               - 2 * ux * ux * uy * k01 + uy * uy * k20 - 2 * ux * uy * uy * k10 + ux * ux * uy * uy * k00;

    /* -- combine second-order moments (operator B) -- */
    double c2s = c20 + c02;
    double c2d = c20 - c02;

    /* -- coefficients of the extended equilibria (App. A) -- */
    const double Pg = 4.0 / (g * g) - 1.0 / g;
    const double Qg = 1.0 / (g * g) - 1.0 / g;
    const double Ug = 2.0 / g + 1.0;
    const double ux2 = ux * ux, uy2 = uy * uy;
    const double txi = 1.0 / wxi - 0.5, tnu = 1.0 / wnu - 0.5;

    double dxux = 0.0, dyuy = 0.0;
    double eq2s_corr = 0.0, eq2d_corr = 0.0, eq11_corr = 0.0;
    if (p->corrections) {
        /* local strain rates from non-equilibrium moments (Eqs. 43-48) */
        double A = 0.5 * (Ug * cs2 - 1.0) * ux;
        double B = 0.5 * (Ug * cs2 - r * r) * uy;
        double e_brho = -A * dxrho - B * dyrho;
        double e_srho = -A * dxrho + B * dyrho;
        /* reading A4: Eq. 45; with appendix_literal, App. A's residuals */
        double R2s, R2d;
        if (p->appendix_literal) {
            R2s = c2s - 2 * cs2 * rho + e_brho;
            R2d = c2d - e_srho;
        } else {
            R2s = c2s - 2 * cs2 * rho - (1.0 / g - 1.0) * (ux2 + uy2) * rho + e_brho;
            R2d = c2d - (1.0 / g - 1.0) * (ux2 - uy2) * rho + e_srho;
        }
        double Cbx = (-2 * cs2 / wxi + (Pg * ux2 + Qg * uy2) / 2 + (3 * cs2 - 1.0) / 2) * rho;
        double Cby = (-2 * cs2 / wxi + (Pg * uy2 + Qg * ux2) / 2 + (3 * cs2 - r * r) / 2) * rho;
        double Csx = (-2 * cs2 / wnu + (Pg * ux2 - Qg * uy2) / 2 + (3 * cs2 - 1.0) / 2) * rho;
        double Csy = (2 * cs2 / wnu + (-Pg * uy2 + Qg * ux2) / 2 - (3 * cs2 - r * r) / 2) * rho;
        dxux = (Csy * R2s - Cby * R2d) / (Cbx * Csy - Csx * Cby);
        dyuy = (R2s - Cbx * dxux) / Cby;

        double theta_bx = -(Pg * ux2 + Qg * uy2 + (3 * cs2 - 1.0)) * rho * txi;
        double theta_by = -(Pg * uy2 + Qg * ux2 + (3 * cs2 - r * r)) * rho * txi;
        double lambda_bx = -(Ug * cs2 - 1.0) * txi * ux;
        double lambda_by = -(Ug * cs2 - r * r) * txi * uy;
        double theta_sx = -(Pg * ux2 - Qg * uy2 + (3 * cs2 - 1.0)) * rho * tnu;
        double theta_sy = (-Pg * uy2 + Qg * ux2 - (3 * cs2 - r * r)) * rho * tnu;
        double lambda_sx = -(Ug * cs2 - 1.0) * tnu * ux;
        double lambda_sy = (Ug * cs2 - r * r) * tnu * uy;
        double ttheta_sx = -Qg * tnu * rho * ux * uy;
        double ttheta_sy = -Qg * tnu * rho * ux * uy;
        double tlambda_sx = -(1.0 / g - 1.0) * tnu * cs2 * uy;
        double tlambda_sy = -(1.0 / g - 1.0) * tnu * cs2 * ux;

        eq2s_corr = theta_bx * dxux + theta_by * dyuy + lambda_bx * dxrho + lambda_by * dyrho;
        eq2d_corr = theta_sx * dxux - theta_sy * dyuy + lambda_sx * dxrho + lambda_sy * dyrho;
        eq11_corr = ttheta_sx * dxux + ttheta_sy * dyuy + tlambda_sx * dxrho + tlambda_sy * dyrho;
    }

    double m00, m10, m01, m20, m02, m11, m21, m12, m22;
    if (p->model == 0) {
        /* -- preconditioned central-moment equilibria (Eq. 14 + corrections), dt = 1 -- */
        double eq10 = 0.0, eq01 = 0.0;
        double eq2s = 2 * cs2 * rho + (1.0 / g - 1.0) * rho * (ux2 + uy2) + eq2s_corr;
        double eq2d = (1.0 / g - 1.0) * rho * (ux2 - uy2) + eq2d_corr;
        double eq11 = (1.0 / g - 1.0) * rho * ux * uy + eq11_corr;
        double eq21 = (1.0 / (g * g) - 3.0 / g + 2.0) * rho * ux2 * uy;
        double eq12 = (1.0 / (g * g) - 3.0 / g + 2.0) * rho * ux * uy2;
        double eq22 = cs2 * cs2 * rho;

        /* -- central moments of the source (Eq. 13-central) -- */
        const double fx = p->fx, fy = p->fy;
        double s10 = fx / g, s01 = fy / g;
        double s20 = (1.0 / (g * g) - 1.0 / g) * 2 * fx * ux;
        double s02 = (1.0 / (g * g) - 1.0 / g) * 2 * fy * uy;
        double s11 = (1.0 / (g * g) - 1.0 / g) * (fx * uy + fy * ux);
        double s2s = s20 + s02, s2d = s20 - s02;

        /* -- relaxation (App. A), dt = 1 -- */
        const double w1 = p->omega_1;
        double t00 = c00;
        double t10 = c10 + w1 * (eq10 - c10) + (1 - w1 / 2) * s10;
        double t01 = c01 + w1 * (eq01 - c01) + (1 - w1 / 2) * s01;
        double t2s = c2s + wxi * (eq2s - c2s) + (1 - wxi / 2) * s2s;
        double t2d = c2d + wnu * (eq2d - c2d) + (1 - wnu / 2) * s2d;
        double t11 = c11 + wnu * (eq11 - c11) + (1 - wnu / 2) * s11;
        double t21 = c21 + p->omega_21 * (eq21 - c21);
        double t12 = c12 + p->omega_12 * (eq12 - c12);
        double t22 = c22 + p->omega_22 * (eq22 - c22);

        /* -- segregate (operator B^-1, reading A2) -- */
        double t20 = 0.5 * (t2s + t2d);
        double t02 = 0.5 * (t2s - t2d);

        /* -- post-collision raw moments m~ = F^-1 m~^c (reading A5) -- */
        m00 = t00;
        m10 = t10 + ux * t00;
        m01 = t01 + uy * t00;
        m20 = t20 + 2 * ux * t10 + ux2 * t00;
        m02 = t02 + 2 * uy * t01 + uy2 * t00;
        m11 = t11 + uy * t10 + ux * t01 + ux * uy * t00;
        m21 = t21 + 2 * ux * t11 + ux2 * t01 + uy * t20 + 2 * ux * uy * t10 + ux2 * uy * t00;
        m12 = t12 + 2 * uy * t11 + uy2 * t10 + ux * t02 + 2 * ux * uy * t01 + ux * uy2 * t00;
        m22 = t22 + 2 * ux * t12 + ux2 * t02 + 2 * uy * t21 + 4 * ux * uy * t11
                   + 2 * ux2 * uy * t01 + uy2 * t20 + 2 * ux * uy2 * t10 + ux2 * uy2 * t00;
    } else {
        /* PRNR-LBM (Eq. LBErawmomentrectangularlattice): relax the combined
           raw moments B m towards the raw equilibria of Eq. 12, whose second
           order carries the same corrections (Sec. 3.4; reading A12: the
           strain rates are those of Eq. 45 as above), with the raw sources of
           Eq. 13 and the rates of Eq. 11 (zero for the conserved moments). */
        const double r2s = k20 + k02, r2d = k20 - k02;
        const double eq2s = 2 * cs2 * rho + rho * (ux2 + uy2) / g + eq2s_corr;
        const double eq2d = rho * (ux2 - uy2) / g + eq2d_corr;
        const double eq11 = rho * ux * uy / g + eq11_corr;
        const double eq21 = rho * (cs2 + ux2 / (g * g)) * uy;
        const double eq12 = rho * (cs2 + uy2 / (g * g)) * ux;
        const double eq22 = rho * cs2 * cs2 + rho * cs2 * (ux2 + uy2) + rho * ux2 * uy2;
        const double fx = p->fx, fy = p->fy;
        const double s10 = fx / g, s01 = fy / g;
        const double s20 = 2 * fx * ux / (g * g), s02 = 2 * fy * uy / (g * g);
        const double s11 = (fx * uy + fy * ux) / (g * g);
        const double t2s = r2s + wxi * (eq2s - r2s) + (1 - wxi / 2) * (s20 + s02);
        const double t2d = r2d + wnu * (eq2d - r2d) + (1 - wnu / 2) * (s20 - s02);
        m00 = k00;
        m10 = k10 + s10;
        m01 = k01 + s01;
        m11 = k11 + wnu * (eq11 - k11) + (1 - wnu / 2) * s11;
        m21 = k21 + p->omega_21 * (eq21 - k21);
        m12 = k12 + p->omega_12 * (eq12 - k12);
        m22 = k22 + p->omega_22 * (eq22 - k22);
        /* segregate (B^-1, reading A2) */
        m20 = 0.5 * (t2s + t2d);
        m02 = 0.5 * (t2s - t2d);
    }

    /* -- inverse scaling: factor r^-n for k~'_mn -- */
    m01 /= r;
    m02 /= r * r;
    m11 /= r;
    m21 /= r;
    m12 /= r * r;
    m22 /= r * r;

    /* -- post-collision populations f~ = P^-1 m~ (Eq. 72) -- */
    ft[0] = m00 - m20 - m02 + m22;
    ft[1] = 0.5 * (m10 + m20 - m12 - m22);
    ft[2] = 0.5 * (m01 + m02 - m21 - m22);
    ft[3] = 0.5 * (-m10 + m20 + m12 - m22);
    ft[4] = 0.5 * (-m01 + m02 + m21 - m22);
    ft[5] = 0.25 * (m11 + m21 + m12 + m22);
    ft[6] = 0.25 * (-m11 + m21 - m12 + m22);
    ft[7] = 0.25 * (m11 - m21 - m12 + m22);
    ft[8] = 0.25 * (-m11 - m21 + m12 + m22);

    if (diag) {
        diag[0] = rho;
        diag[1] = ux;
        diag[2] = uy;
        diag[3] = dxux;
        diag[4] = dyuy;
    }
}

void orc_collide_node(const orc_params *p, const double f[9], double dxrho, double dyrho,
                      double ft[9], double diag[5])
{
    orc_consts c;
    make_consts(p, &c);
    collide(&c, f, dxrho, dyrho, ft, diag);
}

/* ---------------------------------------------------------------------- */
/* Grid helpers */

#define IDX(s, i, y, x) ((size_t)(i) * (size_t)(s)->c.p.ny * (size_t)(s)->c.p.nx + (size_t)(y) * (size_t)(s)->c.p.nx + (size_t)(x))
#define NODE(s, y, x) ((size_t)(y) * (size_t)(s)->c.p.nx + (size_t)(x))

static int periodic_x(int bc) { return bc == ORC_BC_CHANNEL || bc == ORC_BC_PERIODIC; }
static int periodic_y(int bc) { return bc == ORC_BC_PERIODIC; }

static void fields_from_post(orc_state *s);

orc_state *orc_create(const orc_params *p)
{
    if (p->nx < 1 || p->ny < 1) return NULL;
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    make_consts(p, &s->c);
    size_t n = (size_t)p->nx * (size_t)p->ny;
    s->ft = (double *)calloc(9 * n, sizeof(double));
    s->f = (double *)calloc(9 * n, sizeof(double));
    s->rho = (double *)calloc(n, sizeof(double));
    s->ux = (double *)calloc(n, sizeof(double));
    s->uy = (double *)calloc(n, sizeof(double));
    s->ux_snap = (double *)calloc(n, sizeof(double));
    if (!s->ft || !s->f || !s->rho || !s->ux || !s->uy || !s->ux_snap) {
        free(s->ft); free(s->f); free(s->rho); free(s->ux); free(s->uy); free(s->ux_snap);
        free(s);
        return NULL;
    }
    /* uniform rest state: f~ = w(r) rho0 */
    double w[9];
    equilibrium(&s->c, 1.0, 0.0, 0.0, w);
    for (int i = 0; i < 9; i++)
        for (size_t k = 0; k < n; k++) s->ft[(size_t)i * n + k] = w[i];
    fields_from_post(s);
    memcpy(s->ux_snap, s->ux, n * sizeof(double));
    return s;
}

void orc_destroy(orc_state *s)
{
    if (!s) return;
    free(s->ft); free(s->f); free(s->rho); free(s->ux); free(s->uy); free(s->ux_snap);
    free(s);
}

/* Fields of a post-collision state: rho = sum f~ (collision conserves mass);
 * rho u = sum f~ e - F/(2 gamma), which equals the velocity the collision used
 * (its first moments gain F/gamma, App. A relaxation of k10, k01). */
static void fields_from_post(orc_state *s)
{
    const orc_params *p = &s->c.p;
    size_t n = (size_t)p->nx * p->ny;
    for (size_t k = 0; k < n; k++) {
        double rho = 0, jx = 0, jy = 0;
        for (int i = 0; i < 9; i++) {
            double v = s->ft[(size_t)i * n + k];
            rho += v;
            jx += v * EX[i];
            jy += v * EYB[i] * p->r;
        }
        s->rho[k] = rho;
        s->ux[k] = (jx - p->fx / (2 * p->gamma)) / rho;
        s->uy[k] = (jy - p->fy / (2 * p->gamma)) / rho;
    }
}

void orc_set_populations(orc_state *s, const double *ft)
{
    size_t n = (size_t)s->c.p.nx * s->c.p.ny;
    memcpy(s->ft, ft, 9 * n * sizeof(double));
    fields_from_post(s);
    memcpy(s->ux_snap, s->ux, n * sizeof(double));
    s->t = 0;
}

void orc_get_populations(const orc_state *s, double *ft)
{
    size_t n = (size_t)s->c.p.nx * s->c.p.ny;
    memcpy(ft, s->ft, 9 * n * sizeof(double));
}

/* f~ = f^eq(rho, u) at every node (Eq. 12 without corrections). */
void orc_init_fields(orc_state *s, const double *rho, const double *ux, const double *uy)
{
    size_t n = (size_t)s->c.p.nx * s->c.p.ny;
    for (size_t k = 0; k < n; k++) {
        double feq[9];
        equilibrium(&s->c, rho[k], ux[k], uy[k], feq);
        for (int i = 0; i < 9; i++) s->ft[(size_t)i * n + k] = feq[i];
    }
    fields_from_post(s);
    memcpy(s->ux_snap, s->ux, n * sizeof(double));
    s->t = 0;
}

void orc_fields(const orc_state *s, double *rho, double *ux, double *uy)
{
    size_t n = (size_t)s->c.p.nx * s->c.p.ny;
    if (rho) memcpy(rho, s->rho, n * sizeof(double));
    if (ux) memcpy(ux, s->ux, n * sizeof(double));
    if (uy) memcpy(uy, s->uy, n * sizeof(double));
}

long orc_time(const orc_state *s) { return s->t; }

/* Streaming f(x, t+1) = f~(x - e, t) (App. A), with half-way bounce-back at
 * walls (reading A3). */
static double pull(const orc_state *s, int i, int x, int y)
{
    const orc_params *p = &s->c.p;
    int sx = x - EX[i], sy = y - EYB[i];
    if (periodic_x(p->bc)) sx = (sx + p->nx) % p->nx;
    if (periodic_y(p->bc)) sy = (sy + p->ny) % p->ny;
    if (sx >= 0 && sx < p->nx && sy >= 0 && sy < p->ny) return s->ft[IDX(s, i, sy, sx)];
    /* bounce-back: f~_o(x), o = opposite(i), left x towards the wall and
     * comes back reversed */
    int o = OPP[i];
    double v = s->ft[IDX(s, o, y, x)];
    if (sy >= p->ny && p->u_lid != 0.0) {
        /* moving top wall, u_w = (u_lid, 0): f_i = f~_o + f^eq_i(u_w) - f^eq_o(u_w) */
        double feq[9];
        equilibrium(&s->c, 1.0, p->u_lid, 0.0, feq);
        v += feq[i] - feq[o];
    }
    return v;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Density of the node (x, y), with the ghost rule of reading A1 outside. */
static double rho_at(const orc_state *s, int x, int y)
{
    const orc_params *p = &s->c.p;
    if (periodic_x(p->bc)) x = (x + p->nx) % p->nx;
    else x = clampi(x, 0, p->nx - 1);
    if (periodic_y(p->bc)) y = (y + p->ny) % p->ny;
    else y = clampi(y, 0, p->ny - 1);
    return s->rho[NODE(s, y, x)];
}

void orc_density_gradient(const orc_state *s, int x, int y, double *dxrho, double *dyrho)
{
    double rE = rho_at(s, x + 1, y), rW = rho_at(s, x - 1, y);
    double rN = rho_at(s, x, y + 1), rS = rho_at(s, x, y - 1);
    double rNE = rho_at(s, x + 1, y + 1), rNW = rho_at(s, x - 1, y + 1);
    double rSE = rho_at(s, x + 1, y - 1), rSW = rho_at(s, x - 1, y - 1);
    *dxrho = (4 * (rE - rW) + (rNE - rNW) + (rSE - rSW)) / 12.0;
    *dyrho = (4 * (rN - rS) + (rNE - rSE) + (rNW - rSW)) / (12.0 * s->c.p.r);
}

/* Test hook: overwrite the density field (for checking the stencil). */
void orc_set_rho(orc_state *s, const double *rho)
{
    size_t n = (size_t)s->c.p.nx * s->c.p.ny;
    memcpy(s->rho, rho, n * sizeof(double));
}

void orc_step(orc_state *s, long nsteps)
{
    const orc_params *p = &s->c.p;
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny;
    for (long t = 0; t < nsteps; t++) {
        /* stream */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++)
                for (int i = 0; i < 9; i++) s->f[IDX(s, i, y, x)] = pull(s, i, x, y);
        /* hydrodynamic fields */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                size_t k = NODE(s, y, x);
                double rho = 0, jx = 0, jy = 0;
                for (int i = 0; i < 9; i++) {
                    double v = s->f[(size_t)i * n + k];
                    rho += v;
                    jx += v * EX[i];
                    jy += v * EYB[i] * p->r;
                }
                s->rho[k] = rho;
                s->ux[k] = (jx + p->fx / (2 * p->gamma)) / rho;
                s->uy[k] = (jy + p->fy / (2 * p->gamma)) / rho;
            }
        /* density gradient + collision */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                size_t k = NODE(s, y, x);
                double f[9], ft[9], dxr = 0, dyr = 0;
                for (int i = 0; i < 9; i++) f[i] = s->f[(size_t)i * n + k];
                if (!p->drho_off) orc_density_gradient(s, x, y, &dxr, &dyr);
                collide(&s->c, f, dxr, dyr, ft, NULL);
                for (int i = 0; i < 9; i++) s->ft[(size_t)i * n + k] = ft[i];
            }
        s->t++;
    }
}

/* Residual ||u_x(t) - u_x(t-20)||_2 (Sec. 5.2, reading A8); advances the
 * snapshot. */
double orc_residual_update(orc_state *s)
{
    size_t n = (size_t)s->c.p.nx * s->c.p.ny;
    double acc = 0.0;
    for (size_t k = 0; k < n; k++) {
        double d = s->ux[k] - s->ux_snap[k];
        acc += d * d;
        s->ux_snap[k] = s->ux[k];
    }
    return sqrt(acc);
}

/* Run in blocks of 20 steps until the residual falls below tol or max_steps
 * is reached.  Returns the last residual; *steps_done receives the step
 * count.  A non-finite residual stops the run (divergence). */
double orc_run(orc_state *s, double tol, long max_steps, long *steps_done)
{
    double res = INFINITY;
    long done = 0;
    while (done + 20 <= max_steps) {
        orc_step(s, 20);
        done += 20;
        res = orc_residual_update(s);
        if (!(res == res) || isinf(res)) break;
        if (res < tol) break;
    }
    if (steps_done) *steps_done = done;
    return res;
}

double orc_total_mass(const orc_state *s)
{
    size_t n = (size_t)s->c.p.nx * s->c.p.ny;
    double m = 0.0;
    for (size_t k = 0; k < 9 * n; k++) m += s->ft[k];
    return m;
}
