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
 * What one time step computes, node by node, in FP64:
 *   - streaming: each population arrives from the neighbour it points away
 *     from, or is reflected at a wall (half-way bounce-back, the lid adds
 *     momentum; reading A3);
 *   - the density rho and the velocity u (with half the body force, Sec. 4.2);
 *   - the density gradient from the densities of the same step (reading A1);
 *   - the collision (Sec. 3-4): the raw and central moments of the nine
 *     populations by their definitions with the rectangular velocities
 *     (Eq. 3); the gamma-preconditioned central-moment equilibria (Eq. 14)
 *     with the grid-anisotropy and cubic-velocity corrections (Eqs. 30-31,
 *     coefficients of Eqs. 38-40) and the local strain rates (Eqs. 43-48);
 *     relaxation with the rates of Eq. 11 in the combined (2s, 2d) basis
 *     (Eqs. 7-8); raw post-collision moments by the binomial theorem; and the
 *     populations by inverting the moment map, which for the D2Q9 set is a
 *     product of two 3 x 3 Vandermonde systems.
 * The moment transforms are written from their definitions rather than from
 * the matrices P, S, F and their inverses, so that this file and the
 * matrix-form statement (oracle/matrix_form.py) check each other.
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
 *   A13 storage_f32 = 1 keeps the arithmetic in FP64 and rounds only what is
 *       stored between steps, as a reduced-precision run stores it: the
 *       deviation of each post-collision population from the rest state
 *       w_i(r), to the nearest float32.  The paper fixes no precision; this
 *       is the oracle of the FP32 storage format, used where the FP64 run
 *       and an FP32-storage run of an unstable flow part ways.
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
    int model;       /* 0: PRC-LBM (central moments, Sec. 4.2);
                        1: PRNR-LBM (raw moments, Sec. 4.1 and Sec. 5.3)   */
    int appendix_literal; /* 1: the strain-rate residuals exactly as App. A
                             prints them (reading A4 not applied); for
                             reporting the size of that reading only    */
    int storage_f32; /* 1: the stored post-collision populations are
                        rounded, every step, to the nearest float32
                        deviation from the rest state w_i(r) (the
                        shifted FP32 storage of a reduced-precision
                        run); the arithmetic stays FP64            */
} orc_params;

/* Per-run constants derived once from the parameters. */
typedef struct {
    orc_params p;
    double q;        /* Eq. 2: q = min(1, r)                      */
    double cs2;      /* q^2 c_s*^2 with c_s*^2 = 1/3 (Eq. 1-2)     */
    double omega_nu; /* from nu = gamma q^2 c_s*^2 (1/w - 1/2)     */
    double w[9];     /* rest state w_i(r) (storage_f32 only)       */
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
/* Moments of a population set.  The nine D2Q9 velocities are the products of
 * the one-dimensional sets {0, +1, -1} in x and {0, +r, -r} in y (Eq. 3), so a
 * moment sum_i f_i c_ix^a c_iy^b (a, b = 0, 1, 2) is a tensor product of two
 * 3 x 3 Vandermonde maps, and the populations follow from the nine moments
 * by inverting each of them.  Moments here are always taken with the
 * physical velocities (c_ix, c_iy) = (e_ix, r e_iy/r): the "rectangular" raw
 * moments k'_ab that the square-lattice moments P f become after the scaling
 * S (Sec. 4.1). */

/* index of the velocity (vx, vy) with vx in {0, 1, -1} and vy/r in {0, 1, -1} */
static int dir_of(int vx, int vyb)
{
    for (int i = 0; i < 9; i++)
        if (EX[i] == vx && EYB[i] == vyb) return i;
    return -1;
}

/* Populations from their moments m[a][b] = sum_i f_i c_ix^a c_iy^b: solve the
 * x map for every b, then the y map for every x velocity.  With the values
 * v in {0, +h, -h}: F(0) = M0 - M2/h^2, F(+h) = (M1/h + M2/h^2)/2,
 * F(-h) = (M2/h^2 - M1/h)/2 (h = 1 in x, h = r in y). */
static void populations_from_moments(double r, const double m[3][3], double f[9])
{
    double fx[3][3]; /* [x velocity 0, +1, -1][b] */
    for (int b = 0; b < 3; b++) {
        fx[0][b] = m[0][b] - m[2][b];
        fx[1][b] = 0.5 * (m[1][b] + m[2][b]);
        fx[2][b] = 0.5 * (m[2][b] - m[1][b]);
    }
    static const int VAL[3] = {0, 1, -1};
    const double ir = 1.0 / r, ir2 = 1.0 / (r * r);
    for (int k = 0; k < 3; k++) {
        const double *n = fx[k];
        f[dir_of(VAL[k], 0)] = n[0] - n[2] * ir2;
        f[dir_of(VAL[k], 1)] = 0.5 * (n[1] * ir + n[2] * ir2);
        f[dir_of(VAL[k], -1)] = 0.5 * (n[2] * ir2 - n[1] * ir);
    }
}

/* Moments about the velocity (ux, uy) by their definition:
 * m[a][b] = sum_i f_i (c_ix - ux)^a (c_iy - uy)^b; (0, 0) gives the raw moments. */
static void moments_about(double r, const double f[9], double ux, double uy, double m[3][3])
{
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) m[a][b] = 0.0;
    for (int i = 0; i < 9; i++) {
        const double dx = EX[i] - ux, dy = r * EYB[i] - uy;
        const double px[3] = {1.0, dx, dx * dx}, py[3] = {1.0, dy, dy * dy};
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) m[a][b] += f[i] * px[a] * py[b];
    }
}

/* Raw moments from central moments about (ux, uy), by the binomial theorem:
 * c_x^a c_y^b = sum_{p <= a, q <= b} C(a,p) C(b,q) ux^(a-p) uy^(b-q)
 * (c_x - ux)^p (c_y - uy)^q. */
static void raw_from_central(const double c[3][3], double ux, double uy, double m[3][3])
{
    static const double BIN[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}};
    const double pux[3] = {1.0, ux, ux * ux}, puy[3] = {1.0, uy, uy * uy};
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double v = 0.0;
            for (int p = 0; p <= a; p++)
                for (int q = 0; q <= b; q++) v += BIN[a][p] * BIN[b][q] * pux[a - p] * puy[b - q] * c[p][q];
            m[a][b] = v;
        }
}

/* Equilibrium populations f^eq(rho, u): the raw-moment equilibria of Eq. 12
 * (uncorrected) in the physical velocities, mapped to populations.  Used for
 * the rest weights, field initialisation and the equilibrium-difference
 * bounce-back (reading A3). */
static void equilibrium(const orc_consts *c, double rho, double ux, double uy, double feq[9])
{
    const double g = c->p.gamma, cs2 = c->cs2;
    double m[3][3];
    m[0][0] = rho;
    m[1][0] = rho * ux;
    m[0][1] = rho * uy;
    m[2][0] = cs2 * rho + rho * ux * ux / g;
    m[0][2] = cs2 * rho + rho * uy * uy / g;
    m[1][1] = rho * ux * uy / g;
    m[2][1] = rho * (cs2 + ux * ux / (g * g)) * uy;
    m[1][2] = rho * (cs2 + uy * uy / (g * g)) * ux;
    m[2][2] = rho * cs2 * cs2 + rho * cs2 * (ux * ux + uy * uy) + rho * ux * ux * uy * uy;
    populations_from_moments(c->p.r, m, feq);
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
/* One node's collision.  The moments come from their definitions (raw
 * moments of the physical velocities, central moments about the node's
 * velocity), the preconditioned central-moment equilibria of Eq. 14 carry
 * the corrections of Eqs. 30-31 with the coefficients of Eqs. 38-40 and the
 * local strain rates of Eqs. 43-48; the second-order moments relax in the
 * combined (2s, 2d) basis of Sec. 4.2, and the post-collision central
 * moments go back to raw moments by the binomial theorem and to populations
 * by inverting the moment map.  diag (if not NULL) receives rho, u_x, u_y,
 * d_x u_x, d_y u_y. */
static void collide(const orc_consts *c, const double f[9], double dxrho, double dyrho,
                    double ft[9], double *diag)
{
    const orc_params *p = &c->p;
    const double r = p->r, g = p->gamma, cs2 = c->cs2;
    const double wxi = p->omega_xi, wnu = c->omega_nu;

    /* -- raw moments of the physical velocities (what S P f gives) -- */
    double km[3][3];
    moments_about(r, f, 0.0, 0.0, km);
    const double k00 = km[0][0], k10 = km[1][0], k01 = km[0][1];
    const double k20 = km[2][0], k02 = km[0][2], k11 = km[1][1];
    const double k21 = km[2][1], k12 = km[1][2], k22 = km[2][2];

    /* -- hydrodynamic fields: density and velocity with half the force (Sec. 4.2) -- */
    const double rho = k00;
    const double ux = (k10 + p->fx / (2.0 * g)) / rho;
    const double uy = (k01 + p->fy / (2.0 * g)) / rho;

    /* -- central moments about u, by their definition -- */
    double cm[3][3];
    moments_about(r, f, ux, uy, cm);
    const double c00 = cm[0][0], c10 = cm[1][0], c01 = cm[0][1];
    const double c20 = cm[2][0], c02 = cm[0][2], c11 = cm[1][1];
    const double c21 = cm[2][1], c12 = cm[1][2], c22 = cm[2][2];

    /* -- combined second-order moments (the basis of Eqs. 7-8) -- */
    double c2s = c20 + c02;
    double c2d = c20 - c02;

    /* -- coefficients of the corrected equilibria (Eqs. 38-40, prefactors of Sec. 3.4) -- */
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

        /* -- relaxation with the rates of Eq. 11, dt = 1 -- */
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

        /* -- post-collision raw moments by the binomial theorem (reading A5) -- */
        const double tc[3][3] = {{t00, t01, t02}, {t10, t11, t12}, {t20, t21, t22}};
        double tm[3][3];
        raw_from_central(tc, ux, uy, tm);
        m00 = tm[0][0];
        m10 = tm[1][0];
        m01 = tm[0][1];
        m20 = tm[2][0];
        m02 = tm[0][2];
        m11 = tm[1][1];
        m21 = tm[2][1];
        m12 = tm[1][2];
        m22 = tm[2][2];
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

    /* -- post-collision populations from their moments -- */
    const double mt[3][3] = {{m00, m01, m02}, {m10, m11, m12}, {m20, m21, m22}};
    populations_from_moments(r, mt, ft);

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
    equilibrium(&s->c, 1.0, 0.0, 0.0, s->c.w);
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
 * (its first moments gain F/gamma in the relaxation, Sec. 4.2). */
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

/* Streaming f(x, t+1) = f~(x - e, t) (Sec. 2), with half-way bounce-back at
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
                if (p->storage_f32)
                    for (int i = 0; i < 9; i++) ft[i] = s->c.w[i] + (double)(float)(ft[i] - s->c.w[i]);
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
