/*
 * stp_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of one projection time step of the
 * simplified TPLS single-phase channel-flow solver (arXiv 1511.07800).  It is
 * the oracle against which the CUDA path is checked.  It shares no code,
 * header, table or constant generator with the CUDA library; only tests/,
 * the smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * Every loop is written out plainly, one output point at a time, in the order
 * the paper states the method:
 *   Sec. 2.2 (Eq. for nu_t, the van Driest factor phi_w)   -> eddy viscosity
 *   Sec. 3.1 (Eq. momentum half step, the split into the
 *             "convective-like" and "diffusive-like" viscous terms; AB3 for
 *             the former and for u.grad u, Crank-Nicolson for the latter)
 *                                                          -> explicit terms,
 *                                                             diffusion, CN
 *   Sec. 3.1 (Eq. presdiv)                                 -> divergence/RHS
 *   Sec. 3.4 (Eqs. Jacobi, Jacobi-SOR; SRJ cycle)          -> pressure solve
 *   Sec. 3.1 (Eq. project u_p_1)                           -> correction
 *   Sec. 2.1 (periodic x, y; no-slip walls at z=0, Lz)     -> boundaries
 *
 * Readings where the paper is silent (ghost reflection at the walls, edge
 * averages of nu_T, AB start-up, CN solved by point Jacobi, plain l2
 * residual norm checked once per SRJ cycle, tanh wall stretching, constant
 * flux forcing) are the ones listed in the design notes of the repository.
 *
 * Layout: x fastest.  Cell (i,j,k), i<nx, j<ny, k<nz.
 *   u[k][j][i] at x = i*dx,       y = (j+1/2)dy, z = zc[k]
 *   v[k][j][i] at x = (i+1/2)dx,  y = j*dy,      z = zc[k]
 *   w[k][j][i] at x = (i+1/2)dx,  y = (j+1/2)dy, z = zf[k], k = 0..nz
 *   p, nu at the cell centres.
 *
 * Compile with -ffp-contract=off (no fused multiply-add).  OpenMP, when
 * enabled, only splits the z loops of the stencils; every reduction is a
 * serial loop in a fixed order, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    double Lx, Ly, Lz;
    double nu;        /* molecular kinematic viscosity 1/Re                 */
    double dt;
    int forcing;      /* 0: constant body force fx = -dp/dx; 1: constant flux */
    double fx;
    double ubulk;     /* target bulk velocity when forcing == 1              */
    int les;          /* 1: Smagorinsky eddy viscosity with van Driest factor */
    double cs, vd_a, re_tau;
    double stretch;   /* 0: uniform z; gamma > 0: tanh clustering at walls   */
    int cn_sweeps;    /* point-Jacobi sweeps for the Crank-Nicolson system   */
    int srj_m;        /* SRJ cycle length M                                  */
    const double *srj_omega; /* omega_1..omega_M, one per sweep of a cycle   */
    double ptol;      /* relative l2 residual tolerance of the pressure solve */
    int pmaxit;       /* cap on SRJ sweeps per solve                          */
    int zline;        /* 0: point Jacobi-SOR sweeps; 1: z-line Jacobi-SOR      */
    int cn_zline;     /* Crank-Nicolson by 0: point Jacobi; 1: z-line Jacobi  */
} orc_params;

/* ------------------------------------------------------------------------ */
/* grid                                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz;
    double dx, dy;
    double *zf;   /* nz+1 face heights                                      */
    double *zc;   /* nz centre heights                                      */
    double *dz;   /* nz cell widths zf[k+1]-zf[k]                            */
    double *hz;   /* nz+1: centre-to-centre distance across face c;
                     hz[0], hz[nz] = centre-to-wall distance                 */
    double *dzf;  /* nz+1: distance between the two u-values that straddle
                     face c, the ghost at a wall being the mirror image of
                     the first interior centre (so dzf[0] = dz[0])           */
} grid;

void orc_zfaces(const orc_params *P, double *zf)
{
    int k;
    for (k = 0; k <= P->nz; k++) {
        double s = (double)k / (double)P->nz;
        if (P->stretch > 0.0)
            zf[k] = 0.5 * P->Lz * (1.0 + tanh(P->stretch * (2.0 * s - 1.0)) / tanh(P->stretch));
        else
            zf[k] = P->Lz * s;
    }
    zf[0] = 0.0;
    zf[P->nz] = P->Lz;
}

static void grid_make(const orc_params *P, grid *g)
{
    int k, nz = P->nz;
    g->nx = P->nx; g->ny = P->ny; g->nz = nz;
    g->dx = P->Lx / P->nx;
    g->dy = P->Ly / P->ny;
    g->zf = (double *)malloc(sizeof(double) * (nz + 1));
    g->zc = (double *)malloc(sizeof(double) * nz);
    g->dz = (double *)malloc(sizeof(double) * nz);
    g->hz = (double *)malloc(sizeof(double) * (nz + 1));
    g->dzf = (double *)malloc(sizeof(double) * (nz + 1));
    orc_zfaces(P, g->zf);
    for (k = 0; k < nz; k++) {
        g->dz[k] = g->zf[k + 1] - g->zf[k];
        g->zc[k] = 0.5 * (g->zf[k] + g->zf[k + 1]);
    }
    g->hz[0] = g->zc[0] - g->zf[0];
    g->hz[nz] = g->zf[nz] - g->zc[nz - 1];
    for (k = 1; k < nz; k++) g->hz[k] = g->zc[k] - g->zc[k - 1];
    g->dzf[0] = g->dz[0];
    g->dzf[nz] = g->dz[nz - 1];
    for (k = 1; k < nz; k++) g->dzf[k] = g->hz[k];
}

static void grid_free(grid *g)
{
    free(g->zf); free(g->zc); free(g->dz); free(g->hz); free(g->dzf);
}

/* index helpers: centred / u / v arrays have nz levels, w arrays nz+1 */
#define IDX(g, i, j, k) ((((size_t)(k)) * (g)->ny + (size_t)(j)) * (g)->nx + (size_t)(i))

static int wrap(int i, int n) { return (i % n + n) % n; }

/* u or v value with the no-slip ghost: below/above a wall the value is the
   negative of the first interior value (zero on the wall face). */
static double vel_g(const grid *g, const double *a, int i, int j, int k)
{
    i = wrap(i, g->nx); j = wrap(j, g->ny);
    if (k < 0) return -a[IDX(g, i, j, 0)];
    if (k >= g->nz) return -a[IDX(g, i, j, g->nz - 1)];
    return a[IDX(g, i, j, k)];
}

/* centred scalar (nu) with even reflection at the walls */
static double cen_g(const grid *g, const double *a, int i, int j, int k)
{
    i = wrap(i, g->nx); j = wrap(j, g->ny);
    if (k < 0) k = 0;
    if (k >= g->nz) k = g->nz - 1;
    return a[IDX(g, i, j, k)];
}

/* w value, periodic in x,y; k in 0..nz */
static double wv(const grid *g, const double *w, int i, int j, int k)
{
    i = wrap(i, g->nx); j = wrap(j, g->ny);
    return w[IDX(g, i, j, k)];
}

/* distance between centre k and the next centre above (ghost at the top) */
static double dzc_up(const grid *g, int k) { return (k < g->nz - 1) ? g->hz[k + 1] : g->dz[g->nz - 1]; }
static double dzc_dn(const grid *g, int k) { return (k > 0) ? g->hz[k] : g->dz[0]; }

/* ------------------------------------------------------------------------ */
/* viscosity averaged to cell edges                                          */
/* ------------------------------------------------------------------------ */

/* xy-edge at x = i dx, y = j dy, level k */
static double nu_xy(const grid *g, const double *nu, int i, int j, int k)
{
    return 0.25 * (cen_g(g, nu, i - 1, j - 1, k) + cen_g(g, nu, i, j - 1, k) +
                   cen_g(g, nu, i - 1, j, k) + cen_g(g, nu, i, j, k));
}
/* xz-edge at x = i dx, y = (j+1/2) dy, z = zf[c] */
static double nu_xz(const grid *g, const double *nu, int i, int j, int c)
{
    return 0.25 * (cen_g(g, nu, i - 1, j, c - 1) + cen_g(g, nu, i, j, c - 1) +
                   cen_g(g, nu, i - 1, j, c) + cen_g(g, nu, i, j, c));
}
/* yz-edge at x = (i+1/2) dx, y = j dy, z = zf[c] */
static double nu_yz(const grid *g, const double *nu, int i, int j, int c)
{
    return 0.25 * (cen_g(g, nu, i, j - 1, c - 1) + cen_g(g, nu, i, j, c - 1) +
                   cen_g(g, nu, i, j - 1, c) + cen_g(g, nu, i, j, c));
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2: Smagorinsky eddy viscosity with the van Driest wall factor      */
/* ------------------------------------------------------------------------ */

/* strain-rate components on their natural edges */
static double e12(const grid *g, const double *u, const double *v, int i, int j, int k)
{
    return 0.5 * ((vel_g(g, u, i, j, k) - vel_g(g, u, i, j - 1, k)) / g->dy +
                  (vel_g(g, v, i, j, k) - vel_g(g, v, i - 1, j, k)) / g->dx);
}
static double e13(const grid *g, const double *u, const double *w, int i, int j, int c)
{
    return 0.5 * ((vel_g(g, u, i, j, c) - vel_g(g, u, i, j, c - 1)) / g->dzf[c] +
                  (wv(g, w, i, j, c) - wv(g, w, i - 1, j, c)) / g->dx);
}
static double e23(const grid *g, const double *v, const double *w, int i, int j, int c)
{
    return 0.5 * ((vel_g(g, v, i, j, c) - vel_g(g, v, i, j, c - 1)) / g->dzf[c] +
                  (wv(g, w, i, j, c) - wv(g, w, i, j - 1, c)) / g->dy);
}

static void eddy_viscosity(const orc_params *P, const grid *g, const double *u, const double *v,
                           const double *w, double *nu)
{
    int k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < g->nz; k++) {
        int i, j;
        double delta = 2.0 * cbrt(g->dx * g->dy * g->dz[k]);
        double d = g->zc[k] < P->Lz - g->zc[k] ? g->zc[k] : P->Lz - g->zc[k];
        double dplus = d * P->re_tau / (0.5 * P->Lz);
        double phi = 1.0 - exp(-dplus / P->vd_a);
        double lm = P->cs * delta * phi;
        for (j = 0; j < g->ny; j++)
            for (i = 0; i < g->nx; i++) {
                double s11 = (vel_g(g, u, i + 1, j, k) - vel_g(g, u, i, j, k)) / g->dx;
                double s22 = (vel_g(g, v, i, j + 1, k) - vel_g(g, v, i, j, k)) / g->dy;
                double s33 = (wv(g, w, i, j, k + 1) - wv(g, w, i, j, k)) / g->dz[k];
                double s12 = 0.25 * (e12(g, u, v, i, j, k) + e12(g, u, v, i + 1, j, k) +
                                     e12(g, u, v, i, j + 1, k) + e12(g, u, v, i + 1, j + 1, k));
                double s13 = 0.25 * (e13(g, u, w, i, j, k) + e13(g, u, w, i + 1, j, k) +
                                     e13(g, u, w, i, j, k + 1) + e13(g, u, w, i + 1, j, k + 1));
                double s23 = 0.25 * (e23(g, v, w, i, j, k) + e23(g, v, w, i, j + 1, k) +
                                     e23(g, v, w, i, j, k + 1) + e23(g, v, w, i, j + 1, k + 1));
                double smag = sqrt(2.0 * (s11 * s11 + s22 * s22 + s33 * s33) +
                                   4.0 * (s12 * s12 + s13 * s13 + s23 * s23));
                nu[IDX(g, i, j, k)] = P->nu + lm * lm * smag;
            }
    }
}

/* total viscosity nu_T = 1/Re + nu_t (nu_t = 0 without the LES closure) */
static void total_viscosity(const orc_params *P, const grid *g, const double *u, const double *v,
                            const double *w, double *nu)
{
    size_t n = (size_t)g->nx * g->ny * g->nz, q;
    if (P->les) {
        eddy_viscosity(P, g, u, v, w, nu);
    } else {
        for (q = 0; q < n; q++) nu[q] = P->nu;
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: explicit terms  N = -u.grad u + d_j(nu_T d_i u_j) + f            */
/* ------------------------------------------------------------------------ */

/* advective form u_j d_j u_i (Eq. NSE momentum), centred on the MAC grid */
static double adv_u(const grid *g, const double *u, const double *v, const double *w, int i, int j, int k)
{
    double uu = vel_g(g, u, i, j, k);
    double vb = 0.25 * (vel_g(g, v, i - 1, j, k) + vel_g(g, v, i, j, k) +
                        vel_g(g, v, i - 1, j + 1, k) + vel_g(g, v, i, j + 1, k));
    double wb = 0.25 * (wv(g, w, i - 1, j, k) + wv(g, w, i, j, k) +
                        wv(g, w, i - 1, j, k + 1) + wv(g, w, i, j, k + 1));
    double dudx = (vel_g(g, u, i + 1, j, k) - vel_g(g, u, i - 1, j, k)) / (2.0 * g->dx);
    double dudy = (vel_g(g, u, i, j + 1, k) - vel_g(g, u, i, j - 1, k)) / (2.0 * g->dy);
    double dudz = (vel_g(g, u, i, j, k + 1) - vel_g(g, u, i, j, k - 1)) / (dzc_up(g, k) + dzc_dn(g, k));
    return uu * dudx + vb * dudy + wb * dudz;
}

static double adv_v(const grid *g, const double *u, const double *v, const double *w, int i, int j, int k)
{
    double ub = 0.25 * (vel_g(g, u, i, j - 1, k) + vel_g(g, u, i + 1, j - 1, k) +
                        vel_g(g, u, i, j, k) + vel_g(g, u, i + 1, j, k));
    double vv = vel_g(g, v, i, j, k);
    double wb = 0.25 * (wv(g, w, i, j - 1, k) + wv(g, w, i, j, k) +
                        wv(g, w, i, j - 1, k + 1) + wv(g, w, i, j, k + 1));
    double dvdx = (vel_g(g, v, i + 1, j, k) - vel_g(g, v, i - 1, j, k)) / (2.0 * g->dx);
    double dvdy = (vel_g(g, v, i, j + 1, k) - vel_g(g, v, i, j - 1, k)) / (2.0 * g->dy);
    double dvdz = (vel_g(g, v, i, j, k + 1) - vel_g(g, v, i, j, k - 1)) / (dzc_up(g, k) + dzc_dn(g, k));
    return ub * dvdx + vv * dvdy + wb * dvdz;
}

/* w at interior face c (1..nz-1) */
static double adv_w(const grid *g, const double *u, const double *v, const double *w, int i, int j, int c)
{
    double ub = 0.25 * (vel_g(g, u, i, j, c - 1) + vel_g(g, u, i + 1, j, c - 1) +
                        vel_g(g, u, i, j, c) + vel_g(g, u, i + 1, j, c));
    double vb = 0.25 * (vel_g(g, v, i, j, c - 1) + vel_g(g, v, i, j + 1, c - 1) +
                        vel_g(g, v, i, j, c) + vel_g(g, v, i, j + 1, c));
    double ww = wv(g, w, i, j, c);
    double dwdx = (wv(g, w, i + 1, j, c) - wv(g, w, i - 1, j, c)) / (2.0 * g->dx);
    double dwdy = (wv(g, w, i, j + 1, c) - wv(g, w, i, j - 1, c)) / (2.0 * g->dy);
    double dwdz = (wv(g, w, i, j, c + 1) - wv(g, w, i, j, c - 1)) / (g->dz[c] + g->dz[c - 1]);
    return ub * dwdx + vb * dwdy + ww * dwdz;
}

/* "convective-like" viscous term of Eq. more_conv: sum_j d_j(nu_T d_i u_j) */
static double cvisc_u(const grid *g, const double *u, const double *v, const double *w, const double *nu,
                      int i, int j, int k)
{
    double dx = g->dx, dy = g->dy;
    double fxp = cen_g(g, nu, i, j, k) * (vel_g(g, u, i + 1, j, k) - vel_g(g, u, i, j, k)) / dx;
    double fxm = cen_g(g, nu, i - 1, j, k) * (vel_g(g, u, i, j, k) - vel_g(g, u, i - 1, j, k)) / dx;
    double fyp = nu_xy(g, nu, i, j + 1, k) * (vel_g(g, v, i, j + 1, k) - vel_g(g, v, i - 1, j + 1, k)) / dx;
    double fym = nu_xy(g, nu, i, j, k) * (vel_g(g, v, i, j, k) - vel_g(g, v, i - 1, j, k)) / dx;
    double fzp = nu_xz(g, nu, i, j, k + 1) * (wv(g, w, i, j, k + 1) - wv(g, w, i - 1, j, k + 1)) / dx;
    double fzm = nu_xz(g, nu, i, j, k) * (wv(g, w, i, j, k) - wv(g, w, i - 1, j, k)) / dx;
    return (fxp - fxm) / dx + (fyp - fym) / dy + (fzp - fzm) / g->dz[k];
}

static double cvisc_v(const grid *g, const double *u, const double *v, const double *w, const double *nu,
                      int i, int j, int k)
{
    double dx = g->dx, dy = g->dy;
    double fxp = nu_xy(g, nu, i + 1, j, k) * (vel_g(g, u, i + 1, j, k) - vel_g(g, u, i + 1, j - 1, k)) / dy;
    double fxm = nu_xy(g, nu, i, j, k) * (vel_g(g, u, i, j, k) - vel_g(g, u, i, j - 1, k)) / dy;
    double fyp = cen_g(g, nu, i, j, k) * (vel_g(g, v, i, j + 1, k) - vel_g(g, v, i, j, k)) / dy;
    double fym = cen_g(g, nu, i, j - 1, k) * (vel_g(g, v, i, j, k) - vel_g(g, v, i, j - 1, k)) / dy;
    double fzp = nu_yz(g, nu, i, j, k + 1) * (wv(g, w, i, j, k + 1) - wv(g, w, i, j - 1, k + 1)) / dy;
    double fzm = nu_yz(g, nu, i, j, k) * (wv(g, w, i, j, k) - wv(g, w, i, j - 1, k)) / dy;
    return (fxp - fxm) / dx + (fyp - fym) / dy + (fzp - fzm) / g->dz[k];
}

static double cvisc_w(const grid *g, const double *u, const double *v, const double *w, const double *nu,
                      int i, int j, int c)
{
    double dx = g->dx, dy = g->dy, h = g->hz[c];
    double fxp = nu_xz(g, nu, i + 1, j, c) * (vel_g(g, u, i + 1, j, c) - vel_g(g, u, i + 1, j, c - 1)) / h;
    double fxm = nu_xz(g, nu, i, j, c) * (vel_g(g, u, i, j, c) - vel_g(g, u, i, j, c - 1)) / h;
    double fyp = nu_yz(g, nu, i, j + 1, c) * (vel_g(g, v, i, j + 1, c) - vel_g(g, v, i, j + 1, c - 1)) / h;
    double fym = nu_yz(g, nu, i, j, c) * (vel_g(g, v, i, j, c) - vel_g(g, v, i, j, c - 1)) / h;
    double fzp = cen_g(g, nu, i, j, c) * (wv(g, w, i, j, c + 1) - wv(g, w, i, j, c)) / g->dz[c];
    double fzm = cen_g(g, nu, i, j, c - 1) * (wv(g, w, i, j, c) - wv(g, w, i, j, c - 1)) / g->dz[c - 1];
    return (fxp - fxm) / dx + (fyp - fym) / dy + (fzp - fzm) / h;
}

static void explicit_terms(const orc_params *P, const grid *g, const double *u, const double *v,
                           const double *w, const double *nu, double *Nu, double *Nv, double *Nw)
{
    int k, nz = g->nz;
    double f = (P->forcing == 0) ? P->fx : 0.0;
#pragma omp parallel for schedule(static)
    for (k = 0; k < nz; k++) {
        int i, j;
        for (j = 0; j < g->ny; j++)
            for (i = 0; i < g->nx; i++) {
                size_t q = IDX(g, i, j, k);
                Nu[q] = -adv_u(g, u, v, w, i, j, k) + cvisc_u(g, u, v, w, nu, i, j, k) + f;
                Nv[q] = -adv_v(g, u, v, w, i, j, k) + cvisc_v(g, u, v, w, nu, i, j, k);
            }
    }
#pragma omp parallel for schedule(static)
    for (k = 0; k <= nz; k++) {
        int i, j;
        for (j = 0; j < g->ny; j++)
            for (i = 0; i < g->nx; i++) {
                size_t q = IDX(g, i, j, k);
                if (k == 0 || k == nz) Nw[q] = 0.0;
                else Nw[q] = -adv_w(g, u, v, w, i, j, k) + cvisc_w(g, u, v, w, nu, i, j, k);
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: "diffusive-like" term of Eq. more_diff, d_j(nu_T d_j u_i)       */
/* ------------------------------------------------------------------------ */

static double diff_u(const grid *g, const double *u, const double *nu, int i, int j, int k)
{
    double dx = g->dx, dy = g->dy, c = vel_g(g, u, i, j, k);
    double fxp = cen_g(g, nu, i, j, k) * (vel_g(g, u, i + 1, j, k) - c) / dx;
    double fxm = cen_g(g, nu, i - 1, j, k) * (c - vel_g(g, u, i - 1, j, k)) / dx;
    double fyp = nu_xy(g, nu, i, j + 1, k) * (vel_g(g, u, i, j + 1, k) - c) / dy;
    double fym = nu_xy(g, nu, i, j, k) * (c - vel_g(g, u, i, j - 1, k)) / dy;
    double fzp = nu_xz(g, nu, i, j, k + 1) * (vel_g(g, u, i, j, k + 1) - c) / g->dzf[k + 1];
    double fzm = nu_xz(g, nu, i, j, k) * (c - vel_g(g, u, i, j, k - 1)) / g->dzf[k];
    return (fxp - fxm) / dx + (fyp - fym) / dy + (fzp - fzm) / g->dz[k];
}

static double diff_v(const grid *g, const double *v, const double *nu, int i, int j, int k)
{
    double dx = g->dx, dy = g->dy, c = vel_g(g, v, i, j, k);
    double fxp = nu_xy(g, nu, i + 1, j, k) * (vel_g(g, v, i + 1, j, k) - c) / dx;
    double fxm = nu_xy(g, nu, i, j, k) * (c - vel_g(g, v, i - 1, j, k)) / dx;
    double fyp = cen_g(g, nu, i, j, k) * (vel_g(g, v, i, j + 1, k) - c) / dy;
    double fym = cen_g(g, nu, i, j - 1, k) * (c - vel_g(g, v, i, j - 1, k)) / dy;
    double fzp = nu_yz(g, nu, i, j, k + 1) * (vel_g(g, v, i, j, k + 1) - c) / g->dzf[k + 1];
    double fzm = nu_yz(g, nu, i, j, k) * (c - vel_g(g, v, i, j, k - 1)) / g->dzf[k];
    return (fxp - fxm) / dx + (fyp - fym) / dy + (fzp - fzm) / g->dz[k];
}

/* w at interior face c; w is zero on the wall faces */
static double diff_w(const grid *g, const double *w, const double *nu, int i, int j, int c)
{
    double dx = g->dx, dy = g->dy, h = g->hz[c], ctr = wv(g, w, i, j, c);
    double fxp = nu_xz(g, nu, i + 1, j, c) * (wv(g, w, i + 1, j, c) - ctr) / dx;
    double fxm = nu_xz(g, nu, i, j, c) * (ctr - wv(g, w, i - 1, j, c)) / dx;
    double fyp = nu_yz(g, nu, i, j + 1, c) * (wv(g, w, i, j + 1, c) - ctr) / dy;
    double fym = nu_yz(g, nu, i, j, c) * (ctr - wv(g, w, i, j - 1, c)) / dy;
    double fzp = cen_g(g, nu, i, j, c) * (wv(g, w, i, j, c + 1) - ctr) / g->dz[c];
    double fzm = cen_g(g, nu, i, j, c - 1) * (ctr - wv(g, w, i, j, c - 1)) / g->dz[c - 1];
    return (fxp - fxm) / dx + (fyp - fym) / dy + (fzp - fzm) / h;
}

/* diagonal weight S_D of the diffusion operator at a point: D a = sum_nb c a_nb - S_D a_ctr,
   where a wall ghost (-a_ctr) is folded into S_D */
static double diag_u(const grid *g, const double *nu, int i, int j, int k)
{
    double s = (cen_g(g, nu, i, j, k) + cen_g(g, nu, i - 1, j, k)) / (g->dx * g->dx) +
               (nu_xy(g, nu, i, j + 1, k) + nu_xy(g, nu, i, j, k)) / (g->dy * g->dy);
    double gu = (k == g->nz - 1) ? 2.0 : 1.0, gd = (k == 0) ? 2.0 : 1.0;
    s += (gu * nu_xz(g, nu, i, j, k + 1) / g->dzf[k + 1] + gd * nu_xz(g, nu, i, j, k) / g->dzf[k]) / g->dz[k];
    return s;
}

static double diag_v(const grid *g, const double *nu, int i, int j, int k)
{
    double s = (nu_xy(g, nu, i + 1, j, k) + nu_xy(g, nu, i, j, k)) / (g->dx * g->dx) +
               (cen_g(g, nu, i, j, k) + cen_g(g, nu, i, j - 1, k)) / (g->dy * g->dy);
    double gu = (k == g->nz - 1) ? 2.0 : 1.0, gd = (k == 0) ? 2.0 : 1.0;
    s += (gu * nu_yz(g, nu, i, j, k + 1) / g->dzf[k + 1] + gd * nu_yz(g, nu, i, j, k) / g->dzf[k]) / g->dz[k];
    return s;
}

static double diag_w(const grid *g, const double *nu, int i, int j, int c)
{
    return (nu_xz(g, nu, i + 1, j, c) + nu_xz(g, nu, i, j, c)) / (g->dx * g->dx) +
           (nu_yz(g, nu, i, j + 1, c) + nu_yz(g, nu, i, j, c)) / (g->dy * g->dy) +
           (cen_g(g, nu, i, j, c) / g->dz[c] + cen_g(g, nu, i, j, c - 1) / g->dz[c - 1]) / g->hz[c];
}

static void diffusion(const grid *g, const double *u, const double *v, const double *w, const double *nu,
                      double *Du, double *Dv, double *Dw)
{
    int k, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (k = 0; k < nz; k++) {
        int i, j;
        for (j = 0; j < g->ny; j++)
            for (i = 0; i < g->nx; i++) {
                size_t q = IDX(g, i, j, k);
                Du[q] = diff_u(g, u, nu, i, j, k);
                Dv[q] = diff_v(g, v, nu, i, j, k);
            }
    }
#pragma omp parallel for schedule(static)
    for (k = 0; k <= nz; k++) {
        int i, j;
        for (j = 0; j < g->ny; j++)
            for (i = 0; i < g->nx; i++) {
                size_t q = IDX(g, i, j, k);
                Dw[q] = (k == 0 || k == nz) ? 0.0 : diff_w(g, w, nu, i, j, k);
            }
    }
}

static void thomas(int n, const double *lo, const double *di, const double *up, const double *rhs, double *x,
                   double *cp, double *dp);

/* One z-line Jacobi sweep of (I - h D) a = rhs: for every column the
   z-couplings of D are kept implicit and the x-y neighbours are taken from
   the previous iterate a, i.e. per column
     (1 + h S_D) x_k - h cz+_k x_{k+1} - h cz-_k x_{k-1}
         = rhs_k + h sum_{x-y nb} c_nb a_nb,
   solved exactly (Thomas).  S_D is the diagonal weight of D (wall ghosts
   folded in), cz+/- the coefficients of D on the levels above and below,
   c_nb those of the x-y neighbours. */
static void cn_line_sweep(const grid *g, const double *nu, double h, const double *ru, const double *rv,
                          const double *rw, const double *au, const double *av, const double *aw, double *us,
                          double *vs, double *ws)
{
    int j, nz = g->nz;
    double dx2 = g->dx * g->dx, dy2 = g->dy * g->dy;
#pragma omp parallel for schedule(static)
    for (j = 0; j < g->ny; j++) {
        double *lo = (double *)malloc(sizeof(double) * 6 * (nz + 1)), *di = lo + (nz + 1), *up = di + (nz + 1);
        double *rh = up + (nz + 1), *cp = rh + (nz + 1), *dp = cp + (nz + 1);
        double *x = (double *)malloc(sizeof(double) * (nz + 1));
        int i, k;
        for (i = 0; i < g->nx; i++) {
            /* u: levels 0..nz-1 */
            for (k = 0; k < nz; k++) {
                double czp = (k < nz - 1) ? nu_xz(g, nu, i, j, k + 1) / (g->dzf[k + 1] * g->dz[k]) : 0.0;
                double czm = (k > 0) ? nu_xz(g, nu, i, j, k) / (g->dzf[k] * g->dz[k]) : 0.0;
                double xy = (cen_g(g, nu, i, j, k) * vel_g(g, au, i + 1, j, k) +
                             cen_g(g, nu, i - 1, j, k) * vel_g(g, au, i - 1, j, k)) / dx2 +
                            (nu_xy(g, nu, i, j + 1, k) * vel_g(g, au, i, j + 1, k) +
                             nu_xy(g, nu, i, j, k) * vel_g(g, au, i, j - 1, k)) / dy2;
                di[k] = 1.0 + h * diag_u(g, nu, i, j, k);
                up[k] = -h * czp;
                lo[k] = -h * czm;
                rh[k] = ru[IDX(g, i, j, k)] + h * xy;
            }
            thomas(nz, lo, di, up, rh, x, cp, dp);
            for (k = 0; k < nz; k++) us[IDX(g, i, j, k)] = x[k];
            /* v: levels 0..nz-1 */
            for (k = 0; k < nz; k++) {
                double czp = (k < nz - 1) ? nu_yz(g, nu, i, j, k + 1) / (g->dzf[k + 1] * g->dz[k]) : 0.0;
                double czm = (k > 0) ? nu_yz(g, nu, i, j, k) / (g->dzf[k] * g->dz[k]) : 0.0;
                double xy = (nu_xy(g, nu, i + 1, j, k) * vel_g(g, av, i + 1, j, k) +
                             nu_xy(g, nu, i, j, k) * vel_g(g, av, i - 1, j, k)) / dx2 +
                            (cen_g(g, nu, i, j, k) * vel_g(g, av, i, j + 1, k) +
                             cen_g(g, nu, i, j - 1, k) * vel_g(g, av, i, j - 1, k)) / dy2;
                di[k] = 1.0 + h * diag_v(g, nu, i, j, k);
                up[k] = -h * czp;
                lo[k] = -h * czm;
                rh[k] = rv[IDX(g, i, j, k)] + h * xy;
            }
            thomas(nz, lo, di, up, rh, x, cp, dp);
            for (k = 0; k < nz; k++) vs[IDX(g, i, j, k)] = x[k];
            /* w: interior faces 1..nz-1 (row k - 1 of the system); the wall
               faces are zero and couple to nothing */
            ws[IDX(g, i, j, 0)] = 0.0;
            ws[IDX(g, i, j, nz)] = 0.0;
            if (nz >= 2) {
                for (k = 1; k < nz; k++) {
                    double czp = (k < nz - 1) ? cen_g(g, nu, i, j, k) / (g->dz[k] * g->hz[k]) : 0.0;
                    double czm = (k > 1) ? cen_g(g, nu, i, j, k - 1) / (g->dz[k - 1] * g->hz[k]) : 0.0;
                    double xy = (nu_xz(g, nu, i + 1, j, k) * wv(g, aw, i + 1, j, k) +
                                 nu_xz(g, nu, i, j, k) * wv(g, aw, i - 1, j, k)) / dx2 +
                                (nu_yz(g, nu, i, j + 1, k) * wv(g, aw, i, j + 1, k) +
                                 nu_yz(g, nu, i, j, k) * wv(g, aw, i, j - 1, k)) / dy2;
                    di[k - 1] = 1.0 + h * diag_w(g, nu, i, j, k);
                    up[k - 1] = -h * czp;
                    lo[k - 1] = -h * czm;
                    rh[k - 1] = rw[IDX(g, i, j, k)] + h * xy;
                }
                thomas(nz - 1, lo, di, up, rh, x, cp, dp);
                for (k = 1; k < nz; k++) ws[IDX(g, i, j, k)] = x[k - 1];
            }
        }
        free(lo);
        free(x);
    }
}

/* Crank-Nicolson system (I - dt/2 D) a* = rhs by point Jacobi (or, with
   cn_zline, z-line Jacobi), rhs as the first iterate.  One point sweep:
   a_new = (rhs + dt/2 (D a + S_D a)) / (1 + dt/2 S_D). */
static void cn_solve(const orc_params *P, const grid *g, const double *nu, double *ru, double *rv, double *rw,
                     double *us, double *vs, double *ws)
{
    size_t nc = (size_t)g->nx * g->ny * g->nz, nw = (size_t)g->nx * g->ny * (g->nz + 1);
    double *au = (double *)malloc(sizeof(double) * nc), *av = (double *)malloc(sizeof(double) * nc);
    double *aw = (double *)malloc(sizeof(double) * nw);
    double *Du = (double *)malloc(sizeof(double) * nc), *Dv = (double *)malloc(sizeof(double) * nc);
    double *Dw = (double *)malloc(sizeof(double) * nw);
    double h = 0.5 * P->dt;
    int s, k, nz = g->nz;
    memcpy(au, ru, sizeof(double) * nc);
    memcpy(av, rv, sizeof(double) * nc);
    memcpy(aw, rw, sizeof(double) * nw);
    for (s = 0; s < P->cn_sweeps; s++) {
        if (P->cn_zline) {
            cn_line_sweep(g, nu, h, ru, rv, rw, au, av, aw, us, vs, ws);
            memcpy(au, us, sizeof(double) * nc);
            memcpy(av, vs, sizeof(double) * nc);
            memcpy(aw, ws, sizeof(double) * nw);
            continue;
        }
        diffusion(g, au, av, aw, nu, Du, Dv, Dw);
#pragma omp parallel for schedule(static)
        for (k = 0; k < nz; k++) {
            int i, j;
            for (j = 0; j < g->ny; j++)
                for (i = 0; i < g->nx; i++) {
                    size_t q = IDX(g, i, j, k);
                    double su = diag_u(g, nu, i, j, k), sv = diag_v(g, nu, i, j, k);
                    us[q] = (ru[q] + h * (Du[q] + su * au[q])) / (1.0 + h * su);
                    vs[q] = (rv[q] + h * (Dv[q] + sv * av[q])) / (1.0 + h * sv);
                }
        }
#pragma omp parallel for schedule(static)
        for (k = 0; k <= nz; k++) {
            int i, j;
            for (j = 0; j < g->ny; j++)
                for (i = 0; i < g->nx; i++) {
                    size_t q = IDX(g, i, j, k);
                    if (k == 0 || k == nz) { ws[q] = 0.0; continue; }
                    {
                        double sw = diag_w(g, nu, i, j, k);
                        ws[q] = (rw[q] + h * (Dw[q] + sw * aw[q])) / (1.0 + h * sw);
                    }
                }
        }
        memcpy(au, us, sizeof(double) * nc);
        memcpy(av, vs, sizeof(double) * nc);
        memcpy(aw, ws, sizeof(double) * nw);
    }
    if (P->cn_sweeps <= 0) {
        memcpy(us, ru, sizeof(double) * nc);
        memcpy(vs, rv, sizeof(double) * nc);
        memcpy(ws, rw, sizeof(double) * nw);
    }
    free(au); free(av); free(aw); free(Du); free(Dv); free(Dw);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1, Eq. presdiv: discrete divergence and the Poisson operator L=DG  */
/* ------------------------------------------------------------------------ */

static void divergence(const grid *g, const double *u, const double *v, const double *w, double *out)
{
    int k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < g->nz; k++) {
        int i, j;
        for (j = 0; j < g->ny; j++)
            for (i = 0; i < g->nx; i++)
                out[IDX(g, i, j, k)] = (vel_g(g, u, i + 1, j, k) - vel_g(g, u, i, j, k)) / g->dx +
                                       (vel_g(g, v, i, j + 1, k) - vel_g(g, v, i, j, k)) / g->dy +
                                       (wv(g, w, i, j, k + 1) - wv(g, w, i, j, k)) / g->dz[k];
    }
}

/* L p = D(G p): flux form with zero flux through the walls (w fixed at 0) */
static double lap_at(const grid *g, const double *p, int i, int j, int k)
{
    double c = cen_g(g, p, i, j, k);
    double gxp = (cen_g(g, p, i + 1, j, k) - c) / g->dx, gxm = (c - cen_g(g, p, i - 1, j, k)) / g->dx;
    double gyp = (cen_g(g, p, i, j + 1, k) - c) / g->dy, gym = (c - cen_g(g, p, i, j - 1, k)) / g->dy;
    double gzp = (k < g->nz - 1) ? (cen_g(g, p, i, j, k + 1) - c) / g->hz[k + 1] : 0.0;
    double gzm = (k > 0) ? (c - cen_g(g, p, i, j, k - 1)) / g->hz[k] : 0.0;
    return (gxp - gxm) / g->dx + (gyp - gym) / g->dy + (gzp - gzm) / g->dz[k];
}

static void laplacian(const grid *g, const double *p, double *out)
{
    int k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < g->nz; k++) {
        int i, j;
        for (j = 0; j < g->ny; j++)
            for (i = 0; i < g->nx; i++) out[IDX(g, i, j, k)] = lap_at(g, p, i, j, k);
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.4: Scheduled Relaxation Jacobi                                     */
/* ------------------------------------------------------------------------ */

/* Jacobi-SOR sweep (Eq. Jacobi-SOR in 3-D): the Jacobi value p^J solves the
   point equation of L p = b for p_ijk with the neighbours held at their old
   values; the relaxed value is (1-omega) p + omega p^J, written here as
   p + omega (p^J - p). */
static void srj_sweep(const grid *g, const double *p, const double *b, double omega, double *out)
{
    int k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < g->nz; k++) {
        int i, j;
        double cxx = 1.0 / (g->dx * g->dx), cyy = 1.0 / (g->dy * g->dy);
        double cup = (k < g->nz - 1) ? 1.0 / (g->hz[k + 1] * g->dz[k]) : 0.0;
        double cdn = (k > 0) ? 1.0 / (g->hz[k] * g->dz[k]) : 0.0;
        double S = 2.0 * cxx + 2.0 * cyy + cup + cdn;
        for (j = 0; j < g->ny; j++)
            for (i = 0; i < g->nx; i++) {
                double nb = cxx * (cen_g(g, p, i + 1, j, k) + cen_g(g, p, i - 1, j, k)) +
                            cyy * (cen_g(g, p, i, j + 1, k) + cen_g(g, p, i, j - 1, k));
                double pc = p[IDX(g, i, j, k)];
                double pj;
                if (k < g->nz - 1) nb += cup * p[IDX(g, i, j, k + 1)];
                if (k > 0) nb += cdn * p[IDX(g, i, j, k - 1)];
                pj = (nb - b[IDX(g, i, j, k)]) / S;
                out[IDX(g, i, j, k)] = pc + omega * (pj - pc);
            }
    }
}

/* Tridiagonal solve (Thomas algorithm, no pivoting; the matrices here are
   strictly diagonally dominant): lo[k] x[k-1] + di[k] x[k] + up[k] x[k+1]
   = rhs[k], k = 0..n-1 (lo[0], up[n-1] unused).  cp, dp: scratch of n. */
static void thomas(int n, const double *lo, const double *di, const double *up, const double *rhs, double *x,
                   double *cp, double *dp)
{
    int k;
    cp[0] = up[0] / di[0];
    dp[0] = rhs[0] / di[0];
    for (k = 1; k < n; k++) {
        double m = di[k] - lo[k] * cp[k - 1];
        cp[k] = (k < n - 1) ? up[k] / m : 0.0;
        dp[k] = (rhs[k] - lo[k] * dp[k - 1]) / m;
    }
    x[n - 1] = dp[n - 1];
    for (k = n - 2; k >= 0; k--) x[k] = dp[k] - cp[k] * x[k + 1];
}

/* z-line Jacobi-SOR sweep: the line value p^L solves the equations of
   L p = b on a whole z column (i, j) at once, with the x and y neighbours
   held at their old values; relaxed as p + omega (p^L - p).  The column
   equations, multiplied by -1, are
     (2/dx^2 + 2/dy^2 + cup_k + cdn_k) p^L_k - cup_k p^L_{k+1} - cdn_k p^L_{k-1}
        = cxx (p_{i+1} + p_{i-1}) + cyy (p_{j+1} + p_{j-1}) - b_k,
   a tridiagonal system per column (walls: cup = 0 at the top, cdn = 0 at
   the bottom, as in the point sweep). */
static void line_sweep(const grid *g, const double *p, const double *b, double omega, double *out)
{
    int j;
#pragma omp parallel for schedule(static)
    for (j = 0; j < g->ny; j++) {
        int nz = g->nz, i, k;
        double cxx = 1.0 / (g->dx * g->dx), cyy = 1.0 / (g->dy * g->dy);
        double *lo = (double *)malloc(sizeof(double) * nz), *di = (double *)malloc(sizeof(double) * nz);
        double *up = (double *)malloc(sizeof(double) * nz), *rhs = (double *)malloc(sizeof(double) * nz);
        double *x = (double *)malloc(sizeof(double) * nz), *cp = (double *)malloc(sizeof(double) * nz);
        double *dp = (double *)malloc(sizeof(double) * nz);
        for (k = 0; k < nz; k++) {
            double cup = (k < nz - 1) ? 1.0 / (g->hz[k + 1] * g->dz[k]) : 0.0;
            double cdn = (k > 0) ? 1.0 / (g->hz[k] * g->dz[k]) : 0.0;
            di[k] = 2.0 * cxx + 2.0 * cyy + cup + cdn;
            up[k] = -cup;
            lo[k] = -cdn;
        }
        for (i = 0; i < g->nx; i++) {
            for (k = 0; k < nz; k++)
                rhs[k] = cxx * (cen_g(g, p, i + 1, j, k) + cen_g(g, p, i - 1, j, k)) +
                         cyy * (cen_g(g, p, i, j + 1, k) + cen_g(g, p, i, j - 1, k)) - b[IDX(g, i, j, k)];
            thomas(nz, lo, di, up, rhs, x, cp, dp);
            for (k = 0; k < nz; k++) {
                double pc = p[IDX(g, i, j, k)];
                out[IDX(g, i, j, k)] = pc + omega * (x[k] - pc);
            }
        }
        free(lo); free(di); free(up); free(rhs); free(x); free(cp); free(dp);
    }
}

static double norm2(const double *a, size_t n)
{
    double s = 0.0;
    size_t q;
    for (q = 0; q < n; q++) s += a[q] * a[q];
    return sqrt(s);
}

static double residual_norm(const grid *g, const double *p, const double *b, double *tmp)
{
    size_t n = (size_t)g->nx * g->ny * g->nz, q;
    laplacian(g, p, tmp);
    for (q = 0; q < n; q++) tmp[q] = b[q] - tmp[q];
    return norm2(tmp, n);
}

/* SRJ solve of L p = b from the guess in p.  Each cycle: test
   ||b - L p||_2 <= tol ||b||_2, then M sweeps with omega_1..omega_M (point
   sweeps, or z-line sweeps when zline).
   Returns the number of sweeps; *rel gets the final relative residual
   (the absolute norm if ||b|| = 0).  Returns -1-sweeps if maxit was hit. */
static int poisson_srj(const grid *g, double *p, const double *b, int M, const double *omega, double tol,
                       int maxit, int zline, double *rel)
{
    size_t n = (size_t)g->nx * g->ny * g->nz;
    double *tmp = (double *)malloc(sizeof(double) * n);
    double *q2 = (double *)malloc(sizeof(double) * n);
    double nb = norm2(b, n), r;
    int it = 0, m, status;
    for (;;) {
        r = residual_norm(g, p, b, tmp);
        if (r <= tol * nb) { status = it; break; }
        if (it >= maxit) { status = -1 - it; break; }
        for (m = 0; m < M; m++) {
            if (zline)
                line_sweep(g, p, b, omega[m], q2);
            else
                srj_sweep(g, p, b, omega[m], q2);
            memcpy(p, q2, sizeof(double) * n);
            it++;
        }
    }
    *rel = (nb > 0.0) ? r / nb : r;
    free(tmp); free(q2);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1, Eq. project u_p_1: u^{n+1} = u* - dt G p                         */
/* ------------------------------------------------------------------------ */

static void correct(const orc_params *P, const grid *g, const double *p, double *u, double *v, double *w)
{
    int k, nz = g->nz;
    double dt = P->dt;
#pragma omp parallel for schedule(static)
    for (k = 0; k < nz; k++) {
        int i, j;
        for (j = 0; j < g->ny; j++)
            for (i = 0; i < g->nx; i++) {
                size_t q = IDX(g, i, j, k);
                u[q] = u[q] - dt * (cen_g(g, p, i, j, k) - cen_g(g, p, i - 1, j, k)) / g->dx;
                v[q] = v[q] - dt * (cen_g(g, p, i, j, k) - cen_g(g, p, i, j - 1, k)) / g->dy;
            }
    }
#pragma omp parallel for schedule(static)
    for (k = 0; k <= nz; k++) {
        int i, j;
        for (j = 0; j < g->ny; j++)
            for (i = 0; i < g->nx; i++) {
                size_t q = IDX(g, i, j, k);
                if (k == 0 || k == nz) w[q] = 0.0;
                else w[q] = w[q] - dt * (cen_g(g, p, i, j, k) - cen_g(g, p, i, j, k - 1)) / g->hz[k];
            }
    }
}

/* volume-weighted mean of u over the channel */
static double bulk_u(const grid *g, const double *u, double Lz)
{
    double s = 0.0;
    int i, j, k;
    for (k = 0; k < g->nz; k++)
        for (j = 0; j < g->ny; j++)
            for (i = 0; i < g->nx; i++) s += u[IDX(g, i, j, k)] * g->dz[k];
    return s / ((double)g->nx * g->ny * Lz);
}

/* ------------------------------------------------------------------------ */
/* the time step                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    orc_params P;
    double *omega;
    grid g;
    size_t nc, nw;
    double *u, *v, *w, *p, *nu;
    double *Nu[3], *Nv[3], *Nw[3];   /* explicit terms at n, n-1, n-2 */
    int nhist;                         /* how many history levels are valid */
    long step;
    double last_dpdx;                  /* implied -dp/dx of the flux fixup  */
} orc_state;

orc_state *orc_create(const orc_params *P)
{
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    int l;
    s->P = *P;
    s->omega = (double *)malloc(sizeof(double) * (P->srj_m > 0 ? P->srj_m : 1));
    if (P->srj_m > 0) memcpy(s->omega, P->srj_omega, sizeof(double) * P->srj_m);
    s->P.srj_omega = s->omega;
    grid_make(P, &s->g);
    s->nc = (size_t)P->nx * P->ny * P->nz;
    s->nw = (size_t)P->nx * P->ny * (P->nz + 1);
    s->u = (double *)calloc(s->nc, sizeof(double));
    s->v = (double *)calloc(s->nc, sizeof(double));
    s->w = (double *)calloc(s->nw, sizeof(double));
    s->p = (double *)calloc(s->nc, sizeof(double));
    s->nu = (double *)calloc(s->nc, sizeof(double));
    for (l = 0; l < 3; l++) {
        s->Nu[l] = (double *)calloc(s->nc, sizeof(double));
        s->Nv[l] = (double *)calloc(s->nc, sizeof(double));
        s->Nw[l] = (double *)calloc(s->nw, sizeof(double));
    }
    return s;
}

void orc_destroy(orc_state *s)
{
    int l;
    if (!s) return;
    free(s->u); free(s->v); free(s->w); free(s->p); free(s->nu); free(s->omega);
    for (l = 0; l < 3; l++) { free(s->Nu[l]); free(s->Nv[l]); free(s->Nw[l]); }
    grid_free(&s->g);
    free(s);
}

void orc_set_fields(orc_state *s, const double *u, const double *v, const double *w, const double *p)
{
    memcpy(s->u, u, sizeof(double) * s->nc);
    memcpy(s->v, v, sizeof(double) * s->nc);
    memcpy(s->w, w, sizeof(double) * s->nw);
    if (p) memcpy(s->p, p, sizeof(double) * s->nc);
    else memset(s->p, 0, sizeof(double) * s->nc);
    s->nhist = 0;
    s->step = 0;
}

void orc_get_fields(const orc_state *s, double *u, double *v, double *w, double *p, double *nu)
{
    if (u) memcpy(u, s->u, sizeof(double) * s->nc);
    if (v) memcpy(v, s->v, sizeof(double) * s->nc);
    if (w) memcpy(w, s->w, sizeof(double) * s->nw);
    if (p) memcpy(p, s->p, sizeof(double) * s->nc);
    if (nu) memcpy(nu, s->nu, sizeof(double) * s->nc);
}

/* One projection step (Sec. 3.1).  stats[0] = SRJ sweeps, stats[1] = final
   relative residual, stats[2] = max |div u^{n+1}|, stats[3] = bulk velocity,
   stats[4] = max |u|, stats[5] = implied -dp/dx (flux forcing).
   Returns 0, or 1 if the pressure solve hit its sweep cap. */
static int one_step(orc_state *s, double *stats)
{
    const orc_params *P = &s->P;
    const grid *g = &s->g;
    size_t nc = s->nc, nw = s->nw, q;
    double *Nu0, *Nv0, *Nw0;
    double b0, b1, b2;
    double *ru = (double *)malloc(sizeof(double) * nc), *rv = (double *)malloc(sizeof(double) * nc);
    double *rw = (double *)malloc(sizeof(double) * nw);
    double *Du = (double *)malloc(sizeof(double) * nc), *Dv = (double *)malloc(sizeof(double) * nc);
    double *Dw = (double *)malloc(sizeof(double) * nw);
    double *us = (double *)malloc(sizeof(double) * nc), *vs = (double *)malloc(sizeof(double) * nc);
    double *ws = (double *)malloc(sizeof(double) * nw);
    double *b = (double *)malloc(sizeof(double) * nc);
    double rel = 0.0, dmax = 0.0, umax = 0.0;
    int it, status = 0;

    /* rotate the history ring: slot 0 becomes level n */
    Nu0 = s->Nu[2]; Nv0 = s->Nv[2]; Nw0 = s->Nw[2];
    s->Nu[2] = s->Nu[1]; s->Nv[2] = s->Nv[1]; s->Nw[2] = s->Nw[1];
    s->Nu[1] = s->Nu[0]; s->Nv[1] = s->Nv[0]; s->Nw[1] = s->Nw[0];
    s->Nu[0] = Nu0; s->Nv[0] = Nv0; s->Nw[0] = Nw0;

    /* nu_T at time n (Sec. 2.2, frozen over the step) */
    total_viscosity(P, g, s->u, s->v, s->w, s->nu);
    /* explicit terms at time n */
    explicit_terms(P, g, s->u, s->v, s->w, s->nu, s->Nu[0], s->Nv[0], s->Nw[0]);
    if (s->nhist < 3) s->nhist++;
    /* Adams-Bashforth: forward Euler, then AB2, then AB3 (23,-16,5)/12 */
    if (s->nhist == 1) { b0 = 1.0; b1 = 0.0; b2 = 0.0; }
    else if (s->nhist == 2) { b0 = 1.5; b1 = -0.5; b2 = 0.0; }
    else { b0 = 23.0 / 12.0; b1 = -16.0 / 12.0; b2 = 5.0 / 12.0; }
    /* CN right-hand side: u^n + dt*AB + dt/2 D u^n */
    diffusion(g, s->u, s->v, s->w, s->nu, Du, Dv, Dw);
    for (q = 0; q < nc; q++) {
        ru[q] = s->u[q] + P->dt * (b0 * s->Nu[0][q] + b1 * s->Nu[1][q] + b2 * s->Nu[2][q]) + 0.5 * P->dt * Du[q];
        rv[q] = s->v[q] + P->dt * (b0 * s->Nv[0][q] + b1 * s->Nv[1][q] + b2 * s->Nv[2][q]) + 0.5 * P->dt * Dv[q];
    }
    for (q = 0; q < nw; q++)
        rw[q] = s->w[q] + P->dt * (b0 * s->Nw[0][q] + b1 * s->Nw[1][q] + b2 * s->Nw[2][q]) + 0.5 * P->dt * Dw[q];
    /* wall faces of w stay zero */
    for (q = 0; q < (size_t)g->nx * g->ny; q++) { rw[q] = 0.0; rw[nw - 1 - q] = 0.0; }
    /* provisional velocity */
    cn_solve(P, g, s->nu, ru, rv, rw, us, vs, ws);
    /* Poisson right-hand side b = D u* / dt */
    divergence(g, us, vs, ws, b);
    for (q = 0; q < nc; q++) b[q] = b[q] / P->dt;
    /* pressure, previous p as the guess */
    it = poisson_srj(g, s->p, b, P->srj_m, P->srj_omega, P->ptol, P->pmaxit, P->zline, &rel);
    if (it < 0) { status = 1; it = -1 - it; }
    /* projection */
    correct(P, g, s->p, us, vs, ws);
    if (P->forcing == 1) {
        double ub = bulk_u(g, us, P->Lz);
        for (q = 0; q < nc; q++) us[q] += P->ubulk - ub;
        s->last_dpdx = (P->ubulk - ub) / P->dt;
    }
    memcpy(s->u, us, sizeof(double) * nc);
    memcpy(s->v, vs, sizeof(double) * nc);
    memcpy(s->w, ws, sizeof(double) * nw);
    divergence(g, s->u, s->v, s->w, b);
    for (q = 0; q < nc; q++) {
        if (fabs(b[q]) > dmax) dmax = fabs(b[q]);
        if (fabs(s->u[q]) > umax) umax = fabs(s->u[q]);
    }
    s->step++;
    if (stats) {
        stats[0] = it; stats[1] = rel; stats[2] = dmax; stats[3] = bulk_u(g, s->u, P->Lz);
        stats[4] = umax; stats[5] = s->last_dpdx;
    }
    free(ru); free(rv); free(rw); free(Du); free(Dv); free(Dw); free(us); free(vs); free(ws); free(b);
    return status;
}

int orc_step(orc_state *s, int nsteps, double *stats)
{
    int n, st = 0;
    for (n = 0; n < nsteps; n++) st |= one_step(s, stats);
    return st;
}

/* ------------------------------------------------------------------------ */
/* building blocks exposed for the pins (each builds its own grid)           */
/* ------------------------------------------------------------------------ */

void orc_viscosity(const orc_params *P, const double *u, const double *v, const double *w, double *nu)
{
    grid g; grid_make(P, &g); total_viscosity(P, &g, u, v, w, nu); grid_free(&g);
}

void orc_explicit(const orc_params *P, const double *u, const double *v, const double *w, const double *nu,
                  double *Nu, double *Nv, double *Nw)
{
    grid g; grid_make(P, &g); explicit_terms(P, &g, u, v, w, nu, Nu, Nv, Nw); grid_free(&g);
}

/* advective term only (u.grad u), for the pins */
void orc_advection(const orc_params *P, const double *u, const double *v, const double *w,
                   double *Au, double *Av, double *Aw)
{
    grid g; int i, j, k;
    grid_make(P, &g);
    for (k = 0; k < g.nz; k++)
        for (j = 0; j < g.ny; j++)
            for (i = 0; i < g.nx; i++) {
                Au[IDX(&g, i, j, k)] = adv_u(&g, u, v, w, i, j, k);
                Av[IDX(&g, i, j, k)] = adv_v(&g, u, v, w, i, j, k);
            }
    for (k = 0; k <= g.nz; k++)
        for (j = 0; j < g.ny; j++)
            for (i = 0; i < g.nx; i++)
                Aw[IDX(&g, i, j, k)] = (k == 0 || k == g.nz) ? 0.0 : adv_w(&g, u, v, w, i, j, k);
    grid_free(&g);
}

/* convective-like viscous term only */
void orc_cross_viscous(const orc_params *P, const double *u, const double *v, const double *w, const double *nu,
                       double *Cu, double *Cv, double *Cw)
{
    grid g; int i, j, k;
    grid_make(P, &g);
    for (k = 0; k < g.nz; k++)
        for (j = 0; j < g.ny; j++)
            for (i = 0; i < g.nx; i++) {
                Cu[IDX(&g, i, j, k)] = cvisc_u(&g, u, v, w, nu, i, j, k);
                Cv[IDX(&g, i, j, k)] = cvisc_v(&g, u, v, w, nu, i, j, k);
            }
    for (k = 0; k <= g.nz; k++)
        for (j = 0; j < g.ny; j++)
            for (i = 0; i < g.nx; i++)
                Cw[IDX(&g, i, j, k)] = (k == 0 || k == g.nz) ? 0.0 : cvisc_w(&g, u, v, w, nu, i, j, k);
    grid_free(&g);
}

void orc_diffusion(const orc_params *P, const double *u, const double *v, const double *w, const double *nu,
                   double *Du, double *Dv, double *Dw)
{
    grid g; grid_make(P, &g); diffusion(&g, u, v, w, nu, Du, Dv, Dw); grid_free(&g);
}

void orc_diffusion_diag(const orc_params *P, const double *nu, double *Su, double *Sv, double *Sw)
{
    grid g; int i, j, k;
    grid_make(P, &g);
    for (k = 0; k < g.nz; k++)
        for (j = 0; j < g.ny; j++)
            for (i = 0; i < g.nx; i++) {
                Su[IDX(&g, i, j, k)] = diag_u(&g, nu, i, j, k);
                Sv[IDX(&g, i, j, k)] = diag_v(&g, nu, i, j, k);
            }
    for (k = 0; k <= g.nz; k++)
        for (j = 0; j < g.ny; j++)
            for (i = 0; i < g.nx; i++)
                Sw[IDX(&g, i, j, k)] = (k == 0 || k == g.nz) ? 0.0 : diag_w(&g, nu, i, j, k);
    grid_free(&g);
}

void orc_cn_solve(const orc_params *P, const double *nu, double *ru, double *rv, double *rw,
                  double *us, double *vs, double *ws)
{
    grid g; grid_make(P, &g); cn_solve(P, &g, nu, ru, rv, rw, us, vs, ws); grid_free(&g);
}

void orc_divergence(const orc_params *P, const double *u, const double *v, const double *w, double *out)
{
    grid g; grid_make(P, &g); divergence(&g, u, v, w, out); grid_free(&g);
}

void orc_laplacian(const orc_params *P, const double *p, double *out)
{
    grid g; grid_make(P, &g); laplacian(&g, p, out); grid_free(&g);
}

void orc_srj_sweep(const orc_params *P, const double *p, const double *b, double omega, double *out)
{
    grid g; grid_make(P, &g); srj_sweep(&g, p, b, omega, out); grid_free(&g);
}

void orc_line_sweep(const orc_params *P, const double *p, const double *b, double omega, double *out)
{
    grid g; grid_make(P, &g); line_sweep(&g, p, b, omega, out); grid_free(&g);
}

int orc_poisson(const orc_params *P, double *p, const double *b, double tol, int maxit, double *rel)
{
    grid g; int it;
    grid_make(P, &g);
    it = poisson_srj(&g, p, b, P->srj_m, P->srj_omega, tol, maxit, P->zline, rel);
    grid_free(&g);
    return it;
}

void orc_correct(const orc_params *P, const double *p, double *u, double *v, double *w)
{
    grid g; grid_make(P, &g); correct(P, &g, p, u, v, w); grid_free(&g);
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    int n = 1;
#pragma omp parallel
    {
#pragma omp master
        n = omp_get_num_threads();
    }
    return n;
#else
    return 1;
#endif
}
