/*
 * vp_oracle.c -- plain FP64 CPU oracle for the SL-MPP5/7 Vlasov-Poisson
 * method (Tanaka, Yoshikawa, Minoshima & Yoshida 2017).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU baseline, never by the product path.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Style: each function follows the paper's steps in the paper's order with
 * plain loops and no blocking, fusion or reordering beyond what the printed
 * formulas state.  Where the paper is silent or ambiguous the reading taken
 * is stated next to the code (R1..R12, listed again in the design notes).
 * The only parallelism is an OpenMP loop over independent lines.
 */
#include "vp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* unit roundoff of the oracle's arithmetic (FP64) */
static const double VPO_EPS = 1.1102230246251565e-16; /* 2^-53 */

/* ------------------------------------------------------------------------ */
/* small helpers: minmod and median as used by Suresh & Huynh (Appendix A)  */
/* ------------------------------------------------------------------------ */

/* R4: minmod(a, b, ...) is the argument of smallest magnitude when all
 * arguments share one sign, and 0 otherwise. */
static double minmod2(double a, double b) {
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

static double minmod4(double a, double b, double c, double d) {
    if (a > 0.0 && b > 0.0 && c > 0.0 && d > 0.0) {
        double m = a;
        if (b < m) m = b;
        if (c < m) m = c;
        if (d < m) m = d;
        return m;
    }
    if (a < 0.0 && b < 0.0 && c < 0.0 && d < 0.0) {
        double m = a;
        if (b > m) m = b;
        if (c > m) m = c;
        if (d > m) m = d;
        return m;
    }
    return 0.0;
}

static double min3(double a, double b, double c) {
    double m = a;
    if (b < m) m = b;
    if (c < m) m = c;
    return m;
}

static double max3(double a, double b, double c) {
    double m = a;
    if (b > m) m = b;
    if (c > m) m = c;
    return m;
}

/* R4: median(a, b, c) is the middle value of the three. */
static double median3(double a, double b, double c) {
    double lo = a < b ? a : b;
    double hi = a < b ? b : a;
    if (c < lo) return lo;
    if (c > hi) return hi;
    return c;
}

/* ------------------------------------------------------------------------ */
/* CSL flux, Sec. 2.1.2                                                      */
/* ------------------------------------------------------------------------ */
/*
 * Phi_{i-1/2} for a flow from cell i-1 into cell i.  The paper's stencil
 * f_{i-4} .. f_{i+2} maps onto u[-3] .. u[3] with u[0] = f_{i-1} the upwind
 * cell.  CSL5: Phi = sum_{j=0}^{4} C_j zeta^j (Eqs. 29-34); CSL7:
 * Phi = sum_{j=0}^{6} D_j zeta^j (Eqs. 36-43); zeta = nu here.
 */
double vpo_csl_flux(int order, double nu, const double *u) {
    const double fim4 = u[-3], fim3 = u[-2], fim2 = u[-1], fim1 = u[0];
    const double fi = u[1], fip1 = u[2], fip2 = u[3];
    double c[7];
    int nterm;
    if (order == 5) {
        c[0] = fim3 / 30.0 - 13.0 / 60.0 * fim2 + 47.0 / 60.0 * fim1 + 9.0 / 20.0 * fi - fip1 / 20.0;
        c[1] = -fim2 / 24.0 + 5.0 / 8.0 * fim1 - 5.0 / 8.0 * fi + fip1 / 24.0;
        c[2] = -fim3 / 24.0 + fim2 / 4.0 - fim1 / 3.0 + fi / 12.0 + fip1 / 24.0;
        c[3] = fim2 / 24.0 - fim1 / 8.0 + fi / 8.0 - fip1 / 24.0;
        c[4] = fim3 / 120.0 - fim2 / 30.0 + fim1 / 20.0 - fi / 30.0 + fip1 / 120.0;
        nterm = 5;
    } else {
        c[0] = -fim4 / 140.0 + 5.0 / 84.0 * fim3 - 101.0 / 420.0 * fim2 + 319.0 / 420.0 * fim1 +
               107.0 / 210.0 * fi - 19.0 / 210.0 * fip1 + fip2 / 105.0;
        c[1] = fim3 / 180.0 - 5.0 / 72.0 * fim2 + 49.0 / 72.0 * fim1 - 49.0 / 72.0 * fi +
               5.0 / 72.0 * fip1 - fip2 / 180.0;
        c[2] = 7.0 / 720.0 * fim4 - 19.0 / 240.0 * fim3 + 7.0 / 24.0 * fim2 - 23.0 / 72.0 * fim1 +
               fi / 48.0 + 7.0 / 80.0 * fip1 - fip2 / 90.0;
        c[3] = -fim3 / 144.0 + 11.0 / 144.0 * fim2 - 7.0 / 36.0 * fim1 + 7.0 / 36.0 * fi -
               11.0 / 144.0 * fip1 + fip2 / 144.0;
        c[4] = -fim4 / 360.0 + fim3 / 48.0 - 13.0 / 240.0 * fim2 + 23.0 / 360.0 * fim1 - fi / 30.0 +
               fip1 / 240.0 + fip2 / 720.0;
        c[5] = fim3 / 720.0 - fim2 / 144.0 + fim1 / 72.0 - fi / 72.0 + fip1 / 144.0 - fip2 / 720.0;
        c[6] = fim4 / 5040.0 - fim3 / 840.0 + fim2 / 336.0 - fim1 / 252.0 + fi / 336.0 -
               fip1 / 840.0 + fip2 / 5040.0;
        nterm = 7;
    }
    double phi = 0.0, zj = 1.0;
    for (int j = 0; j < nterm; ++j) {
        phi += c[j] * zj;
        zj *= nu;
    }
    return phi;
}

/* ------------------------------------------------------------------------ */
/* MP constraint, Appendix A (Suresh & Huynh 1997)                           */
/* ------------------------------------------------------------------------ */
/*
 * Interface between u[0] (the paper's f_i) and u[1] (f_{i+1}); uses
 * u[-2..2] = f_{i-2} .. f_{i+2}; phi is step 1's interpolated value.
 * vpo_mp_bounds returns f^min and f^max of steps 4-6.
 */
void vpo_mp_bounds(const double *u, double alpha, double *fmin_out, double *fmax_out) {
    const double fim2 = u[-2], fim1 = u[-1], fi = u[0], fip1 = u[1], fip2 = u[2];
    /* step 4: d_k = f_{k-1} + f_{k+1} - 2 f_k */
    double d_im1 = fim2 + fi - 2.0 * fim1;
    double d_i = fim1 + fip1 - 2.0 * fi;
    double d_ip1 = fi + fip2 - 2.0 * fip1;
    double dm4_p = minmod4(4.0 * d_i - d_ip1, 4.0 * d_ip1 - d_i, d_i, d_ip1);   /* d^M4_{i+1/2} */
    double dm4_m = minmod4(4.0 * d_im1 - d_i, 4.0 * d_i - d_im1, d_im1, d_i);   /* d^M4_{i-1/2} */
    /* step 5 */
    double f_ul = fi + alpha * (fi - fim1);
    double f_av = (fi + fip1) / 2.0;
    double f_md = f_av - dm4_p / 2.0;
    double f_lc = fi + (fi - fim1) / 2.0 + 4.0 * dm4_m / 3.0;
    /* step 6 */
    double a = min3(fi, fip1, f_md), b = min3(fi, f_ul, f_lc);
    *fmin_out = a > b ? a : b;
    a = max3(fi, fip1, f_md);
    b = max3(fi, f_ul, f_lc);
    *fmax_out = a < b ? a : b;
}

double vpo_mp_constraint(double phi, const double *u, double alpha) {
    const double fim1 = u[-1], fi = u[0], fip1 = u[1];
    /* step 2 */
    double fstar = fi + minmod2(fip1 - fi, alpha * (fi - fim1));
    /* step 3 (R3: the strict "< 0" as printed) */
    if ((phi - fi) * (phi - fstar) < 0.0) return phi;
    /* steps 4-6 */
    double f_min, f_max;
    vpo_mp_bounds(u, alpha, &f_min, &f_max);
    /* step 7 */
    return median3(phi, f_min, f_max);
}

/* ------------------------------------------------------------------------ */
/* PP flux limiter, Sec. 2.1.1 Eqs. (15)-(23), used as Eqs. (47)-(48)        */
/* ------------------------------------------------------------------------ */
/*
 * PP(phibar, f_i, f_{i+1}) with u0 = f_i upwind, u1 = f_{i+1} downwind.
 * The upwind interface value is f^UP_{i+1/2} = f_i (Eq. 16 with c > 0).
 * R5: when theta binds it is scaled by (1 - 8 eps) so that the two halves
 * of Eq. (19) stay >= 0 after rounding, and it is clamped to [0, 1]; a
 * non-positive denominator (possible only for negative input data) gives
 * theta = 0, i.e. the upwind flux.
 */
double vpo_pp_limiter(double phibar, double u0, double u1, double nu) {
    double u_plus = u0 - 2.0 * nu * phibar;      /* U^+_i          */
    double u_up_plus = u0 - 2.0 * nu * u0;       /* U^{UP,+}_i     */
    double u_minus = u1 + 2.0 * nu * phibar;     /* U^-_{i+1}      */
    double u_up_minus = u1 + 2.0 * nu * u0;      /* U^{UP,-}_{i+1} */
    double th_plus = 1.0, th_minus = 1.0;
    int binds = 0;
    if (u_plus < 0.0) {
        double den = u_up_plus - u_plus;
        th_plus = den > 0.0 ? u_up_plus / den : 0.0;
        binds = 1;
    }
    if (u_minus < 0.0) {
        double den = u_up_minus - u_minus;
        th_minus = den > 0.0 ? u_up_minus / den : 0.0;
        binds = 1;
    }
    double theta = th_plus < th_minus ? th_plus : th_minus;
    if (binds) theta *= (1.0 - 8.0 * VPO_EPS);
    if (theta < 0.0) theta = 0.0;
    if (theta > 1.0) theta = 1.0;
    return theta * phibar + (1.0 - theta) * u0;
}

double vpo_interface_flux(int order, int mp, int pp, double alpha, double nu, const double *u) {
    double phi = vpo_csl_flux(order, nu, u);
    if (mp) phi = vpo_mp_constraint(phi, u, alpha);
    if (pp) phi = vpo_pp_limiter(phi, u[0], u[1], nu);
    return phi;
}

/* ------------------------------------------------------------------------ */
/* shift decomposition and the SL update of one line                        */
/* ------------------------------------------------------------------------ */
/*
 * R2: a shift of s = c dt / Delta cells is split as s = N + zeta with N the
 * nearest integer (halves away from zero) and zeta in [-1/2, 1/2].  The
 * integer part is an exact copy of cells; the fractional part is one SL-MPP
 * step with CFL number nu = |zeta| in the direction sign(zeta).
 */
void vpo_shift_split(double s, long *n_int, double *zeta) {
    double n = round(s);
    *n_int = (long)n;
    *zeta = s - n;
}

static double fetch(const double *g, long L, int bc, long i) {
    if (bc == VPO_BC_PERIODIC) {
        long m = i % L;
        if (m < 0) m += L;
        return g[m];
    }
    return (i >= 0 && i < L) ? g[i] : 0.0; /* R6: zero ghost cells */
}

/*
 * Eq. (49): f^{n+1}_i = f^n_i - nu (Phi^_{i+1/2} - Phi^_{i-1/2}) on the
 * line shifted by N cells.  For zeta < 0 the stencil is mirrored (the
 * paper treats c > 0 without loss of generality, Sec. 2.1): the cell's
 * outgoing interface is then its left one and the upwind neighbour of its
 * incoming interface is its right neighbour.
 */
void vpo_advect_line(int order, int mp, int pp, double alpha, int bc, long L,
                     double *line, long stride, double s) {
    long n_int;
    double zeta;
    vpo_shift_split(s, &n_int, &zeta);
    const long sigma = zeta < 0.0 ? -1 : 1;
    const double nu = fabs(zeta);

    double stack_g[2048], stack_o[2048];
    double *g = stack_g, *out = stack_o;
    if (L > 2048) {
        g = (double *)malloc(sizeof(double) * L);
        out = (double *)malloc(sizeof(double) * L);
    }
    for (long i = 0; i < L; ++i) g[i] = line[i * stride];

    for (long i = 0; i < L; ++i) {
        /* w[k+4] = value, after the integer shift, of the cell k steps
         * upwind-ordered from cell i: f^n_{i - N + sigma k}, k = -4..4 */
        double w[9];
        for (int k = -4; k <= 4; ++k) w[k + 4] = fetch(g, L, bc, i - n_int + sigma * k);
        double phi_out = vpo_interface_flux(order, mp, pp, alpha, nu, &w[4]); /* upwind cell: i      */
        double phi_in = vpo_interface_flux(order, mp, pp, alpha, nu, &w[3]);  /* upwind cell: i - sg */
        out[i] = w[4] - nu * (phi_out - phi_in);
    }
    for (long i = 0; i < L; ++i) line[i * stride] = out[i];
    if (g != stack_g) {
        free(g);
        free(out);
    }
}

/* ------------------------------------------------------------------------ */
/* RK--MPP5, Sec. 2.1.1: Eq. (8) interface value, Eq. (9) MP, the PP limiter  */
/* of Eqs. (15)-(23), three-stage TVD Runge-Kutta, Eq. (10)                   */
/* ------------------------------------------------------------------------ */
/*
 * Interface value between u[0] = f_i (upwind) and u[1] = f_{i+1}: Eq. (8)
 * written for the interface i+1/2, i.e. on f_{i-2} .. f_{i+2}.
 */
static double rk_interface(int mp, int pp, double alpha, double nu, const double *u) {
    double phi = (2.0 * u[-2] - 13.0 * u[-1] + 47.0 * u[0] + 27.0 * u[1] - 3.0 * u[2]) / 60.0;
    if (mp) phi = vpo_mp_constraint(phi, u, alpha);
    if (pp) phi = vpo_pp_limiter(phi, u[0], u[1], nu);
    return phi;
}

/* one Euler stage out_i = g_i - nu L_i(g), L_i = f^_{i+1/2} - f^_{i-1/2};
 * for c < 0 the stencil is mirrored (sigma = -1) */
static void rk_stage(int mp, int pp, double alpha, int bc, long L, const double *g, long sigma, double nu,
                     double *out) {
    for (long i = 0; i < L; ++i) {
        double w[7];
        for (int k = -3; k <= 3; ++k) w[k + 3] = fetch(g, L, bc, i + sigma * k);
        double flux_out = rk_interface(mp, pp, alpha, nu, &w[3]); /* upwind cell i          */
        double flux_in = rk_interface(mp, pp, alpha, nu, &w[2]);  /* upwind cell i - sigma  */
        out[i] = w[3] - nu * (flux_out - flux_in);
    }
}

/* One RK--MPP5 step of a line with CFL number cnu = c dt / dx (signed);
 * returns -1 (line untouched) unless |cnu| < 1/2, the PP limiter's condition. */
int vpo_rk_mpp5_line(int mp, int pp, double alpha, int bc, long L, double *line, long stride, double cnu) {
    const long sigma = cnu < 0.0 ? -1 : 1;
    const double nu = fabs(cnu);
    if (!(nu < 0.5)) return -1;
    double *f0 = (double *)malloc(sizeof(double) * 4 * L);
    double *f1 = f0 + L, *f2 = f1 + L, *e = f2 + L;
    for (long i = 0; i < L; ++i) f0[i] = line[i * stride];
    rk_stage(mp, pp, alpha, bc, L, f0, sigma, nu, f1);                 /* f^(1) */
    rk_stage(mp, pp, alpha, bc, L, f1, sigma, nu, e);
    for (long i = 0; i < L; ++i) f2[i] = 0.75 * f0[i] + 0.25 * e[i];   /* f^(2) */
    rk_stage(mp, pp, alpha, bc, L, f2, sigma, nu, e);
    for (long i = 0; i < L; ++i) line[i * stride] = f0[i] / 3.0 + 2.0 / 3.0 * e[i];
    free(f0);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* grid helpers                                                             */
/* ------------------------------------------------------------------------ */
long vpo_nx_total(const vpo_grid *g) {
    long n = 1;
    for (int d = 0; d < g->dx; ++d) n *= g->nx[d];
    return n;
}

long vpo_nv_total(const vpo_grid *g) {
    long n = 1;
    for (int d = 0; d < g->dv; ++d) n *= g->nv[d];
    return n;
}

static double dxd(const vpo_grid *g, int d) { return (g->xhi[d] - g->xlo[d]) / g->nx[d]; }
static double dvd(const vpo_grid *g, int d) { return (g->vhi[d] - g->vlo[d]) / g->nv[d]; }
static double xc(const vpo_grid *g, int d, long i) { return g->xlo[d] + (i + 0.5) * dxd(g, d); }
static double vc(const vpo_grid *g, int d, long j) { return g->vlo[d] + (j + 0.5) * dvd(g, d); }

static int grid_ok(const vpo_grid *g) {
    if (g->dx < 1 || g->dx > 3 || g->dv != g->dx) return 0;
    if (g->order != 5 && g->order != 7) return 0;
    for (int d = 0; d < g->dx; ++d)
        if (g->nx[d] < 1 || g->nv[d] < 1) return 0;
    return 1;
}

static int nthreads_req = 0;
void vpo_set_threads(int n) {
    nthreads_req = n;
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#endif
}
int vpo_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* directional sweeps, Eqs. (4)-(5)                                          */
/* ------------------------------------------------------------------------ */
/* Advection along x_dim with speed v_dim (the cell centre of that velocity
 * index), Eq. (4): every line along x_dim, s = v dt / Delta x. */
int vpo_drift_sweep(const vpo_grid *g, double *f, int dim, double dt) {
    if (!grid_ok(g) || dim < 0 || dim >= g->dx) return -1;
    const long NV = vpo_nv_total(g);
    long outer = 1, inner = NV, vstride = 1;
    for (int k = 0; k < dim; ++k) outer *= g->nx[k];
    for (int k = dim + 1; k < g->dx; ++k) inner *= g->nx[k];
    for (int k = dim + 1; k < g->dv; ++k) vstride *= g->nv[k];
    const long L = g->nx[dim];
    const double h = dxd(g, dim);
    const long nlines = outer * inner;
#pragma omp parallel for schedule(static)
    for (long line = 0; line < nlines; ++line) {
        long o = line / inner, c = line % inner;
        long vid = ((c % NV) / vstride) % g->nv[dim];
        double s = vc(g, dim, vid) * dt / h;
        vpo_advect_line(g->order, g->mp, g->pp, g->alpha, g->xbc, L, f + o * L * inner + c, inner, s);
    }
    return 0;
}

/* Advection along v_dim with the acceleration of the line's spatial point,
 * Eq. (5): s = a dt / Delta v; velocity boundaries never let mass in (R6). */
int vpo_kick_sweep(const vpo_grid *g, double *f, int dim, double dt, const double *accel_dim) {
    if (!grid_ok(g) || dim < 0 || dim >= g->dv) return -1;
    const long NX = vpo_nx_total(g);
    long vouter = 1, inner = 1;
    for (int k = 0; k < dim; ++k) vouter *= g->nv[k];
    for (int k = dim + 1; k < g->dv; ++k) inner *= g->nv[k];
    const long L = g->nv[dim];
    const double h = dvd(g, dim);
    const long nlines = NX * vouter * inner;
#pragma omp parallel for schedule(static)
    for (long line = 0; line < nlines; ++line) {
        long o = line / inner, c = line % inner;
        long xpt = o / vouter;
        double s = accel_dim[xpt] * dt / h;
        vpo_advect_line(g->order, g->mp, g->pp, g->alpha, VPO_BC_OUTFLOW, L, f + o * L * inner + c,
                        inner, s);
    }
    return 0;
}

/* Unsplit advection in physical space (Sec. 3.1, Test-1d; Sec. 2.4 names it
 * as the alternative to directional splitting).  R23: the paper does not print
 * the update it timed; the reading taken is the flux form with every
 * direction's SL-MPP fluxes taken from f^n in one conservative update,
 *   f^{n+1} = f^n + sum_d (A_d f^n - f^n),
 * A_d f^n the 1D line update along x_d (Eq. 49, exactly what vpo_drift_sweep
 * along d makes of f^n).  Each increment A_d f^n - f^n is a difference of
 * interface masses along d, so the update conserves mass; it needs f^n kept
 * whole while the increments are formed (the extra storage the paper cites).
 * Positivity is not guaranteed: each direction's PP limiter allows a cell to
 * lose half of itself through each face, i.e. up to D times its content over
 * all 2D faces; the paper keeps the CFL number below 0.1 for this reason. */
int vpo_drift_unsplit(const vpo_grid *g, double *f, double dt) {
    if (!grid_ok(g)) return -1;
    const long n = vpo_nx_total(g) * vpo_nv_total(g);
    double *a = (double *)malloc(sizeof(double) * n);   /* A_d f^n */
    double *inc = (double *)calloc(n, sizeof(double));  /* sum_d (A_d f^n - f^n) */
    if (!a || !inc) {
        free(a);
        free(inc);
        return -1;
    }
    for (int d = 0; d < g->dx; ++d) {
        memcpy(a, f, sizeof(double) * n);
        vpo_drift_sweep(g, a, d, dt);
        for (long i = 0; i < n; ++i) inc[i] += a[i] - f[i];
    }
    for (long i = 0; i < n; ++i) f[i] += inc[i];
    free(a);
    free(inc);
    return 0;
}

/* The sweeps above with RK--MPP5 in place of the SL update (Sec. 2.1.1);
 * -1 if any line's |c dt / Delta| >= 1/2 (those lines are left unchanged). */
int vpo_drift_sweep_rk(const vpo_grid *g, double *f, int dim, double dt) {
    if (!grid_ok(g) || dim < 0 || dim >= g->dx) return -1;
    const long NV = vpo_nv_total(g);
    long outer = 1, inner = NV, vstride = 1;
    for (int k = 0; k < dim; ++k) outer *= g->nx[k];
    for (int k = dim + 1; k < g->dx; ++k) inner *= g->nx[k];
    for (int k = dim + 1; k < g->dv; ++k) vstride *= g->nv[k];
    const long L = g->nx[dim];
    const double h = dxd(g, dim);
    const long nlines = outer * inner;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long line = 0; line < nlines; ++line) {
        long o = line / inner, c = line % inner;
        long vid = ((c % NV) / vstride) % g->nv[dim];
        double cnu = vc(g, dim, vid) * dt / h;
        bad |= vpo_rk_mpp5_line(g->mp, g->pp, g->alpha, g->xbc, L, f + o * L * inner + c, inner, cnu) != 0;
    }
    return bad ? -1 : 0;
}

int vpo_kick_sweep_rk(const vpo_grid *g, double *f, int dim, double dt, const double *accel_dim) {
    if (!grid_ok(g) || dim < 0 || dim >= g->dv) return -1;
    const long NX = vpo_nx_total(g);
    long vouter = 1, inner = 1;
    for (int k = 0; k < dim; ++k) vouter *= g->nv[k];
    for (int k = dim + 1; k < g->dv; ++k) inner *= g->nv[k];
    const long L = g->nv[dim];
    const double h = dvd(g, dim);
    const long nlines = NX * vouter * inner;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long line = 0; line < nlines; ++line) {
        long o = line / inner, c = line % inner;
        long xpt = o / vouter;
        double cnu = accel_dim[xpt] * dt / h;
        bad |= vpo_rk_mpp5_line(g->mp, g->pp, g->alpha, VPO_BC_OUTFLOW, L, f + o * L * inner + c, inner,
                                cnu) != 0;
    }
    return bad ? -1 : 0;
}

/* rho(x) = integral of f over velocity space (Eq. 3) on the mesh. */
void vpo_density_moment(const vpo_grid *g, const double *f, double *rho) {
    const long NX = vpo_nx_total(g), NV = vpo_nv_total(g);
    double dV = 1.0;
    for (int d = 0; d < g->dv; ++d) dV *= dvd(g, d);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < NX; ++x) {
        double s = 0.0;
        for (long v = 0; v < NV; ++v) s += f[x * NV + v];
        rho[x] = s * dV;
    }
}

/* ------------------------------------------------------------------------ */
/* plain discrete Fourier transform (Eq. C4 convention: no 1/N forward)     */
/* ------------------------------------------------------------------------ */
void vpo_dft_lines(long n, long nlines, const long *line_base, long stride, double *re,
                   double *im, int sign) {
    double *cr = (double *)malloc(sizeof(double) * n);
    double *ci = (double *)malloc(sizeof(double) * n);
    double *tr = (double *)malloc(sizeof(double) * n);
    double *ti = (double *)malloc(sizeof(double) * n);
    for (long k = 0; k < n; ++k) {
        cr[k] = cos(2.0 * M_PI * (double)k / (double)n);
        ci[k] = sin(2.0 * M_PI * (double)k / (double)n);
    }
    for (long l = 0; l < nlines; ++l) {
        const long b = line_base[l];
        for (long k = 0; k < n; ++k) {
            double sr = 0.0, si = 0.0;
            for (long j = 0; j < n; ++j) {
                long m = (j * k) % n; /* exp(sign * 2 pi i j k / n) */
                double wr = cr[m], wi = sign * ci[m];
                double xr = re[b + j * stride], xi = im[b + j * stride];
                sr += xr * wr - xi * wi;
                si += xr * wi + xi * wr;
            }
            tr[k] = sr;
            ti[k] = si;
        }
        for (long k = 0; k < n; ++k) {
            re[b + k * stride] = tr[k];
            im[b + k * stride] = ti[k];
        }
    }
    free(cr);
    free(ci);
    free(tr);
    free(ti);
}

/* DFT along every axis of a row-major D-dimensional complex array */
static void dft_nd(int D, const long *n, double *re, double *im, int sign) {
    for (int a = 0; a < D; ++a) {
        long outer = 1, inner = 1;
        for (int k = 0; k < a; ++k) outer *= n[k];
        for (int k = a + 1; k < D; ++k) inner *= n[k];
        long nl = outer * inner;
        long *base = (long *)malloc(sizeof(long) * nl);
        for (long o = 0; o < outer; ++o)
            for (long c = 0; c < inner; ++c) base[o * inner + c] = o * n[a] * inner + c;
        vpo_dft_lines(n[a], nl, base, inner, re, im, sign);
        free(base);
    }
}

/* ------------------------------------------------------------------------ */
/* Poisson solver, Sec. 2.2 and Appendix C                                   */
/* ------------------------------------------------------------------------ */
/*
 * Eigenvalue, times Delta^2, of the 2nd/4th/6th-order discrete Laplacian
 * (Eqs. C1, C5, C6) for the discrete wavenumber theta = k Delta.  These are
 * the denominators of the Green functions (Eqs. 51-53 / C3, C7, C8):
 * G(k) = 4 pi G Delta^2 / mu(theta), summed over axes.
 */
static double lap_eig(int order, double theta) {
    double s1 = sin(theta / 2.0), s2 = sin(theta), s3 = sin(1.5 * theta);
    if (order == 2) return -4.0 * s1 * s1;
    if (order == 4) return (s2 * s2 - 16.0 * s1 * s1) / 3.0;
    return -(2.0 * s3 * s3 - 27.0 * s2 * s2 + 270.0 * s1 * s1) / 45.0;
}

/*
 * d phi / dx at point i by the 2-, 4- or 6-point FDA (Eqs. C9-C11).
 * R8: Eq. (C10) as printed has the opposite overall sign to Eqs. (C9) and
 * (C11); the central difference consistent with those two is used.
 * `at(k)` returns phi k points from i.
 */
static double fda(int order, const double *p /* p[-3..3] */, double h) {
    if (order == 2) return (p[1] - p[-1]) / (2.0 * h);
    if (order == 4) return (-p[2] + 8.0 * p[1] - 8.0 * p[-1] + p[-2]) / (12.0 * h);
    return (p[3] - 9.0 * p[2] + 45.0 * p[1] - 45.0 * p[-1] + 9.0 * p[-2] - p[-3]) / (60.0 * h);
}

/* a = -grad phi on a periodic (or padded) grid of extent m[], sampled for
 * the box indices 0..nbox-1 along each axis. */
static void force_from_phi(const vpo_grid *g, const double *phi_grid, const long *m,
                           double *accel) {
    const int D = g->dx;
    const long NX = vpo_nx_total(g);
    for (int a = 0; a < D; ++a) {
        const double h = dxd(g, a);
        for (long x = 0; x < NX; ++x) {
            long idx[3] = {0, 0, 0}, r = x;
            for (int d = D - 1; d >= 0; --d) {
                idx[d] = r % g->nx[d];
                r /= g->nx[d];
            }
            double p[7];
            for (int k = -3; k <= 3; ++k) {
                long j[3] = {idx[0], idx[1], idx[2]};
                j[a] = ((idx[a] + k) % m[a] + m[a]) % m[a];
                long lin = 0;
                for (int d = 0; d < D; ++d) lin = lin * m[d] + j[d];
                p[k + 3] = phi_grid[lin];
            }
            accel[a * NX + x] = -fda(g->pois_order, &p[3], h);
        }
    }
}

/*
 * R7: lap(phi) = S (rho - rho_bg) with S = g->coupling (4 pi G for gravity,
 * Eq. 3; -1 with rho_bg = 1 for electrons, Eq. 74 in units e = m = omega_pe
 * = 1, where the acceleration is -d phi_s / dx, Eq. 73).  Periodic: the
 * k = 0 mode of phi is zero.  Isolated (3D only, cubic cells): the
 * doubling-up method of Sec. 2.2 with G(r) = -(S / 4 pi) dV / r (R9: the
 * attractive sign for S > 0, and the r = 0 entry is the mean of 1/r over one
 * cell, (3 ln(2 + sqrt 3) - pi / 2) / Delta); R10: the FDA stencil at the
 * box edge reads the padded-grid potential with cyclic indices.
 * phi: NX values; accel: dx * NX values, axis-major.
 */
int vpo_poisson_solve(const vpo_grid *g, const double *rho, double *phi, double *accel) {
    const int D = g->dx;
    const long NX = vpo_nx_total(g);
    const double S = g->coupling;
    if (g->pois_order != 2 && g->pois_order != 4 && g->pois_order != 6) return -1;
    if (g->poisson == VPO_POIS_PERIODIC) {
        long n[3] = {1, 1, 1};
        for (int d = 0; d < D; ++d) n[d] = g->nx[d];
        double *re = (double *)malloc(sizeof(double) * NX);
        double *im = (double *)calloc(NX, sizeof(double));
        for (long x = 0; x < NX; ++x) re[x] = rho[x] - g->rho_bg;
        dft_nd(D, n, re, im, -1);
        for (long x = 0; x < NX; ++x) {
            long r = x, allzero = 1;
            double lam = 0.0;
            for (int d = D - 1; d >= 0; --d) {
                long nk = r % n[d];
                r /= n[d];
                if (nk) allzero = 0;
                double h = dxd(g, d);
                lam += lap_eig(g->pois_order, 2.0 * M_PI * (double)nk / (double)n[d]) / (h * h);
            }
            if (allzero) {
                re[x] = 0.0;
                im[x] = 0.0;
            } else {
                re[x] = S * re[x] / lam;
                im[x] = S * im[x] / lam;
            }
        }
        dft_nd(D, n, re, im, +1);
        for (long x = 0; x < NX; ++x) phi[x] = re[x] / (double)NX;
        force_from_phi(g, phi, n, accel);
        free(re);
        free(im);
        return 0;
    }
    /* isolated */
    if (D != 3) return -1;
    const double h = dxd(g, 0);
    if (fabs(dxd(g, 1) - h) > 1e-12 * h || fabs(dxd(g, 2) - h) > 1e-12 * h) return -1;
    long m[3];
    for (int d = 0; d < 3; ++d) m[d] = 2L * g->nx[d];
    const long MT = m[0] * m[1] * m[2];
    double *gr = (double *)malloc(sizeof(double) * MT);
    double *gi = (double *)calloc(MT, sizeof(double));
    double *rr = (double *)calloc(MT, sizeof(double));
    double *ri = (double *)calloc(MT, sizeof(double));
    const double dV = h * h * h;
    const double self = (3.0 * log(2.0 + sqrt(3.0)) - M_PI / 2.0) / h;
    for (long a = 0; a < m[0]; ++a)
        for (long b = 0; b < m[1]; ++b)
            for (long c = 0; c < m[2]; ++c) {
                double ra = (double)(a < m[0] - a ? a : m[0] - a) * h;
                double rb = (double)(b < m[1] - b ? b : m[1] - b) * h;
                double rc = (double)(c < m[2] - c ? c : m[2] - c) * h;
                double r = sqrt(ra * ra + rb * rb + rc * rc);
                double inv_r = (a == 0 && b == 0 && c == 0) ? self : 1.0 / r;
                gr[(a * m[1] + b) * m[2] + c] = -(S / (4.0 * M_PI)) * dV * inv_r;
            }
    for (long a = 0; a < g->nx[0]; ++a)
        for (long b = 0; b < g->nx[1]; ++b)
            for (long c = 0; c < g->nx[2]; ++c)
                rr[(a * m[1] + b) * m[2] + c] =
                    rho[(a * g->nx[1] + b) * g->nx[2] + c] - g->rho_bg;
    dft_nd(3, m, gr, gi, -1);
    dft_nd(3, m, rr, ri, -1);
    for (long x = 0; x < MT; ++x) {
        double pr = gr[x] * rr[x] - gi[x] * ri[x];
        double pi = gr[x] * ri[x] + gi[x] * rr[x];
        rr[x] = pr;
        ri[x] = pi;
    }
    dft_nd(3, m, rr, ri, +1);
    for (long x = 0; x < MT; ++x) rr[x] /= (double)MT;
    for (long a = 0; a < g->nx[0]; ++a)
        for (long b = 0; b < g->nx[1]; ++b)
            for (long c = 0; c < g->nx[2]; ++c)
                phi[(a * g->nx[1] + b) * g->nx[2] + c] = rr[(a * m[1] + b) * m[2] + c];
    force_from_phi(g, rr, m, accel);
    free(gr);
    free(gi);
    free(rr);
    free(ri);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* diagnostics                                                              */
/* ------------------------------------------------------------------------ */
/*
 * out[0] mass  = sum f dX dV
 * out[1] ke    = 1/2 sum f |v|^2 dX dV
 * out[2] fe    = 1/2 sum_x |a|^2 dX          (electric energy for plasmas)
 * out[3] pe    = 1/2 sum_x (rho - rho_bg) phi dX   (potential energy)
 * out[4] min f, out[5] max f
 * out[6] mode_amp = (2 / NX) |sum_x a_1(x) exp(-2 pi i mode j_1 / n_1)|
 *                   (amplitude of Fourier mode `mode` of the field along x_1)
 * out[7] l1 = sum |f| dX dV, out[8] l2 = sum f^2 dX dV
 */
void vpo_diagnostics(const vpo_grid *g, const double *f, const double *rho, const double *phi,
                     const double *accel, int mode, double *out) {
    const long NX = vpo_nx_total(g), NV = vpo_nv_total(g);
    double dX = 1.0, dV = 1.0;
    for (int d = 0; d < g->dx; ++d) dX *= dxd(g, d);
    for (int d = 0; d < g->dv; ++d) dV *= dvd(g, d);
    double mass = 0.0, ke = 0.0, l1 = 0.0, l2 = 0.0, fmn = INFINITY, fmx = -INFINITY;
    for (long x = 0; x < NX; ++x)
        for (long v = 0; v < NV; ++v) {
            double val = f[x * NV + v];
            long r = v;
            double v2 = 0.0;
            for (int d = g->dv - 1; d >= 0; --d) {
                double vv = vc(g, d, r % g->nv[d]);
                r /= g->nv[d];
                v2 += vv * vv;
            }
            mass += val;
            ke += 0.5 * val * v2;
            l1 += fabs(val);
            l2 += val * val;
            if (val < fmn) fmn = val;
            if (val > fmx) fmx = val;
        }
    double fe = 0.0, pe = 0.0, cr = 0.0, ci = 0.0;
    for (long x = 0; x < NX; ++x) {
        for (int d = 0; d < g->dx; ++d) fe += 0.5 * accel[d * NX + x] * accel[d * NX + x];
        pe += 0.5 * (rho[x] - g->rho_bg) * phi[x];
        long j1 = x;
        for (int d = g->dx - 1; d >= 1; --d) j1 /= g->nx[d];
        double ang = -2.0 * M_PI * (double)((mode * j1) % g->nx[0]) / (double)g->nx[0];
        cr += accel[x] * cos(ang);
        ci += accel[x] * sin(ang);
    }
    out[0] = mass * dX * dV;
    out[1] = ke * dX * dV;
    out[2] = fe * dX;
    out[3] = pe * dX;
    out[4] = fmn;
    out[5] = fmx;
    out[6] = 2.0 / (double)NX * sqrt(cr * cr + ci * ci);
    out[7] = l1 * dX * dV;
    out[8] = l2 * dX * dV;
}

/* ------------------------------------------------------------------------ */
/* Strang-split step, Sec. 2.4 Eq. (55)                                      */
/* ------------------------------------------------------------------------ */
/*
 * R11: KDK follows Eq. (55): T_v(dt/2) [v_1, v_2, v_3 in that order], then
 * T_x(dt) [x_3, x_2, x_1], then rho and the Poisson solve, then T_v(dt/2).
 * DKD: T_x(dt/2), rho + Poisson, T_v(dt), T_x(dt/2) with the same axis
 * orders.  The field solved after the drifts serves the following kicks,
 * including KDK's first half kick of the next step.  accel (dx * NX) holds
 * on entry the field for KDK's first half kick and on exit the last field
 * solved.  diag (optional, nsteps * VPO_NDIAG) gets the diagnostics of the
 * f reached after each step, with its own density and field computed in
 * separate buffers (so asking for diagnostics never changes the run).
 */
int vpo_step(const vpo_grid *g, double *f, double dt, int split, int nsteps, double *accel,
             int mode, double *diag) {
    if (!grid_ok(g)) return -1;
    const long NX = vpo_nx_total(g);
    double *rho = (double *)malloc(sizeof(double) * NX);
    double *phi = (double *)malloc(sizeof(double) * NX);
    double *acc_d = (double *)malloc(sizeof(double) * NX * g->dx);
    for (int n = 0; n < nsteps; ++n) {
        if (split == VPO_SPLIT_KDK) {
            for (int d = 0; d < g->dv; ++d) vpo_kick_sweep(g, f, d, 0.5 * dt, accel + d * NX);
            for (int d = g->dx - 1; d >= 0; --d) vpo_drift_sweep(g, f, d, dt);
            vpo_density_moment(g, f, rho);
            vpo_poisson_solve(g, rho, phi, accel);
            for (int d = 0; d < g->dv; ++d) vpo_kick_sweep(g, f, d, 0.5 * dt, accel + d * NX);
        } else {
            for (int d = g->dx - 1; d >= 0; --d) vpo_drift_sweep(g, f, d, 0.5 * dt);
            vpo_density_moment(g, f, rho);
            vpo_poisson_solve(g, rho, phi, accel);
            for (int d = 0; d < g->dv; ++d) vpo_kick_sweep(g, f, d, dt, accel + d * NX);
            for (int d = g->dx - 1; d >= 0; --d) vpo_drift_sweep(g, f, d, 0.5 * dt);
        }
        if (diag) {
            vpo_density_moment(g, f, rho);
            vpo_poisson_solve(g, rho, phi, acc_d);
            vpo_diagnostics(g, f, rho, phi, acc_d, mode, diag + (long)n * VPO_NDIAG);
        }
    }
    free(rho);
    free(phi);
    free(acc_d);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* initial conditions (point values at cell centres, R1)                    */
/* ------------------------------------------------------------------------ */
/*
 * VPO_IC_LANDAU   params {alpha, k1, k2, k3, sigma, amp}:
 *     amp (1 + alpha sum_d cos(k_d x_d)) prod_d exp(-v_d^2 / 2 sigma^2) / sqrt(2 pi sigma^2)
 *     (Eq. 75 for electrons, Eq. 69 for the self-gravitating slab)
 * VPO_IC_TWOSTREAM params {alpha, k}:
 *     v_1^2 exp(-|v|^2 / 2) / (2 pi)^{D/2} (1 + alpha cos(k x_1))
 * VPO_IC_PLUMMER  params {G, M, a}: isotropic Plummer distribution
 *     F(E) = 24 sqrt(2) / (7 pi^3) a^2 / (G^5 M^4) (-E)^{7/2}, E < 0,
 *     E = |v|^2 / 2 - G M / sqrt(r^2 + a^2), r from the box centre
 * VPO_IC_SPHERE   params {G, M, R}: Sec. 3.4 (Eq. 77): a sphere of mass M and
 *     radius 2R about the box centre of uniform density rho0 = M / (4 pi (2R)^3 / 3),
 *     rho0 (2 pi sigma^2)^{-3/2} exp(-|v|^2 / 2 sigma^2), sigma^2 = G M / (20 R),
 *     inside (r < 2R), zero outside
 * VPO_IC_ADVECT   params {shape}: Test-1 profiles in x on [0, 1)^D,
 *     0: rectangle (Eqs. 60, 65), 1: 1 + (1/D) sum sin(2 pi x_d) (Eqs. 62, 66),
 *     2: sum sin^4(4 pi x_d) (Eqs. 63, 67); constant in v.
 */
int vpo_init_f(const vpo_grid *g, int kind, const double *p, int np, double *f) {
    if (!grid_ok(g)) return -1;
    const long NX = vpo_nx_total(g), NV = vpo_nv_total(g);
    const int D = g->dx;
    for (long x = 0; x < NX; ++x) {
        double xs[3] = {0, 0, 0};
        long r = x;
        for (int d = D - 1; d >= 0; --d) {
            xs[d] = xc(g, d, r % g->nx[d]);
            r /= g->nx[d];
        }
        for (long v = 0; v < NV; ++v) {
            double vs[3] = {0, 0, 0};
            long q = v;
            for (int d = D - 1; d >= 0; --d) {
                vs[d] = vc(g, d, q % g->nv[d]);
                q /= g->nv[d];
            }
            double val = 0.0;
            if (kind == VPO_IC_LANDAU) {
                if (np < 6) return -1;
                double alpha = p[0], sig = p[4], amp = p[5];
                double sp = 1.0, mv = 1.0;
                for (int d = 0; d < D; ++d) {
                    sp += alpha * cos(p[1 + d] * xs[d]);
                    mv *= exp(-vs[d] * vs[d] / (2.0 * sig * sig)) / sqrt(2.0 * M_PI * sig * sig);
                }
                val = amp * sp * mv;
            } else if (kind == VPO_IC_TWOSTREAM) {
                if (np < 2) return -1;
                double v2 = 0.0;
                for (int d = 0; d < D; ++d) v2 += vs[d] * vs[d];
                val = vs[0] * vs[0] * exp(-v2 / 2.0) / pow(2.0 * M_PI, 0.5 * D) *
                      (1.0 + p[0] * cos(p[1] * xs[0]));
            } else if (kind == VPO_IC_PLUMMER) {
                if (np < 3 || D != 3) return -1;
                double G = p[0], M = p[1], a = p[2], r2 = 0.0, v2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double c = 0.5 * (g->xlo[d] + g->xhi[d]);
                    r2 += (xs[d] - c) * (xs[d] - c);
                    v2 += vs[d] * vs[d];
                }
                double E = 0.5 * v2 - G * M / sqrt(r2 + a * a);
                val = E < 0.0 ? 24.0 * sqrt(2.0) / (7.0 * M_PI * M_PI * M_PI) * a * a /
                                    (pow(G, 5.0) * pow(M, 4.0)) * pow(-E, 3.5)
                              : 0.0;
            } else if (kind == VPO_IC_SPHERE) {
                if (np < 3 || D != 3) return -1;
                double G = p[0], M = p[1], R = p[2], r2 = 0.0, v2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double c = 0.5 * (g->xlo[d] + g->xhi[d]);
                    r2 += (xs[d] - c) * (xs[d] - c);
                    v2 += vs[d] * vs[d];
                }
                double rho0 = M / (4.0 * M_PI * pow(2.0 * R, 3.0) / 3.0);
                double s2 = G * M / (20.0 * R);
                val = r2 < (2.0 * R) * (2.0 * R) ? rho0 * exp(-v2 / (2.0 * s2)) / pow(2.0 * M_PI * s2, 1.5) : 0.0;
            } else if (kind == VPO_IC_ADVECT) {
                if (np < 1) return -1;
                int shape = (int)p[0];
                if (shape == 0) {
                    val = 1.0;
                    for (int d = 0; d < D; ++d)
                        if (!(xs[d] >= 0.25 && xs[d] <= 0.75)) val = 0.0;
                } else if (shape == 1) {
                    val = 1.0;
                    for (int d = 0; d < D; ++d) val += sin(2.0 * M_PI * xs[d]) / D;
                } else {
                    for (int d = 0; d < D; ++d) {
                        double sn = sin(4.0 * M_PI * xs[d]);
                        val += sn * sn * sn * sn;
                    }
                }
            } else {
                return -1;
            }
            f[x * NV + v] = val;
        }
    }
    return 0;
}

/* CFL time step, Eqs. (56)-(58) */
double vpo_cfl_dt(const vpo_grid *g, double nu, const double *accel) {
    double dtp = INFINITY, dtv = INFINITY;
    const long NX = vpo_nx_total(g);
    for (int d = 0; d < g->dx; ++d) {
        double vmax = fabs(g->vlo[d]) > fabs(g->vhi[d]) ? fabs(g->vlo[d]) : fabs(g->vhi[d]);
        if (vmax > 0.0) {
            double t = nu * dxd(g, d) / vmax;
            if (t < dtp) dtp = t;
        }
    }
    if (accel)
        for (int d = 0; d < g->dv; ++d)
            for (long x = 0; x < NX; ++x) {
                double a = fabs(accel[d * NX + x]);
                if (a > 0.0) {
                    double t = nu * dvd(g, d) / a;
                    if (t < dtv) dtv = t;
                }
            }
    return dtp < dtv ? dtp : dtv;
}
