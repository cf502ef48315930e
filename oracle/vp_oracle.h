/*
 * vp_oracle.h -- plain FP64 CPU oracle for the SL-MPP5/7 Vlasov-Poisson
 * method of Tanaka, Yoshikawa, Minoshima & Yoshida (2017).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load this library.  It shares
 * no source, header, table or constant with the CUDA library and is never on
 * the product path.
 *
 * Every function restates one step of the paper in its own order and
 * notation, in double precision, with plain loops:
 *   - CSL5/CSL7 flux            : Sec. 2.1.2, Eqs. (29)-(43)
 *   - MP constraint             : Appendix A, steps 1-7 (applied as Eqs. (44)-(45))
 *   - PP flux limiter           : Sec. 2.1.1, Eqs. (15)-(23) (applied as Eqs. (47)-(48))
 *   - SL-MPP update             : Eq. (49)
 *   - directional splitting     : Sec. 2, Eqs. (4)-(5); Sec. 2.4, Eq. (55)
 *   - Poisson solver, FDA force : Sec. 2.2, Eqs. (50)-(54); Appendix C
 *   - CFL time step             : Sec. 2.4, Eqs. (56)-(58)
 * Layout of f: row-major [x_1..x_D][v_1..v_D], velocity innermost (Sec. 2.3:
 * each spatial point holds its whole velocity grid).
 */
#ifndef VP_ORACLE_H
#define VP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define VPO_BC_PERIODIC 0
#define VPO_BC_OUTFLOW 1 /* zero ghost cells: nothing flows in */

#define VPO_POIS_PERIODIC 0
#define VPO_POIS_ISOLATED 1

#define VPO_SPLIT_KDK 0
#define VPO_SPLIT_DKD 1

#define VPO_IC_LANDAU 0
#define VPO_IC_TWOSTREAM 1
#define VPO_IC_PLUMMER 2
#define VPO_IC_ADVECT 3
#define VPO_IC_SPHERE 4

#define VPO_NDIAG 9 /* mass, ke, fe, pe, min_f, max_f, mode_amp, l1, l2 */

typedef struct {
    int dx, dv;                       /* spatial / velocity dimensions, dx == dv in 1..3 */
    int nx[3], nv[3];                 /* cells per axis */
    double xlo[3], xhi[3];            /* spatial box */
    double vlo[3], vhi[3];            /* velocity box */
    int xbc;                          /* VPO_BC_PERIODIC or VPO_BC_OUTFLOW */
    int order;                        /* 5 (CSL5) or 7 (CSL7) */
    int mp;                           /* 1: MP constraint on, 0: plain CSL */
    int pp;                           /* 1: PP limiter on */
    double alpha;                     /* MP parameter, 4 in the paper */
    int poisson;                      /* VPO_POIS_PERIODIC or VPO_POIS_ISOLATED */
    int pois_order;                   /* 2, 4 or 6 */
    double coupling;                  /* S in lap(phi) = S (rho - rho_bg); 4 pi G for gravity, -1 for electrons */
    double rho_bg;                    /* neutralising background */
} vpo_grid;

/* ---- one interface ------------------------------------------------------
 * u points at the upwind cell of the interface (u[0]); u[-3..3] must be
 * readable.  The interface lies between u[0] and u[1]; the flow goes from
 * u[0] towards u[1]; nu in [0, 1] is the fractional CFL number. */
double vpo_csl_flux(int order, double nu, const double *u);
double vpo_mp_constraint(double phi, const double *u, double alpha);
/* f^min, f^max of Appendix A steps 4-6 (the bounds step 7 applies) */
void vpo_mp_bounds(const double *u, double alpha, double *fmin_out, double *fmax_out);
double vpo_pp_limiter(double phibar, double u0, double u1, double nu);
double vpo_interface_flux(int order, int mp, int pp, double alpha, double nu, const double *u);

/* ---- shift decomposition and one line ----------------------------------- */
void vpo_shift_split(double s, long *n_int, double *zeta);
/* Advance one line of L cells (element stride `stride`) by a shift of s cells. */
void vpo_advect_line(int order, int mp, int pp, double alpha, int bc, long L,
                     double *line, long stride, double s);

/* ---- sweeps, moments, Poisson, diagnostics, step ------------------------ */
long vpo_nx_total(const vpo_grid *g);
long vpo_nv_total(const vpo_grid *g);
int vpo_rk_mpp5_line(int mp, int pp, double alpha, int bc, long L, double *line, long stride, double cnu);
int vpo_drift_sweep_rk(const vpo_grid *g, double *f, int dim, double dt);
int vpo_kick_sweep_rk(const vpo_grid *g, double *f, int dim, double dt, const double *accel_dim);
int vpo_drift_sweep(const vpo_grid *g, double *f, int dim, double dt);
int vpo_kick_sweep(const vpo_grid *g, double *f, int dim, double dt, const double *accel_dim);
int vpo_drift_unsplit(const vpo_grid *g, double *f, double dt);
void vpo_density_moment(const vpo_grid *g, const double *f, double *rho);
int vpo_poisson_solve(const vpo_grid *g, const double *rho, double *phi, double *accel);
void vpo_diagnostics(const vpo_grid *g, const double *f, const double *rho, const double *phi,
                     const double *accel, int mode, double *out);
int vpo_step(const vpo_grid *g, double *f, double dt, int split, int nsteps, double *accel,
             int mode, double *diag);
int vpo_init_f(const vpo_grid *g, int kind, const double *params, int nparams, double *f);
double vpo_cfl_dt(const vpo_grid *g, double nu, const double *accel);

/* plain O(n^2) discrete Fourier transform along one axis of a strided batch */
void vpo_dft_lines(long n, long nlines, const long *line_base, long stride, double *re,
                   double *im, int sign);

void vpo_set_threads(int n);
int vpo_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
