/*
 * vlasov.h -- C ABI of the GB300 (sm_103a) SL-MPP5/7 Vlasov-Poisson library.
 *
 * The method is that of Tanaka, Yoshikawa, Minoshima & Yoshida (2017),
 * "Multidimensional Vlasov-Poisson simulations with high-order monotonicity-
 * and positivity-preserving schemes": a Strang-split sequence of 1D
 * semi-Lagrangian advections of the phase-space distribution f, each one a
 * conservative flux update (Sec. 2.1.2) whose fluxes pass through the MP
 * constraint (Appendix A) and the positivity-preserving flux limiter
 * (Sec. 2.1.1), with the acceleration from an FFT Poisson solve (Sec. 2.2).
 *
 * Conventions shared by every call:
 *   - Return value: VP_OK (0) or a negative VP_E* code; vp_last_error()
 *     returns a one-line description of the last failure on that context.
 *   - Asynchrony: work is enqueued on the CUDA stream given to vp_create and
 *     returns without waiting, except where a call says it synchronises.
 *   - Memory: the distribution function f and every array passed as a
 *     "_dev" pointer are device memory owned by the caller (the library never
 *     frees them).  The library owns only small internal tables and FFT
 *     buffers (allocated at vp_create, freed at vp_destroy).
 *   - Layout of f: row-major [x_1 .. x_D][v_1 .. v_D], velocity innermost,
 *     i.e. every spatial cell holds its whole velocity grid contiguously
 *     (Sec. 2.3).  Element type float (VP_F32) or double (VP_F64).
 *   - Spatial arrays (rho, phi, one acceleration component): NX = prod nx
 *     doubles, row-major [x_1 .. x_D].  An acceleration field is D such
 *     arrays back to back (axis-major, D * NX doubles).
 *   - Cells are uniform; cell i of an axis covers [lo + i h, lo + (i+1) h].
 */
#ifndef VLASOV_H
#define VLASOV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define VP_OK 0
#define VP_EINVAL (-1)      /* bad argument (message in vp_last_error) */
#define VP_ECUDA (-2)       /* a CUDA call failed */
#define VP_ENOMEM (-3)      /* a library-internal allocation failed */
#define VP_ETIMEOUT (-4)    /* a bounded device-side wait gave up */
#define VP_ENONFINITE (-5)  /* diagnostics found NaN or Inf in f */
#define VP_ENOTSUP (-6)     /* configuration not supported */
#define VP_ECFL (-7)        /* a sweep's CFL number is outside the scheme's range (RK-MPP5: |nu| < 1/2) */

/* ---- enumerations ------------------------------------------------------ */
#define VP_F32 0
#define VP_F64 1
#define VP_BC_PERIODIC 0
#define VP_BC_OUTFLOW 1 /* zero ghost cells: nothing flows in */
#define VP_POIS_PERIODIC 0
#define VP_POIS_ISOLATED 1
#define VP_SPLIT_KDK 0
#define VP_SPLIT_DKD 1
#define VP_SCHEME_SL 0
#define VP_SCHEME_RK 1
#define VP_IC_LANDAU 0
#define VP_IC_TWOSTREAM 1
#define VP_IC_PLUMMER 2
#define VP_IC_ADVECT 3
#define VP_IC_SPHERE 4
#define VP_NDIAG 9

/* ---- grid and scheme --------------------------------------------------- */
typedef struct {
    int dx, dv;            /* spatial / velocity dimensions; dx == dv in 1..3 */
    int nx[3], nv[3];      /* cells per axis (entries beyond dx/dv ignored) */
    double xlo[3], xhi[3]; /* spatial box per axis */
    double vlo[3], vhi[3]; /* velocity box per axis */
    int xbc;               /* VP_BC_PERIODIC or VP_BC_OUTFLOW (spatial axes);
                              velocity axes are always zero-inflow */
    int order;             /* 5: CSL5 flux (Eqs. 29-34); 7: CSL7 (Eqs. 36-43) */
    int mp;                /* 1: MP constraint (Appendix A) on, 0: off */
    int pp;                /* 1: PP flux limiter (Eqs. 15-23) on, 0: off */
    double alpha;          /* MP parameter (4 in the paper) */
    int precision;         /* VP_F32 or VP_F64: storage and arithmetic of f */
    int poisson;           /* VP_POIS_PERIODIC or VP_POIS_ISOLATED (3D, cubic cells) */
    int pois_order;        /* 2, 4 or 6: Green function and FDA order (App. C) */
    double coupling;       /* S in lap(phi) = S (rho - rho_bg): 4 pi G for
                              gravity (Eq. 3), -1 for electrons (Eq. 74) */
    double rho_bg;         /* neutralising background density */
    int scheme;            /* VP_SCHEME_SL: semi-Lagrangian SL-MPP (Eq. 49, any CFL);
                              VP_SCHEME_RK: RK-MPP5 (Eqs. 8-10, order 5, |nu| < 1/2) */
} vp_grid;

/* diagnostics of one state, all double precision */
typedef struct {
    double mass;     /* sum f dX dV */
    double ke;       /* 1/2 sum f |v|^2 dX dV */
    double fe;       /* 1/2 sum_x |a|^2 dX  (field energy) */
    double pe;       /* 1/2 sum_x (rho - rho_bg) phi dX  (potential energy) */
    double min_f;    /* minimum of f */
    double max_f;    /* maximum of f */
    double mode_amp; /* (2/NX) |sum_x a_1(x) exp(-2 pi i m j_1 / n_1)|, m = `mode` */
    double l1;       /* sum |f| dX dV */
    double l2;       /* sum f^2 dX dV */
} vp_diag;

typedef struct vp_ctx vp_ctx; /* opaque: grid, stream, tables, FFT plans */

/*
 * vp_create -- validate the grid (Sec. 2: uniform Cartesian phase-space
 * mesh) and build a context bound to `cuda_stream` (a cudaStream_t; NULL
 * for the legacy default stream) on the current device.  Precomputes the
 * CSL weight polynomials, the Green function of the Poisson solver (Eqs.
 * 50-54) and allocates the library's small FFT/scratch buffers.
 * *out receives the context; on failure *out is NULL.
 */
int vp_create(const vp_grid *grid, void *cuda_stream, vp_ctx **out);

/* Free the context and its internal buffers (not f).  NULL is accepted. */
void vp_destroy(vp_ctx *ctx);

/* Message of the last failure on ctx ("" if none).  Never NULL. */
const char *vp_last_error(const vp_ctx *ctx);

/* Number of cells of f (NX * NV) and bytes per element (4 or 8). */
long long vp_num_cells(const vp_ctx *ctx);
int vp_elem_size(const vp_ctx *ctx);

/*
 * vp_bind_f -- attach the caller-owned device array holding f
 * (vp_num_cells elements of the grid's precision, 16-byte aligned).  All
 * later calls read and write it in place.
 */
int vp_bind_f(vp_ctx *ctx, void *f_dev);

/*
 * vp_init_f -- fill f with an analytic initial condition sampled at cell
 * centres (point values):
 *   VP_IC_LANDAU    params {alpha, k1, k2, k3, sigma, amp}:
 *                   amp (1 + alpha sum_d cos k_d x_d) prod_d N(v_d; 0, sigma^2)
 *                   (Eq. 75; Eq. 69 for the gravitating slab)
 *   VP_IC_TWOSTREAM params {alpha, k}: v_1^2 exp(-|v|^2/2)/(2 pi)^{D/2} (1 + alpha cos k x_1)
 *   VP_IC_PLUMMER   params {G, M, a}: isotropic Plummer distribution function
 *   VP_IC_ADVECT    params {shape}: Test-1 profiles in x (Eqs. 60, 62, 63, 65-67)
 *   VP_IC_SPHERE    params {G, M, R}: uniform sphere of mass M and radius 2R about
 *                   the box centre, Maxwellian with sigma^2 = G M / (20 R) (Eq. 77)
 */
int vp_init_f(vp_ctx *ctx, int kind, const double *params, int nparams);

/* Host <-> device copies of f on the context stream (host memory should be
 * pinned for asynchrony); `bytes` must equal vp_num_cells * vp_elem_size. */
int vp_upload_f(vp_ctx *ctx, const void *host, size_t bytes);
int vp_download_f(vp_ctx *ctx, void *host, size_t bytes);

/*
 * vp_host_alloc -- page-locked host memory for the copies above, backed by
 * transparent huge pages where the kernel provides them: an anonymous
 * mapping aligned to the huge-page size, advised for huge pages and
 * registered with the CUDA driver (cudaHostRegister).  Copies from and to
 * it need one address translation per huge page instead of one per base
 * page; with f of tens of GB and the sweeps touching all of device memory
 * between copies, a cudaHostAlloc buffer of base pages was seen to copy at
 * half the rate.  The paper has no counterpart (its runs stay on the
 * machine).  *out receives the pointer (host-readable and writable, zero
 * filled); VP_EINVAL for bytes == 0 or out == NULL, VP_ENOMEM if the mapping
 * fails, VP_ECUDA if registration fails (nothing is left allocated).
 * vp_host_free unregisters and unmaps a pointer vp_host_alloc returned
 * (VP_EINVAL for any other pointer).  Both synchronise with the device.
 */
int vp_host_alloc(size_t bytes, void **out);
int vp_host_free(void *p);

/*
 * vp_drift_sweep -- advance f by the 1D advection along spatial axis `dim`
 * (0-based) at speed v_dim for a time dt (Eq. 4): every line along x_dim is
 * shifted by s = v dt / dx_dim cells, split as s = N + zeta with N the
 * nearest integer (an exact copy) and |zeta| <= 1/2 the CFL number of one
 * SL-MPP update (Eq. 49).  In place.
 */
int vp_drift_sweep(vp_ctx *ctx, int dim, double dt);

/*
 * vp_kick_sweep -- same along velocity axis `dim` with the acceleration
 * accel_dev[x] (NX doubles, device) of each spatial cell (Eq. 5), shift
 * s = a dt / dv_dim; zero inflow at the velocity boundaries.  In place.
 */
int vp_kick_sweep(vp_ctx *ctx, int dim, double dt, const double *accel_dev);

/*
 * vp_drift_unsplit -- nsteps unsplit steps of the advection in physical space
 * (the alternative to directional splitting of Sec. 2.4, compared in Test-1d
 * of Sec. 3.1): every step forms both directions' SL-MPP increments from the
 * same f^n,
 *     f^{n+1} = f^n + (A_1 f^n - f^n) + (A_2 f^n - f^n),
 * A_d the line update of vp_drift_sweep(d, dt) (Eq. 49 with the grid's MP
 * constraint and PP limiter).  Mass is conserved on a periodic box;
 * positivity is not guaranteed (each direction's PP limiter bounds what a
 * face takes, not what four faces take together), which is why the paper runs
 * it at CFL numbers below 0.1.
 * scratch_dev: caller-owned device array of vp_num_cells elements of the
 * grid's precision, 16-byte aligned, not overlapping f; the steps alternate
 * between f and scratch_dev and the result ends in f (an odd nsteps adds one
 * device copy).  scratch_dev's contents afterwards are unspecified.
 * VP_ENOTSUP unless the grid has two spatial dimensions and the SL scheme, or
 * if a line moves by more than 4 whole cells per step; VP_EINVAL for a NULL,
 * misaligned or overlapping scratch_dev, nsteps < 0 or a non-finite dt.
 */
int vp_drift_unsplit(vp_ctx *ctx, double dt, int nsteps, void *scratch_dev);

/* rho_dev[x] = sum_v f dV (Eq. 3 on the mesh), NX doubles, computed from the
 * float/double f with double-precision accumulation. */
int vp_density_moment(vp_ctx *ctx, double *rho_dev);

/*
 * vp_poisson_solve -- lap(phi) = S (rho - rho_bg) by FFT convolution
 * (Sec. 2.2): periodic with the 2nd/4th/6th-order Green function (Eqs.
 * 51-53, k = 0 mode zero) or isolated by doubling-up with G(r) = -(S/4pi)
 * dV / r (Eq. 54); then accel = -grad phi by the 2/4/6-point FDA (Eqs.
 * C9-C11).  rho_dev: NX doubles in; phi_dev: NX doubles out (may be NULL);
 * accel_dev: dx * NX doubles out.
 */
int vp_poisson_solve(vp_ctx *ctx, const double *rho_dev, double *phi_dev, double *accel_dev);

/*
 * vp_diagnostics -- compute the density, field and the vp_diag quantities of
 * the current f (mode index `mode` for mode_amp) and copy them to *out.
 * Synchronises the stream.  Returns VP_ENONFINITE if f holds NaN or Inf.
 */
int vp_diagnostics(vp_ctx *ctx, int mode, vp_diag *out);

/*
 * vp_step -- nsteps Strang-split steps (Sec. 2.4, Eq. 55).  KDK: kicks
 * v_1..v_D by dt/2 with accel, drifts x_D..x_1 by dt, density + Poisson ->
 * accel, kicks by dt/2.  DKD: drifts by dt/2, density + Poisson -> accel,
 * kicks by dt, drifts by dt/2.  accel_dev (dx * NX doubles, device) holds on
 * entry the field used by KDK's first half kick and on exit the last field
 * solved.  If diag_dev is not NULL it receives nsteps * VP_NDIAG doubles
 * (vp_diag order) describing f after each step.  Captured once into a CUDA
 * graph per (dt, split, diag) and replayed.
 */
int vp_step(vp_ctx *ctx, double dt, int split, int nsteps, double *accel_dev, int mode,
            double *diag_dev);

/* Kernel launches the library issued on this context since creation. */
long long vp_launch_count(const vp_ctx *ctx);

/*
 * vp_sync -- wait for the context stream and check the device status word
 * that bounded device-side waits (TMA completion barriers) write when they
 * give up.  Returns VP_ETIMEOUT (and clears the word) if one did.
 */
int vp_sync(vp_ctx *ctx);

/*
 * vp_set_option -- implementation choices (no effect on results):
 *   VP_OPT_SWEEP_IMPL: 0 automatic, 1 staged-load kernels only, 2 prefer the
 *                      TMA-pipelined strided-axis kernel, 3 prefer the
 *                      staged-load strided kernel that walks two lines per
 *                      thread with packed FP32 pair arithmetic (FP32 grids;
 *                      the same bits as 1);
 *   VP_OPT_AUTOTUNE:   1 (default) times candidate tile shapes of each sweep
 *                      geometry on its first use, with that sweep's shifts,
 *                      on a copy of a window of f (at most 256 MB of whole
 *                      lines, centred on the box's central spatial cell so
 *                      that it holds the populated part of phase space;
 *                      allocated for the tuning and freed; f is left
 *                      unchanged; without room for it the defaults stay),
 *                      and of the unsplit
 *                      step (f -> scratch_dev), and keeps the fastest; 0 uses
 *                      fixed defaults;
 *   VP_OPT_WAIT_LIMIT: iterations of each bounded device-side wait in the
 *                      sweeps (the TMA kernel's tile barriers; default 2^26,
 *                      seconds).  A wait that runs out makes the kernel drain
 *                      its own copies, return, and vp_sync report
 *                      VP_ETIMEOUT; 0 makes every such wait give up at once
 *                      (a test of that path).
 * Changing an option forgets tuned shapes and the captured step graph.
 */
#define VP_OPT_SWEEP_IMPL 1
#define VP_OPT_AUTOTUNE 2
#define VP_OPT_WAIT_LIMIT 3
int vp_set_option(vp_ctx *ctx, int option, long long value);

/* Tile shape in use for sweep (kick, dim): out4 = {impl, W or R, segments,
 * CTAs per SM (0 = occupancy maximum)}; impl 0 means not tuned yet. */
int vp_get_tuning(const vp_ctx *ctx, int kick, int dim, int *out4);

/* ---- batched ensembles ---------------------------------------------------
 * Many independent 1D1V / 2D2V runs of uneven size (FP32, MP5 or MP7 with
 * MP and PP, periodic space, zero-inflow velocity, periodic Poisson) advanced
 * together: one KDK step (Eq. 55) of every run is one persistent kernel
 * launch working through a queue of (run, stage, tile) items with per-run
 * stage counters (bounded waits), captured once in a CUDA graph.  All runs'
 * f live in one caller-owned FP32 pool (run r at its f_offset, layout as for
 * a single run); the library owns the per-run fields and the work plan.
 */
typedef struct {
    int dims;               /* 1 or 2 (dv == dx) */
    int nx[2], nv[2];       /* spatial axes: powers of two <= 256, NX <= 4096; nv <= 4096 */
    double xlo[2], xhi[2], vlo[2], vhi[2];
    double coupling, rho_bg;/* as in vp_grid */
    int pois_order;         /* 2, 4 or 6 */
} vp_run_desc;

typedef struct vp_ens vp_ens;

int vp_ensemble_create(const vp_run_desc *runs, int nruns, int order, void *cuda_stream, vp_ens **out);
void vp_ensemble_destroy(vp_ens *ens);
const char *vp_ensemble_last_error(const vp_ens *ens);
/* cells of the pool (sum of the runs' cells, each run padded to 32 floats) */
long long vp_ensemble_num_cells(const vp_ens *ens);
/* element offset of run `run` in the pool and of its field in the field array */
int vp_ensemble_run_layout(const vp_ens *ens, int run, long long *f_offset, long long *acc_offset);
/* attach the caller's FP32 pool (vp_ensemble_num_cells floats, 128-byte aligned) */
int vp_ensemble_bind(vp_ens *ens, float *pool_dev);
/* analytic initial condition of one run (VP_IC_LANDAU or VP_IC_TWOSTREAM, as vp_init_f) */
int vp_ensemble_init_run(vp_ens *ens, int run, int kind, const double *params, int nparams);
/* density + Poisson of every run from the current f (needed once before the first step); synchronises */
int vp_ensemble_field(vp_ens *ens);
/* device pointer to the field array (sum over runs of dims * NX doubles) */
int vp_ensemble_accel(const vp_ens *ens, const double **accel_dev);
/* tile shapes: W columns per strided tile, R lines per contiguous tile (both
 * dividing 256), CTAs per SM of the persistent grid (0 = occupancy maximum) */
int vp_ensemble_set_tiles(vp_ens *ens, int W, int R, int ctas_per_sm);
int vp_ensemble_get_tiles(const vp_ens *ens, int *out3);
/* Whether the line walkers of the ensemble vote, warp by warp, on flat
 * stencils (u_{-1} = u_0 = u_1 on every lane) and then skip the interpolant
 * and the MP bounds (1, the default), or leave the vote out (0).  The results
 * are the same bits either way (the constrained flux of a flat stencil is u_0
 * exactly); the vote pays where f has flat (e.g. empty) regions and only
 * costs where it has none.  set: VP_EINVAL for other values; forgets the
 * captured step graph. */
int vp_ensemble_set_flat_vote(vp_ens *ens, int on);
int vp_ensemble_get_flat_vote(const vp_ens *ens, int *on);
/* time candidate tile shapes (W, R, CTAs per SM), with and without the
 * flat-stencil vote, with whole steps at dt from a snapshot of f and the
 * field (allocated for the tuning, restored after every timed step, freed:
 * the ensemble's state is unchanged); keep the fastest; synchronises.
 * VP_ENOMEM without room for the snapshot. */
int vp_ensemble_autotune(vp_ens *ens, double dt);
/* nsteps KDK steps of every run (one persistent launch each, graph replay) */
int vp_ensemble_step(vp_ens *ens, double dt, int nsteps);
/* wait for the stream; VP_ETIMEOUT if a bounded wait in the kernel gave up */
int vp_ensemble_sync(vp_ens *ens);
/* polls of each stage-dependency wait in the kernel before it gives up
 * (default 2^24, about a second); a CTA whose wait runs out records
 * VP_ETIMEOUT for vp_ensemble_sync and leaves the kernel, and the step's f is
 * then undefined.  0 makes every dependency wait give up at once (a test of
 * that path).  Forgets the captured step graph. */
int vp_ensemble_set_wait_limit(vp_ens *ens, long long iterations);
long long vp_ensemble_launch_count(const vp_ens *ens);

/* ---- learned flux correction (not in the paper) --------------------------
 * A 25 -> 32 -> 32 -> 32 -> 1 ReLU network g corrects the mass that a
 * spatial sweep (drift) on a coarse velocity grid moves through each
 * interface: M = nu Phi_MP + s g(x), where Phi_MP is the CSL7 flux after the
 * MP constraint (App. A), s = max |u_k| + 1e-30 over the upwind-ordered 8-cell
 * stencil u_{-3..4} of the interface and x = ((u_k - u_0) / s for k = -3..4,
 * (u+_k - u-_k) / (2 s) and (u+_k + u-_k - 2 u_k) / (2 s) for k = -3..4, nu);
 * u+ / u- are the same cells of the
 * lines in the neighbouring velocity cells along the sweep's axis (+: larger
 * |v|; a neighbour outside the velocity box is zero).  The velocity
 * difference is what a coarse velocity cell loses: its sub-cell spread of
 * speeds moves the sub-cell gradient of f across x, also where the cell's
 * own fractional shift nu is zero, hence a mass rather than a flux value.
 * The PP limiter (Sec. 2.1.1) then acts on the total mass (u_0 - 2M >= 0,
 * u_1 + 2M >= 0: the clamp of M into [-u_1/2, u_0/2]) and the update keeps
 * the flux form f'_i = f_{i-n} - (M_out - M_in) (Eq. 49), so mass conservation
 * and f >= 0 hold as for the plain scheme.  With use_net = 2 the corrected
 * mass first passes the MP bounds of App. A again (the clamp into
 * [nu f_min, nu f_max]); a network trained without that clamp loses its
 * gain under it, so use_net = 1 (PP only) is the default of vp_learned_step.  Weights and matrix inputs are rounded to bfloat16, sums are
 * FP32.  Parameters: VP_NET_NPARAM floats, W1[32][25] b1[32] W2[32][32]
 * b2[32] W3[32][32] b3[32] w4[32] b4[1] (FP32 master copy; rounded when used).
 * Training pairs come from fine-grid runs of the method (vp_fine_flux,
 * vp_fluxnet_line_map, vp_group_mean, vp_restrict_velocity, vp_make_samples).
 */
#define VP_NET_NPARAM 2977

/* one sweep of the grid of ctx (FP32, order 7) with the network correction
 * (use_net = 1: PP on the corrected mass; use_net = 2: MP bounds then PP;
 * drifts only) or without it (use_net = 0: the same call as vp_drift_sweep /
 * vp_kick_sweep); wts_dev: VP_NET_NPARAM floats (device); f is updated in
 * place as seen by the caller.  With the network on, the walk reads f^n as it
 * is (a line's velocity neighbours included) and writes the new lines to a
 * buffer of f's size that the library owns, then copies that buffer back
 * into f on the context's stream; the buffer is allocated by the first
 * learned sweep or step of the context (not inside a stream capture) and
 * freed with it.  f_snap_dev is not read (kept in the signature; may be
 * NULL).  At most 128 velocity cells on the sweep's velocity axis (one
 * 128-row MMA operand per interface step; VP_ENOTSUP beyond, f unchanged).
 * VP_ENOTSUP for use_net with kick = 1, VP_EINVAL for use_net outside 0..2. */
int vp_learned_sweep(vp_ctx *ctx, int kick, int dim, double dt, const double *accel_dev,
                     const float *wts_dev, int use_net, const float *f_snap_dev);

/*
 * vp_learned_step -- vp_step with every drift (spatial sweep) replaced by
 * vp_learned_sweep(ctx, 0, d, h, NULL, wts_dev, 1, NULL): the same Strang
 * sequence (Sec. 2.4, Eq. 55), kicks and field solves unchanged, captured
 * into a CUDA graph per (dt, split, wts_dev) and replayed.  The network
 * weights are read at every replay (training may update them in place).
 * Arguments as vp_step; wts_dev: VP_NET_NPARAM device floats.  VP_ENOTSUP
 * unless the grid is FP32 with CSL7.
 */
int vp_learned_step(vp_ctx *ctx, double dt, int split, int nsteps, double *accel_dev, const float *wts_dev,
                    int mode, double *diag_dev);

/* Mass that the sweep (kick, dim, dt) of ctx's current f moves through every
 * `every`-th interface of every line, in cell units: G[line][j] for the
 * interface before cell j * every (j = 0 .. L / every); f' = f + G_{i-1/2} -
 * G_{i+1/2} reproduces the sweep.  f is not modified.  G_dev: device doubles. */
int vp_fine_flux(vp_ctx *ctx, int kick, int dim, double dt, const double *accel_dev, int every,
                 double *G_dev);

/* For a coarse grid whose velocity cells are factor^D fine cells (same
 * spatial grid, D <= 2): the fine lines averaged by every coarse line of the
 * sweep (kick, dim).  map_host (host, n_coarse_lines * group entries) may be
 * NULL to query the sizes. */
int vp_fluxnet_line_map(const vp_grid *fine, const vp_grid *coarse, int factor, int kick, int dim,
                        long long *map_host, long long *n_coarse_lines, int *group);

/* Coefficients of the cell-pair training loss: for pair t with left and
 * right interface samples li[t], ri[t] (indices into sc, the samples' scales
 * s from vp_make_samples) coef[2t] = -s_l / m, coef[2t + 1] = s_r / m,
 * m = max(s_l, s_r), and (weight not NULL) weight[t] = m^importance, the
 * pair's draw weight.  Device arrays; asynchronous on `stream`. */
int vp_pair_coefs(const float *sc, const long long *li, const long long *ri, long long n, double importance,
                  float *coef, double *weight, void *stream);

/* G_coarse[l][j] = scale * mean_g G_fine[map[l][g]][j] (device arrays) */
int vp_group_mean(const double *G_fine, long long n_coarse_lines, int nout, const long long *map_dev,
                  int group, double scale, double *G_coarse, void *cuda_stream);

/* coarse f = mean over factor1 x factor2 fine velocity cells ([NX][nf1][nf2]
 * -> [NX][nf1/factor1][nf2/factor2]; nf2 = factor2 = 1 for one velocity
 * dimension); device arrays */
int vp_restrict_velocity(const float *f_fine, float *f_coarse, long long NX, int nf1, int nf2, int factor1,
                         int factor2, void *cuda_stream);

/* Training pairs on the coarse grid of ctx: for every line and interface
 * (L + 1 per line), X (25 floats, zero velocity features for kick = 1) and
 * y = (Gc - whole coarse cells swept - nu Phi_MP) / s, the mass the network
 * should add; y = NaN where |zeta| < zmin or the interface is the duplicate
 * periodic end.  scale_dev (may be
 * NULL) receives s per sample (0 where y is NaN), so that a caller can weight
 * samples by the mass flux nu s they carry. */
int vp_make_samples(vp_ctx *coarse, int kick, int dim, double dt, const double *accel_dev,
                    const double *Gc_dev, double zmin, float *X_dev, float *y_dev, float *scale_dev);

/* loss += mean over groups of r^2 and grad += its gradient, where the nsamp
 * samples form consecutive groups of `group` (1, or 2 for the two interfaces
 * of one cell) with residual r = sum_k a_k (g(X_k) - y_k), a_k = coef_dev[k]
 * (all 1 when coef_dev is NULL); straight-through bfloat16 rounding; all
 * device arrays; nsamp must be a multiple of group. */
int vp_net_grad(const float *X_dev, const float *y_dev, const float *coef_dev, long long nsamp, int group,
                const float *wts_dev, float *grad_dev, float *loss_dev, void *cuda_stream);

/* one Adam step (beta 0.9 / 0.999, eps 1e-8) on the FP32 parameters; zeroes grad */
int vp_net_adam(float *wts_dev, float *m_dev, float *v_dev, float *grad_dev, int step, float lr,
                void *cuda_stream);

/*
 * vp_poisson_periodic_noalloc -- the periodic Poisson solve and force of
 * vp_poisson_solve (same arguments and results for a grid with
 * poisson == VP_POIS_PERIODIC), for callers that cannot allocate device
 * memory while they run: code whose device memory is all owned by its own
 * pool or caching allocator and budgeted up front, and latency-critical
 * loops that cannot afford the device-wide synchronisation of cudaMalloc and
 * cudaFree.  It needs no context and allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.  The paper has no counterpart;
 * this is a library entry point only.
 *   grid:     the grid (only dx, nx, xlo, xhi, pois_order, coupling, rho_bg
 *             and poisson are read); rho_dev: NX doubles in; phi_dev: NX
 *             doubles out or NULL; accel_dev: dx * NX doubles out (device).
 *   Limits:   NX = prod nx <= VP_NOALLOC_MAX_POINTS (262144), each axis
 *             <= 4096 cells; larger grids return VP_EINVAL.
 *   Scratch:  a 4 MiB static device array (VP_NOALLOC_MAX_POINTS complex
 *             doubles) held by every GPU that loads the library until the
 *             process exits.  Every call uses the same array and leaves its
 *             contents behind; calls that overlap on the GPU (two streams,
 *             two threads) race on it and must be serialised by the caller.
 *   Set-up:   the first call on each device looks up the array's device
 *             address (with that device current) and sets a kernel
 *             attribute; make that first call before any stream capture.
 *             The address is kept for the life of the process: it assumes
 *             the device's primary context is not reset (cudaDeviceReset)
 *             between calls.
 * Returns VP_OK, VP_EINVAL (bad or too large grid, NULL array) or VP_ECUDA,
 * also when a CUDA error from earlier work is pending on the calling thread
 * (it is left pending, not cleared, and nothing is launched).
 */
#define VP_NOALLOC_MAX_POINTS 262144
int vp_poisson_periodic_noalloc(const vp_grid *grid, void *cuda_stream, const double *rho_dev,
                                double *phi_dev, double *accel_dev);

#ifdef __cplusplus
}
#endif
#endif
