// vp_api.cu -- the C ABI (include/vlasov.h): argument checks, context
// lifetime, the Strang step and its CUDA graph.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "vp_internal.cuh"

int vp_fail(vp_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

namespace {

// CSL weight polynomials from the definition of the SL flux (Sec. 2.1.2,
// Eqs. 26-27): Phi(nu) is the mean over the departure interval of the
// derivative of the primitive P(x) = int f, where P is the interpolating
// polynomial of the cumulative cell sums at the stencil's interfaces.
// Interfaces x_m = m + 1/2 (m = -h-1 .. h, cells -h .. h, h = (order-1)/2),
// measured by y = 1/2 - x so that the flux interface is y = 0 and the
// departure point is y = nu.  With Q_k(y) = sum_{m >= k} l_m(y) (l_m the
// Lagrange basis on the nodes y_m = -m), w_k(nu) = -(Q_k(nu) - Q_k(0)) / nu.
}  // namespace

WPoly vp_csl_weight_polys(int order) {
    WPoly wp{};
    const int h = (order - 1) / 2;
    const int npt = 2 * h + 2;          // interfaces
    const int deg = npt - 1;            // degree of the primitive
    double node[8];
    for (int i = 0; i < npt; ++i) node[i] = -(double)(i - h - 1);  // m = i - h - 1
    double lag[8][8] = {};              // lag[i][j]: coefficient of y^j in l_i
    for (int i = 0; i < npt; ++i) {
        double poly[8] = {1.0};
        int d = 0;
        double den = 1.0;
        for (int l = 0; l < npt; ++l) {
            if (l == i) continue;
            // poly *= (y - node[l])
            double nxt[8] = {};
            for (int j = 0; j <= d; ++j) {
                nxt[j + 1] += poly[j];
                nxt[j] -= node[l] * poly[j];
            }
            ++d;
            for (int j = 0; j <= d; ++j) poly[j] = nxt[j];
            den *= node[i] - node[l];
        }
        for (int j = 0; j <= deg; ++j) lag[i][j] = poly[j] / den;
    }
    wp.nterm = deg;  // Phi has degree deg - 1 in nu
    for (int k = -h; k <= h; ++k) {
        // Q_k = sum over interfaces m >= k, i.e. i = m + h + 1 >= k + h + 1
        double q[8] = {};
        for (int i = k + h + 1; i < npt; ++i)
            for (int j = 0; j <= deg; ++j) q[j] += lag[i][j];
        for (int j = 1; j <= deg; ++j) wp.c[j - 1][k + 3] = -q[j];
    }
    return wp;
}

namespace {

bool is_fin(double x) { return std::isfinite(x); }

int check_ctx(vp_ctx *c, bool need_f) {
    if (!c) return VP_EINVAL;
    if (need_f && !c->f) return vp_fail(c, VP_EINVAL, "no distribution function bound (vp_bind_f)");
    return VP_OK;
}

int validate(const vp_grid *g, char *msg, size_t n) {
    if (g->dx < 1 || g->dx > 3 || g->dv != g->dx) {
        snprintf(msg, n, "dx must equal dv and lie in 1..3");
        return VP_EINVAL;
    }
    for (int d = 0; d < g->dx; ++d) {
        if (g->nx[d] < 1 || g->nv[d] < 1) {
            snprintf(msg, n, "cell counts must be >= 1");
            return VP_EINVAL;
        }
        if (!(g->xhi[d] > g->xlo[d]) || !(g->vhi[d] > g->vlo[d]) || !is_fin(g->xlo[d]) ||
            !is_fin(g->xhi[d]) || !is_fin(g->vlo[d]) || !is_fin(g->vhi[d])) {
            snprintf(msg, n, "boxes must be finite with hi > lo");
            return VP_EINVAL;
        }
    }
    if (g->order != 5 && g->order != 7) {
        snprintf(msg, n, "order must be 5 or 7");
        return VP_EINVAL;
    }
    if (g->precision != VP_F32 && g->precision != VP_F64) {
        snprintf(msg, n, "precision must be VP_F32 or VP_F64");
        return VP_EINVAL;
    }
    if (g->xbc != VP_BC_PERIODIC && g->xbc != VP_BC_OUTFLOW) {
        snprintf(msg, n, "xbc must be VP_BC_PERIODIC or VP_BC_OUTFLOW");
        return VP_EINVAL;
    }
    if (g->scheme != VP_SCHEME_SL && g->scheme != VP_SCHEME_RK) {
        snprintf(msg, n, "scheme must be VP_SCHEME_SL or VP_SCHEME_RK");
        return VP_EINVAL;
    }
    if (g->scheme == VP_SCHEME_RK && g->order != 5) {
        snprintf(msg, n, "RK-MPP5 is fifth order: order must be 5");
        return VP_ENOTSUP;
    }
    if (g->pois_order != 2 && g->pois_order != 4 && g->pois_order != 6) {
        snprintf(msg, n, "pois_order must be 2, 4 or 6");
        return VP_EINVAL;
    }
    if (!(g->alpha >= 0.0) || !is_fin(g->alpha) || !is_fin(g->coupling) || !is_fin(g->rho_bg)) {
        snprintf(msg, n, "alpha, coupling and rho_bg must be finite (alpha >= 0)");
        return VP_EINVAL;
    }
    if (g->poisson == VP_POIS_ISOLATED) {
        if (g->dx != 3) {
            snprintf(msg, n, "isolated Poisson needs three spatial dimensions");
            return VP_ENOTSUP;
        }
        const double h = (g->xhi[0] - g->xlo[0]) / g->nx[0];
        for (int d = 1; d < 3; ++d) {
            const double hd = (g->xhi[d] - g->xlo[d]) / g->nx[d];
            if (std::fabs(hd - h) > 1e-12 * h) {
                snprintf(msg, n, "isolated Poisson needs cubic cells");
                return VP_ENOTSUP;
            }
        }
    } else if (g->poisson != VP_POIS_PERIODIC) {
        snprintf(msg, n, "poisson must be VP_POIS_PERIODIC or VP_POIS_ISOLATED");
        return VP_EINVAL;
    }
    int nmax = 0;
    for (int d = 0; d < g->dx; ++d) {
        nmax = g->nx[d] > nmax ? g->nx[d] : nmax;
        if (g->poisson == VP_POIS_ISOLATED) nmax = 2 * g->nx[d] > nmax ? 2 * g->nx[d] : nmax;
    }
    if (nmax > 4096) {
        snprintf(msg, n, "spatial axes are limited to 4096 cells (2048 isolated)");
        return VP_ENOTSUP;
    }
    return VP_OK;
}

void free_buffers(vp_ctx *c) {
    cudaFree(c->d_shift);
    cudaFree(c->d_rho);
    cudaFree(c->d_phi);
    cudaFree(c->d_acc);
    cudaFree(c->d_rho_s);
    cudaFree(c->d_phi_s);
    cudaFree(c->d_fft);
    cudaFree(c->d_green);
    cudaFree(c->d_ghat);
    cudaFree(c->d_part);
    cudaFree(c->d_diag);
    cudaFree(c->d_flag);
    cudaFree(c->d_status);
    cudaFree(c->d_netfrag);
    cudaFree(c->d_learn_out);
    if (c->graph.valid) cudaGraphExecDestroy(c->graph.exec);
}

bool capturing(const vp_ctx *c) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &st) != cudaSuccess) {
        cudaGetLastError();
        return true;  // legacy stream while another stream captures: do not sync
    }
    return st != cudaStreamCaptureStatusNone;
}

int sweep_all(vp_ctx *c, int kick, int dim, double dt, const double *accel) {
    int rc;
    // RK-MPP5 (Eq. 10): three stages fused in one launch, default tiles (its
    // stages do not leave f bit-for-bit unchanged at dt = 0, which the tuner needs)
    if (c->g.scheme == VP_SCHEME_RK) return vp_launch_rk_sweep(c, kick, dim, dt, accel);
    if (c->opt_autotune && !c->tune[kick][dim].valid && !capturing(c))
        if ((rc = vp_tune_sweep(c, kick, dim, dt, accel))) return rc;
    rc = vp_launch_shift_table(c, kick, dim, dt, accel);
    if (rc) return rc;
    return vp_launch_sweep(c, kick, dim);
}

// one Strang step (Eq. 55) on the context stream
// one Strang step; with wts the drifts are learned sweeps of that network
int enqueue_step(vp_ctx *c, double dt, int split, double *acc, const float *wts) {
    const vp_grid &g = c->g;
    const long long NX = c->NX;
    int rc;
    // the drifts x_D ... x_1 of a stage; learned drifts alternate between f
    // and the library's second array (each reads f^n whole and writes the
    // new lines apart), with the network operands made once per stage and
    // one copy back into f only after an odd number of drifts
    auto drifts = [&](double h) {
        if (!wts) {
            for (int d = g.dx - 1; d >= 0; --d)
                if ((rc = sweep_all(c, 0, d, h, nullptr))) return rc;
            return VP_OK;
        }
        float *src = static_cast<float *>(c->f), *dst = static_cast<float *>(c->d_learn_out);
        for (int d = g.dx - 1; d >= 0; --d) {
            if ((rc = vp_learned_drift_io(c, d, h, wts, 1, src, dst, d == g.dx - 1))) return rc;
            float *t = src;
            src = dst;
            dst = t;
        }
        if (src != c->f)
            VP_CUDA_TRY(c, cudaMemcpyAsync(c->f, src, (size_t)c->ncell * sizeof(float), cudaMemcpyDeviceToDevice,
                                           c->stream));
        return VP_OK;
    };
    if (split == VP_SPLIT_KDK) {
        for (int d = 0; d < g.dv; ++d)
            if ((rc = sweep_all(c, 1, d, 0.5 * dt, acc + d * NX))) return rc;
        if ((rc = drifts(dt))) return rc;
        if ((rc = vp_launch_moment(c, c->d_rho_s))) return rc;
        if ((rc = vp_launch_poisson(c, c->d_rho_s, c->d_phi_s, acc))) return rc;
        for (int d = 0; d < g.dv; ++d)
            if ((rc = sweep_all(c, 1, d, 0.5 * dt, acc + d * NX))) return rc;
    } else {
        if ((rc = drifts(0.5 * dt))) return rc;
        if ((rc = vp_launch_moment(c, c->d_rho_s))) return rc;
        if ((rc = vp_launch_poisson(c, c->d_rho_s, c->d_phi_s, acc))) return rc;
        for (int d = 0; d < g.dv; ++d)
            if ((rc = sweep_all(c, 1, d, dt, acc + d * NX))) return rc;
        if ((rc = drifts(0.5 * dt))) return rc;
    }
    return VP_OK;
}

}  // namespace

bool vp_capturing(const vp_ctx *c) { return capturing(c); }

extern "C" {

int vp_create(const vp_grid *grid, void *cuda_stream, vp_ctx **out) {
    if (!out) return VP_EINVAL;
    *out = nullptr;
    if (!grid) return VP_EINVAL;
    vp_ctx *c = new (std::nothrow) vp_ctx();
    if (!c) return VP_ENOMEM;
    c->g = *grid;
    for (int d = grid->dx; d < 3; ++d) {
        c->g.nx[d] = c->g.nv[d] = 1;
        c->g.xlo[d] = c->g.vlo[d] = 0.0;
        c->g.xhi[d] = c->g.vhi[d] = 1.0;
    }
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    int rc = validate(&c->g, c->err, sizeof(c->err));
    if (rc) {
        fprintf(stderr, "vp_create: %s\n", c->err);
        delete c;
        return rc;
    }
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return VP_ECUDA;
    }
    c->NX = c->NV = 1;
    for (int d = 0; d < c->g.dx; ++d) {
        c->NX *= c->g.nx[d];
        c->NV *= c->g.nv[d];
    }
    c->ncell = c->NX * c->NV;
    c->esize = c->g.precision == VP_F32 ? 4 : 8;
    c->wp = vp_csl_weight_polys(c->g.order);
    long long ncls = c->NX;
    for (int d = 0; d < c->g.dv; ++d) ncls = c->g.nv[d] > ncls ? c->g.nv[d] : ncls;
    long long nvsum = 0;  // the unsplit step's tables of every drift axis
    for (int d = 0; d < c->g.dv; ++d) nvsum += c->g.nv[d];
    ncls = nvsum > ncls ? nvsum : ncls;
    c->shift_cap = ncls;
    const size_t shift_bytes = (size_t)ncls * (c->esize == 4 ? sizeof(LineShift<float>) : sizeof(LineShift<double>));
#define ALLOC(p, bytes)                                                     \
    if (cudaMalloc((void **)&(p), (bytes)) != cudaSuccess) {                \
        free_buffers(c);                                                    \
        delete c;                                                           \
        cudaGetLastError();                                                 \
        return VP_ENOMEM;                                                   \
    }
    ALLOC(c->d_shift, shift_bytes);
    ALLOC(c->d_rho, sizeof(double) * c->NX);
    ALLOC(c->d_phi, sizeof(double) * c->NX);
    ALLOC(c->d_acc, sizeof(double) * c->NX * c->g.dx);
    ALLOC(c->d_rho_s, sizeof(double) * c->NX);
    ALLOC(c->d_phi_s, sizeof(double) * c->NX);
    ALLOC(c->d_part, sizeof(double) * c->NX * 6);
    ALLOC(c->d_diag, sizeof(double) * VP_NDIAG);
    ALLOC(c->d_flag, sizeof(int));
    ALLOC(c->d_status, sizeof(int));
#undef ALLOC
    c->opt_autotune = 1;
    c->opt_wait_limit = 1u << 26;
    if (cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess) {
        free_buffers(c);
        delete c;
        return VP_ECUDA;
    }
    if ((rc = vp_sweep_setup(c)) || (rc = vp_field_setup(c)) || (rc = vp_rk_setup())) {
        fprintf(stderr, "vp_create: %s\n", c->err);
        free_buffers(c);
        delete c;
        return rc;
    }
    *out = c;
    return VP_OK;
}

void vp_destroy(vp_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_buffers(c);
    delete c;
}

const char *vp_last_error(const vp_ctx *c) { return c ? c->err : "null context"; }

long long vp_num_cells(const vp_ctx *c) { return c ? c->ncell : 0; }

int vp_elem_size(const vp_ctx *c) { return c ? c->esize : 0; }

long long vp_launch_count(const vp_ctx *c) { return c ? c->launches : 0; }

int vp_bind_f(vp_ctx *c, void *f_dev) {
    if (!c) return VP_EINVAL;
    if (!f_dev) return vp_fail(c, VP_EINVAL, "f_dev is NULL");
    if (reinterpret_cast<uintptr_t>(f_dev) & 15)
        return vp_fail(c, VP_EINVAL, "f_dev must be 16-byte aligned");
    c->f = f_dev;
    return VP_OK;
}

int vp_init_f(vp_ctx *c, int kind, const double *params, int nparams) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    static const int need[5] = {6, 2, 3, 1, 3};
    if (kind < 0 || kind > 4) return vp_fail(c, VP_EINVAL, "unknown initial condition %d", kind);
    if (!params || nparams < need[kind])
        return vp_fail(c, VP_EINVAL, "initial condition %d needs %d parameters", kind, need[kind]);
    if ((kind == VP_IC_PLUMMER || kind == VP_IC_SPHERE) && c->g.dx != 3)
        return vp_fail(c, VP_EINVAL, "the Plummer and uniform spheres need 3D3V");
    for (int i = 0; i < nparams; ++i)
        if (!is_fin(params[i])) return vp_fail(c, VP_EINVAL, "non-finite parameter");
    return vp_launch_init(c, kind, params, nparams);
}

int vp_upload_f(vp_ctx *c, const void *host, size_t bytes) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    if (!host || bytes != (size_t)c->ncell * c->esize)
        return vp_fail(c, VP_EINVAL, "upload needs %lld bytes", (long long)c->ncell * c->esize);
    VP_CUDA_TRY(c, cudaMemcpyAsync(c->f, host, bytes, cudaMemcpyHostToDevice, c->stream));
    return VP_OK;
}

int vp_download_f(vp_ctx *c, void *host, size_t bytes) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    if (!host || bytes != (size_t)c->ncell * c->esize)
        return vp_fail(c, VP_EINVAL, "download needs %lld bytes", (long long)c->ncell * c->esize);
    VP_CUDA_TRY(c, cudaMemcpyAsync(host, c->f, bytes, cudaMemcpyDeviceToHost, c->stream));
    return VP_OK;
}

int vp_drift_sweep(vp_ctx *c, int dim, double dt) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    if (dim < 0 || dim >= c->g.dx) return vp_fail(c, VP_EINVAL, "dim %d out of range", dim);
    if (!is_fin(dt)) return vp_fail(c, VP_EINVAL, "dt must be finite");
    const double h = (c->g.xhi[dim] - c->g.xlo[dim]) / c->g.nx[dim];
    const double vmax = std::fmax(std::fabs(c->g.vlo[dim]), std::fabs(c->g.vhi[dim]));
    if (vmax * std::fabs(dt) / h > 1e9) return vp_fail(c, VP_EINVAL, "shift too large");
    return sweep_all(c, 0, dim, dt, nullptr);
}

int vp_kick_sweep(vp_ctx *c, int dim, double dt, const double *accel_dev) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    if (dim < 0 || dim >= c->g.dv) return vp_fail(c, VP_EINVAL, "dim %d out of range", dim);
    if (!is_fin(dt)) return vp_fail(c, VP_EINVAL, "dt must be finite");
    if (!accel_dev) return vp_fail(c, VP_EINVAL, "accel_dev is NULL");
    return sweep_all(c, 1, dim, dt, accel_dev);
}

int vp_density_moment(vp_ctx *c, double *rho_dev) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    if (!rho_dev) return vp_fail(c, VP_EINVAL, "rho_dev is NULL");
    return vp_launch_moment(c, rho_dev);
}

int vp_poisson_solve(vp_ctx *c, const double *rho_dev, double *phi_dev, double *accel_dev) {
    int rc = check_ctx(c, false);
    if (rc) return rc;
    if (!rho_dev || !accel_dev) return vp_fail(c, VP_EINVAL, "rho_dev and accel_dev are required");
    return vp_launch_poisson(c, rho_dev, phi_dev ? phi_dev : c->d_phi, accel_dev);
}

int vp_set_option(vp_ctx *c, int option, long long value) {
    if (!c) return VP_EINVAL;
    if (option == VP_OPT_SWEEP_IMPL) {
        if (value < 0 || value > 3) return vp_fail(c, VP_EINVAL, "sweep implementation must be 0 .. 3");
        c->opt_impl = (int)value;
    } else if (option == VP_OPT_AUTOTUNE) {
        c->opt_autotune = value != 0;
    } else if (option == VP_OPT_WAIT_LIMIT) {
        if (value < 0 || value > 0xffffffffLL) return vp_fail(c, VP_EINVAL, "wait limit must fit 32 bits");
        c->opt_wait_limit = (unsigned)value;
    } else {
        return vp_fail(c, VP_EINVAL, "unknown option %d", option);
    }
    for (int k = 0; k < 2; ++k)
        for (int d = 0; d < 3; ++d) c->tune[k][d].valid = 0;
    c->utune[0].valid = c->utune[1].valid = 0;
    if (c->graph.valid) {
        cudaGraphExecDestroy(c->graph.exec);
        c->graph.valid = 0;
    }
    return VP_OK;
}

int vp_get_tuning(const vp_ctx *c, int kick, int dim, int *out4) {
    if (!c || !out4 || kick < 0 || kick > 1 || dim < 0 || dim > 2) return VP_EINVAL;
    const SweepTune &t = c->tune[kick][dim];
    out4[0] = t.valid ? t.impl : 0;
    out4[1] = t.W;
    out4[2] = t.nseg;
    out4[3] = t.ctas_per_sm;
    return VP_OK;
}

int vp_sync(vp_ctx *c) {
    if (!c) return VP_EINVAL;
    VP_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    int st = 0;
    VP_CUDA_TRY(c, cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
        cudaMemset(c->d_status, 0, sizeof(int));
        if (st == VP_ETIMEOUT) return vp_fail(c, VP_ETIMEOUT, "a device-side wait gave up");
        if (st == VP_ECFL) return vp_fail(c, VP_ECFL, "an RK-MPP5 sweep had |nu| >= 1/2 (Sec. 2.1.1)");
        return vp_fail(c, VP_ECUDA, "a kernel's self-check failed (status %d)", st);
    }
    return VP_OK;
}

int vp_diagnostics(vp_ctx *c, int mode, vp_diag *out) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    if (!out) return vp_fail(c, VP_EINVAL, "out is NULL");
    VP_CUDA_TRY(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
    if ((rc = vp_launch_diag(c, mode, c->d_diag))) return rc;
    double h[VP_NDIAG];
    int flag = 0;
    VP_CUDA_TRY(c, cudaMemcpyAsync(h, c->d_diag, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    VP_CUDA_TRY(c, cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if ((rc = vp_sync(c))) return rc;
    memcpy(out, h, sizeof(h));
    if (flag) return vp_fail(c, VP_ENONFINITE, "f holds NaN or Inf");
    return VP_OK;
}

// nsteps Strang steps, captured once per (dt, split, f, accel, network) in a CUDA graph
static int run_steps(vp_ctx *c, double dt, int split, int nsteps, double *accel_dev, int mode, double *diag_dev,
              const float *wts) {
    int rc;
    if (!accel_dev) return vp_fail(c, VP_EINVAL, "accel_dev is NULL");
    if (split != VP_SPLIT_KDK && split != VP_SPLIT_DKD) return vp_fail(c, VP_EINVAL, "bad split");
    if (nsteps < 0 || !is_fin(dt)) return vp_fail(c, VP_EINVAL, "bad dt or nsteps");
    // graph path needs a capturable (non-legacy) stream
    const bool use_graph = c->stream != nullptr && c->stream != cudaStreamLegacy;
    vp_graph_cache &gc = c->graph;
    if (c->opt_autotune && !capturing(c)) {
        // each sweep tuned at the step it appears in: KDK kicks by dt/2 and
        // drifts by dt, DKD the other way round
        const double hd = split == VP_SPLIT_KDK ? dt : 0.5 * dt, hk = split == VP_SPLIT_KDK ? 0.5 * dt : dt;
        for (int d = 0; d < c->g.dx; ++d)
            if ((rc = vp_tune_sweep(c, 0, d, hd, nullptr))) return rc;
        for (int d = 0; d < c->g.dv; ++d)
            if ((rc = vp_tune_sweep(c, 1, d, hk, accel_dev + d * c->NX))) return rc;
    }
    if (use_graph && !(gc.valid && gc.dt == dt && gc.split == split && gc.f == c->f && gc.acc == accel_dev &&
                      gc.wts == wts)) {
        if (gc.valid) {
            cudaGraphExecDestroy(gc.exec);
            gc.valid = 0;
        }
        const long long before = c->launches;
        VP_CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_step(c, dt, split, accel_dev, wts);
        cudaGraph_t graph;
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        const long long per_step_captured = c->launches - before;
        c->launches = before;  // captured, not launched
        if (rc) {
            if (e == cudaSuccess) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return vp_fail(c, VP_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&gc.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return vp_fail(c, VP_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        gc.valid = 1;
        gc.dt = dt;
        gc.split = split;
        gc.f = c->f;
        gc.acc = accel_dev;
        gc.wts = wts;
        gc.per_step = per_step_captured;
    }
    for (int s = 0; s < nsteps; ++s) {
        if (use_graph) {
            VP_CUDA_TRY(c, cudaGraphLaunch(gc.exec, c->stream));
            c->launches += gc.per_step;
        } else if ((rc = enqueue_step(c, dt, split, accel_dev, wts))) {
            return rc;
        }
        if (diag_dev && (rc = vp_launch_diag(c, mode, diag_dev + (long long)s * VP_NDIAG))) return rc;
    }
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

int vp_step(vp_ctx *c, double dt, int split, int nsteps, double *accel_dev, int mode,
            double *diag_dev) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    return run_steps(c, dt, split, nsteps, accel_dev, mode, diag_dev, nullptr);
}

int vp_learned_step(vp_ctx *c, double dt, int split, int nsteps, double *accel_dev, const float *wts_dev,
                    int mode, double *diag_dev) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    if (!wts_dev) return vp_fail(c, VP_EINVAL, "wts_dev is NULL");
    if (c->g.precision != VP_F32 || c->g.order != 7)
        return vp_fail(c, VP_ENOTSUP, "the learned sweep runs on FP32 CSL7 grids");
    if ((rc = vp_learned_prepare(c))) return rc;
    return run_steps(c, dt, split, nsteps, accel_dev, mode, diag_dev, wts_dev);
}

}  // extern "C"
