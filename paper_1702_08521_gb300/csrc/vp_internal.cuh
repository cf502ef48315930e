// vp_internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>

#include "vlasov.h"

// Per line class (one velocity index for a drift, one spatial cell for a
// kick): the integer shift n, the direction sigma = sign(zeta), the CFL number
// nu = |zeta| and the CSL weights w_k(nu) on the upwind-ordered stencil
// u[-3..3] (u[0] = upwind cell of the interface).  For CSL5 w[0] = w[6] = 0.
template <typename T>
struct __align__(16) LineShift {
    T w[7];
    T nu;
    int n;
    int sigma;
};

// Geometry of one sweep: f viewed as [outer][L][inner].
// Division of 32-bit unsigned values by a divisor fixed before the launch
// (Granlund & Montgomery 1994, Fig. 4.1): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (t + ((n - t) >> s1)) >> s2
// where t = high word of m n, s1 = min(l, 1), s2 = max(l - 1, 0).
struct FastDiv {
    unsigned d, m;
    int s1, s2;
};

inline FastDiv make_fastdiv(unsigned d) {
    int l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    FastDiv f;
    f.d = d;
    f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}

#ifdef __CUDACC__
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv &f) {
    const unsigned t = __umulhi(n, f.m);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}
__device__ __forceinline__ unsigned fmod_u(unsigned n, const FastDiv &f) { return n - fdiv(n, f) * f.d; }
#endif

struct SweepGeo {
    long long outer, inner;
    int L;
    int periodic;
    // class of a line: cls_from_inner ? (c / cdiv) % cmod : o / cdiv
    int cls_from_inner;
    long long cdiv, cmod;
    // column-kernel tile (W columns x full line), row-kernel lines per CTA
    int W, nseg, R;
    // divisors of the launch: cdiv, cmod, tiles per outer index, W (or R),
    // nseg, L, 16-byte pieces per tile row
    FastDiv fd_cdiv, fd_cmod, fd_tpo, fd_w, fd_nseg, fd_l, fd_wv, fd_w2;
    unsigned tpo;
};

// zero rows staged on each side of an outflow line (a shift |n| <= VP_GHOST - 4
// walks the line without bounds handling)
#define VP_GHOST 8

// tile configuration of one sweep geometry (chosen by the autotuner)
struct SweepTune {
    int valid;
    int impl;   // 1: staged loads (k_sweep_cols / k_sweep_rows), 2: TMA pipeline,
                // 3: staged loads with two lines per thread (FP32 strided sweeps)
    int W, nseg, ctas_per_sm;
};

// tile of the unsplit step (T1 x1 rows x T2 x2 cells x TV velocity cells,
// `threads` per CTA), one per halo width (4 or 8 cells)
struct UnsplitTune {
    int valid;
    int T1, T2, TV, threads;
};

struct LimParams {
    double alpha;
    int mp, pp;
};

// CSL weight polynomials: w_k(nu) = sum_j c[j][k] nu^j.
struct WPoly {
    double c[7][7];
    int nterm;  // 5 or 7 polynomial terms
};

struct vp_graph_cache {
    cudaGraphExec_t exec;
    double dt;
    int split;
    void *f;
    double *acc;
    long long per_step;  // kernels in one captured step
    const float *wts;    // network of the learned drifts (NULL: plain step)
    int valid;
};

struct vp_ctx {
    vp_grid g;
    cudaStream_t stream;
    int device, sm_count;
    long long NX, NV, ncell;
    int esize;
    void *f;
    WPoly wp;
    // library-owned device buffers
    void *d_shift;
    long long shift_cap;
    double *d_rho, *d_phi, *d_acc;      // diagnostics scratch
    double *d_rho_s, *d_phi_s;          // step scratch
    double2 *d_fft;
    double *d_green;                    // periodic: S / lambda(k)
    double2 *d_ghat;                    // isolated: DFT of the padded Green function
    long long MT;
    int m[3];
    double *d_part;                     // diagnostics partial sums [NX * 6]
    double *d_diag;                     // VP_NDIAG doubles
    int *d_flag;                        // non-finite flag
    long long launches;
    int *d_status;                      // device-side error word (bounded waits)
    void *d_netfrag;                    // network weights in MMA fragment order (allocated on first use)
    void *d_learn_out;                  // learned sweep: the updated lines (allocated on first use)
    int learned_ready;                  // learned-sweep buffers allocated, kernel attributes set
    int opt_impl;                       // 0 auto, 1 staged, 2 TMA
    int opt_autotune;                   // 1: time candidate tiles on first use
    unsigned opt_wait_limit;            // iterations of each bounded device-side wait
    SweepTune tune[2][3];               // [kick][dim]
    UnsplitTune utune[2];               // unsplit step, [halo of 8 cells]
    vp_graph_cache graph;
    char err[256];
};

// error helpers
int vp_fail(vp_ctx *c, int code, const char *fmt, ...);

// line geometry of the sweep (kick, dim): lines of L cells at stride
// `inner`, `outer` blocks of them, and the class of a line (its velocity index
// for drifts, its spatial point for kicks) that selects its shift
inline SweepGeo vp_make_geo(const vp_ctx *c, int kick, int dim) {

    const vp_grid &g = c->g;
    SweepGeo geo{};
    if (!kick) {
        long long outer = 1, inner = c->NV, vstride = 1;
        for (int k = 0; k < dim; ++k) outer *= g.nx[k];
        for (int k = dim + 1; k < g.dx; ++k) inner *= g.nx[k];
        for (int k = dim + 1; k < g.dv; ++k) vstride *= g.nv[k];
        geo.outer = outer;
        geo.inner = inner;
        geo.L = g.nx[dim];
        geo.periodic = g.xbc == VP_BC_PERIODIC;
        geo.cls_from_inner = 1;
        geo.cdiv = vstride;
        geo.cmod = g.nv[dim];
    } else {
        long long vouter = 1, inner = 1;
        for (int k = 0; k < dim; ++k) vouter *= g.nv[k];
        for (int k = dim + 1; k < g.dv; ++k) inner *= g.nv[k];
        geo.outer = c->NX * vouter;
        geo.inner = inner;
        geo.L = g.nv[dim];
        geo.periodic = 0;
        geo.cls_from_inner = 0;
        geo.cdiv = vouter;
        geo.cmod = 1;
    }
    geo.fd_cdiv = make_fastdiv((unsigned)geo.cdiv);
    geo.fd_cmod = make_fastdiv((unsigned)geo.cmod);
    return geo;
}

#define VP_CUDA_TRY(ctx, call)                                                         \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return vp_fail((ctx), VP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

// launchers implemented in the kernel files; all enqueue on ctx->stream
int vp_launch_shift_table(vp_ctx *c, int kick, int dim, double dt, const double *accel);
// the context stream is being captured into a graph (no synchronising calls)
bool vp_capturing(const vp_ctx *c);
// buffers and kernel attributes of the learned sweep (outside any stream capture)
int vp_learned_prepare(vp_ctx *c);
// one learned drift along dim from fin to fout (distinct arrays of f's size);
// net: make the network operands from wts first
int vp_learned_drift_io(vp_ctx *c, int dim, double dt, const float *wts, int use_net, const float *fin,
                        float *fout, bool net);
// RK-MPP5 sweeps: kernel attributes once per process, one sweep (table + fused stages)
int vp_rk_setup();
int vp_launch_rk_sweep(vp_ctx *c, int kick, int dim, double dt, const double *accel);
int vp_launch_sweep(vp_ctx *c, int kick, int dim);
// autotune sweep (kick, dim) at its own shifts (dt, accel); outside stream capture only
int vp_tune_sweep(vp_ctx *c, int kick, int dim, double dt, const double *accel);
int vp_launch_moment(vp_ctx *c, double *rho);
int vp_launch_poisson(vp_ctx *c, const double *rho, double *phi, double *acc);
int vp_launch_diag(vp_ctx *c, int mode, double *out_dev);
int vp_launch_init(vp_ctx *c, int kind, const double *p, int np);
int vp_field_setup(vp_ctx *c);          // Green function tables (at create)
// CSL weight polynomials of the given order (5 or 7), from the definition of the SL flux
WPoly vp_csl_weight_polys(int order);
// learned flux correction network: 9 features, 3 hidden layers of 32
#define VP_NET_FEATURES 25
#define VP_NET_HIDDEN 32
// analytic initial condition into any f array of grid g (precision from g)
int vp_launch_init_ptr(void *f, const vp_grid &g, int kind, const double *p, int np, cudaStream_t st);
int vp_sweep_setup(vp_ctx *c);          // kernel attributes (at create)
