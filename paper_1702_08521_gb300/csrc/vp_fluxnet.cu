// vp_fluxnet.cu -- learned flux correction on a coarser velocity grid
// (an addition to the method, not in the paper).
//
// A 25 -> 32 -> 32 -> 32 -> 1 ReLU network g corrects the mass that a
// coarse-grid spatial sweep moves through an interface:
//   M = nu Phi_MP + s g(x),
// Phi_MP the CSL7 flux after the MP constraint, s = max |u| over the 8-cell
// upwind-ordered stencil u_{-3..4}, x = ((u_k - u_0) / s, (u+_k - u-_k) / (2 s),
// (u+_k + u-_k - 2 u_k) / (2 s), nu) with u+ / u- the same cells of the lines in
// the neighbouring velocity cells (+: larger |v|).  The correction is a mass, not a flux value: the
// sub-cell spread of speeds inside a coarse velocity cell moves mass even
// where the cell's own fractional shift nu is small.  The corrected mass
// passes the PP limiter (f_i - 2 M >= 0, f_{i+1} + 2 M >= 0) and, on request
// (use_net = 2), the MP bounds of App. A before it (the clamp into
// [nu f_min, nu f_max]); the update keeps the flux form
// f'_i = f_{i-n} - (M_out - M_in), so conservation and f >= 0 hold exactly as
// for the plain scheme.  Weights and matrix inputs are bfloat16, sums FP32.
//
// Training data come from fine-grid runs of the method itself: for a sweep,
// the fine-grid mass through every coarse interface (mean over the fine
// lines a coarse line aggregates), minus the coarse integer-shift part and
// the coarse MP-limited fractional mass, over s, is the target of g.
// Training: per-sample forward/backward (FP32, bfloat16-rounded weights and
// activations, straight-through backward), per-CTA weight-gradient
// reductions, Adam.
#include <cuda_bf16.h>

#include <cmath>

#include "vp_internal.cuh"
#include "vp_sweep_core.cuh"
#include "vp_umma.cuh"

namespace {

constexpr int H = VP_NET_HIDDEN;
constexpr int NF = VP_NET_FEATURES;

// parameter layout (floats): W1[H][NF] b1[H] W2[H][H] b2[H] W3[H][H] b3[H] w4[H] b4[1]
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + H * NF;
constexpr int OFF_W2 = OFF_B1 + H;
constexpr int OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H;
constexpr int OFF_B3 = OFF_W3 + H * H;
constexpr int OFF_W4 = OFF_B3 + H;
constexpr int OFF_B4 = OFF_W4 + H;
constexpr int NPARAM = OFF_B4 + 1;
static_assert(NPARAM == VP_NET_NPARAM, "parameter count");

__device__ __forceinline__ float bfr(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// ---- network on one sample (SIMT, weights in shared memory, rounded) -------------

struct NetAct {
    float x[NF], h1[H], h2[H], h3[H];
    float z1[H], z2[H], z3[H];
};

__device__ __forceinline__ float net_forward(const float *__restrict__ w, const float *xin, float *h1,
                                             float *h2, float *h3) {
    float x[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) x[k] = bfr(xin[k]);
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
        float a = w[OFF_B1 + j];
#pragma unroll
        for (int k = 0; k < NF; ++k) a = fmaf(w[OFF_W1 + j * NF + k], x[k], a);
        h1[j] = bfr(fmaxf(a, 0.f));
    }
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
        float a = w[OFF_B2 + j];
#pragma unroll
        for (int k = 0; k < H; ++k) a = fmaf(w[OFF_W2 + j * H + k], h1[k], a);
        h2[j] = bfr(fmaxf(a, 0.f));
    }
    float g = w[OFF_B4];
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
        float a = w[OFF_B3 + j];
#pragma unroll
        for (int k = 0; k < H; ++k) a = fmaf(w[OFF_W3 + j * H + k], h2[k], a);
        const float v = bfr(fmaxf(a, 0.f));
        if (h3) h3[j] = v;
        g = fmaf(w[OFF_W4 + j], v, g);
    }
    return g;
}

// features of the upwind-ordered stencil u[0..7] = u_{-3..4} and of the same
// cells up / um of the velocity-neighbour lines (+: larger |v|): velocity
// difference and curvature
__device__ __forceinline__ float net_features(const float *u, const float *up, const float *um, float nu,
                                              float *x) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s = fmaxf(s, fabsf(u[k]));
    s += 1e-30f;
    const float inv = 1.0f / s;
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (u[k] - u[3]) * inv;
#pragma unroll
    for (int k = 0; k < 8; ++k) x[8 + k] = (up[k] - um[k]) * (0.5f * inv);
#pragma unroll
    for (int k = 0; k < 8; ++k) x[16 + k] = fmaf(0.5f, up[k] + um[k], -u[k]) * inv;
    x[24] = nu;
    return s;
}

// ---- training ----------------------------------------------------------------------

constexpr int kTrainThreads = 128;

// One CTA: kTrainThreads samples.  Samples come in consecutive groups of
// `group` (1 or 2; a pair = the two interfaces of one cell) whose residual is
// r = sum_k a_k (g_k - y_k) (a_k = coef[k], 1 without coef); the loss is the
// mean of r^2 over groups.  The two threads of a pair exchange their terms by
// a warp shuffle.  Loss and weight gradients accumulated in global FP32
// (per-CTA reductions, then one atomic per parameter).
__global__ void __launch_bounds__(kTrainThreads) k_net_grad(const float *__restrict__ X,
                                                            const float *__restrict__ y,
                                                            const float *__restrict__ coef,
                                                            const float *__restrict__ wts, long long nsamp,
                                                            int group, float *__restrict__ grad,
                                                            float *__restrict__ loss) {
    __shared__ float w[NPARAM];
    __shared__ float A0[kTrainThreads][NF + 1];
    __shared__ float A1[kTrainThreads][H + 1];
    __shared__ float A2[kTrainThreads][H + 1];
    __shared__ float D[kTrainThreads][H + 1];  // delta of the current layer
    __shared__ float red[kTrainThreads];
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x)
        w[i] = (i >= OFF_B4 || (i >= OFF_B1 && i < OFF_W2) || (i >= OFF_B2 && i < OFF_W3) ||
                (i >= OFF_B3 && i < OFF_W4))
                   ? wts[i]
                   : bfr(wts[i]);
    __syncthreads();
    const long long sidx = (long long)blockIdx.x * kTrainThreads + threadIdx.x;
    const bool valid = sidx < nsamp;
    const int t = threadIdx.x;
    float x[NF], h1[H], h2[H], h3[H];
    float term = 0.f, a = 0.f;
    if (valid) {
        for (int k = 0; k < NF; ++k) x[k] = X[sidx * NF + k];
        const float g = net_forward(w, x, h1, h2, h3);
        a = coef ? coef[sidx] : 1.f;
        term = a * (g - y[sidx]);
    } else {
        for (int k = 0; k < NF; ++k) x[k] = 0.f;
        for (int j = 0; j < H; ++j) h1[j] = h2[j] = h3[j] = 0.f;
    }
    // group residual (pairs are threads 2k, 2k + 1 of the same warp)
    float r = term;
    if (group == 2) r += __shfl_xor_sync(0xffffffffu, term, 1);
    const float ngroups = (float)(nsamp / group);
    const float dg = valid ? 2.0f * r * a / ngroups : 0.f;
    red[t] = (valid && (group == 1 || (t & 1) == 0)) ? r * r / ngroups : 0.f;
    for (int k = 0; k < NF; ++k) A0[t][k] = bfr(x[k]);
    for (int j = 0; j < H; ++j) {
        A1[t][j] = h1[j];
        A2[t][j] = h2[j];
    }
    // layer 4: g = w4 . h3 + b4
    for (int j = 0; j < H; ++j) D[t][j] = h3[j];  // temporarily hold h3
    __syncthreads();
    // grads of w4, b4: sum_s dg_s h3_s
    {
        __shared__ float dgs[kTrainThreads];
        dgs[t] = dg;
        __syncthreads();
        if (t < H) {
            float a = 0.f;
            for (int s = 0; s < kTrainThreads; ++s) a = fmaf(dgs[s], D[s][t], a);
            atomicAdd(grad + OFF_W4 + t, a);
        }
        if (t == H) {
            float a = 0.f, l = 0.f;
            for (int s = 0; s < kTrainThreads; ++s) {
                a += dgs[s];
                l += red[s];
            }
            atomicAdd(grad + OFF_B4, a);
            atomicAdd(loss, l);
        }
        __syncthreads();
    }
    // delta3 = dg * w4 * [h3 > 0] (h3 > 0 iff its pre-activation was > 0)
    float d3[H];
    for (int j = 0; j < H; ++j) d3[j] = (h3[j] > 0.f) ? dg * w[OFF_W4 + j] : 0.f;
    __syncthreads();
    for (int j = 0; j < H; ++j) D[t][j] = d3[j];
    __syncthreads();
    // grads W3 = sum_s d3_s h2_s^T, b3 = sum_s d3_s
    for (int e = t; e < H * H; e += blockDim.x) {
        const int i = e / H, k = e % H;
        float a = 0.f;
        for (int s = 0; s < kTrainThreads; ++s) a = fmaf(D[s][i], A2[s][k], a);
        atomicAdd(grad + OFF_W3 + e, a);
    }
    if (t < H) {
        float a = 0.f;
        for (int s = 0; s < kTrainThreads; ++s) a += D[s][t];
        atomicAdd(grad + OFF_B3 + t, a);
    }
    // delta2 = (W3^T d3) * [h2 > 0]
    float d2[H];
    for (int k = 0; k < H; ++k) {
        float a = 0.f;
        for (int j = 0; j < H; ++j) a = fmaf(w[OFF_W3 + j * H + k], d3[j], a);
        d2[k] = (h2[k] > 0.f) ? a : 0.f;
    }
    __syncthreads();
    for (int j = 0; j < H; ++j) D[t][j] = d2[j];
    __syncthreads();
    for (int e = t; e < H * H; e += blockDim.x) {
        const int i = e / H, k = e % H;
        float a = 0.f;
        for (int s = 0; s < kTrainThreads; ++s) a = fmaf(D[s][i], A1[s][k], a);
        atomicAdd(grad + OFF_W2 + e, a);
    }
    if (t < H) {
        float a = 0.f;
        for (int s = 0; s < kTrainThreads; ++s) a += D[s][t];
        atomicAdd(grad + OFF_B2 + t, a);
    }
    float d1[H];
    for (int k = 0; k < H; ++k) {
        float a = 0.f;
        for (int j = 0; j < H; ++j) a = fmaf(w[OFF_W2 + j * H + k], d2[j], a);
        d1[k] = (h1[k] > 0.f) ? a : 0.f;
    }
    __syncthreads();
    for (int j = 0; j < H; ++j) D[t][j] = d1[j];
    __syncthreads();
    for (int e = t; e < H * NF; e += blockDim.x) {
        const int i = e / NF, k = e % NF;
        float a = 0.f;
        for (int s = 0; s < kTrainThreads; ++s) a = fmaf(D[s][i], A0[s][k], a);
        atomicAdd(grad + OFF_W1 + e, a);
    }
    if (t < H) {
        float a = 0.f;
        for (int s = 0; s < kTrainThreads; ++s) a += D[s][t];
        atomicAdd(grad + OFF_B1 + t, a);
    }
}

__global__ void k_adam(float *__restrict__ wts, float *__restrict__ m, float *__restrict__ v,
                       float *__restrict__ grad, int n, float lr, float b1, float b2, float eps, float bc1,
                       float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    wts[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    grad[i] = 0.f;
}

// ---- training data -----------------------------------------------------------------

// Mass through interfaces of fine lines, in fine-cell units, for one sweep:
// G_{i+1/2} = sum of the N whole cells swept through + nu Phi_hat at the
// shifted interface (the flux form of the SL update: f'_i = f_i + G_{i-1/2}
// - G_{i+1/2}).  Lines: f viewed as [outer][L][inner]; one thread per line;
// the line's class (speed) as in the sweeps.  Output: G at interfaces
// j * every - 1/2 for j = 0 .. L/every (boundary interfaces included).
__global__ void k_fine_flux(const float *__restrict__ f, long long outer, int L, long long inner,
                            int periodic, int kick, int from_inner, long long cdiv, long long cmod,
                            const double *__restrict__ accel, double lo, double dvel, double dt,
                            double h, WPoly wp, int every, double *__restrict__ G, float alpha) {
    extern __shared__ double fx[];  // [L][blockDim] prefix sums (FP64)
    const long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int T = blockDim.x;
    const bool ok = line < outer * inner;
    const long long o = ok ? line / inner : 0, c = ok ? line % inner : 0;
    const float *base = f + o * L * inner + c;
    const long long cls = from_inner ? (c / cdiv) % cmod : o / cdiv;
    const double speed = kick ? accel[cls] : vp_core::cell_centre(lo, dvel, (int)cls);
    const LineShift<float> sh = vp_core::make_shift<float>(speed, dt, h, wp);
    const int sg = sh.sigma;
    // value of the line in the upwind frame (reversed when sigma < 0)
    auto val = [&](long long k) -> float {
        if (periodic) {
            k %= L;
            if (k < 0) k += L;
        } else if (k < 0 || k >= L) {
            return 0.f;
        }
        const long long kk = sg > 0 ? k : L - 1 - k;
        return base[kk * inner];
    };
    // prefix sums S(k) = sum_{m < k} u_m in the upwind frame
    double acc = 0.0;
    if (ok)
        for (int k = 0; k < L; ++k) {
            fx[k * T + threadIdx.x] = acc;
            acc += val(k);
        }
    const double total = acc;
    auto S = [&](long long k) -> double {  // sum_{m < k}, extended beyond the line
        if (periodic) {
            long long q = k / L, r = k % L;
            if (r < 0) {
                r += L;
                q -= 1;
            }
            return fx[r * T + threadIdx.x] + (double)q * total;
        }
        if (k <= 0) return 0.0;
        if (k >= L) return total;
        return fx[k * T + threadIdx.x];
    };
    if (!ok) return;
    const int n = sh.n * sg;  // whole cells swept, in the upwind frame (>= 0)
    const int nout = L / every + 1;
    for (int j = 0; j < nout; ++j) {
        // interface between cells (i - 1) and i of the original line, i = j * every
        const int i = j * every;
        // in the upwind frame the interface sits between cells ip - 1 and ip
        const int ip = sg > 0 ? i : L - i;
        // G' = sum_{m = ip - n}^{ip - 1} u_m + nu Phi(upwind cell ip - 1 - n)
        const long long up = (long long)ip - 1 - n;
        float u[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) u[k] = val(up - 3 + k);
        const float M = vp_core::flux<float, 7, true>(sh, u[0], u[1], u[2], u[3], u[4], u[5], u[6], alpha, 1, 1);
        const double g = (S(ip) - S(ip - n)) + (double)M;
        G[line * nout + j] = sg > 0 ? g : -g;
    }
}

// coarse state: mean over the (factor1 x factor2) fine velocity cells of a
// velocity grid [nf1][nf2] (nf2 = factor2 = 1 for one velocity dimension)
__global__ void k_restrict_v2(const float *__restrict__ ff, float *__restrict__ fc, long long NX, int nf1,
                              int nf2, int factor1, int factor2) {
    const int nc1 = nf1 / factor1, nc2 = nf2 / factor2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NX * nc1 * nc2) return;
    const long long x = t / (nc1 * nc2);
    const int J = (int)(t % (nc1 * nc2));
    const int J1 = J / nc2, J2 = J % nc2;
    double s = 0.0;
    for (int a = 0; a < factor1; ++a)
        for (int b = 0; b < factor2; ++b)
            s += ff[x * nf1 * nf2 + (long long)(J1 * factor1 + a) * nf2 + (J2 * factor2 + b)];
    fc[t] = (float)(s / (factor1 * factor2));
}

// Samples on coarse lines: for every coarse interface with |zeta| >= zmin,
// features of the coarse stencil and the normalised target
// y = (Phi_target - Phi_CSL7) / s.  Gc: coarse-unit masses through the
// coarse interfaces ([coarse line][L + 1]).  Invalid samples get y = NaN.
__global__ void k_make_samples(const float *__restrict__ fc, long long outer, int L, long long inner,
                               int periodic, int kick, int from_inner, long long cdiv, long long cmod,
                               const double *__restrict__ accel, double lo, double dvel, double dt,
                               double h, WPoly wp, const double *__restrict__ Gc, double zmin,
                               float *__restrict__ X, float *__restrict__ y, float *__restrict__ sc,
                               float alpha) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nlines = outer * inner;
    if (t >= nlines * (L + 1)) return;
    const long long line = t / (L + 1);
    const int i = (int)(t % (L + 1));  // interface between cells i - 1 and i
    const long long o = line / inner, c = line % inner;
    const float *base = fc + o * L * inner + c;
    const long long cls = from_inner ? (c / cdiv) % cmod : o / cdiv;
    const double speed = kick ? accel[cls] : vp_core::cell_centre(lo, dvel, (int)cls);
    const LineShift<float> sh = vp_core::make_shift<float>(speed, dt, h, wp);
    const double s_full = speed * dt / h;
    const double zeta = s_full - round(s_full);
    float *xo = X + t * NF;
    if (fabs(zeta) < zmin || (periodic && i == L)) {
        for (int k = 0; k < NF; ++k) xo[k] = 0.f;
        y[t] = __int_as_float(0x7fc00000);
        if (sc) sc[t] = 0.f;
        return;
    }
    const int sg = sh.sigma;
    auto val = [&](long long k) -> float {
        if (periodic) {
            k %= L;
            if (k < 0) k += L;
        } else if (k < 0 || k >= L) {
            return 0.f;
        }
        const long long kk = sg > 0 ? k : L - 1 - k;
        return base[kk * inner];
    };
    const int ip = sg > 0 ? i : L - i;
    const int n = sh.n * sg;
    const long long up = (long long)ip - 1 - n;
    float u[8], unp[8], unm[8];
    for (int k = 0; k < 8; ++k) u[k] = val(up - 3 + k);
    // velocity-neighbour lines of a spatial sweep (+: larger |v|), zero
    // outside the velocity box; none for a velocity sweep
    for (int k = 0; k < 8; ++k) unp[k] = unm[k] = 0.f;
    if (!kick) {
        const int sp = speed >= 0.0 ? 1 : -1;
        const long long J = (c / cdiv) % cmod;
        auto nval = [&](long long dj, long long k) -> float {
            const long long Jn = J + dj;
            if (Jn < 0 || Jn >= cmod) return 0.f;
            if (periodic) {
                k %= L;
                if (k < 0) k += L;
            } else if (k < 0 || k >= L) {
                return 0.f;
            }
            const long long kk = sg > 0 ? k : L - 1 - k;
            return base[kk * inner + dj * cdiv];
        };
        for (int k = 0; k < 8; ++k) {
            unp[k] = nval(sp, up - 3 + k);
            unm[k] = nval(-sp, up - 3 + k);
        }
    }
    // whole cells swept in the upwind frame, signed: sum_{m = ip - n}^{ip - 1} u_m
    // (n < 0 when the integer shift opposes the fractional one)
    double whole = 0.0;
    if (n >= 0)
        for (long long m = ip - n; m < ip; ++m) whole += val(m);
    else
        for (long long m = ip; m < ip - n; ++m) whole -= val(m);
    const double g = sg > 0 ? Gc[line * (L + 1) + i] : -Gc[line * (L + 1) + i];
    // coarse fractional mass as the plain sweep computes it: CSL7, then MP
    float phi = sh.w[0] * u[0];
    for (int k = 1; k < 7; ++k) phi = fmaf(sh.w[k], u[k], phi);
    phi = vp_core::mp_limit(phi, u[1], u[2], u[3], u[4], u[5], alpha);
    float x[NF];
    const float s = net_features(u, unp, unm, sh.nu, x);
    for (int k = 0; k < NF; ++k) xo[k] = x[k];
    y[t] = (float)((g - whole - (double)sh.nu * (double)phi) / (double)s);
    if (sc) sc[t] = s;
}

// cell pairs of the training loss: the residual of the cell between
// interfaces l and r is (s_r (g_r - y_r) - s_l (g_l - y_l)) / max(s_l, s_r),
// so the pair's coefficients are (-s_l / m, s_r / m), m = max(s_l, s_r); the
// draw weight of the pair is m^importance (1 for importance 0)
__global__ void k_pair_coefs(const float *__restrict__ sc, const long long *__restrict__ li,
                             const long long *__restrict__ ri, long long n, double importance,
                             float *__restrict__ coef, double *__restrict__ weight) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double sl = sc[li[t]], sr = sc[ri[t]];
    const double m = sl > sr ? sl : sr;
    coef[2 * t] = (float)(-(sl / m));
    coef[2 * t + 1] = (float)(sr / m);
    if (weight) weight[t] = importance > 0.0 ? pow(m, importance) : 1.0;
}

// coarse-interface masses from fine ones: mean over `group` fine lines of
// every fine value, scaled by `scale` (fine -> coarse cell units)
__global__ void k_group_mean(const double *__restrict__ Gf, long long ncl, int nout, const long long *map,
                             int group, double scale, double *__restrict__ Gc) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncl * nout) return;
    const long long cl = t / nout;
    const int j = (int)(t % nout);
    double s = 0.0;
    for (int g = 0; g < group; ++g) s += Gf[map[cl * group + g] * nout + j];
    Gc[t] = scale * s / group;
}

// ---- inference: the learned coarse sweep, network on the tensor cores -------------------
//
// A CTA stages a tile of lines of the drift along x_d in shared memory: all L
// cells of each line, for every velocity index j of the axis v_d (the line
// class) times a block of the other indices, so that the velocity neighbours
// of every line (j +- 1, the +/- lines of the features) are in the tile and no
// other CTA reads the tile's lines: the update is written to f in place,
// without a snapshot.  Each lane then walks one line upwind -> downwind as the
// plain line walker does (8-cell windows of the line and of its velocity
// difference and curvature in registers, one new row per interface, the MP
// curvature and d^{M4} carried), and at every interface the warp's 32 lanes
// form one 32-row feature tile for the network on the tensor cores.  The
// interface mass (plain MP mass plus s g, MP bounds when asked, PP) leaves the
// upwind cell and enters the next, so each cell is written once:
// f' = (u - M_out) + M_in.

constexpr int kTcThreads = 128;  // one line per thread, one 128-row MMA operand per interface step

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// bf16(max(lo, 0)) in the low half, bf16(max(hi, 0)) in the high half
__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// tile of a learned sweep: columns col = (g cmod + j) T + t hold the line with
// inner index c = c_tile + g cmod cdiv + j cdiv + t (class j); tiles per outer
// index: (inner / (G cmod cdiv)) (cdiv / T)
struct LTile {
    long long outer, inner, cdiv, cmod;
    int L, T, G, NC, pitch;  // NC = G cmod T columns, row pitch in floats
    long long tpo;           // tiles per outer index
    long long tblocks;       // t blocks per group block: cdiv / T
};

// Network operands for the tensor cores, prepared once per call from the
// FP32 master weights: W1, W2, W3 (32 outputs x 48 inputs) and w4 (row 0 of a
// 16 x 48 matrix) as bf16 in the canonical K-major layout.  Inputs 0-31 are
// the layer's inputs (W1 zero beyond its 25 features); every A row carries
// the constant 1 in columns 32 and 33, and the operands hold the bias there
// as a bf16 pair, b = bf16(b) + bf16(b - bf16(b)), so the accumulator starts
// from the bias to 16 significant bits and no epilogue adds it.
constexpr int kOpW = 32 * vp_umma::kK * 2;    // bytes of one 32-row bf16 operand
constexpr int kOpW4 = 16 * vp_umma::kK * 2;   // 16 rows
constexpr int kOpBytes = 3 * kOpW + kOpW4;
constexpr int kOpAlloc = (kOpBytes + 127) / 128 * 128;

__global__ void k_net_umma(const float *__restrict__ wts, unsigned char *__restrict__ out) {
    constexpr int K = vp_umma::kK;
    for (int e = threadIdx.x; e < 3 * 32 * K + 16 * K; e += blockDim.x) {
        int layer, n, k;
        if (e < 3 * 32 * K) {
            layer = e / (32 * K);
            n = (e / K) % 32;
            k = e % K;
        } else {
            layer = 3;
            n = (e - 3 * 32 * K) / K;
            k = (e - 3 * 32 * K) % K;
        }
        const int kin = layer == 0 ? NF : H;
        float w = 0.f, b = 0.f;
        if (layer < 3) {
            const int base = layer == 0 ? OFF_W1 : (layer == 1 ? OFF_W2 : OFF_W3);
            w = k < kin ? wts[base + n * kin + k] : 0.f;
            b = wts[(layer == 0 ? OFF_B1 : (layer == 1 ? OFF_B2 : OFF_B3)) + n];
        } else if (n == 0) {
            w = k < H ? wts[OFF_W4 + k] : 0.f;
            b = wts[OFF_B4];
        }
        const float bh = __bfloat162float(__float2bfloat16_rn(b));
        const float v = k < 32 ? w : k == 32 ? bh : k == 33 ? b - bh : 0.f;
        const uint32_t off = (uint32_t)(layer * kOpW) + vp_umma::kmajor_offset(n, k);
        *reinterpret_cast<__nv_bfloat16 *>(out + off) = __float2bfloat16_rn(v);
    }
}

constexpr int kABytes = 128 * vp_umma::kK * 2;  // one 128 x 48 bf16 feature operand
// interfaces per line in one network batch: three operands and the weights
// take 46.5 KB of shared memory and 128 tensor-memory columns, so four CTAs
// share an SM (all 512 columns)
constexpr int kLC = 3;
// tensor-memory columns of a CTA: the power of two >= 32 that holds LC
// accumulators of 32 columns
__host__ __device__ constexpr uint32_t tmem_cols(int lc) {
    return lc <= 1 ? 32u : (lc <= 2 ? 64u : (lc <= 4 ? 128u : 256u));
}

// bf16 columns 0-31 of row r (in w) of an operand in the canonical layout
__device__ __forceinline__ void store_row(unsigned char *op, int r, const uint32_t (&w)[16]) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
        *reinterpret_cast<uint4 *>(op + vp_umma::kmajor_offset(r, 8 * kk)) =
            make_uint4(w[4 * kk], w[4 * kk + 1], w[4 * kk + 2], w[4 * kk + 3]);
}

// The three hidden layers and the output layer for `nb` operands of 128
// feature rows (operand b at A + b kABytes, accumulator columns 32 b .. 32 b
// + 31), on the tensor cores: one thread issues each layer's MMAs (three
// k-blocks of 16) and commits them to the mbarrier; every thread then reads
// its own row back from tensor memory, applies ReLU, rounds to bf16 and
// writes it as the next layer's A row.  Returns g of this thread's row of
// each operand.  Bounded waits: on a timeout the status word is set.
template <int LC>
__device__ __forceinline__ void net_tc(unsigned char *A, const unsigned char *ops, uint32_t tmem, uint64_t *bar,
                                       uint32_t &phase, int nb, float (&g)[LC], int *status) {
    const int warp = threadIdx.x >> 5;
    const uint32_t a_s = vp_tma::saddr(A), w_s = vp_tma::saddr(ops);
    const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
    for (int layer = 0; layer < 4; ++layer) {
        vp_umma::fence_proxy_async();
        vp_umma::fence_before_sync();
        __syncthreads();
        if (threadIdx.x == 0) {
            vp_umma::fence_after_sync();
            const uint32_t idesc = vp_umma::idesc_bf16_f32(128, layer < 3 ? 32 : 16);
            const uint64_t bd = vp_umma::smem_desc(w_s + (uint32_t)(layer * kOpW), 128, vp_umma::kSBO);
            for (int b = 0; b < nb; ++b) {
                const uint64_t ad = vp_umma::smem_desc(a_s + (uint32_t)(b * kABytes), 128, vp_umma::kSBO);
#pragma unroll
                for (int s = 0; s < vp_umma::kK / 16; ++s)  // 256 bytes per k-block: 16 to the address field
                    vp_umma::mma_bf16(tmem + (uint32_t)(32 * b), ad + (uint64_t)(16 * s), bd + (uint64_t)(16 * s),
                                      idesc, (uint32_t)s);
            }
            vp_umma::commit(bar);
        }
        const bool done = vp_tma::mbar_wait(bar, phase, 1u << 24);
        phase ^= 1u;
        if (!done) atomicExch(status, VP_ETIMEOUT);
        vp_umma::fence_after_sync();
        if (layer < 3) {
            for (int b = 0; b < nb; ++b) {
                float v[32];
                vp_umma::ld32(tl + (uint32_t)(32 * b), v);
                uint32_t w[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) w[i] = pack_relu_bf16(v[2 * i], v[2 * i + 1]);
                store_row(A + b * kABytes, threadIdx.x, w);
            }
        } else {
#pragma unroll
            for (int b = 0; b < LC; ++b) g[b] = b < nb ? vp_umma::ld1(tl + (uint32_t)(32 * b)) : 0.f;
        }
    }
}

// Reads f^n (fin, not written during the launch) through L2 and writes the
// updated lines to fout; a thread reads its line and the two lines of the
// neighbouring velocity cells row by row as it walks.
template <bool PERIODIC, int LC>
__global__ void __launch_bounds__(kTcThreads) k_learned_walk(const float *__restrict__ fin, float *__restrict__ fout,
                                                             LTile tl, const LineShift<float> *__restrict__ tab,
                                                             const uint4 *__restrict__ netops, double lo,
                                                             double dvel, float alpha, int mode,
                                                             int *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    unsigned char *A = tsm;                                // LC operands of 128 x 48 bf16
    unsigned char *ops = tsm + LC * kABytes;               // W1 W2 W3 w4, biases
    const int L = tl.L, NC = tl.NC, T = tl.T;
    const int cmod = (int)tl.cmod;
    const long long o = (long long)blockIdx.x / tl.tpo;
    const long long tin = (long long)blockIdx.x - o * tl.tpo;
    const long long gb = tin / tl.tblocks, tb = tin - gb * tl.tblocks;
    // inner index of column col
    auto col_c = [&](int col) -> long long {
        const int t = col % T, jg = col / T;
        const int j = jg % cmod, g = jg / cmod;
        return (gb * tl.G + g) * tl.cmod * tl.cdiv + (long long)j * tl.cdiv + tb * T + t;
    };
    const long long obase = o * (long long)L * tl.inner;
    // phase 0: network operands, tensor memory, mbarrier
    for (int e = threadIdx.x; e < kOpAlloc / 16; e += blockDim.x)
        reinterpret_cast<uint4 *>(ops)[e] = netops[e];
    // columns 32-47 of every A row: 1, 1 (the bias pair), then zeros
    for (int b = 0; b < LC; ++b)
#pragma unroll
        for (int kk = 4; kk < vp_umma::kK / 8; ++kk)
            *reinterpret_cast<uint4 *>(A + b * kABytes + vp_umma::kmajor_offset(threadIdx.x, 8 * kk)) =
                kk == 4 ? make_uint4(pack_bf16(1.f, 1.f), 0u, 0u, 0u) : make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x < 32) vp_umma::tmem_alloc(&tslot, tmem_cols(LC));
    if (threadIdx.x == 0) {
        vp_tma::mbar_init(&bar, 1);
        vp_tma::fence_mbar_init();
    }
    vp_umma::fence_before_sync();
    __syncthreads();
    vp_umma::fence_after_sync();
    const uint32_t tmem = tslot;
    uint32_t phase = 0;
    const int col = threadIdx.x;
    const bool ok = col < NC;
    const int colc = ok ? col : 0;
    // the line's shift and its velocity neighbours (+: larger |v|)
    const int j = (colc / T) % cmod;
    const LineShift<float> sh = tab[j];
    const int sg = sh.sigma;
    const float nu = sh.nu;
    const int sp = vp_core::cell_centre(lo, dvel, j) >= 0.0 ? 1 : -1;
    const int cp = (j + sp >= 0 && j + sp < cmod) ? colc + sp * T : -1;
    const int cm = (j - sp >= 0 && j - sp < cmod) ? colc - sp * T : -1;
    int n = sh.n;
    if (PERIODIC) {  // the shift modulo L
        n %= L;
        if (n < 0) n += L;
    }
    // source row of the upwind cell of interface 0 (the cell before the
    // walk's first cell), unwrapped for zero-inflow lines
    const int q = (sg > 0 ? 0 : L - 1) - n - sg;
    auto wrap = [&](int r) -> int {
        if (PERIODIC) {
            r %= L;
            if (r < 0) r += L;
        }
        return r;
    };
    // the line and its velocity neighbours in f^n (row r at r inner)
    const float *pu = fin + obase + col_c(colc);
    const float *pp = fin + obase + col_c(cp >= 0 ? cp : colc);
    const float *pm = fin + obase + col_c(cm >= 0 ? cm : colc);
    // cell value, velocity difference and velocity curvature at row r (wrapped
    // for periodic lines; outside [0, L) zero for zero-inflow lines)
    auto fetch_w = [&](int r, float &u, float &dv, float &cv) {
        const bool in = ok && (PERIODIC || (r >= 0 && r < L));
        const long long o = (long long)r * tl.inner;
        u = in ? __ldg(pu + o) : 0.f;
        const float up = in && cp >= 0 ? __ldg(pp + o) : 0.f;
        const float um = in && cm >= 0 ? __ldg(pm + o) : 0.f;
        dv = up - um;
        cv = fmaf(0.5f, up + um, -u);
    };
    float u[8], dv[8], cv[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) fetch_w(wrap(q + (m - 3) * sg), u[m], dv[m], cv[m]);
    // the row entering the window after interface k: q + (5 + k) sg, wrapped
    // incrementally.  Rows enter as raw values (u, u+, u-) loaded one batch
    // ahead: the next batch's rows are requested before this batch's network
    // round trips, which hide the L2 latency.
    int rn = wrap(q + 5 * sg);
    auto load_raw = [&](float &a, float &ap, float &am) {
        const bool in = ok && (PERIODIC || (rn >= 0 && rn < L));
        const long long o = (long long)rn * tl.inner;
        a = in ? __ldg(pu + o) : 0.f;
        ap = in && cp >= 0 ? __ldg(pp + o) : 0.f;
        am = in && cm >= 0 ? __ldg(pm + o) : 0.f;
        rn += sg;
        if (PERIODIC) {
            rn = rn == L ? 0 : rn;
            rn = rn < 0 ? L - 1 : rn;
        }
    };
    float ru[LC], rp[LC], rm[LC];
#pragma unroll
    for (int b = 0; b < LC; ++b) load_raw(ru[b], rp[b], rm[b]);
    // MP carries: curvature of the upwind cell, d^{M4} at its upwind face
    float dc = vp_core::curv(u[2], u[3], u[4]);
    float m4m = vp_core::dm4(vp_core::curv(u[1], u[2], u[3]), dc);
    float Min = 0.f;
    const long long cbase = obase + col_c(colc);
#pragma unroll 1
    for (int k0 = 0; k0 <= L; k0 += LC) {
        const int nb = L + 1 - k0 < LC ? L + 1 - k0 : LC;
        float xu[LC], xp[LC], xm[LC];  // the next batch's rows
#pragma unroll
        for (int b = 0; b < LC; ++b) load_raw(xu[b], xp[b], xm[b]);
        float Mp[LC], sc[LC], mlo[LC], mhi[LC], u3[LC], u4[LC];
#pragma unroll
        for (int b = 0; b < LC; ++b) {
            if (b >= nb) break;
            // plain mass of interface k0 + b (CSL7, MP bounds as a clamp)
            const float dp = vp_core::curv(u[3], u[4], u[5]);
            const float m4p = vp_core::dm4(dc, dp);
            float phi = sh.w[0] * u[0];
#pragma unroll
            for (int m = 1; m < 7; ++m) phi = fmaf(sh.w[m], u[m], phi);
            vp_core::mp_lohi_carried(u[2], u[3], u[4], alpha, m4m, m4p, mlo[b], mhi[b]);
            Mp[b] = vp_core::mul_rn(nu, fminf(fmaxf(phi, mlo[b]), mhi[b]));
            u3[b] = u[3];
            u4[b] = u[4];
            // feature row (columns 0-7 stencil, 8-15 velocity difference,
            // 16-23 velocity curvature, 24 nu, 25-31 zero), as net_features
            float s = 0.f;
#pragma unroll
            for (int m = 0; m < 8; ++m) s = fmaxf(s, fabsf(u[m]));
            s += 1e-30f;
            sc[b] = s;
            const float inv = 1.0f / s;
            const float hinv = 0.5f * inv;
            uint32_t w[16];
#pragma unroll
            for (int m = 0; m < 4; ++m) w[m] = pack_bf16((u[2 * m] - u[3]) * inv, (u[2 * m + 1] - u[3]) * inv);
            w[1] = pack_bf16((u[2] - u[3]) * inv, 0.f);
#pragma unroll
            for (int m = 0; m < 4; ++m) w[4 + m] = pack_bf16(dv[2 * m] * hinv, dv[2 * m + 1] * hinv);
#pragma unroll
            for (int m = 0; m < 4; ++m) w[8 + m] = pack_bf16(cv[2 * m] * inv, cv[2 * m + 1] * inv);
            w[12] = pack_bf16(nu, 0.f);
            w[13] = w[14] = w[15] = 0u;
            store_row(A + b * kABytes, threadIdx.x, w);
            // advance the window and the MP carries
            dc = dp;
            m4m = m4p;
            const float un = ru[b], dvn = rp[b] - rm[b], cvn = fmaf(0.5f, rp[b] + rm[b], -un);
#pragma unroll
            for (int m = 0; m < 7; ++m) {
                u[m] = u[m + 1];
                dv[m] = dv[m + 1];
                cv[m] = cv[m + 1];
            }
            u[7] = un;
            dv[7] = dvn;
            cv[7] = cvn;
        }
        float g[LC];
        net_tc<LC>(A, ops, tmem, &bar, phase, nb, g, status);
#pragma unroll
        for (int b = 0; b < LC; ++b) {
            ru[b] = xu[b];
            rp[b] = xp[b];
            rm[b] = xm[b];
        }
#pragma unroll
        for (int b = 0; b < LC; ++b) {
            if (b >= nb) break;
            float M = fmaf(sc[b], g[b], Mp[b]);
            if (mode == 2) M = fminf(fmaxf(M, vp_core::mul_rn(nu, mlo[b])), vp_core::mul_rn(nu, mhi[b]));
            M = vp_core::pp_clamp(M, vp_core::half_rd(u3[b]), vp_core::half_rd(u4[b]));
            // the cell whose source is u3 takes M in from the previous interface
            const int k = k0 + b;
            if (ok && k >= 1) {
                const int i = sg > 0 ? k - 1 : L - k;
                fout[cbase + (long long)i * tl.inner] = (u3[b] - M) + Min;
            }
            Min = M;
        }
    }
    vp_umma::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        vp_umma::fence_after_sync();
        vp_umma::tmem_dealloc(tmem, tmem_cols(LC));
    }
}

}  // namespace

// ---- host entry points ------------------------------------------------------------------

extern "C" {

int vp_net_grad(const float *X, const float *y, const float *coef, long long nsamp, int group, const float *wts,
                float *grad, float *loss, void *stream) {
    if (!X || !y || !wts || !grad || !loss || nsamp < 1 || (group != 1 && group != 2) || nsamp % group)
        return VP_EINVAL;
    const long long blocks = (nsamp + kTrainThreads - 1) / kTrainThreads;
    k_net_grad<<<(unsigned)blocks, kTrainThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        X, y, coef, wts, nsamp, group, grad, loss);
    return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ECUDA;
}

int vp_net_adam(float *wts, float *m, float *v, float *grad, int step, float lr, void *stream) {
    if (!wts || !m || !v || !grad || step < 1 || !(lr > 0.f)) return VP_EINVAL;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    k_adam<<<(NPARAM + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(wts, m, v, grad, NPARAM, lr, b1,
                                                                               b2, 1e-8f, bc1, bc2);
    return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ECUDA;
}

}  // extern "C"

// geometry helpers shared with the context-level entry points below
namespace {
struct LineGeo {
    long long outer, inner;
    int L, periodic, kick, from_inner;
    long long cdiv, cmod;
    double lo, dvel, h;
};

LineGeo line_geo(const vp_grid &g, long long NX, long long NV, int kick, int dim) {
    LineGeo q{};
    if (!kick) {
        long long outer = 1, inner = NV, vstride = 1;
        for (int k = 0; k < dim; ++k) outer *= g.nx[k];
        for (int k = dim + 1; k < g.dx; ++k) inner *= g.nx[k];
        for (int k = dim + 1; k < g.dv; ++k) vstride *= g.nv[k];
        q.outer = outer;
        q.inner = inner;
        q.L = g.nx[dim];
        q.periodic = g.xbc == VP_BC_PERIODIC;
        q.from_inner = 1;
        q.cdiv = vstride;
        q.cmod = g.nv[dim];
        q.h = (g.xhi[dim] - g.xlo[dim]) / g.nx[dim];
    } else {
        long long vouter = 1, inner = 1;
        for (int k = 0; k < dim; ++k) vouter *= g.nv[k];
        for (int k = dim + 1; k < g.dv; ++k) inner *= g.nv[k];
        q.outer = NX * vouter;
        q.inner = inner;
        q.L = g.nv[dim];
        q.periodic = 0;
        q.from_inner = 0;
        q.cdiv = vouter;
        q.cmod = 1;
        q.h = (g.vhi[dim] - g.vlo[dim]) / g.nv[dim];
    }
    q.kick = kick;
    q.lo = g.vlo[dim];
    q.dvel = (g.vhi[dim] - g.vlo[dim]) / g.nv[dim];
    return q;
}
}  // namespace

int vp_learned_prepare(vp_ctx *c) {
    if (c->learned_ready) return VP_OK;
    if (!c->d_netfrag) VP_CUDA_TRY(c, cudaMalloc(&c->d_netfrag, kOpAlloc));
    // the updated lines of a learned sweep (copied back into f after the walk)
    if (!c->d_learn_out) VP_CUDA_TRY(c, cudaMalloc(&c->d_learn_out, (size_t)c->ncell * sizeof(float)));
    VP_CUDA_TRY(c, cudaFuncSetAttribute(k_learned_walk<true, kLC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        200 * 1024));
    VP_CUDA_TRY(c, cudaFuncSetAttribute(k_learned_walk<false, kLC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        200 * 1024));
    c->learned_ready = 1;
    return VP_OK;
}

// one learned drift along dim from fin (f^n, not written) to fout; with
// net = true the network operands are made from wts first (a stage of
// several drifts with one network makes them once)
int vp_learned_drift_io(vp_ctx *c, int dim, double dt, const float *wts, int use_net, const float *fin,
                        float *fout, bool net) {
    const LineGeo q = line_geo(c->g, c->NX, c->NV, 0, dim);
    // tile: every class j of its lines times a block of the other indices,
    // about 128 lines (columns)
    LTile tl{};
    tl.outer = q.outer;
    tl.inner = q.inner;
    tl.cdiv = q.cdiv;
    tl.cmod = q.cmod;
    tl.L = q.L;
    const long long NG = q.inner / (q.cmod * q.cdiv);
    const int target = 128;
    if (q.cmod > kTcThreads)
        return vp_fail(c, VP_ENOTSUP, "more than %d velocity cells on the sweep's axis", kTcThreads);
    if (q.cmod * q.cdiv <= target) {
        tl.T = (int)q.cdiv;
        long long G = target / (q.cmod * q.cdiv);
        while (G > 1 && NG % G) --G;
        tl.G = (int)(G < 1 ? 1 : G);
    } else {
        tl.G = 1;
        long long T = target / q.cmod;
        if (T < 1) T = 1;
        while (T > 1 && q.cdiv % T) --T;
        tl.T = (int)T;
    }
    tl.NC = (int)(tl.G * q.cmod * tl.T);
    tl.pitch = 0;
    tl.tblocks = q.cdiv / tl.T;
    tl.tpo = (NG / tl.G) * tl.tblocks;
    const int threads = kTcThreads;  // one 128-row operand: a thread per row, rows >= NC are idle
    const size_t smem = (size_t)kLC * kABytes + kOpAlloc;
    const long long blocks = q.outer * tl.tpo;
    if (blocks >= (1LL << 31)) return vp_fail(c, VP_ENOTSUP, "learned sweep has too many tiles");
    int rc = vp_launch_shift_table(c, 0, dim, dt, nullptr);
    if (rc != VP_OK) return rc;
    if (net) {
        k_net_umma<<<1, 256, 0, c->stream>>>(wts, static_cast<unsigned char *>(c->d_netfrag));
        c->launches++;
    }
    const LineShift<float> *tab = static_cast<const LineShift<float> *>(c->d_shift);
    const uint4 *ops = static_cast<const uint4 *>(c->d_netfrag);
    if (q.periodic)
        k_learned_walk<true, kLC><<<(unsigned)blocks, threads, smem, c->stream>>>(
            fin, fout, tl, tab, ops, q.lo, q.dvel, (float)c->g.alpha, use_net, c->d_status);
    else
        k_learned_walk<false, kLC><<<(unsigned)blocks, threads, smem, c->stream>>>(
            fin, fout, tl, tab, ops, q.lo, q.dvel, (float)c->g.alpha, use_net, c->d_status);
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

extern "C" {

int vp_learned_sweep(vp_ctx *c, int kick, int dim, double dt, const double *accel_dev, const float *wts,
                     int use_net, const float *f_snap) {
    (void)f_snap;  // the walk reads f^n as it is and writes the new lines to a buffer of its own
    if (!c || !c->f) return VP_EINVAL;
    if (c->g.precision != VP_F32 || c->g.order != 7)
        return vp_fail(c, VP_ENOTSUP, "the learned sweep runs on FP32 CSL7 grids");
    if (use_net < 0 || use_net > 2) return vp_fail(c, VP_EINVAL, "use_net must be 0, 1 or 2");
    if (use_net && kick) return vp_fail(c, VP_ENOTSUP, "the learned correction applies to spatial sweeps");
    if (dim < 0 || dim >= c->g.dx || (kick && !accel_dev) || (use_net && !wts) || !std::isfinite(dt))
        return vp_fail(c, VP_EINVAL, "bad learned-sweep arguments");
    if (!use_net) return kick ? vp_kick_sweep(c, dim, dt, accel_dev) : vp_drift_sweep(c, dim, dt);
    int rc = vp_learned_prepare(c);
    if (rc != VP_OK) return rc;
    float *fout = static_cast<float *>(c->d_learn_out);
    if ((rc = vp_learned_drift_io(c, dim, dt, wts, use_net, static_cast<const float *>(c->f), fout, true)))
        return rc;
    VP_CUDA_TRY(c, cudaMemcpyAsync(c->f, fout, (size_t)c->ncell * sizeof(float), cudaMemcpyDeviceToDevice,
                                   c->stream));
    return VP_OK;
}

int vp_fine_flux(vp_ctx *c, int kick, int dim, double dt, const double *accel_dev, int every,
                 double *G_dev) {
    if (!c || !c->f || !G_dev || every < 1) return VP_EINVAL;
    if (c->g.precision != VP_F32 || c->g.order != 7)
        return vp_fail(c, VP_ENOTSUP, "fine fluxes are computed for FP32 CSL7 grids");
    if (dim < 0 || dim >= c->g.dx || (kick && !accel_dev)) return vp_fail(c, VP_EINVAL, "bad fine-flux arguments");
    const LineGeo q = line_geo(c->g, c->NX, c->NV, kick, dim);
    if (q.L % every) return vp_fail(c, VP_EINVAL, "line length must be a multiple of `every`");
    const int T = 64;
    const size_t smem = (size_t)q.L * T * sizeof(double);
    if (smem > 200 * 1024) return vp_fail(c, VP_ENOTSUP, "line too long");
    cudaFuncSetAttribute(k_fine_flux, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    const long long nl = q.outer * q.inner;
    k_fine_flux<<<(unsigned)((nl + T - 1) / T), T, smem, c->stream>>>(
        static_cast<const float *>(c->f), q.outer, q.L, q.inner, q.periodic, kick, q.from_inner, q.cdiv, q.cmod,
        accel_dev, q.lo, q.dvel, dt, q.h, c->wp, every, G_dev, (float)c->g.alpha);
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

int vp_restrict_velocity(const float *f_fine, float *f_coarse, long long NX, int nf1, int nf2, int factor1,
                         int factor2, void *stream) {
    if (!f_fine || !f_coarse || factor1 < 1 || factor2 < 1 || nf1 % factor1 || nf2 % factor2) return VP_EINVAL;
    const long long n = NX * (nf1 / factor1) * (nf2 / factor2);
    k_restrict_v2<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        f_fine, f_coarse, NX, nf1, nf2, factor1, factor2);
    return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ECUDA;
}

int vp_pair_coefs(const float *sc, const long long *li, const long long *ri, long long n, double importance,
                  float *coef, double *weight, void *stream) {
    if (!sc || !li || !ri || !coef || n < 0 || !(importance >= 0.0)) return VP_EINVAL;
    if (n == 0) return VP_OK;
    k_pair_coefs<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(sc, li, ri, n,
                                                                                            importance, coef, weight);
    return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ECUDA;
}

int vp_group_mean(const double *G_fine, long long n_coarse_lines, int nout, const long long *map_dev,
                  int group, double scale, double *G_coarse, void *stream) {
    if (!G_fine || !map_dev || !G_coarse || group < 1 || nout < 1) return VP_EINVAL;
    const long long n = n_coarse_lines * nout;
    k_group_mean<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        G_fine, n_coarse_lines, nout, map_dev, group, scale, G_coarse);
    return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ECUDA;
}

// Fine lines aggregated by every coarse line of a sweep, for a coarse grid
// whose velocity cells are factor^D fine cells (same spatial grid).
int vp_fluxnet_line_map(const vp_grid *fine, const vp_grid *coarse, int factor, int kick, int dim,
                        long long *map_host, long long *n_coarse_lines, int *group) {
    if (!fine || !coarse || factor < 1 || fine->dx != coarse->dx || fine->dx < 1 || fine->dx > 2) return VP_EINVAL;
    const int D = fine->dx;
    long long NXf = 1, NVf = 1, NVc = 1;
    for (int k = 0; k < D; ++k) {
        if (fine->nx[k] != coarse->nx[k] || fine->nv[k] != factor * coarse->nv[k]) return VP_EINVAL;
        NXf *= fine->nx[k];
        NVf *= fine->nv[k];
        NVc *= coarse->nv[k];
    }
    const LineGeo qc = line_geo(*coarse, NXf, NVc, kick, dim);
    const LineGeo qf = line_geo(*fine, NXf, NVf, kick, dim);
    const long long ncl = qc.outer * qc.inner;
    // velocity cells of the coarse line's other axes, expanded
    int g = 1;
    for (int k = 0; k < D; ++k)
        if (!(kick && k == dim)) g *= factor;
    if (n_coarse_lines) *n_coarse_lines = ncl;
    if (group) *group = g;
    if (!map_host) return VP_OK;
    for (long long cl = 0; cl < ncl; ++cl) {
        const long long O = cl / qc.inner, C = cl % qc.inner;
        // full coarse index of the line's first cell, decomposed [x..][J..]
        const long long lin = O * (long long)qc.L * qc.inner + C;
        long long x = lin / NVc, J = lin % NVc;
        int Jv[2] = {0, 0};
        for (int k = D - 1; k >= 0; --k) {
            Jv[k] = (int)(J % coarse->nv[k]);
            J /= coarse->nv[k];
        }
        int idx = 0;
        for (int a = 0; a < (D > 0 ? factor : 1); ++a)
            for (int b = 0; b < (D > 1 ? factor : 1); ++b) {
                int jf[2] = {Jv[0] * factor + a, D > 1 ? Jv[1] * factor + b : 0};
                // along the swept velocity axis every fine line starts at cell 0
                if (kick) {
                    if (dim == 0 && a) continue;
                    if (dim == 1 && b) continue;
                    jf[dim] = 0;
                }
                long long jl = 0;
                for (int k = 0; k < D; ++k) jl = jl * fine->nv[k] + jf[k];
                const long long flin = x * NVf + jl;  // fine index of the line's first cell
                const long long Of = flin / ((long long)qf.L * qf.inner);
                const long long Cf = flin % qf.inner;
                map_host[cl * g + idx++] = Of * qf.inner + Cf;
            }
    }
    return VP_OK;
}

int vp_make_samples(vp_ctx *coarse, int kick, int dim, double dt, const double *accel_dev,
                    const double *Gc_dev, double zmin, float *X_dev, float *y_dev, float *scale_dev) {
    vp_ctx *c = coarse;
    if (!c || !c->f || !Gc_dev || !X_dev || !y_dev) return VP_EINVAL;
    if (dim < 0 || dim >= c->g.dx || (kick && !accel_dev)) return vp_fail(c, VP_EINVAL, "bad sample arguments");
    const LineGeo q = line_geo(c->g, c->NX, c->NV, kick, dim);
    const long long n = q.outer * q.inner * (q.L + 1);
    k_make_samples<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(
        static_cast<const float *>(c->f), q.outer, q.L, q.inner, q.periodic, kick, q.from_inner, q.cdiv, q.cmod,
        accel_dev, q.lo, q.dvel, dt, q.h, c->wp, Gc_dev, zmin, X_dev, y_dev, scale_dev, (float)c->g.alpha);
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

}  // extern "C"
