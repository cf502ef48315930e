// vp_fluxnet.cu -- learned flux correction on a coarser velocity grid
// (a spec addition to the method, not in the paper).
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
    for (int k = 0; k < 8; ++k) x[16 + k] = (0.5f * (up[k] + um[k]) - u[k]) * inv;
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
// A CTA takes NL consecutive lines of the sweep.  Phase 0 stages the lines
// and, from the snapshot, their velocity-difference lines (u+ - u-) / 2 and
// velocity-curvature lines (u+ + u-) / 2 - u in shared memory (consecutive
// threads read consecutive lines: coalesced for strided sweeps), with the
// lines' shift decompositions.  Phase 1 computes every interface's limited
// mass: the plain MP mass, plus s g from the network on the tensor cores
// (described at the loop), then (use_net = 2) the MP bounds, and the PP
// limiter.  Phase 2: one thread per
// cell writes the flux-form update.  Interface k of a line is the k-th one
// the upwind walk meets: its upwind cell is q_k = q_0 + k sigma,
// q_0 = (sigma > 0 ? 0 : L - 1) - n - sigma; the k-th cell of the walk
// (k >= 1) takes M_{k-1} in and M_k out.

constexpr int kTcThreads = 128;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// D = A B + C with C = (c.x, c.y) in both row halves of the lane's fragment
__device__ __forceinline__ void mma_bf16_c(float (&d)[4], const uint32_t (&a)[4], uint2 b, float2 c) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%10,%11};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y), "f"(c.x), "f"(c.y));
}

// bf16(max(lo, 0)) in the low half, bf16(max(hi, 0)) in the high half
__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// four 8x8 bf16 matrices from shared memory, one row address per lane
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr)
                 : "memory");
}

// ReLU, round to bf16 and re-pack accumulators as the next layer's A fragments
__device__ __forceinline__ void relu_pack(const float (&acc)[4][4], uint32_t (&a)[2][4]) {
#pragma unroll
    for (int kb = 0; kb < 2; ++kb) {
        a[kb][0] = pack_relu_bf16(acc[2 * kb][0], acc[2 * kb][1]);
        a[kb][1] = pack_relu_bf16(acc[2 * kb][2], acc[2 * kb][3]);
        a[kb][2] = pack_relu_bf16(acc[2 * kb + 1][0], acc[2 * kb + 1][1]);
        a[kb][3] = pack_relu_bf16(acc[2 * kb + 1][2], acc[2 * kb + 1][3]);
    }
}

// per-line data of a learned-sweep CTA
struct LLine {
    long long base;  // offset of row 0
    int sp;          // +1 / -1: the velocity neighbour with larger |v| is at +sp
    int has_p, has_m;
    int q0;          // upwind cell of the walk's first interface (unwrapped)
};

constexpr int kLG = 8;   // staged rows on each side of a learned-sweep line
constexpr int kFS = 80;  // bytes per feature row (32 bf16 + 16 pad: conflict-free ldmatrix)

// network weights in the order the learned sweep keeps them in shared memory:
// B fragments of the three hidden layers [layer][k block][n tile][lane][2],
// the w4 fragments [k block][lane] (w4 in column 0 of B), then b1 b2 b3,
// bf16(w4) and b4 (129 floats, padded to 132)
constexpr int kFragWords = 3 * 2 * 4 * 32 * 2 + 2 * 32 * 2 + 132;
static_assert(kFragWords % 4 == 0, "fragment block is copied in 16-byte units");

__global__ void k_net_frags(const float *__restrict__ wts, uint32_t *__restrict__ out) {
    uint2 *w4f = reinterpret_cast<uint2 *>(out + 3 * 2 * 4 * 32 * 2);
    float *wvec = reinterpret_cast<float *>(w4f + 2 * 32);
    for (int e = threadIdx.x; e < 3 * 2 * 4 * 32; e += blockDim.x) {
        const int lane = e & 31, frag = e >> 5;  // frag = (layer * 2 + kb) * 4 + nt
        const int nt = frag & 3, kb = (frag >> 2) & 1, layer = frag >> 3;
        const int off = layer == 0 ? OFF_W1 : (layer == 1 ? OFF_W2 : OFF_W3);
        const int kin = layer == 0 ? NF : H;
        const int n = 8 * nt + (lane >> 2), k0 = 16 * kb + 2 * (lane & 3), k1 = k0 + 8;
        auto wv = [&](int k) { return k < kin ? wts[off + n * kin + k] : 0.f; };
        out[2 * e] = pack_bf16(wv(k0), wv(k0 + 1));
        out[2 * e + 1] = pack_bf16(wv(k1), wv(k1 + 1));
    }
    for (int e = threadIdx.x; e < 2 * 32; e += blockDim.x) {
        const int lane = e & 31, kb = e >> 5, k0 = 16 * kb + 2 * (lane & 3);
        const float *w4 = wts + OFF_W4;
        w4f[e] = (lane >> 2) == 0 ? make_uint2(pack_bf16(w4[k0], w4[k0 + 1]), pack_bf16(w4[k0 + 8], w4[k0 + 9]))
                                  : make_uint2(0u, 0u);
    }
    for (int e = threadIdx.x; e < 132; e += blockDim.x) {
        const int grp = e / H, n = e - grp * H;
        wvec[e] = grp == 0   ? wts[OFF_B1 + n]
                  : grp == 1 ? wts[OFF_B2 + n]
                  : grp == 2 ? wts[OFF_B3 + n]
                  : grp == 3 ? bfr(wts[OFF_W4 + n])
                  : e == 4 * H ? wts[OFF_B4]
                               : 0.f;
    }
}

// divisors of the line index (host-precomputed; used when every line index fits 32 bits)
struct LineDiv {
    FastDiv inner, cdiv, cmod;
    int fast;
};

template <bool PERIODIC>
__global__ void __launch_bounds__(kTcThreads) k_learned_sweep(float *__restrict__ f, long long outer, int L,
                                                              long long inner, int from_inner, long long cdiv,
                                                              long long cmod,
                                                              const LineShift<float> *__restrict__ tab,
                                                              const uint4 *__restrict__ netfrag, double lo,
                                                              double dvel, float alpha,
                                                              int use_net, const float *__restrict__ fsnap,
                                                              int lgNL, LineDiv ldv) {
    extern __shared__ __align__(16) unsigned char tsm[];
    const int NL = 1 << lgNL;
    const int NI = NL * (L + 1);  // interface e = k * NL + l (line l, k-th interface of its walk)
    const int LP = L + 2 * kLG;   // staged rows: -kLG .. L + kLG - 1
    uint32_t *wfrag = reinterpret_cast<uint32_t *>(tsm);  // [3][2][4][32 lanes][2] B fragments
    uint2 *w4f = reinterpret_cast<uint2 *>(wfrag + 3 * 2 * 4 * 32 * 2);  // [2][32 lanes] w4 in column 0
    float *wvec = reinterpret_cast<float *>(w4f + 2 * 32);  // b1 b2 b3 w4(bf16) b4: 129
    LineShift<float> *shs = reinterpret_cast<LineShift<float> *>(wvec + 132);
    LLine *lls = reinterpret_cast<LLine *>(shs + NL);
    float *lines = reinterpret_cast<float *>(lls + NL);  // [LP][NL], row r at (r + kLG)
    float *dvl = lines + NL * LP;                         // [LP][NL] velocity differences
    float *cvl = dvl + NL * LP;                           // [LP][NL] velocity curvatures
    float *mass = cvl + NL * LP;                          // [L + 1][NL] interface masses
    // per warp: 32 feature rows of kFS bytes
    unsigned char *fbuf = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(mass + (size_t)NL * (L + 1)) + 15) & ~static_cast<uintptr_t>(15));
    const long long nlines = outer * inner;
    const long long l0 = (long long)blockIdx.x * NL;
    const int nl = (int)(nlines - l0 < NL ? nlines - l0 : NL);
    // phase 0: network fragments, per-line data, then the lines and their
    // velocity-difference and velocity-curvature lines
    if (use_net) {
        uint4 *dst = reinterpret_cast<uint4 *>(tsm);
        for (int e = threadIdx.x; e < kFragWords / 4; e += blockDim.x) dst[e] = netfrag[e];
    }
    for (int l = threadIdx.x; l < NL; l += blockDim.x) {
        LLine ll{0, 1, 0, 0, 0};
        LineShift<float> sh{};
        sh.sigma = 1;
        if (l < nl) {
            const long long line = l0 + l;
            long long o, c, cls;
            if (ldv.fast) {
                const unsigned ou = fdiv((unsigned)line, ldv.inner);
                o = ou;
                c = (unsigned)line - ou * ldv.inner.d;
                cls = from_inner ? fmod_u(fdiv((unsigned)c, ldv.cdiv), ldv.cmod) : fdiv(ou, ldv.cdiv);
            } else {
                o = line / inner;
                c = line % inner;
                cls = from_inner ? (c / cdiv) % cmod : o / cdiv;
            }
            sh = tab[cls];
            ll.base = o * L * inner + c;
            if (use_net) {  // drift lines: +sp is the neighbour with larger |v|
                ll.sp = vp_core::cell_centre(lo, dvel, (int)cls) >= 0.0 ? 1 : -1;
                ll.has_p = cls + ll.sp >= 0 && cls + ll.sp < cmod;
                ll.has_m = cls - ll.sp >= 0 && cls - ll.sp < cmod;
            }
            int n = sh.n;
            if (PERIODIC) {  // the shift modulo L, nearest to zero
                n %= L;
                if (n > L / 2) n -= L;
                if (n < -(L / 2)) n += L;
                sh.n = n;
            }
            ll.q0 = (sh.sigma > 0 ? 0 : L - 1) - n - sh.sigma;
        }
        shs[l] = sh;
        lls[l] = ll;
    }
    __syncthreads();
    const int lt = threadIdx.x & (NL - 1), rt = threadIdx.x >> lgNL, rstep = blockDim.x >> lgNL;
    if (lt < nl) {
        // four rows per thread in flight: all loads first, then the stores
        const LLine ll = lls[lt];
        const long long pofs = ll.sp * cdiv;
        constexpr int B = 4;
        for (int r0 = rt; r0 < LP; r0 += B * rstep) {
            float v[B], up[B], um[B];
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const int r = r0 + j * rstep;
                int rr = r - kLG;  // line row
                if (PERIODIC) {
                    if (L >= kLG) {  // staged rows reach at most kLG beyond either end
                        rr += rr < 0 ? L : 0;
                        rr -= rr >= L ? L : 0;
                    } else {
                        while (rr < 0) rr += L;
                        while (rr >= L) rr -= L;
                    }
                }
                const bool in = r < LP && (PERIODIC || (rr >= 0 && rr < L));
                const long long a = ll.base + (long long)rr * inner;
                v[j] = in ? f[a] : 0.f;
                up[j] = in && use_net && ll.has_p ? fsnap[a + pofs] : 0.f;
                um[j] = in && use_net && ll.has_m ? fsnap[a - pofs] : 0.f;
            }
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const int r = r0 + j * rstep;
                if (r < LP) {
                    lines[r * NL + lt] = v[j];
                    if (use_net) {
                        dvl[r * NL + lt] = 0.5f * (up[j] - um[j]);
                        cvl[r * NL + lt] = 0.5f * (up[j] + um[j]) - v[j];
                    }
                }
            }
        }
    }
    __syncthreads();
    // row q of staged line l: direct inside the staged rows, wrapped (periodic)
    // or zero (outflow) beyond them (only for shifts of more than kLG - 5 cells)
    auto row = [&](const float *ln, int l, int q) -> float {
        if (q < -kLG || q >= L + kLG) {
            if constexpr (PERIODIC) {
                while (q < 0) q += L;
                while (q >= L) q -= L;
            } else {
                return 0.f;
            }
        }
        return ln[(q + kLG) * NL + l];
    };
    if (!use_net) {
        // phase 1 without the network: limited mass of every interface (CSL7, MP, PP)
        for (int e = threadIdx.x; e < NI; e += blockDim.x) {
            const int l = e & (NL - 1), k = e >> lgNL;
            if (l >= nl) continue;
            const LineShift<float> &sh = shs[l];
            const int sg = sh.sigma;
            const int q = lls[l].q0 + k * sg;
            const int qa = q - 3 * sg, qb = q + 3 * sg;
            float u[7];
            if (min(qa, qb) >= -kLG && max(qa, qb) < L + kLG) {
                const int st = sg * NL;
                const float *pu = lines + (qa + kLG) * NL + l;
#pragma unroll
                for (int m = 0; m < 7; ++m) u[m] = pu[m * st];
            } else {
#pragma unroll
                for (int m = 0; m < 7; ++m) u[m] = row(lines, l, qa + m * sg);
            }
            float phi = sh.w[0] * u[0];
#pragma unroll
            for (int m = 1; m < 7; ++m) phi = fmaf(sh.w[m], u[m], phi);
            phi = vp_core::mp_limit(phi, u[1], u[2], u[3], u[4], u[5], alpha);
            mass[e] = vp_core::pp_clamp(vp_core::mul_rn(sh.nu, phi), vp_core::half_rd(u[3]),
                                        vp_core::half_rd(u[4]));
        }
    } else {
        // phase 1 with the network: a warp takes 32 interfaces (two 16-row MMA
        // tiles).  Lane i computes interface i's plain MP mass and its feature
        // row (bf16, columns 0-7 stencil, 8-15 velocity difference, 16-23
        // velocity curvature, 24 nu, 25-31 zero) into the warp's buffer;
        // ldmatrix turns the rows into A fragments; the layers run with
        // mma.sync (biases as the C operand, FP32 accumulation, ReLU and bf16
        // rounding in one conversion); the output layer is an MMA with w4 in
        // column 0 of B; lane i then adds s g and applies the PP limiter (after
        // the MP bounds when use_net = 2).
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, t = lane & 3;
        unsigned char *fb = fbuf + warp * 32 * kFS;
        const uint32_t fb_s = static_cast<uint32_t>(__cvta_generic_to_shared(fb));
        // this lane's ldmatrix row: matrix lane >> 3 holds rows +8 (odd) and columns +8 (>= 2)
        const uint32_t ldm = fb_s + (uint32_t)(((lane & 7) + 8 * ((lane >> 3) & 1)) * kFS + 16 * (lane >> 4));
        const uint2 *wf2 = reinterpret_cast<const uint2 *>(wfrag);
        const float2 b4c = make_float2(t == 0 ? wvec[4 * H] : 0.f, 0.f);
        const int nit = (NI + 31) >> 5;
        for (int it = warp; it < nit; it += blockDim.x >> 5) {
            const int e = (it << 5) + lane;
            const int l = e & (NL - 1), k = e >> lgNL;
            const bool ok = e < NI && l < nl;
            float Mp = 0.f, s = 1.f, u3 = 0.f, u4 = 0.f, nu = 0.f, mlo = 0.f, mhi = 0.f;
            uint4 p0 = make_uint4(0u, 0u, 0u, 0u), p1 = p0, p2 = p0, p3 = p0;
            if (ok) {
                const LineShift<float> &sh = shs[l];
                const int sg = sh.sigma;
                const int q = lls[l].q0 + k * sg;
                nu = sh.nu;
                float u[8], dv[8], cv[8];
                const int qa = q - 3 * sg, qb = q + 4 * sg;
                if (min(qa, qb) >= -kLG && max(qa, qb) < L + kLG) {
                    const int st = sg * NL;
                    const float *pu = lines + (qa + kLG) * NL + l;
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        u[m] = pu[m * st];
                        dv[m] = pu[NL * LP + m * st];
                        cv[m] = pu[2 * NL * LP + m * st];
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        u[m] = row(lines, l, qa + m * sg);
                        dv[m] = row(dvl, l, qa + m * sg);
                        cv[m] = row(cvl, l, qa + m * sg);
                    }
                }
                float phi = sh.w[0] * u[0];
#pragma unroll
                for (int m = 1; m < 7; ++m) phi = fmaf(sh.w[m], u[m], phi);
                // MP bounds of this stencil (App. A steps 4-6); the plain
                // mass and, after the network, the corrected one are clamped
                // into them (the constraint equals the clamp, see mp_clamp)
                vp_core::mp_lohi(u[1], u[2], u[3], u[4], u[5], alpha, mlo, mhi);
                mlo = vp_core::mul_rn(nu, mlo);
                mhi = vp_core::mul_rn(nu, mhi);
                Mp = fminf(fmaxf(vp_core::mul_rn(nu, phi), mlo), mhi);
                u3 = u[3];
                u4 = u[4];
                s = 0.f;
#pragma unroll
                for (int m = 0; m < 8; ++m) s = fmaxf(s, fabsf(u[m]));
                s += 1e-30f;
                const float inv = 1.0f / s;
                p0 = make_uint4(pack_bf16((u[0] - u3) * inv, (u[1] - u3) * inv),
                                pack_bf16((u[2] - u3) * inv, 0.f), pack_bf16((u[4] - u3) * inv, (u[5] - u3) * inv),
                                pack_bf16((u[6] - u3) * inv, (u[7] - u3) * inv));
                p1 = make_uint4(pack_bf16(dv[0] * inv, dv[1] * inv), pack_bf16(dv[2] * inv, dv[3] * inv),
                                pack_bf16(dv[4] * inv, dv[5] * inv), pack_bf16(dv[6] * inv, dv[7] * inv));
                p2 = make_uint4(pack_bf16(cv[0] * inv, cv[1] * inv), pack_bf16(cv[2] * inv, cv[3] * inv),
                                pack_bf16(cv[4] * inv, cv[5] * inv), pack_bf16(cv[6] * inv, cv[7] * inv));
                p3.x = pack_bf16(nu, 0.f);
            }
            uint4 *fr = reinterpret_cast<uint4 *>(fb + lane * kFS);
            fr[0] = p0;
            fr[1] = p1;
            fr[2] = p2;
            fr[3] = p3;
            __syncwarp();
            uint32_t a[2][2][4];  // [tile][k block][fragment]
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int kb = 0; kb < 2; ++kb) ldsm_x4(a[j][kb], ldm + (uint32_t)(j * 16 * kFS + kb * 32));
            __syncwarp();
            float acc[2][4][4];
#pragma unroll
            for (int layer = 0; layer < 3; ++layer) {
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const float2 b = *reinterpret_cast<const float2 *>(wvec + layer * H + 8 * nt + 2 * t);
                    const uint2 bb0 = wf2[((layer * 2 + 0) * 4 + nt) * 32 + lane];
                    const uint2 bb1 = wf2[((layer * 2 + 1) * 4 + nt) * 32 + lane];
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        mma_bf16_c(acc[j][nt], a[j][0], bb0, b);
                        mma_bf16(acc[j][nt], a[j][1], bb1.x, bb1.y);
                    }
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) relu_pack(acc[j], a[j]);
            }
            float g[2][4];
            const uint2 w40 = w4f[lane], w41 = w4f[32 + lane];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                mma_bf16_c(g[j], a[j][0], w40, b4c);
                mma_bf16(g[j], a[j][1], w41.x, w41.y);
            }
            // row r of tile j sits in lane 4 (r mod 8), element 0 (r < 8) or 2
            const int src = (lane & 7) << 2;
            const float g00 = __shfl_sync(0xffffffffu, g[0][0], src);
            const float g02 = __shfl_sync(0xffffffffu, g[0][2], src);
            const float g10 = __shfl_sync(0xffffffffu, g[1][0], src);
            const float g12 = __shfl_sync(0xffffffffu, g[1][2], src);
            const float gi = (lane & 16) ? ((lane & 8) ? g12 : g10) : ((lane & 8) ? g02 : g00);
            if (ok) {
                float M = fmaf(s, gi, Mp);
                if (use_net == 2) M = fminf(fmaxf(M, mlo), mhi);
                mass[e] = vp_core::pp_clamp(M, vp_core::half_rd(u3), vp_core::half_rd(u4));
            }
        }
    }
    __syncthreads();
    // phase 2: the flux-form update, one thread per cell (consecutive
    // threads: consecutive lines)
    if (lt < nl) {
        const int sg = shs[lt].sigma, q0 = lls[lt].q0;
        const long long base = lls[lt].base;
        for (int kr = rt; kr < L; kr += rstep) {
            const int k = kr + 1;                  // the cell between interfaces k - 1 and k
            const int i = sg > 0 ? k - 1 : L - k;  // the k-th cell of the walk
            const float v = row(lines, lt, q0 + k * sg) - (mass[k * NL + lt] - mass[(k - 1) * NL + lt]);
            f[base + (long long)i * inner] = v;
        }
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
    if (!c->d_snap) VP_CUDA_TRY(c, cudaMalloc(&c->d_snap, (size_t)c->ncell * sizeof(float)));
    if (!c->d_netfrag) VP_CUDA_TRY(c, cudaMalloc(&c->d_netfrag, kFragWords * sizeof(uint32_t)));
    VP_CUDA_TRY(c, cudaFuncSetAttribute(k_learned_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        200 * 1024));
    VP_CUDA_TRY(c, cudaFuncSetAttribute(k_learned_sweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        200 * 1024));
    c->learned_ready = 1;
    return VP_OK;
}

extern "C" {

int vp_learned_sweep(vp_ctx *c, int kick, int dim, double dt, const double *accel_dev, const float *wts,
                     int use_net, const float *f_snap) {
    if (!c || !c->f) return VP_EINVAL;
    if (c->g.precision != VP_F32 || c->g.order != 7)
        return vp_fail(c, VP_ENOTSUP, "the learned sweep runs on FP32 CSL7 grids");
    if (use_net < 0 || use_net > 2) return vp_fail(c, VP_EINVAL, "use_net must be 0, 1 or 2");
    if (use_net && kick) return vp_fail(c, VP_ENOTSUP, "the learned correction applies to spatial sweeps");
    if (dim < 0 || dim >= c->g.dx || (kick && !accel_dev) || (use_net && !wts) || !std::isfinite(dt))
        return vp_fail(c, VP_EINVAL, "bad learned-sweep arguments");
    int rc = vp_learned_prepare(c);
    if (rc != VP_OK) return rc;
    if (use_net && !f_snap) {
        // snapshot of f before the sweep in the library-owned buffer
        VP_CUDA_TRY(c, cudaMemcpyAsync(c->d_snap, c->f, (size_t)c->ncell * sizeof(float),
                                       cudaMemcpyDeviceToDevice, c->stream));
        f_snap = static_cast<const float *>(c->d_snap);
    }
    const LineGeo q = line_geo(c->g, c->NX, c->NV, kick, dim);
    rc = vp_launch_shift_table(c, kick, dim, dt, accel_dev);
    if (rc != VP_OK) return rc;
    if (use_net) {
        k_net_frags<<<1, 256, 0, c->stream>>>(wts, static_cast<uint32_t *>(c->d_netfrag));
        c->launches++;
    }
    // lines per CTA: a power of two, at most 16; the largest that leaves room
    // for 7 CTAs per SM (28 warps, as many as the registers allow), else the
    // largest within 48 KB of shared memory
    auto smem_for = [&](int nl) {
        return (size_t)kFragWords * sizeof(uint32_t) + nl * (sizeof(LineShift<float>) + sizeof(LLine)) +
               3 * (size_t)nl * (q.L + 2 * kLG) * sizeof(float) + (size_t)nl * (q.L + 1) * sizeof(float) + 16 +
               (size_t)(kTcThreads / 32) * 32 * kFS;
    };
    int lgNL = 4;
    while (lgNL > 0 && smem_for(1 << lgNL) > 31 * 1024) --lgNL;
    if (smem_for(1 << lgNL) > 31 * 1024) {
        lgNL = 4;
        while (lgNL > 0 && smem_for(1 << lgNL) > 48 * 1024) --lgNL;
    }
    const int NL = 1 << lgNL;
    const size_t smem = smem_for(NL);
    if (smem > 200 * 1024) return vp_fail(c, VP_ENOTSUP, "line too long for the learned sweep");
    const long long nl = q.outer * q.inner;
    const unsigned blocks = (unsigned)((nl + NL - 1) / NL);
    const LineShift<float> *tab = static_cast<const LineShift<float> *>(c->d_shift);
    const uint4 *frag = static_cast<const uint4 *>(c->d_netfrag);
    LineDiv ldv{};
    ldv.fast = nl <= 0xFFFFFFFFll && q.inner <= 0xFFFFFFFFll && q.cdiv <= 0xFFFFFFFFll && q.cmod <= 0xFFFFFFFFll;
    if (ldv.fast) {
        ldv.inner = make_fastdiv((unsigned)q.inner);
        ldv.cdiv = make_fastdiv((unsigned)q.cdiv);
        ldv.cmod = make_fastdiv((unsigned)q.cmod);
    }
    if (q.periodic)
        k_learned_sweep<true><<<blocks, kTcThreads, smem, c->stream>>>(
            static_cast<float *>(c->f), q.outer, q.L, q.inner, q.from_inner, q.cdiv, q.cmod, tab, frag, q.lo,
            q.dvel, (float)c->g.alpha, use_net, f_snap, lgNL, ldv);
    else
        k_learned_sweep<false><<<blocks, kTcThreads, smem, c->stream>>>(
            static_cast<float *>(c->f), q.outer, q.L, q.inner, q.from_inner, q.cdiv, q.cmod, tab, frag, q.lo,
            q.dvel, (float)c->g.alpha, use_net, f_snap, lgNL, ldv);
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
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
