// vp_sweep.cu -- the SL-MPP5/7 advection sweep (shift decomposition, CSL
// flux, MP constraint, PP limiter, conservative update) for sm_103a.
//
// A sweep advances every 1D line of f along one phase-space axis.  f is seen
// as [outer][L][inner]: the line runs along the middle index with element
// stride `inner`.  Two kernels stage whole lines in shared memory so that
// every cell of f is read from HBM once and written once, in place:
//   * k_sweep_cols: inner > 1 (strided axes).  A CTA owns a tile of W
//     consecutive columns (W lines) x the full line; global loads and stores
//     are row-contiguous (coalesced, 16-byte vectors when aligned).
//   * k_sweep_rows: inner == 1 (the contiguous last velocity axis).  A CTA
//     owns R consecutive lines, one contiguous block of memory, staged with
//     an odd row pitch so that 32 lanes walking 32 lines hit 32 banks.
// Each thread walks a segment of one line in the upwind direction with a
// sliding register window, so each interface flux is computed once and the
// incoming flux of a cell is the outgoing flux of its upwind neighbour.
#include <cmath>

#include "vp_internal.cuh"

namespace {

// ---- limiter arithmetic (Appendix A and Sec. 2.1.1) -------------------------

template <typename T>
__device__ __forceinline__ T mm2(T a, T b) {
    // minmod: smallest magnitude if both share a sign, else 0
    if (a > T(0) && b > T(0)) return a < b ? a : b;
    if (a < T(0) && b < T(0)) return a > b ? a : b;
    return T(0);
}

template <typename T>
__device__ __forceinline__ T mm4(T a, T b, T c, T d) {
    if (a > T(0) && b > T(0) && c > T(0) && d > T(0)) return fmin(fmin(a, b), fmin(c, d));
    if (a < T(0) && b < T(0) && c < T(0) && d < T(0)) return fmax(fmax(a, b), fmax(c, d));
    return T(0);
}

template <typename T>
__device__ __forceinline__ T mid3(T a, T b, T c) {
    // middle value of three
    return fmax(fmin(a, b), fmin(fmax(a, b), c));
}

// MP bound of the interface value phi between cells u0 (upwind) and u1,
// neighbours um2, um1 upwind and u2 downwind.
template <typename T>
__device__ __forceinline__ T mp_bound(T phi, T um2, T um1, T u0, T u1, T u2, T alpha) {
    const T back = u0 - um1;
    const T fstar = u0 + mm2(u1 - u0, alpha * back);
    const T a = phi - u0, b = phi - fstar;
    if ((a > T(0) && b < T(0)) || (a < T(0) && b > T(0))) return phi;  // strictly between
    if (um1 == u0 && u0 == u1) return u0;  // all bounds collapse onto u0
    const T dm = um2 + u0 - T(2) * um1;   // curvature at the upwind neighbour
    const T dc = um1 + u1 - T(2) * u0;    // at the upwind cell
    const T dp = u0 + u2 - T(2) * u1;     // at the downwind cell
    const T m4p = mm4(T(4) * dc - dp, T(4) * dp - dc, dc, dp);
    const T m4m = mm4(T(4) * dm - dc, T(4) * dc - dm, dm, dc);
    const T ful = u0 + alpha * back;
    const T fmd = T(0.5) * (u0 + u1) - T(0.5) * m4p;
    const T flc = u0 + T(0.5) * back + (T(4) / T(3)) * m4m;
    const T lo = fmax(fmin(fmin(u0, u1), fmd), fmin(fmin(u0, ful), flc));
    const T hi = fmin(fmax(fmax(u0, u1), fmd), fmax(fmax(u0, ful), flc));
    return mid3(phi, lo, hi);
}

template <typename T>
struct Eps;
template <>
struct Eps<float> {
    static constexpr float safety = 1.0f - 8.0f * 5.9604644775390625e-08f;  // 1 - 8 * 2^-24
};
template <>
struct Eps<double> {
    static constexpr double safety = 1.0 - 8.0 * 1.1102230246251565e-16;  // 1 - 8 * 2^-53
};

// Positivity blend: keep both halves f_i - 2 nu phi >= 0 (outflow side) and
// f_{i+1} + 2 nu phi >= 0 (inflow side of the downwind cell).
template <typename T>
__device__ __forceinline__ T pp_blend(T phi, T u0, T u1, T nu) {
    const T two_nu = T(2) * nu;
    const T up = u0 - two_nu * phi;
    const T um = u1 + two_nu * phi;
    if (!(up < T(0)) && !(um < T(0))) return phi;
    T th = T(1);
    if (up < T(0)) {
        const T base = u0 - two_nu * u0;
        const T den = base - up;
        th = den > T(0) ? base / den : T(0);
    }
    if (um < T(0)) {
        const T base = u1 + two_nu * u0;
        const T den = base - um;
        const T t2 = den > T(0) ? base / den : T(0);
        th = t2 < th ? t2 : th;
    }
    th *= Eps<T>::safety;
    th = th < T(0) ? T(0) : (th > T(1) ? T(1) : th);
    return th * phi + (T(1) - th) * u0;
}

template <typename T, int ORDER>
__device__ __forceinline__ T iface(const T *u, const LineShift<T> &sh, T alpha, int mp, int pp) {
    // u points at the upwind cell (u[0]); u[-3..3] valid
    T phi;
    if (ORDER == 7) {
        phi = sh.w[0] * u[-3];
        phi = fma(sh.w[1], u[-2], phi);
        phi = fma(sh.w[2], u[-1], phi);
        phi = fma(sh.w[3], u[0], phi);
        phi = fma(sh.w[4], u[1], phi);
        phi = fma(sh.w[5], u[2], phi);
        phi = fma(sh.w[6], u[3], phi);
    } else {
        phi = sh.w[1] * u[-2];
        phi = fma(sh.w[2], u[-1], phi);
        phi = fma(sh.w[3], u[0], phi);
        phi = fma(sh.w[4], u[1], phi);
        phi = fma(sh.w[5], u[2], phi);
    }
    if (mp) phi = mp_bound(phi, u[-2], u[-1], u[0], u[1], u[2], alpha);
    if (pp) phi = pp_blend(phi, u[0], u[1], sh.nu);
    return phi;
}

// Advance cells [r0, r1) of one staged line.  sm: line in shared memory with
// element stride ss; out: the same line in global memory, element stride gs.
template <typename T, int ORDER>
__device__ __forceinline__ void sweep_segment(const T *__restrict__ sm, int ss, int L, int periodic,
                                              const LineShift<T> &sh, int r0, int r1,
                                              T *__restrict__ out, long long gs, T alpha, int mp,
                                              int pp) {
    if (r0 >= r1) return;
    const int sg = sh.sigma;
    int n = sh.n;
    if (periodic) {
        n %= L;
        if (n < 0) n += L;
    }
    const T nu = sh.nu;
    // walk in the upwind-to-downwind direction
    int i = sg > 0 ? r0 : r1 - 1;
    const int cnt = r1 - r0;
    // window u[k+4] = value of the shifted line at cell i + sg*k, k = -4..3
    T win[8];
    int p = i - n - 4 * sg;  // source position of u[-4]
    if (periodic) {
        p %= L;
        if (p < 0) p += L;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        T v;
        if (periodic) {
            v = sm[p * ss];
        } else {
            v = (p >= 0 && p < L) ? sm[p * ss] : T(0);
        }
        win[k] = v;
        p += sg;
        if (periodic) {
            if (p >= L) p -= L;
            if (p < 0) p += L;
        }
    }
    // p now points at the source of u[4] (the next value to enter)
    T fin = iface<T, ORDER>(&win[3], sh, alpha, mp, pp);  // upwind cell i - sg
    for (int t = 0; t < cnt; ++t) {
        const T fout = iface<T, ORDER>(&win[4], sh, alpha, mp, pp);
        out[(long long)i * gs] = win[4] - nu * (fout - fin);
        fin = fout;
        i += sg;
        T v;
        if (periodic) {
            v = sm[p * ss];
        } else {
            v = (p >= 0 && p < L) ? sm[p * ss] : T(0);
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) win[k] = win[k + 1];
        win[7] = v;
        p += sg;
        if (periodic) {
            if (p >= L) p -= L;
            if (p < 0) p += L;
        }
    }
}

__device__ __forceinline__ long long line_class(const SweepGeo &g, long long o, long long c) {
    return g.cls_from_inner ? (c / g.cdiv) % g.cmod : o / g.cdiv;
}

template <typename T, int ORDER>
__global__ void __launch_bounds__(512) k_sweep_cols(T *__restrict__ f,
                                                    const LineShift<T> *__restrict__ tab,
                                                    SweepGeo geo, LimParams lp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    const int W = geo.W, L = geo.L;
    const long long tpo = (geo.inner + W - 1) / W;
    const long long o = blockIdx.x / tpo;
    const long long c0 = (blockIdx.x % tpo) * W;
    const int wc = (int)((geo.inner - c0) < W ? (geo.inner - c0) : W);
    T *base = f + o * (long long)L * geo.inner + c0;
    // stage the tile [L][W]
    constexpr int VEC = 16 / sizeof(T);
    const bool vec = (wc == W) && (geo.inner % VEC == 0) && (W % VEC == 0);
    if (vec) {
        const int wv = W / VEC;
        for (int e = threadIdx.x; e < L * wv; e += blockDim.x) {
            const int r = e / wv, cv = e - r * wv;
            const float4 x = *reinterpret_cast<const float4 *>(base + (long long)r * geo.inner + cv * VEC);
            *reinterpret_cast<float4 *>(sm + r * W + cv * VEC) = x;
        }
    } else {
        for (int e = threadIdx.x; e < L * W; e += blockDim.x) {
            const int r = e / W, cc = e - r * W;
            sm[e] = cc < wc ? base[(long long)r * geo.inner + cc] : T(0);
        }
    }
    __syncthreads();
    const int cc = threadIdx.x % W;
    const int seg = threadIdx.x / W;
    if (cc < wc && seg < geo.nseg) {
        const LineShift<T> sh = tab[line_class(geo, o, c0 + cc)];
        const int r0 = (int)((long long)seg * L / geo.nseg);
        const int r1 = (int)((long long)(seg + 1) * L / geo.nseg);
        sweep_segment<T, ORDER>(sm + cc, W, L, geo.periodic, sh, r0, r1, base + cc, geo.inner,
                                (T)lp.alpha, lp.mp, lp.pp);
    }
}

template <typename T, int ORDER>
__global__ void __launch_bounds__(512) k_sweep_rows(T *__restrict__ f,
                                                    const LineShift<T> *__restrict__ tab,
                                                    SweepGeo geo, LimParams lp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    const int L = geo.L, R = geo.R;
    const int P = L | 1;  // odd pitch: 32 lines -> 32 banks
    const long long l0 = (long long)blockIdx.x * R;
    const int nl = (int)((geo.outer - l0) < R ? (geo.outer - l0) : R);
    T *base = f + l0 * L;
    const int tot = nl * L;
    constexpr int VEC = 16 / sizeof(T);
    if ((L % VEC) == 0) {
        for (int e = threadIdx.x * VEC; e < tot; e += blockDim.x * VEC) {
            const float4 x = *reinterpret_cast<const float4 *>(base + e);
            const T *xv = reinterpret_cast<const T *>(&x);
            const int r = e / L, pos = e - r * L;
#pragma unroll
            for (int k = 0; k < VEC; ++k) sm[r * P + pos + k] = xv[k];
        }
    } else {
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int r = e / L, pos = e - r * L;
            sm[r * P + pos] = base[e];
        }
    }
    __syncthreads();
    const int line = threadIdx.x % R;
    const int seg = threadIdx.x / R;
    if (line < nl && seg < geo.nseg) {
        const LineShift<T> sh = tab[line_class(geo, l0 + line, 0)];
        const int r0 = (int)((long long)seg * L / geo.nseg);
        const int r1 = (int)((long long)(seg + 1) * L / geo.nseg);
        sweep_segment<T, ORDER>(sm + line * P, 1, L, geo.periodic, sh, r0, r1,
                                base + (long long)line * L, 1, (T)lp.alpha, lp.mp, lp.pp);
    }
}

// Shift decomposition of every line class, in double precision so that the
// integer part is exact: s = c dt / h, n = nearest integer (halves away from
// zero), zeta = s - n, nu = |zeta|; the weights are the CSL polynomials at nu.
template <typename T>
__global__ void k_shift_table(LineShift<T> *__restrict__ tab, int nclass, int kick, double lo,
                              double dvel, const double *__restrict__ accel, double dt, double h,
                              WPoly wp) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nclass) return;
    double speed;
    if (kick) {
        speed = accel[c];
    } else {
        speed = __dadd_rn(lo, __dmul_rn((double)c + 0.5, dvel));
    }
    const double s = __ddiv_rn(__dmul_rn(speed, dt), h);
    const double n = round(s);
    const double z = __dadd_rn(s, -n);
    const double nu = fabs(z);
    LineShift<T> sh;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        double acc = 0.0;
        for (int j = wp.nterm - 1; j >= 0; --j) acc = fma(acc, nu, wp.c[j][k]);
        sh.w[k] = (T)acc;
    }
    sh.nu = (T)nu;
    sh.n = (int)n;
    sh.sigma = z < 0.0 ? -1 : 1;
    tab[c] = sh;
}

template <typename T, int ORDER>
void set_attrs() {
    cudaFuncSetAttribute(k_sweep_cols<T, ORDER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(k_sweep_rows<T, ORDER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
}

// geometry of the sweep along axis `dim` (kick: velocity axis, else spatial)
SweepGeo make_geo(const vp_ctx *c, int kick, int dim) {
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
    return geo;
}

template <typename T>
int launch_sweep_t(vp_ctx *c, int kick, int dim) {
    SweepGeo geo = make_geo(c, kick, dim);
    const LineShift<T> *tab = static_cast<const LineShift<T> *>(c->d_shift);
    LimParams lp{c->g.alpha, c->g.mp, c->g.pp};
    T *f = static_cast<T *>(c->f);
    const int L = geo.L;
    const int order = c->g.order;
    if (geo.inner > 1) {
        int W = (int)(8192 / sizeof(T) * 4 / L);  // ~32 KB tile for float
        W = W > 128 ? 128 : W;
        W = W < 32 ? 32 : W;
        if (geo.inner < W) W = (int)geo.inner;
        int nseg = L / 8;
        const int maxseg = 256 / W > 0 ? 256 / W : 1;
        nseg = nseg > maxseg ? maxseg : nseg;
        nseg = nseg < 1 ? 1 : nseg;
        geo.W = W;
        geo.nseg = nseg;
        const long long tiles = geo.outer * ((geo.inner + W - 1) / W);
        const size_t smem = (size_t)L * W * sizeof(T);
        if (smem > 200 * 1024) return vp_fail(c, VP_ENOTSUP, "line of %d cells too long to stage", L);
        const int threads = ((W * nseg + 31) / 32) * 32;
        if (order == 7)
            k_sweep_cols<T, 7><<<(unsigned)tiles, threads, smem, c->stream>>>(f, tab, geo, lp);
        else
            k_sweep_cols<T, 5><<<(unsigned)tiles, threads, smem, c->stream>>>(f, tab, geo, lp);
    } else {
        int R = 4096 / L;
        R = R < 32 ? 32 : (R > 128 ? 128 : R);
        if (geo.outer < R) R = (int)geo.outer;
        int nseg = L / 16;
        const int maxseg = 256 / R > 0 ? 256 / R : 1;
        nseg = nseg > maxseg ? maxseg : nseg;
        nseg = nseg < 1 ? 1 : nseg;
        geo.R = R;
        geo.nseg = nseg;
        const long long blocks = (geo.outer + R - 1) / R;
        const size_t smem = (size_t)R * (L | 1) * sizeof(T);
        if (smem > 200 * 1024) return vp_fail(c, VP_ENOTSUP, "line of %d cells too long to stage", L);
        const int threads = ((R * nseg + 31) / 32) * 32;
        if (order == 7)
            k_sweep_rows<T, 7><<<(unsigned)blocks, threads, smem, c->stream>>>(f, tab, geo, lp);
        else
            k_sweep_rows<T, 5><<<(unsigned)blocks, threads, smem, c->stream>>>(f, tab, geo, lp);
    }
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

}  // namespace

int vp_sweep_setup(vp_ctx *c) {
    set_attrs<float, 5>();
    set_attrs<float, 7>();
    set_attrs<double, 5>();
    set_attrs<double, 7>();
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

int vp_launch_shift_table(vp_ctx *c, int kick, int dim, double dt, const double *accel) {
    const vp_grid &g = c->g;
    const int nclass = kick ? (int)c->NX : g.nv[dim];
    const double h = kick ? (g.vhi[dim] - g.vlo[dim]) / g.nv[dim] : (g.xhi[dim] - g.xlo[dim]) / g.nx[dim];
    const double lo = g.vlo[dim];
    const double dvel = (g.vhi[dim] - g.vlo[dim]) / g.nv[dim];
    const int th = 128;
    const int bl = (nclass + th - 1) / th;
    if (g.precision == VP_F32)
        k_shift_table<float><<<bl, th, 0, c->stream>>>(static_cast<LineShift<float> *>(c->d_shift),
                                                       nclass, kick, lo, dvel, accel, dt, h, c->wp);
    else
        k_shift_table<double><<<bl, th, 0, c->stream>>>(static_cast<LineShift<double> *>(c->d_shift),
                                                        nclass, kick, lo, dvel, accel, dt, h, c->wp);
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

int vp_launch_sweep(vp_ctx *c, int kick, int dim) {
    if (c->g.precision == VP_F32) return launch_sweep_t<float>(c, kick, dim);
    return launch_sweep_t<double>(c, kick, dim);
}
