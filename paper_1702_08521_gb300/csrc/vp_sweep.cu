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
//   * k_sweep_cols_tma: the strided-axis sweep as a persistent kernel fed by
//     TMA: one elected thread streams [L x W] tiles global -> shared with
//     cp.async.bulk.tensor (two input stages, mbarrier completion), all
//     threads compute into a shared output tile, which TMA stores back while
//     the next tile is computed.  No per-thread global loads or stores.
// Each thread walks a segment of one line in the upwind direction with a
// sliding register window, so each interface flux is computed once and the
// incoming flux of a cell is the outgoing flux of its upwind neighbour.
#include <cudaTypedefs.h>

#include <cmath>

#include "vp_internal.cuh"
#include "vp_tma.cuh"

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

template <typename T, int ORDER>
__global__ void __launch_bounds__(512) k_sweep_cols_tma(const __grid_constant__ CUtensorMap tmap,
                                                        const LineShift<T> *__restrict__ tab,
                                                        SweepGeo geo, LimParams lp,
                                                        int *__restrict__ status) {
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar[2];
    const int W = geo.W, L = geo.L;
    const int tile = L * W;
    // TMA tensor copies need 128-byte aligned shared-memory buffers: align
    // the dynamic region explicitly (the launch reserves 128 spare bytes)
    const uint32_t base = vp_tma::saddr(smraw);
    const uint32_t pad = (128u - (base & 127u)) & 127u;
    T *in_buf = reinterpret_cast<T *>(smraw + pad);  // [2][L][W]
    T *out_buf = in_buf + 2 * tile;                   // [2][L][W]
    const long long tpo = (geo.inner + W - 1) / W;
    const long long ntiles = geo.outer * tpo;
    const uint32_t bytes = (uint32_t)(tile * sizeof(T));
    // self-check of every alignment the copies rely on; on failure report and
    // leave before issuing any copy
    if (((vp_tma::saddr(in_buf) | vp_tma::saddr(out_buf) | bytes) & 127u) != 0 ||
        ((W * sizeof(T)) & 15u) != 0) {
        if (threadIdx.x == 0) atomicExch(status, VP_EINVAL);
        return;
    }
    if (threadIdx.x == 0) {
        vp_tma::mbar_init(&bar[0], 1);
        vp_tma::mbar_init(&bar[1], 1);
        vp_tma::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            const long long t = blockIdx.x + (long long)s * gridDim.x;
            if (t < ntiles) {
                vp_tma::mbar_expect_tx(&bar[s], bytes);
                vp_tma::load_3d(in_buf + s * tile, &tmap, &bar[s], (int)((t % tpo) * W), 0, (int)(t / tpo));
            }
        }
    }
    const int cc = threadIdx.x % W;
    const int seg = threadIdx.x / W;
    const int r0 = (int)((long long)seg * L / geo.nseg);
    const int r1 = (int)((long long)(seg + 1) * L / geo.nseg);
    int k = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = k & 1;
        T *in = in_buf + s * tile;
        T *out = out_buf + s * tile;
        if (!vp_tma::mbar_wait(&bar[s], (uint32_t)((k >> 1) & 1))) {
            // the tile never arrived: report, drain our stores, leave
            if (threadIdx.x == 0) {
                atomicExch(status, VP_ETIMEOUT);
                vp_tma::mbar_wait(&bar[s ^ 1], (uint32_t)(((k + 1) >> 1) & 1), 1u << 20);
                vp_tma::wait_all<0>();
            }
            return;
        }
        const long long o = t / tpo;
        const long long c0 = (t % tpo) * W;
        const int wc = (int)((geo.inner - c0) < W ? (geo.inner - c0) : W);
        if (cc < wc && seg < geo.nseg) {
            const LineShift<T> sh = tab[line_class(geo, o, c0 + cc)];
            sweep_segment<T, ORDER>(in + cc, W, L, geo.periodic, sh, r0, r1, out + cc, W,
                                    (T)lp.alpha, lp.mp, lp.pp);
        }
        vp_tma::fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            vp_tma::store_3d(&tmap, out, (int)c0, 0, (int)o);
            vp_tma::commit();
            const long long tn = t + 2LL * gridDim.x;
            if (tn < ntiles) {
                vp_tma::mbar_expect_tx(&bar[s], bytes);
                vp_tma::load_3d(in, &tmap, &bar[s], (int)((tn % tpo) * W), 0, (int)(tn / tpo));
            }
            vp_tma::wait_read<1>();  // the other output tile is free again
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) vp_tma::wait_all<0>();
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
    cudaFuncSetAttribute(k_sweep_cols_tma<T, ORDER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

template <typename T>
bool tma_eligible(const vp_ctx *c, const SweepGeo &geo, int W) {
    constexpr int VEC = 16 / sizeof(T);
    return geo.inner > 1 && geo.inner % VEC == 0 && W % VEC == 0 && geo.inner < (1LL << 31) &&
           geo.outer < (1LL << 31) && geo.L <= 256 && W <= 256 &&
           ((size_t)geo.L * W * sizeof(T)) % 128 == 0 &&
           (size_t)4 * geo.L * W * sizeof(T) + 128 <= 200 * 1024 && tensor_map_encoder() != nullptr &&
           (reinterpret_cast<uintptr_t>(c->f) & 15) == 0;
}

template <typename T>
int launch_cols(vp_ctx *c, SweepGeo geo, const SweepTune &tu) {
    const LineShift<T> *tab = static_cast<const LineShift<T> *>(c->d_shift);
    const LimParams lp{c->g.alpha, c->g.mp, c->g.pp};
    T *f = static_cast<T *>(c->f);
    const int L = geo.L;
    int W = tu.W;
    if (geo.inner < W) W = (int)geo.inner;
    geo.W = W;
    geo.nseg = tu.nseg;
    const int threads = ((W * tu.nseg + 31) / 32) * 32;
    const long long tiles = geo.outer * ((geo.inner + W - 1) / W);
    const bool seven = c->g.order == 7;
    if (tu.impl == 2 && tma_eligible<T>(c, geo, W)) {
        CUtensorMap map;
        const cuuint64_t dims[3] = {(cuuint64_t)geo.inner, (cuuint64_t)L, (cuuint64_t)geo.outer};
        const cuuint64_t strides[2] = {(cuuint64_t)geo.inner * sizeof(T),
                                       (cuuint64_t)geo.inner * L * sizeof(T)};
        const cuuint32_t box[3] = {(cuuint32_t)W, (cuuint32_t)L, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = tensor_map_encoder()(&map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                                          3, f, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return vp_fail(c, VP_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        const size_t smem = (size_t)4 * L * W * sizeof(T) + 128;
        int per_sm = tu.ctas_per_sm;
        if (per_sm <= 0) {
            if (seven)
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_cols_tma<T, 7>, threads, smem);
            else
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_cols_tma<T, 5>, threads, smem);
            per_sm = per_sm < 1 ? 1 : per_sm;
        }
        long long grid = (long long)per_sm * c->sm_count;
        grid = grid > tiles ? tiles : grid;
        if (seven)
            k_sweep_cols_tma<T, 7><<<(unsigned)grid, threads, smem, c->stream>>>(map, tab, geo, lp, c->d_status);
        else
            k_sweep_cols_tma<T, 5><<<(unsigned)grid, threads, smem, c->stream>>>(map, tab, geo, lp, c->d_status);
    } else {
        const size_t smem = (size_t)L * W * sizeof(T);
        if (smem > 200 * 1024) return vp_fail(c, VP_ENOTSUP, "line of %d cells too long to stage", L);
        if (seven)
            k_sweep_cols<T, 7><<<(unsigned)tiles, threads, smem, c->stream>>>(f, tab, geo, lp);
        else
            k_sweep_cols<T, 5><<<(unsigned)tiles, threads, smem, c->stream>>>(f, tab, geo, lp);
    }
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

template <typename T>
int launch_rows(vp_ctx *c, SweepGeo geo, const SweepTune &tu) {
    const LineShift<T> *tab = static_cast<const LineShift<T> *>(c->d_shift);
    const LimParams lp{c->g.alpha, c->g.mp, c->g.pp};
    T *f = static_cast<T *>(c->f);
    const int L = geo.L;
    int R = tu.W;
    if (geo.outer < R) R = (int)geo.outer;
    geo.R = R;
    geo.nseg = tu.nseg;
    const long long blocks = (geo.outer + R - 1) / R;
    const size_t smem = (size_t)R * (L | 1) * sizeof(T);
    if (smem > 200 * 1024) return vp_fail(c, VP_ENOTSUP, "line of %d cells too long to stage", L);
    const int threads = ((R * tu.nseg + 31) / 32) * 32;
    if (c->g.order == 7)
        k_sweep_rows<T, 7><<<(unsigned)blocks, threads, smem, c->stream>>>(f, tab, geo, lp);
    else
        k_sweep_rows<T, 5><<<(unsigned)blocks, threads, smem, c->stream>>>(f, tab, geo, lp);
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

// default tile choice when the autotuner has not run
template <typename T>
SweepTune default_tune(const vp_ctx *c, const SweepGeo &geo) {
    SweepTune tu{};
    tu.valid = 1;
    const int L = geo.L;
    if (geo.inner > 1) {
        int W = (int)(32768 / sizeof(T) / L);  // ~32 KB staged tile
        W = W > 128 ? 128 : (W < 32 ? 32 : W);
        W &= ~3;
        int nseg = L / 8;
        const int maxseg = 256 / W > 0 ? 256 / W : 1;
        nseg = nseg > maxseg ? maxseg : (nseg < 1 ? 1 : nseg);
        tu.W = W;
        tu.nseg = nseg;
        const int want = c->opt_impl ? c->opt_impl : 2;
        tu.impl = (want == 2 && tma_eligible<T>(c, geo, W < geo.inner ? W : (int)geo.inner)) ? 2 : 1;
    } else {
        int R = 4096 / L;
        R = R < 32 ? 32 : (R > 128 ? 128 : R);
        int nseg = L / 16;
        const int maxseg = 256 / R > 0 ? 256 / R : 1;
        nseg = nseg > maxseg ? maxseg : (nseg < 1 ? 1 : nseg);
        tu.W = R;
        tu.nseg = nseg;
        tu.impl = 1;
    }
    return tu;
}

template <typename T>
int launch_sweep_t(vp_ctx *c, int kick, int dim) {
    const SweepGeo geo = make_geo(c, kick, dim);
    SweepTune tu = c->tune[kick][dim];
    if (!tu.valid || (c->opt_impl && geo.inner > 1 && tu.impl != c->opt_impl)) tu = default_tune<T>(c, geo);
    if (c->opt_impl == 1) tu.impl = 1;
    if (geo.inner > 1) return launch_cols<T>(c, geo, tu);
    return launch_rows<T>(c, geo, tu);
}

// Autotuner: time candidate tile shapes of one sweep geometry on the bound
// f with a zero shift (n = 0, nu = 0 leaves f bit-for-bit unchanged) and keep
// the fastest.  Runs once per (kind, axis), never inside a stream capture.
template <typename T>
int tune_t(vp_ctx *c, int kick, int dim) {
    const SweepGeo geo = make_geo(c, kick, dim);
    SweepTune best = default_tune<T>(c, geo);
    if (kick) VP_CUDA_TRY(c, cudaMemsetAsync(c->d_acc, 0, sizeof(double) * c->NX, c->stream));
    int rc = vp_launch_shift_table(c, kick, dim, 0.0, kick ? c->d_acc : nullptr);
    if (rc) return rc;
    SweepTune cand[32];
    int nc = 0;
    if (geo.inner > 1) {
        const int impls[2] = {2, 1};
        for (int ii = 0; ii < 2; ++ii) {
            if (c->opt_impl && impls[ii] != c->opt_impl) continue;
            for (int W = 32; W <= 128; W *= 2)
                for (int nseg = 1; nseg <= 8; nseg *= 2) {
                    const int th = W * nseg;
                    if (th < 64 || th > 512 || nseg > geo.L) continue;
                    const int Weff = geo.inner < W ? (int)geo.inner : W;
                    if (impls[ii] == 2 && !tma_eligible<T>(c, geo, Weff)) continue;
                    if (impls[ii] == 1 && (size_t)geo.L * W * sizeof(T) > 200 * 1024) continue;
                    if (nc < 32) cand[nc++] = SweepTune{1, impls[ii], W, nseg, 0};
                }
        }
    } else {
        for (int R = 32; R <= 128; R *= 2)
            for (int nseg = 1; nseg <= 8; nseg *= 2) {
                const int th = R * nseg;
                if (th < 64 || th > 512 || nseg > geo.L) continue;
                if ((size_t)R * (geo.L | 1) * sizeof(T) > 200 * 1024) continue;
                if (nc < 32) cand[nc++] = SweepTune{1, 1, R, nseg, 0};
            }
    }
    if (nc == 0) {
        c->tune[kick][dim] = best;
        return VP_OK;
    }
    cudaEvent_t e0, e1;
    VP_CUDA_TRY(c, cudaEventCreate(&e0));
    VP_CUDA_TRY(c, cudaEventCreate(&e1));
    float best_ms = 1e30f;
    for (int i = 0; i < nc; ++i) {
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, c->stream);
            rc = geo.inner > 1 ? launch_cols<T>(c, geo, cand[i]) : launch_rows<T>(c, geo, cand[i]);
            cudaEventRecord(e1, c->stream);
            if (rc) break;
            const cudaError_t se = cudaEventSynchronize(e1);
            if (se != cudaSuccess) {
                rc = vp_fail(c, VP_ECUDA, "sweep candidate failed: %s", cudaGetErrorString(se));
                break;
            }
            float m = 0.f;
            cudaEventElapsedTime(&m, e0, e1);
            ms = m < ms ? m : ms;
        }
        if (rc) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rc;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = cand[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    best.valid = 1;
    c->tune[kick][dim] = best;
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

int vp_tune_sweep(vp_ctx *c, int kick, int dim) {
    if (c->tune[kick][dim].valid) return VP_OK;
    if (c->g.precision == VP_F32) return tune_t<float>(c, kick, dim);
    return tune_t<double>(c, kick, dim);
}
