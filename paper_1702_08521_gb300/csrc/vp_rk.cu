// vp_rk.cu -- RK-MPP5 sweeps (Sec. 2.1.1): the spatially fifth-order
// finite-volume scheme with the MP constraint and the PP limiter, integrated
// with the three-stage TVD Runge-Kutta method (Eq. 10), the scheme the paper
// compares SL-MPP5 against.
//
// One Euler stage f - nu L(f) is the line walker with no integer shift and
// the MP5 interface value of Eq. 8 in place of the CSL interpolant: upwind
// cell u0, f^{int,5} = (2 u_-2 - 13 u_-1 + 47 u0 + 27 u1 - 3 u2) / 60, then the
// MP constraint and the PP limiter with the stage's CFL number nu = |c| dt /
// dx.  A CTA stages its lines once, runs the three stages in shared memory
// (f^n, f^(1), f^(2) side by side, a barrier between stages) and writes
// f^{n+1} = f^n / 3 + 2/3 (f^(2) - nu L(f^(2))) once: one HBM pass for three
// stages.  FP32 strided sweeps walk two adjacent lines per thread with the
// packed pair arithmetic, as the SL sweeps do.  The scheme is Eulerian: it needs |nu| < 1/2 (the PP limiter's
// condition); the shift table flags a larger one in the context's status
// word, which vp_sync reports.
#include "vp_sweep_core.cuh"
#include "vp_tma.cuh"

using vp_core::mul_rn;

namespace {

// f^{int,5} of Eq. 8 as weights on the walker's stencil (um3 .. u3)
template <typename T>
__device__ __forceinline__ void mp5_weights(T (&w)[7]) {
    w[0] = T(0);
    w[1] = T(2) / T(60);
    w[2] = T(-13) / T(60);
    w[3] = T(47) / T(60);
    w[4] = T(27) / T(60);
    w[5] = T(-3) / T(60);
    w[6] = T(0);
}

template <typename T>
__global__ void k_rk_table(LineShift<T> *__restrict__ tab, int nclass, int kick, double lo, double dvel,
                           const double *__restrict__ accel, double dt, double h, int *status) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nclass) return;
    const double speed = kick ? accel[c] : vp_core::cell_centre(lo, dvel, c);
    const double s = __ddiv_rn(__dmul_rn(speed, dt), h);
    LineShift<T> sh;
    mp5_weights(sh.w);
    sh.n = 0;
    sh.sigma = s < 0.0 ? -1 : 1;
    const double nu = fabs(s);
    if (!(nu < 0.5)) atomicExch(status, VP_ECFL);
    sh.nu = (T)nu;
    tab[c] = sh;
}

// store of one stage: row i of the stage gets ca * a_i + cv * v (a_i: the
// line's f^n at the same row); ca = 0, cv = 1 stores v itself
template <typename T>
struct StageStore {
    T *p;
    const T *a;
    long long step, astep;
    T ca, cv;
    __device__ __forceinline__ void operator()(int, T v) {
        *p = fma(cv, v, mul_rn(ca, *a));
        a += astep;
        p += step;
    }
};

// Strided lines: a tile of W consecutive lines (columns), rows at pitch W.
// PAIR (FP32): a thread walks two adjacent columns with the packed FP32 pair
// arithmetic (each half rounds as the scalar instruction: the same bits); a
// pair whose lines move in opposite directions is walked one line at a time.
template <typename T, bool PERIODIC, bool FULL, bool PAIR>
__global__ void __launch_bounds__(512) k_rk_cols(T *__restrict__ f, const LineShift<T> *__restrict__ tab,
                                                 SweepGeo geo, LimParams lp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int GP = PERIODIC ? 0 : VP_GHOST;
    const int W = geo.W, L = geo.L, LP = L + 2 * GP;
    T *A = reinterpret_cast<T *>(smraw);  // f^n
    T *B = A + LP * W;                    // f^(1)
    T *C = B + LP * W;                    // f^(2)
    const unsigned o = fdiv(blockIdx.x, geo.fd_tpo);
    const unsigned c0 = (blockIdx.x - o * geo.tpo) * (unsigned)W;
    const int wc = (int)((geo.inner - c0) < W ? (geo.inner - c0) : W);
    T *base = f + (long long)o * L * geo.inner + c0;
    for (int e = threadIdx.x; e < GP * W; e += blockDim.x) {
        A[e] = B[e] = C[e] = T(0);
        A[(GP + L) * W + e] = B[(GP + L) * W + e] = C[(GP + L) * W + e] = T(0);
    }
    T *a0 = A + GP * W, *b0 = B + GP * W, *c0p = C + GP * W;
    constexpr int VEC = 16 / sizeof(T);
    const int wv = W / VEC;
    if (wc == W && geo.inner % VEC == 0 && W % VEC == 0 && fmod_u(blockDim.x, geo.fd_wv) == 0) {
        const int r = (int)fdiv(threadIdx.x, geo.fd_wv);
        const int cv = threadIdx.x - r * wv;
        const int rstep = (int)fdiv(blockDim.x, geo.fd_wv);
        const T *src = base + (long long)r * geo.inner + cv * VEC;
        T *dst = a0 + r * W + cv * VEC;
        const long long sstep = (long long)rstep * geo.inner;
        for (int rr = r; rr < L; rr += rstep) {
            vp_tma::cp_async16(dst, src);
            src += sstep;
            dst += rstep * W;
        }
        vp_tma::cp_async_wait_all();
    } else {
        for (int e = threadIdx.x; e < L * W; e += blockDim.x) {
            const int r = (int)fdiv(e, geo.fd_w), cc = e - r * W;
            a0[e] = cc < wc ? base[(long long)r * geo.inner + cc] : T(0);
        }
    }
    __syncthreads();
    const T alpha_t = (T)lp.alpha;
    constexpr int GW = PERIODIC ? 1 : VP_GHOST;
    if constexpr (PAIR) {
        using vp_core::P2;
        const unsigned seg = fdiv(threadIdx.x, geo.fd_w2);
        const int cc = 2 * (int)(threadIdx.x - seg * (unsigned)(W >> 1));
        const bool act = cc < wc && (int)seg < geo.nseg;
        LineShift<float> sa{}, sb{};
        int r0 = 0, r1 = 0;
        bool both = false;
        if (act) {
            sa = tab[vp_core::line_class(geo, o, c0 + cc)];
            sb = cc + 1 < wc ? tab[vp_core::line_class(geo, o, c0 + cc + 1)] : sa;
            both = cc + 1 < wc && sa.sigma == sb.sigma;  // RK lines have no integer shift
            r0 = (int)fdiv(seg * (unsigned)L, geo.fd_nseg);
            r1 = (int)fdiv((seg + 1) * (unsigned)L, geo.fd_nseg);
        }
#pragma unroll 1
        for (int stage = 0; stage < 3; ++stage) {
            if (act) {
                const float ca = stage == 0 ? 0.f : (stage == 1 ? 0.75f : 1.f / 3.f);
                const float cv = stage == 0 ? 1.f : (stage == 1 ? 0.25f : 2.f / 3.f);
                const float *src = stage == 0 ? a0 : (stage == 1 ? b0 : c0p);
                float *sdst = stage == 0 ? b0 : c0p;  // stages 0, 1 write shared memory
                if (both) {
                    const vp_core::LineShiftP2 sh = vp_core::pair_shift(sa, sb);
                    const int i0 = sh.sigma > 0 ? r0 : r1 - 1;
                    P2 *dst = stage == 2 ? reinterpret_cast<P2 *>(base + cc + (long long)i0 * geo.inner)
                                         : reinterpret_cast<P2 *>(sdst + cc + i0 * W);
                    const long long dstep = stage == 2 ? (long long)sh.sigma * (geo.inner >> 1)
                                                       : (long long)sh.sigma * (W >> 1);
                    StageStore<P2> sto{dst, reinterpret_cast<const P2 *>(a0 + cc + i0 * W), dstep,
                                       (long long)sh.sigma * (W >> 1), P2(ca), P2(cv)};
                    vp_core::walk<P2, 5, PERIODIC, FULL, GW>(reinterpret_cast<const P2 *>(src + cc), W >> 1, L, sh,
                                                             r0, r1, P2((float)lp.alpha), lp.mp, lp.pp, sto);
                } else {
                    for (int k = (cc + 1 < wc ? 1 : 0); k >= 0; --k) {
                        const LineShift<float> &sl = k ? sb : sa;
                        const int i0 = sl.sigma > 0 ? r0 : r1 - 1;
                        float *dst = stage == 2 ? base + cc + k + (long long)i0 * geo.inner : sdst + cc + k + i0 * W;
                        const long long dstep = stage == 2 ? (long long)sl.sigma * geo.inner : (long long)sl.sigma * W;
                        StageStore<float> sto{dst, a0 + cc + k + i0 * W, dstep, (long long)sl.sigma * W, ca, cv};
                        vp_core::walk<float, 5, PERIODIC, FULL, GW>(src + cc + k, W, L, sl, r0, r1, (float)lp.alpha,
                                                                    lp.mp, lp.pp, sto);
                    }
                }
            }
            __syncthreads();
        }
        return;
    }
    (void)alpha_t;
    const unsigned seg = fdiv(threadIdx.x, geo.fd_w);
    const int cc = (int)(threadIdx.x - seg * (unsigned)W);
    const bool act = cc < wc && (int)seg < geo.nseg;
    LineShift<T> sh{};
    int r0 = 0, r1 = 0, i0 = 0;
    if (act) {
        sh = tab[vp_core::line_class(geo, o, c0 + cc)];
        r0 = (int)fdiv(seg * (unsigned)L, geo.fd_nseg);
        r1 = (int)fdiv((seg + 1) * (unsigned)L, geo.fd_nseg);
        i0 = sh.sigma > 0 ? r0 : r1 - 1;
    }
    const long long st = (long long)sh.sigma * W;
    const T alpha = (T)lp.alpha;
    constexpr int G = PERIODIC ? 1 : VP_GHOST;
    // stage k stores cv E(g) + ca f^n with E(g) = g - nu L(g) (Eq. 10):
    // f^(1) = E(f^n) (ca = 0), f^(2) = 3/4 f^n + 1/4 E(f^(1)),
    // f^{n+1} = 1/3 f^n + 2/3 E(f^(2)); one walker instance runs all three
#pragma unroll 1
    for (int stage = 0; stage < 3; ++stage) {
        if (act) {
            const T *src = stage == 0 ? a0 : (stage == 1 ? b0 : c0p);
            T *dst = stage == 0 ? b0 + cc + i0 * W : (stage == 1 ? c0p + cc + i0 * W : base + cc + (long long)i0 * geo.inner);
            const long long dstep = stage == 2 ? (long long)sh.sigma * geo.inner : st;
            const T ca = stage == 0 ? T(0) : (stage == 1 ? T(0.75) : T(1) / T(3));
            const T cv = stage == 0 ? T(1) : (stage == 1 ? T(0.25) : T(2) / T(3));
            StageStore<T> sto{dst, a0 + cc + i0 * W, dstep, st, ca, cv};
            vp_core::walk<T, 5, PERIODIC, FULL, G>(src + cc, W, L, sh, r0, r1, alpha, lp.mp, lp.pp, sto);
        }
        __syncthreads();
    }
}

// Contiguous lines: R lines per CTA, each a row at odd pitch P (ghosts on
// both sides); the result goes to a fourth tile at pitch Q and out in rows.
template <typename T, bool FULL>
__global__ void __launch_bounds__(512) k_rk_rows(T *__restrict__ f, const LineShift<T> *__restrict__ tab,
                                                 SweepGeo geo, LimParams lp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int GP = VP_GHOST;  // contiguous lines are velocity lines: zero inflow
    const int L = geo.L, R = geo.R;
    const int P = (L + 2 * GP) | 1;
    const int Q = L | 1;
    T *A = reinterpret_cast<T *>(smraw);
    T *B = A + R * P;
    T *C = B + R * P;
    T *out = C + R * P;
    const long long l0 = (long long)blockIdx.x * R;
    const int nl = (int)((geo.outer - l0) < R ? (geo.outer - l0) : R);
    T *base = f + l0 * L;
    const int tot = nl * L;
    for (int e = threadIdx.x; e < nl * GP; e += blockDim.x) {
        const int r = e / GP, k = e - r * GP;
        A[r * P + k] = B[r * P + k] = C[r * P + k] = T(0);
        A[r * P + GP + L + k] = B[r * P + GP + L + k] = C[r * P + GP + L + k] = T(0);
    }
    constexpr int VEC = 16 / sizeof(T);
    const bool vec = (L % VEC) == 0;  // rows start on 16-byte boundaries of f
    if (vec) {
        for (int e = threadIdx.x * VEC; e < tot; e += blockDim.x * VEC) {
            const float4 x = *reinterpret_cast<const float4 *>(base + e);
            const T *xv = reinterpret_cast<const T *>(&x);
            const int r = (int)fdiv(e, geo.fd_l), pos = e - r * L;
#pragma unroll
            for (int k = 0; k < VEC; ++k) A[r * P + GP + pos + k] = xv[k];
        }
    } else {
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int r = (int)fdiv(e, geo.fd_l), pos = e - r * L;
            A[r * P + GP + pos] = base[e];
        }
    }
    __syncthreads();
    const unsigned seg = fdiv(threadIdx.x, geo.fd_w);
    const int line = (int)(threadIdx.x - seg * (unsigned)R);
    const bool act = line < nl && (int)seg < geo.nseg;
    LineShift<T> sh{};
    int r0 = 0, r1 = 0, i0 = 0;
    if (act) {
        sh = tab[vp_core::line_class(geo, (unsigned)(l0 + line), 0u)];
        r0 = (int)fdiv(seg * (unsigned)L, geo.fd_nseg);
        r1 = (int)fdiv((seg + 1) * (unsigned)L, geo.fd_nseg);
        i0 = sh.sigma > 0 ? r0 : r1 - 1;
    }
    const T alpha = (T)lp.alpha;
    const long long sg = sh.sigma;
    T *a0 = A + line * P + GP, *b0 = B + line * P + GP, *c0p = C + line * P + GP;
    // the three stages of Eq. 10 through one walker instance (see k_rk_cols)
#pragma unroll 1
    for (int stage = 0; stage < 3; ++stage) {
        if (act) {
            const T *src = stage == 0 ? a0 : (stage == 1 ? b0 : c0p);
            T *dst = stage == 0 ? b0 + i0 : (stage == 1 ? c0p + i0 : out + line * Q + i0);
            const T ca = stage == 0 ? T(0) : (stage == 1 ? T(0.75) : T(1) / T(3));
            const T cv = stage == 0 ? T(1) : (stage == 1 ? T(0.25) : T(2) / T(3));
            StageStore<T> sto{dst, a0 + i0, sg, sg, ca, cv};
            vp_core::walk<T, 5, false, FULL, VP_GHOST>(src, 1, L, sh, r0, r1, alpha, lp.mp, lp.pp, sto);
        }
        __syncthreads();
    }
    if (vec) {
        for (int e = threadIdx.x * VEC; e < tot; e += blockDim.x * VEC) {
            float4 x;
            T *xv = reinterpret_cast<T *>(&x);
            const int r = (int)fdiv(e, geo.fd_l), pos = e - r * L;
#pragma unroll
            for (int k = 0; k < VEC; ++k) xv[k] = out[r * Q + pos + k];
            *reinterpret_cast<float4 *>(base + e) = x;
        }
    } else {
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int r = (int)fdiv(e, geo.fd_l), pos = e - r * L;
            base[e] = out[r * Q + pos];
        }
    }
}


template <typename T>
int launch_rk(vp_ctx *c, int kick, int dim) {
    SweepGeo geo = vp_make_geo(c, kick, dim);
    if (geo.outer >= (1LL << 32) || geo.inner >= (1LL << 32))
        return vp_fail(c, VP_ENOTSUP, "sweep geometry exceeds 32-bit line indexing");
    const LineShift<T> *tab = static_cast<const LineShift<T> *>(c->d_shift);
    const LimParams lp{c->g.alpha, c->g.mp, c->g.pp};
    T *f = static_cast<T *>(c->f);
    const int L = geo.L;
    if (geo.inner > 1) {
        const int gp = geo.periodic ? 0 : VP_GHOST;
        // up to 128 lines per tile within 100 KB, narrower for long lines;
        // segments of at least 16 cells (each stage restarts the walk at every
        // segment), up to 512 threads (measured best of four tile rules on the
        // Plummer 32^3 x 64^3 state)
        int W = 128;
        while (W > 32 && (size_t)3 * (L + 2 * gp) * W * sizeof(T) > 100 * 1024) W /= 2;
        while (W > 4 && (size_t)3 * (L + 2 * gp) * W * sizeof(T) > 200 * 1024) W /= 2;
        if (geo.inner < W) W = (int)geo.inner;
        const size_t smem = (size_t)3 * (L + 2 * gp) * W * sizeof(T);
        if (smem > 200 * 1024) return vp_fail(c, VP_ENOTSUP, "line of %d cells too long to stage", L);
        int nseg = L / 16;
        const int maxseg = 512 / W > 0 ? 512 / W : 1;
        nseg = nseg > maxseg ? maxseg : (nseg < 1 ? 1 : nseg);
        geo.W = W;
        geo.nseg = nseg;
        const long long tiles = geo.outer * ((geo.inner + W - 1) / W);
        if (tiles >= (1LL << 31)) return vp_fail(c, VP_ENOTSUP, "sweep has too many tiles");
        geo.tpo = (unsigned)((geo.inner + W - 1) / W);
        geo.fd_tpo = make_fastdiv(geo.tpo);
        geo.fd_w = make_fastdiv((unsigned)W);
        geo.fd_nseg = make_fastdiv((unsigned)nseg);
        geo.fd_wv = make_fastdiv((unsigned)(W / (16 / sizeof(T)) > 0 ? W / (16 / sizeof(T)) : 1));
        // FP32: two adjacent lines per thread unless the staged-load one-line
        // kernels are requested (the same bits either way)
        const bool pair = sizeof(T) == 4 && c->opt_impl != 1 && W % 2 == 0 && geo.inner % 2 == 0 &&
                          (reinterpret_cast<uintptr_t>(c->f) & 7) == 0;
        geo.fd_w2 = make_fastdiv((unsigned)(W >> 1 > 0 ? W >> 1 : 1));
        const int threads = (((pair ? W >> 1 : W) * nseg + 31) / 32) * 32;
        const bool full = c->g.mp && c->g.pp;
#define VP_RK_COLS(PER, FULL)                                                                                  \
    do {                                                                                                       \
        if (pair)                                                                                              \
            k_rk_cols<T, PER, FULL, sizeof(T) == 4><<<(unsigned)tiles, threads, smem, c->stream>>>(f, tab, geo, lp); \
        else                                                                                                   \
            k_rk_cols<T, PER, FULL, false><<<(unsigned)tiles, threads, smem, c->stream>>>(f, tab, geo, lp);    \
    } while (0)
        if (geo.periodic && full)
            VP_RK_COLS(true, true);
        else if (geo.periodic)
            VP_RK_COLS(true, false);
        else if (full)
            VP_RK_COLS(false, true);
        else
            VP_RK_COLS(false, false);
#undef VP_RK_COLS
    } else {
        const int P = (L + 2 * VP_GHOST) | 1, Q = L | 1;
        int R = 4096 / L;
        R = R < 32 ? 32 : (R > 128 ? 128 : R);
        while (R > 1 && (size_t)R * (3 * P + Q) * sizeof(T) > 96 * 1024) R /= 2;
        if (geo.outer < R) R = (int)geo.outer;
        const size_t smem = (size_t)R * (3 * P + Q) * sizeof(T);
        if (smem > 200 * 1024) return vp_fail(c, VP_ENOTSUP, "line of %d cells too long to stage", L);
        int nseg = L / 16;
        const int maxseg = 256 / R > 0 ? 256 / R : 1;
        nseg = nseg > maxseg ? maxseg : (nseg < 1 ? 1 : nseg);
        geo.R = R;
        geo.nseg = nseg;
        geo.fd_w = make_fastdiv((unsigned)R);
        geo.fd_nseg = make_fastdiv((unsigned)nseg);
        geo.fd_l = make_fastdiv((unsigned)L);
        const long long blocks = (geo.outer + R - 1) / R;
        if (blocks >= (1LL << 31)) return vp_fail(c, VP_ENOTSUP, "sweep has too many tiles");
        const int threads = ((R * nseg + 31) / 32) * 32;
        if (c->g.mp && c->g.pp)
            k_rk_rows<T, true><<<(unsigned)blocks, threads, smem, c->stream>>>(f, tab, geo, lp);
        else
            k_rk_rows<T, false><<<(unsigned)blocks, threads, smem, c->stream>>>(f, tab, geo, lp);
    }
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

template <typename T, bool FULL>
void rk_attrs_one() {
    cudaFuncSetAttribute(k_rk_cols<T, true, FULL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_rk_cols<T, false, FULL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if constexpr (sizeof(T) == 4) {
        cudaFuncSetAttribute(k_rk_cols<T, true, FULL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_rk_cols<T, false, FULL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
    cudaFuncSetAttribute(k_rk_rows<T, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <typename T>
void rk_attrs() {
    rk_attrs_one<T, true>();
    rk_attrs_one<T, false>();
}

}  // namespace

int vp_rk_setup() {
    rk_attrs<float>();
    rk_attrs<double>();
    return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ECUDA;
}

int vp_launch_rk_sweep(vp_ctx *c, int kick, int dim, double dt, const double *accel) {
    const vp_grid &g = c->g;
    const int nclass = kick ? (int)c->NX : g.nv[dim];
    const double h = kick ? (g.vhi[dim] - g.vlo[dim]) / g.nv[dim] : (g.xhi[dim] - g.xlo[dim]) / g.nx[dim];
    const double lo = g.vlo[dim];
    const double dvel = (g.vhi[dim] - g.vlo[dim]) / g.nv[dim];
    const int th = 128, bl = (nclass + th - 1) / th;
    if (g.precision == VP_F32)
        k_rk_table<float><<<bl, th, 0, c->stream>>>(static_cast<LineShift<float> *>(c->d_shift), nclass, kick, lo,
                                                   dvel, accel, dt, h, c->d_status);
    else
        k_rk_table<double><<<bl, th, 0, c->stream>>>(static_cast<LineShift<double> *>(c->d_shift), nclass, kick,
                                                    lo, dvel, accel, dt, h, c->d_status);
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return g.precision == VP_F32 ? launch_rk<float>(c, kick, dim) : launch_rk<double>(c, kick, dim);
}
