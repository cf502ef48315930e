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
#include "vp_sweep_core.cuh"
#include "vp_tma.cuh"

namespace {

using vp_core::line_class;
using vp_core::walk;

// running-pointer store of one line's new values (element stride `step`
// between consecutive cells of the walk)
template <typename T>
struct PtrStore {
    T *p;
    long long step;
    __device__ __forceinline__ void operator()(int, T v) {
        *p = v;
        p += step;
    }
};

// staged-load strided sweep: tile = W columns x the whole line, staged as
// rows GP..GP+L-1 of a [(L + 2 GP)][W] shared tile; zero-inflow lines get GP =
// VP_GHOST zero rows on each side, periodic lines none.  PAIR (FP32 only): a
// thread walks two adjacent columns at once with the packed pair arithmetic
// (W / 2 threads per segment row); a pair whose lines differ in their integer
// shift or direction is walked one line after the other.
// largest CTA of the two-line kernels and the CTAs per SM their register
// budget must allow
#define VP_PAIR_THREADS 512
#define VP_PAIR_MINB 1

template <typename T, int ORDER, bool PERIODIC, bool FULL, bool PAIR>
__global__ void __launch_bounds__(PAIR ? VP_PAIR_THREADS : 512, PAIR ? VP_PAIR_MINB : 1)
    k_sweep_cols(T *__restrict__ f,
                                                    const LineShift<T> *__restrict__ tab,
                                                    SweepGeo geo, LimParams lp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int GP = PERIODIC ? 0 : VP_GHOST;
    T *sm = reinterpret_cast<T *>(smraw);
    const int W = geo.W, L = geo.L;
    const unsigned o = fdiv(blockIdx.x, geo.fd_tpo);
    const unsigned c0 = (blockIdx.x - o * geo.tpo) * (unsigned)W;
    const int wc = (int)((geo.inner - c0) < W ? (geo.inner - c0) : W);
    T *base = f + (long long)o * L * geo.inner + c0;
    T *data = sm + GP * W;  // row 0 of the line
    for (int e = threadIdx.x; e < GP * W; e += blockDim.x) {
        sm[e] = T(0);
        data[L * W + e] = T(0);
    }
    constexpr int VEC = 16 / sizeof(T);
    const int wv = W / VEC;
    if (wc == W && geo.inner % VEC == 0 && W % VEC == 0 && fmod_u(blockDim.x, geo.fd_wv) == 0) {
        // every 16-byte piece of the tile in flight at once (cp.async), so the
        // staging is not limited by one outstanding load per thread
        const int r = (int)fdiv(threadIdx.x, geo.fd_wv);
        const int cv = threadIdx.x - r * wv;
        const int rstep = (int)fdiv(blockDim.x, geo.fd_wv);
        const T *src = base + (long long)r * geo.inner + cv * VEC;
        T *dst = data + r * W + cv * VEC;
        const long long sstep = (long long)rstep * geo.inner;
        for (int rr = r; rr < L; rr += rstep) {
            vp_tma::cp_async16(dst, src);
            src += sstep;
            dst += rstep * W;
        }
        vp_tma::cp_async_wait_all();
    } else {
        // row / column of element e advanced incrementally (no division per element)
        const int dr = (int)fdiv(blockDim.x, geo.fd_w), dc = blockDim.x - dr * W;
        int r = (int)fdiv(threadIdx.x, geo.fd_w), cc = threadIdx.x - r * W;
        for (int e = threadIdx.x; e < L * W; e += blockDim.x) {
            data[e] = cc < wc ? base[(long long)r * geo.inner + cc] : T(0);
            r += dr;
            cc += dc;
            if (cc >= W) {
                cc -= W;
                ++r;
            }
        }
    }
    __syncthreads();
    constexpr int G1 = PERIODIC ? 1 : VP_GHOST;
    if constexpr (PAIR) {
        const unsigned seg = fdiv(threadIdx.x, geo.fd_w2);
        const int cc = 2 * (int)(threadIdx.x - seg * (unsigned)(W >> 1));
        if (cc >= wc || (int)seg >= geo.nseg) return;
        const int r0 = (int)fdiv(seg * (unsigned)L, geo.fd_nseg);
        const int r1 = (int)fdiv((seg + 1) * (unsigned)L, geo.fd_nseg);
        const LineShift<float> sa = tab[line_class(geo, o, c0 + cc)];
        if (cc + 1 < wc) {
            const LineShift<float> sb = tab[line_class(geo, o, c0 + cc + 1)];
            if (sa.n == sb.n && sa.sigma == sb.sigma) {
                const vp_core::LineShiftP2 sh = vp_core::pair_shift(sa, sb);
                const int i0 = sh.sigma > 0 ? r0 : r1 - 1;
                PtrStore<vp_core::P2> st{reinterpret_cast<vp_core::P2 *>(base + cc + (long long)i0 * geo.inner),
                                         (long long)sh.sigma * (geo.inner >> 1)};
                walk<vp_core::P2, ORDER, PERIODIC, FULL, G1>(reinterpret_cast<const vp_core::P2 *>(data + cc),
                                                             W >> 1, L, sh, r0, r1, vp_core::P2((float)lp.alpha),
                                                             lp.mp, lp.pp, st);
                return;
            }
            const int i1 = sb.sigma > 0 ? r0 : r1 - 1;
            PtrStore<T> st{base + cc + 1 + (long long)i1 * geo.inner, (long long)sb.sigma * geo.inner};
            walk<T, ORDER, PERIODIC, FULL, G1>(data + cc + 1, W, L, sb, r0, r1, (T)lp.alpha, lp.mp, lp.pp, st);
        }
        const int i0 = sa.sigma > 0 ? r0 : r1 - 1;
        PtrStore<T> st{base + cc + (long long)i0 * geo.inner, (long long)sa.sigma * geo.inner};
        walk<T, ORDER, PERIODIC, FULL, G1>(data + cc, W, L, sa, r0, r1, (T)lp.alpha, lp.mp, lp.pp, st);
    } else {
        const unsigned seg = fdiv(threadIdx.x, geo.fd_w);
        const int cc = (int)(threadIdx.x - seg * (unsigned)W);
        if (cc < wc && (int)seg < geo.nseg) {
            const LineShift<T> sh = tab[line_class(geo, o, c0 + cc)];
            const int r0 = (int)fdiv(seg * (unsigned)L, geo.fd_nseg);
            const int r1 = (int)fdiv((seg + 1) * (unsigned)L, geo.fd_nseg);
            const int i0 = sh.sigma > 0 ? r0 : r1 - 1;
            PtrStore<T> st{base + cc + (long long)i0 * geo.inner, (long long)sh.sigma * geo.inner};
            walk<T, ORDER, PERIODIC, FULL, G1>(data + cc, W, L, sh, r0, r1, (T)lp.alpha, lp.mp, lp.pp, st);
        }
    }
}

// contiguous-axis sweep: R lines per CTA.  Input rows at odd pitch P with a
// zero ghost on each side, results to a second shared tile (odd pitch Q), then
// copied out with 16-byte coalesced stores.  PAIR (FP32 only): lines 2q and
// 2q + 1 are interleaved element by element in shared memory (pair pitch 2P,
// 2Q) so that one thread walks both with 8-byte loads and stores and the
// packed pair arithmetic; a pair whose lines differ in their integer shift or
// direction, and the odd last line of a ragged tile, are walked one line at
// a time (element stride 2).  The 16-lane phases of 8-byte accesses stay
// conflict-free because P is odd.
template <typename T, int ORDER, bool PERIODIC, bool FULL, bool PAIR>
__global__ void __launch_bounds__(PAIR ? VP_PAIR_THREADS : 512, PAIR ? VP_PAIR_MINB : 1)
    k_sweep_rows(T *__restrict__ f,
                                                    const LineShift<T> *__restrict__ tab,
                                                    SweepGeo geo, LimParams lp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int GP = PERIODIC ? 0 : VP_GHOST;
    const int L = geo.L, R = geo.R;
    const int P = (L + 2 * GP) | 1;
    const int Q = L | 1;
    T *in = reinterpret_cast<T *>(smraw);
    T *out = in + R * P;
    const long long l0 = (long long)blockIdx.x * R;
    const int nl = (int)((geo.outer - l0) < R ? (geo.outer - l0) : R);
    T *base = f + l0 * L;
    const int tot = nl * L;
    // shared-memory index of cell pos of line r in the input / output tile
    auto iidx = [&](int r, int pos) -> int {
        return PAIR ? (r >> 1) * (2 * P) + 2 * (GP + pos) + (r & 1) : r * P + GP + pos;
    };
    auto oidx = [&](int r, int pos) -> int { return PAIR ? (r >> 1) * (2 * Q) + 2 * pos + (r & 1) : r * Q + pos; };
    if (GP > 0) {
        constexpr int G = GP > 0 ? GP : 1;
        for (int e = threadIdx.x; e < nl * G; e += blockDim.x) {
            const int r = e / G, k = e - r * G;
            in[iidx(r, k - G)] = T(0);
            in[iidx(r, L + k)] = T(0);
        }
    }
    constexpr int VEC = 16 / sizeof(T);
    const bool vec = (L % VEC) == 0;
    // Element e = r L + pos of the tile: a thread starts at e = VEC t (or t)
    // and advances by a fixed (rows, positions) step, so no division per element.
    if (vec) {
        constexpr int U = 4;  // 16-byte loads in flight per thread
        const int st = blockDim.x * VEC;
        const int dr = (int)fdiv(st, geo.fd_l), dp = st - dr * L;
        int r = (int)fdiv(threadIdx.x * VEC, geo.fd_l), pos = threadIdx.x * VEC - r * L;
        int e = threadIdx.x * VEC;
        for (; e + (U - 1) * st < tot; e += U * st) {
            float4 x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) x[u] = *reinterpret_cast<const float4 *>(base + e + u * st);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const T *xv = reinterpret_cast<const T *>(&x[u]);
                const int i0 = iidx(r, pos);
#pragma unroll
                for (int k = 0; k < VEC; ++k) in[i0 + (PAIR ? 2 * k : k)] = xv[k];
                r += dr;
                pos += dp;
                if (pos >= L) {
                    pos -= L;
                    ++r;
                }
            }
        }
        for (; e < tot; e += st) {
            const float4 x = *reinterpret_cast<const float4 *>(base + e);
            const T *xv = reinterpret_cast<const T *>(&x);
            const int i0 = iidx(r, pos);
#pragma unroll
            for (int k = 0; k < VEC; ++k) in[i0 + (PAIR ? 2 * k : k)] = xv[k];
            r += dr;
            pos += dp;
            if (pos >= L) {
                pos -= L;
                ++r;
            }
        }
    } else {
        const int dr = (int)fdiv(blockDim.x, geo.fd_l), dp = blockDim.x - dr * L;
        int r = (int)fdiv(threadIdx.x, geo.fd_l), pos = threadIdx.x - r * L;
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            in[iidx(r, pos)] = base[e];
            r += dr;
            pos += dp;
            if (pos >= L) {
                pos -= L;
                ++r;
            }
        }
    }
    __syncthreads();
    constexpr int G1 = PERIODIC ? 1 : VP_GHOST;
    if constexpr (PAIR) {
        const unsigned seg = fdiv(threadIdx.x, geo.fd_w2);
        const int line = 2 * (int)(threadIdx.x - seg * (unsigned)(R >> 1));
        if (line < nl && (int)seg < geo.nseg) {
            const int r0 = (int)fdiv(seg * (unsigned)L, geo.fd_nseg);
            const int r1 = (int)fdiv((seg + 1) * (unsigned)L, geo.fd_nseg);
            const LineShift<float> sa = tab[line_class(geo, (unsigned)(l0 + line), 0u)];
            bool paired = false;
            if (line + 1 < nl) {
                const LineShift<float> sb = tab[line_class(geo, (unsigned)(l0 + line + 1), 0u)];
                if (sa.n == sb.n && sa.sigma == sb.sigma) {
                    const vp_core::LineShiftP2 sh = vp_core::pair_shift(sa, sb);
                    const int i0 = sh.sigma > 0 ? r0 : r1 - 1;
                    PtrStore<vp_core::P2> st{reinterpret_cast<vp_core::P2 *>(out + oidx(line, i0)), sh.sigma};
                    walk<vp_core::P2, ORDER, PERIODIC, FULL, G1>(
                        reinterpret_cast<const vp_core::P2 *>(in + iidx(line, 0)), 1, L, sh, r0, r1,
                        vp_core::P2((float)lp.alpha), lp.mp, lp.pp, st);
                    paired = true;
                } else {
                    const int i1 = sb.sigma > 0 ? r0 : r1 - 1;
                    PtrStore<T> st{out + oidx(line + 1, i1), 2LL * sb.sigma};
                    walk<T, ORDER, PERIODIC, FULL, G1>(in + iidx(line + 1, 0), 2, L, sb, r0, r1, (T)lp.alpha,
                                                       lp.mp, lp.pp, st);
                }
            }
            if (!paired) {
                const int i0 = sa.sigma > 0 ? r0 : r1 - 1;
                PtrStore<T> st{out + oidx(line, i0), 2LL * sa.sigma};
                walk<T, ORDER, PERIODIC, FULL, G1>(in + iidx(line, 0), 2, L, sa, r0, r1, (T)lp.alpha, lp.mp,
                                                   lp.pp, st);
            }
        }
    } else {
        const unsigned seg = fdiv(threadIdx.x, geo.fd_w);
        const int line = (int)(threadIdx.x - seg * (unsigned)R);
        if (line < nl && (int)seg < geo.nseg) {
            const LineShift<T> sh = tab[line_class(geo, (unsigned)(l0 + line), 0u)];
            const int r0 = (int)fdiv(seg * (unsigned)L, geo.fd_nseg);
            const int r1 = (int)fdiv((seg + 1) * (unsigned)L, geo.fd_nseg);
            const int i0 = sh.sigma > 0 ? r0 : r1 - 1;
            PtrStore<T> st{out + line * Q + i0, (long long)sh.sigma};
            walk<T, ORDER, PERIODIC, FULL, G1>(in + line * P + GP, 1, L, sh, r0, r1, (T)lp.alpha, lp.mp, lp.pp,
                                               st);
        }
    }
    __syncthreads();
    if (vec) {
        const int st = blockDim.x * VEC;
        const int dr = (int)fdiv(st, geo.fd_l), dp = st - dr * L;
        int r = (int)fdiv(threadIdx.x * VEC, geo.fd_l), pos = threadIdx.x * VEC - r * L;
        for (int e = threadIdx.x * VEC; e < tot; e += st) {
            float4 x;
            T *xv = reinterpret_cast<T *>(&x);
            const int o0 = oidx(r, pos);
#pragma unroll
            for (int k = 0; k < VEC; ++k) xv[k] = out[o0 + (PAIR ? 2 * k : k)];
            *reinterpret_cast<float4 *>(base + e) = x;
            r += dr;
            pos += dp;
            if (pos >= L) {
                pos -= L;
                ++r;
            }
        }
    } else {
        const int dr = (int)fdiv(blockDim.x, geo.fd_l), dp = blockDim.x - dr * L;
        int r = (int)fdiv(threadIdx.x, geo.fd_l), pos = threadIdx.x - r * L;
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            base[e] = out[oidx(r, pos)];
            r += dr;
            pos += dp;
            if (pos >= L) {
                pos -= L;
                ++r;
            }
        }
    }
}

// TMA-fed persistent strided sweep (two input and two output stages)
template <typename T, int ORDER, bool PERIODIC, bool FULL>
__global__ void __launch_bounds__(512) k_sweep_cols_tma(const __grid_constant__ CUtensorMap tmap,
                                                        const LineShift<T> *__restrict__ tab,
                                                        SweepGeo geo, LimParams lp,
                                                        int *__restrict__ status, unsigned wait_limit) {
    extern __shared__ __align__(128) unsigned char smraw_tma[];
    unsigned char *smraw = smraw_tma;
    __shared__ __align__(8) uint64_t bar[2];
    constexpr int GP = PERIODIC ? 0 : VP_GHOST;
    const int W = geo.W, L = geo.L;
    const int itile = (L + 2 * GP) * W;  // input stage: GP zero rows, L rows, GP zero rows
    const int otile = L * W;
    // TMA tensor copies need 128-byte aligned shared-memory buffers: align
    // the dynamic region explicitly (the launch reserves 128 spare bytes)
    const uint32_t sbase = vp_tma::saddr(smraw);
    const uint32_t pad = (128u - (sbase & 127u)) & 127u;
    T *in_buf = reinterpret_cast<T *>(smraw + pad);  // [2][L + 2 GP][W]
    T *out_buf = in_buf + 2 * itile;                  // [2][L][W]
    const unsigned tpo = geo.tpo;
    const unsigned ntiles = (unsigned)geo.outer * tpo;
    const uint32_t bytes = (uint32_t)(otile * sizeof(T));
    // self-check of every alignment the copies rely on; on failure report and
    // leave before issuing any copy
    if (((vp_tma::saddr(in_buf + GP * W) | vp_tma::saddr(in_buf + itile + GP * W) | vp_tma::saddr(out_buf) |
          vp_tma::saddr(out_buf + otile)) & 127u) != 0 ||
        ((W * sizeof(T)) & 127u) != 0) {
        if (threadIdx.x == 0) atomicExch(status, VP_EINVAL);
        return;
    }
    for (int e = threadIdx.x; e < GP * W; e += blockDim.x) {
        in_buf[e] = T(0);
        in_buf[(GP + L) * W + e] = T(0);
        in_buf[itile + e] = T(0);
        in_buf[itile + (GP + L) * W + e] = T(0);
    }
    if (threadIdx.x == 0) {
        vp_tma::mbar_init(&bar[0], 1);
        vp_tma::mbar_init(&bar[1], 1);
        vp_tma::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            const unsigned t = blockIdx.x + (unsigned)s * gridDim.x;
            if (t < ntiles) {
                vp_tma::mbar_expect_tx(&bar[s], bytes);
                vp_tma::load_3d(in_buf + s * itile + GP * W, &tmap, &bar[s], (int)((t % tpo) * W), 0,
                                (int)(t / tpo));
            }
        }
    }
    const unsigned seg = fdiv(threadIdx.x, geo.fd_w);
    const int cc = (int)(threadIdx.x - seg * (unsigned)W);
    const int r0 = (int)fdiv(seg * (unsigned)L, geo.fd_nseg);
    const int r1 = (int)fdiv((seg + 1) * (unsigned)L, geo.fd_nseg);
    int k = 0;
    for (unsigned t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = k & 1;
        T *in = in_buf + s * itile;
        T *out = out_buf + s * otile;
        const bool arrived = vp_tma::mbar_wait(&bar[s], (uint32_t)((k >> 1) & 1), wait_limit);
        if (__syncthreads_or(!arrived)) {
            // a thread gave up on the tile: report, wait (bounded) for this
            // CTA's loads still in flight (this tile's and the next one's)
            // and for its stores, leave
            if (threadIdx.x == 0) {
                atomicExch(status, VP_ETIMEOUT);
                vp_tma::mbar_wait(&bar[s], (uint32_t)((k >> 1) & 1), 1u << 22);
                if (t + gridDim.x < ntiles) vp_tma::mbar_wait(&bar[s ^ 1], (uint32_t)(((k + 1) >> 1) & 1), 1u << 22);
                vp_tma::wait_all<0>();
            }
            return;
        }
        const unsigned o = fdiv(t, geo.fd_tpo);
        const unsigned c0 = (t - o * tpo) * (unsigned)W;
        const int wc = (int)((geo.inner - c0) < W ? (geo.inner - c0) : W);
        if (cc < wc && (int)seg < geo.nseg) {
            const LineShift<T> sh = tab[line_class(geo, o, c0 + cc)];
            const int i0 = sh.sigma > 0 ? r0 : r1 - 1;
            PtrStore<T> st{out + cc + i0 * W, (long long)sh.sigma * W};
            walk<T, ORDER, PERIODIC, FULL, PERIODIC ? 1 : VP_GHOST>(in + GP * W + cc, W, L, sh, r0, r1,
                                                                     (T)lp.alpha, lp.mp, lp.pp, st);
        }
        vp_tma::fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            vp_tma::store_3d(&tmap, out, (int)c0, 0, (int)o);
            vp_tma::commit();
            const unsigned tn = t + 2u * gridDim.x;
            if (tn < ntiles) {
                vp_tma::mbar_expect_tx(&bar[s], bytes);
                const unsigned on = fdiv(tn, geo.fd_tpo);
                vp_tma::load_3d(in + GP * W, &tmap, &bar[s], (int)((tn - on * tpo) * W), 0, (int)on);
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
    const double speed = kick ? accel[c] : vp_core::cell_centre(lo, dvel, c);
    tab[c] = vp_core::make_shift<T>(speed, dt, h, wp);
}

template <typename T, int ORDER, bool PER, bool FULL>
void set_attrs_one() {
    cudaFuncSetAttribute(k_sweep_cols<T, ORDER, PER, FULL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    if constexpr (sizeof(T) == 4)
        cudaFuncSetAttribute(k_sweep_cols<T, ORDER, PER, FULL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
    cudaFuncSetAttribute(k_sweep_rows<T, ORDER, PER, FULL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    if constexpr (sizeof(T) == 4)
        cudaFuncSetAttribute(k_sweep_rows<T, ORDER, PER, FULL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
    cudaFuncSetAttribute(k_sweep_cols_tma<T, ORDER, PER, FULL>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <typename T, int ORDER>
void set_attrs() {
    set_attrs_one<T, ORDER, true, true>();
    set_attrs_one<T, ORDER, false, true>();
    set_attrs_one<T, ORDER, true, false>();
    set_attrs_one<T, ORDER, false, false>();
}

// compile-time dispatch on the scheme order, the line's periodicity and
// whether both limiters are on
#define VP_DISPATCH(ORDER_, PER_, FULL_, CALL)                         \
    do {                                                               \
        if ((ORDER_) == 7) {                                           \
            if (PER_) {                                                \
                if (FULL_) { CALL(7, true, true); }                    \
                else { CALL(7, true, false); }                         \
            } else {                                                   \
                if (FULL_) { CALL(7, false, true); }                   \
                else { CALL(7, false, false); }                        \
            }                                                          \
        } else {                                                       \
            if (PER_) {                                                \
                if (FULL_) { CALL(5, true, true); }                    \
                else { CALL(5, true, false); }                         \
            } else {                                                   \
                if (FULL_) { CALL(5, false, true); }                   \
                else { CALL(5, false, false); }                        \
            }                                                          \
        }                                                              \
    } while (0)

// geometry of the sweep along axis `dim` (kick: velocity axis, else spatial)

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

// ghost rows staged on each side of a line
inline int ghost_rows(const SweepGeo &geo) { return geo.periodic ? 0 : VP_GHOST; }

template <typename T>
size_t tma_smem(int L, int W, int gp) {
    return (size_t)(2 * (L + 2 * gp) * W + 2 * L * W) * sizeof(T) + 128;
}

template <typename T>
bool tma_eligible(const vp_ctx *c, const SweepGeo &geo, int W) {
    constexpr int VEC = 16 / sizeof(T);
    return geo.inner > 1 && geo.inner % VEC == 0 && W % VEC == 0 && geo.inner < (1LL << 31) &&
           geo.outer < (1LL << 31) && geo.L <= 256 && W <= 256 &&
           (W * sizeof(T)) % 128 == 0 && tma_smem<T>(geo.L, W, ghost_rows(geo)) <= 200 * 1024 &&
           tensor_map_encoder() != nullptr &&
           (reinterpret_cast<uintptr_t>(c->f) & 15) == 0;
}

// the pair walker: FP32, even columns per tile and row stride (8-byte pairs)
template <typename T>
bool pair_eligible(const vp_ctx *c, const SweepGeo &geo, int W) {
    return sizeof(T) == 4 && geo.inner > 1 && geo.inner % 2 == 0 && W % 2 == 0 &&
           (reinterpret_cast<uintptr_t>(c->f) & 7) == 0;
}

// line classes and tile coordinates are computed in 32-bit arithmetic
inline bool geo_fits_32(const SweepGeo &geo) { return geo.outer < (1LL << 32) && geo.inner < (1LL << 32); }

template <typename T>
int launch_cols(vp_ctx *c, SweepGeo geo, const SweepTune &tu) {
    if (!geo_fits_32(geo)) return vp_fail(c, VP_ENOTSUP, "sweep geometry exceeds 32-bit line indexing");
    const LineShift<T> *tab = static_cast<const LineShift<T> *>(c->d_shift);
    const LimParams lp{c->g.alpha, c->g.mp, c->g.pp};
    T *f = static_cast<T *>(c->f);
    const int L = geo.L;
    int W = tu.W;
    if (geo.inner < W) W = (int)geo.inner;
    const bool pair = tu.impl == 3 && pair_eligible<T>(c, geo, W);
    // walkers per segment row: W lines, or W / 2 line pairs; at most 512 threads
    const int per_row = pair ? W >> 1 : W;
    int nseg = tu.nseg;
    while (nseg > 1 && per_row * nseg > (pair ? VP_PAIR_THREADS : 512)) nseg >>= 1;
    geo.W = W;
    geo.nseg = nseg;
    const int threads = ((per_row * nseg + 31) / 32) * 32;
    const long long tiles = geo.outer * ((geo.inner + W - 1) / W);
    if (tiles >= (1LL << 31)) return vp_fail(c, VP_ENOTSUP, "sweep has too many tiles");
    geo.tpo = (unsigned)((geo.inner + W - 1) / W);
    geo.fd_tpo = make_fastdiv(geo.tpo);
    geo.fd_w = make_fastdiv((unsigned)W);
    geo.fd_nseg = make_fastdiv((unsigned)nseg);
    geo.fd_wv = make_fastdiv((unsigned)(W / (16 / sizeof(T)) > 0 ? W / (16 / sizeof(T)) : 1));
    const int order = c->g.order;
    const bool per = geo.periodic != 0;
    const bool full = c->g.mp && c->g.pp;
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
        const size_t smem = tma_smem<T>(L, W, ghost_rows(geo));
        int per_sm = tu.ctas_per_sm;
        if (per_sm <= 0) {
#define VP_OCC(O, P, F) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_cols_tma<T, O, P, F>, threads, smem)
            VP_DISPATCH(order, per, full, VP_OCC);
#undef VP_OCC
            per_sm = per_sm < 1 ? 1 : per_sm;
        }
        long long grid = (long long)per_sm * c->sm_count;
        grid = grid > tiles ? tiles : grid;
#define VP_LAUNCH(O, P, F) \
    k_sweep_cols_tma<T, O, P, F><<<(unsigned)grid, threads, smem, c->stream>>>(map, tab, geo, lp, c->d_status, \
                                                                                c->opt_wait_limit)
        VP_DISPATCH(order, per, full, VP_LAUNCH);
#undef VP_LAUNCH
    } else if (pair) {
        const size_t smem = (size_t)(L + 2 * ghost_rows(geo)) * W * sizeof(T);
        if (smem > 200 * 1024) return vp_fail(c, VP_ENOTSUP, "line of %d cells too long to stage", L);
        const int pthreads = threads;
        geo.fd_w2 = make_fastdiv((unsigned)(W >> 1));
#define VP_LAUNCH(O, P, F) \
    k_sweep_cols<T, O, P, F, sizeof(T) == 4><<<(unsigned)tiles, pthreads, smem, c->stream>>>(f, tab, geo, lp)
        VP_DISPATCH(order, per, full, VP_LAUNCH);
#undef VP_LAUNCH
    } else {
        const size_t smem = (size_t)(L + 2 * ghost_rows(geo)) * W * sizeof(T);
        if (smem > 200 * 1024) return vp_fail(c, VP_ENOTSUP, "line of %d cells too long to stage", L);
#define VP_LAUNCH(O, P, F) \
    k_sweep_cols<T, O, P, F, false><<<(unsigned)tiles, threads, smem, c->stream>>>(f, tab, geo, lp)
        VP_DISPATCH(order, per, full, VP_LAUNCH);
#undef VP_LAUNCH
    }
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

template <typename T>
size_t rows_smem(int L, int R, int gp) {
    return (size_t)R * (((L + 2 * gp) | 1) + (L | 1)) * sizeof(T);
}

template <typename T>
int launch_rows(vp_ctx *c, SweepGeo geo, const SweepTune &tu) {
    if (!geo_fits_32(geo)) return vp_fail(c, VP_ENOTSUP, "sweep geometry exceeds 32-bit line indexing");
    const LineShift<T> *tab = static_cast<const LineShift<T> *>(c->d_shift);
    const LimParams lp{c->g.alpha, c->g.mp, c->g.pp};
    T *f = static_cast<T *>(c->f);
    const int L = geo.L;
    int R = tu.W;
    if (geo.outer < R) R = (int)geo.outer;
    const bool pair = tu.impl == 3 && sizeof(T) == 4;
    if (pair && (R & 1)) ++R;  // a single ragged tile keeps an empty slot
    // walkers per segment row: R lines, or R / 2 line pairs; at most 512 threads
    const int per_row = pair ? R >> 1 : R;
    int nseg = tu.nseg;
    while (nseg > 1 && per_row * nseg > (pair ? VP_PAIR_THREADS : 512)) nseg >>= 1;
    geo.R = R;
    geo.nseg = nseg;
    geo.fd_w = make_fastdiv((unsigned)R);
    geo.fd_nseg = make_fastdiv((unsigned)nseg);
    geo.fd_l = make_fastdiv((unsigned)L);
    const long long blocks = (geo.outer + R - 1) / R;
    if (blocks >= (1LL << 31)) return vp_fail(c, VP_ENOTSUP, "sweep has too many tiles");
    const size_t smem = rows_smem<T>(L, R, ghost_rows(geo));
    if (smem > 200 * 1024) return vp_fail(c, VP_ENOTSUP, "line of %d cells too long to stage", L);
    const int threads = ((per_row * nseg + 31) / 32) * 32;
    const bool per = geo.periodic != 0;
    const bool full = c->g.mp && c->g.pp;
    if (pair) {
        geo.fd_w2 = make_fastdiv((unsigned)(R >> 1));
        const int pthreads = threads;
#define VP_LAUNCH(O, P, F) \
    k_sweep_rows<T, O, P, F, sizeof(T) == 4><<<(unsigned)blocks, pthreads, smem, c->stream>>>(f, tab, geo, lp)
        VP_DISPATCH(c->g.order, per, full, VP_LAUNCH);
#undef VP_LAUNCH
    } else {
#define VP_LAUNCH(O, P, F) \
    k_sweep_rows<T, O, P, F, false><<<(unsigned)blocks, threads, smem, c->stream>>>(f, tab, geo, lp)
        VP_DISPATCH(c->g.order, per, full, VP_LAUNCH);
#undef VP_LAUNCH
    }
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
        // long lines: narrower tiles (down to 4 columns) so the staged lines fit
        while (W > 4 && (size_t)(L + 2 * ghost_rows(geo)) * W * sizeof(T) > 200 * 1024) W /= 2;
        int nseg = L / 8;
        const int maxseg = 256 / W > 0 ? 256 / W : 1;
        nseg = nseg > maxseg ? maxseg : (nseg < 1 ? 1 : nseg);
        tu.W = W;
        tu.nseg = nseg;
        const int want = c->opt_impl ? c->opt_impl : 3;
        const int Weff = W < geo.inner ? W : (int)geo.inner;
        tu.impl = (want == 2 && tma_eligible<T>(c, geo, Weff)) ? 2 : (want == 3 && pair_eligible<T>(c, geo, Weff)) ? 3 : 1;
    } else {
        int R = 4096 / L;
        R = R < 32 ? 32 : (R > 128 ? 128 : R);
        while (R > 1 && rows_smem<T>(L, R, ghost_rows(geo)) > 96 * 1024) R /= 2;  // long lines
        int nseg = L / 16;
        const int maxseg = 256 / R > 0 ? 256 / R : 1;
        nseg = nseg > maxseg ? maxseg : (nseg < 1 ? 1 : nseg);
        tu.W = R;
        tu.nseg = nseg;
        const int want = c->opt_impl ? c->opt_impl : 3;
        tu.impl = want == 3 && sizeof(T) == 4 && R % 2 == 0 ? 3 : 1;
    }
    return tu;
}

template <typename T>
int launch_sweep_t(vp_ctx *c, int kick, int dim) {
    const SweepGeo geo = vp_make_geo(c, kick, dim);
    SweepTune tu = c->tune[kick][dim];
    if (!tu.valid || (c->opt_impl && tu.impl != c->opt_impl)) tu = default_tune<T>(c, geo);
    if (c->opt_impl == 1) tu.impl = 1;
    if (geo.inner > 1) return launch_cols<T>(c, geo, tu);
    return launch_rows<T>(c, geo, tu);
}

// Autotuner: time candidate tile shapes of one sweep geometry with the
// sweep's own shifts (dt, accel) on a copy of a window at the centre of f --
// whole outer blocks, or where one block exceeds the budget the middle
// columns of every row -- of at most kTuneBytes (larger than L2, so the
// timing sees HBM), and keep the fastest.  The window keeps every line's
// shift class (its offset is a whole number of class periods; a kick window
// reads the shift table from its first spatial point), so the limiter paths
// are timed on the state at hand where the distribution is, not on an empty
// corner of phase space; f is left untouched.  Without room for the copy the
// defaults stay.  Runs once per (kind, axis), never inside a stream capture.
constexpr size_t kTuneBytes = size_t(256) << 20;

template <typename T>
int tune_on(vp_ctx *c, int kick, int dim, const SweepGeo &geo, const SweepGeo &sub, SweepTune best);

template <typename T>
int tune_t(vp_ctx *c, int kick, int dim, double dt, const double *accel) {
    const SweepGeo geo = vp_make_geo(c, kick, dim);
    SweepTune best = default_tune<T>(c, geo);
    SweepGeo sub = geo;
    const size_t block = (size_t)geo.L * (size_t)geo.inner * sizeof(T);
    size_t bytes;
    bool pitched = false;
    long long o0 = 0, c0 = 0;  // window offset: outer blocks, columns
    // flattened index of the central cell of spatial axes [a, b)
    auto centre = [&](int a, int b) {
        long long i = 0;
        for (int k = a; k < b; ++k) i = i * c->g.nx[k] + c->g.nx[k] / 2;
        return i;
    };
    auto clampll = [](long long x, long long lo, long long hi) { return x < lo ? lo : (x > hi ? hi : x); };
    // the window's middle: the central spatial cell (and middle velocity)
    const long long o_mid = kick ? centre(0, c->g.dx) * geo.cdiv + geo.cdiv / 2 : centre(0, dim);
    const long long c_mid = kick ? 0 : centre(dim + 1, c->g.dx) * c->NV + c->NV / 2;
    if (block <= kTuneBytes) {
        const long long no = (long long)(kTuneBytes / block);
        sub.outer = no < geo.outer ? no : geo.outer;
        o0 = clampll(o_mid - sub.outer / 2, 0, geo.outer - sub.outer);
        if (!geo.cls_from_inner) o0 -= o0 % geo.cdiv;  // whole spatial points
        bytes = (size_t)sub.outer * block;
    } else {
        long long ni = (long long)(kTuneBytes / ((size_t)geo.L * sizeof(T)));
        if (ni >= 128) ni &= ~127LL;
        if (ni < 1) ni = 1;
        sub.outer = 1;
        sub.inner = ni < geo.inner ? ni : geo.inner;
        o0 = clampll(o_mid, 0, geo.outer - 1);
        if (!geo.cls_from_inner) o0 -= o0 % geo.cdiv;
        // whole velocity periods of the line classes, and 16-byte rows
        const long long per = 4 * (geo.cls_from_inner ? geo.cdiv * geo.cmod : 1);
        c0 = clampll(c_mid - sub.inner / 2, 0, geo.inner - sub.inner);
        c0 -= c0 % per;
        bytes = (size_t)geo.L * (size_t)sub.inner * sizeof(T);
        pitched = true;
    }
    const T *src = static_cast<const T *>(c->f) + (o0 * geo.L * geo.inner + c0);
    void *scratch = nullptr;
    if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        c->tune[kick][dim] = best;
        return VP_OK;
    }
    int rc = VP_OK;
    if (pitched)
        rc = cudaMemcpy2DAsync(scratch, (size_t)sub.inner * sizeof(T), src, (size_t)geo.inner * sizeof(T),
                               (size_t)sub.inner * sizeof(T), (size_t)geo.L, cudaMemcpyDeviceToDevice,
                               c->stream) == cudaSuccess ? VP_OK : vp_fail(c, VP_ECUDA, "tuning copy failed");
    else
        rc = cudaMemcpyAsync(scratch, src, bytes, cudaMemcpyDeviceToDevice, c->stream) == cudaSuccess
                 ? VP_OK : vp_fail(c, VP_ECUDA, "tuning copy failed");
    if (rc == VP_OK) rc = vp_launch_shift_table(c, kick, dim, dt, accel);
    if (rc == VP_OK) {
        void *f = c->f, *tab = c->d_shift;
        c->f = scratch;
        if (!geo.cls_from_inner) c->d_shift = static_cast<LineShift<T> *>(c->d_shift) + o0 / geo.cdiv;
        rc = tune_on<T>(c, kick, dim, geo, sub, best);
        c->f = f;
        c->d_shift = tab;
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(scratch);
    return rc;
}

// time the candidates of geometry geo on sub (the tuning copy bound as f)
template <typename T>
int tune_on(vp_ctx *c, int kick, int dim, const SweepGeo &geo, const SweepGeo &sub, SweepTune best) {
    int rc = VP_OK;
    constexpr int kMaxCand = 48;
    SweepTune cand[kMaxCand];
    int nc = 0;
    if (geo.inner > 1) {
        const int impls[3] = {3, 2, 1};
        // lines too long for a 32-column tile take 4-16 columns and more segments
        const bool longl = (size_t)(geo.L + 2 * ghost_rows(geo)) * 32 * sizeof(T) > 200 * 1024;
        for (int ii = 0; ii < 3; ++ii) {
            if (c->opt_impl && impls[ii] != c->opt_impl) continue;
            for (int W = longl ? 4 : 32; W <= (longl ? 16 : 128); W *= 2)
                for (int nseg = 1; nseg <= (longl ? 64 : 8); nseg *= 2) {
                    const int th = (impls[ii] == 3 ? W / 2 : W) * nseg;
                    if (th < (impls[ii] == 3 ? 32 : 64) || th > (impls[ii] == 3 ? VP_PAIR_THREADS : 512) ||
                        nseg > geo.L || (longl && nseg * 8 > geo.L))
                        continue;
                    const int Weff = geo.inner < W ? (int)geo.inner : W;
                    if (impls[ii] == 2 && !tma_eligible<T>(c, geo, Weff)) continue;
                    if (impls[ii] == 3 && !pair_eligible<T>(c, geo, Weff)) continue;
                    if (impls[ii] != 2 && (size_t)(geo.L + 2 * ghost_rows(geo)) * W * sizeof(T) > 200 * 1024)
                        continue;
                    if (nc < kMaxCand) cand[nc++] = SweepTune{1, impls[ii], W, nseg, 0};
                }
        }
    } else {
        // long lines take fewer lines per CTA (the staged tile must fit) and
        // more segments per line (segments of at least 8 cells)
        for (int impl = 1; impl <= 3; impl += 2) {
            if ((c->opt_impl == 1 && impl != 1) || (c->opt_impl == 3 && impl != 3) || (impl == 3 && sizeof(T) != 4))
                continue;
            for (int R = 8; R <= 128; R *= 2)
                for (int nseg = 1; nseg <= 64; nseg *= 2) {
                    const int th = (impl == 3 ? R / 2 : R) * nseg;
                    if (th < (impl == 3 ? 32 : 64) || th > (impl == 3 ? VP_PAIR_THREADS : 512) || nseg * 8 > geo.L)
                        continue;
                    if (rows_smem<T>(geo.L, R, ghost_rows(geo)) > 200 * 1024) continue;
                    if (nc < kMaxCand) cand[nc++] = SweepTune{1, impl, R, nseg, 0};
                }
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
            rc = geo.inner > 1 ? launch_cols<T>(c, sub, cand[i]) : launch_rows<T>(c, sub, cand[i]);
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

int vp_tune_sweep(vp_ctx *c, int kick, int dim, double dt, const double *accel) {
    if (c->tune[kick][dim].valid) return VP_OK;
    if (c->g.precision == VP_F32) return tune_t<float>(c, kick, dim, dt, accel);
    return tune_t<double>(c, kick, dim, dt, accel);
}
