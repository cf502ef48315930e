// vp_ensemble.cu -- batched ensembles of independent 1D1V / 2D2V
// Vlasov-Poisson runs (uneven sizes) advanced one KDK step per persistent
// kernel launch, the step captured in a CUDA graph.
//
// Work queue: one step of every run is a list of items (run, stage, tile)
// sorted by stage.  Each CTA of a persistent grid pops items with an atomic
// counter (the next one while it works on the current one), waits (bounded)
// until the previous stage of that run has finished all its tiles, processes
// the tile and counts it done.  Items are popped in queue order by running
// CTAs only, and a CTA takes up its popped item right after its current one,
// which comes earlier in the queue; every item's dependencies come earlier
// still, so the earliest unfinished item is always being worked on: no
// deadlock, whatever the residency.
//
// Stages of a KDK step (Eq. 55), per run:
//   1D1V: kick v (dt/2) | drift x (dt) | density + Poisson | kick v (dt/2)
//   2D2V: kick v1, kick v2 (dt/2) | drift x2, drift x1 (dt) | density |
//         Poisson | kick v1, kick v2 (dt/2)
// Sweeps reuse the line walker of the single-run kernels.  A kick tile's
// lines share one spatial point, so thread 0 decomposes its shift in FP64
// once per tile; drift shifts depend only on dt and come from a table made
// once per dt (k_ens_drift_table).  Data written by other CTAs inside
// the launch (f of the previous stage, density, field) is read with L1-bypass
// loads (ld.global.cg).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "vp_internal.cuh"
#include "vp_sweep_core.cuh"
#include "vp_tma.cuh"

namespace {

// threads of a CTA: 128, so that many independent items are in flight per
// SM (256-thread CTAs, 4 per SM, left their staging waits exposed: 3.47
// against 3.07 ms per step); launch bounds for 6 CTAs per SM, which the
// staged tiles' shared memory allows anyway, leave 80 registers (no spills)
constexpr int kThreads = 128;
constexpr int kMaxStages = 8;
// shared-memory budget of one staged sweep tile (wider tiles are halved)
constexpr size_t kTileBytes = 56 * 1024;

enum StageKind { ST_COLS = 0, ST_ROWS = 1, ST_MOMENT = 2, ST_POISSON = 3 };

struct StageDesc {
    int kind;
    int kick;        // 1: velocity axis (speed = acceleration), 0: spatial axis
    int axis;        // axis index within x or v
    int half;        // 1: dt/2
    long long outer, inner;
    int L;
    int periodic;
    int cls_from_inner;
    long long cdiv, cmod;
    int tiles;
    int tw;          // tile width: columns (strided sweep) or lines (contiguous sweep)
    int done_slot;   // index of this stage's completion counter
};

struct RunDesc {
    long long f_off;
    int dims;
    int nx[2], nv[2];
    long long NX, NV;
    double xlo[2], hx[2], vlo[2], hv[2];
    long long acc_off, rho_off;
    long long dsh_off;  // drift shifts: axis 0 at [dsh_off, dsh_off + nv[0]), axis 1 after
    double coupling, rho_bg;
    int pois_order;
    int nstage;
    StageDesc st[kMaxStages];
};

struct EnsItem {
    int run, stage, tile, pad;
};

struct EnsParams {
    double dt;
    double alpha;
    int mp, pp, order;
    int W, R;          // tile widths of strided / contiguous sweeps
    int xpt;           // spatial points per density tile
    unsigned wait_limit;  // iterations of each dependency wait before it gives up
    WPoly wp;
    float wpf[7][7];   // the weight polynomials' coefficients in FP32 (wp.c)
};

// ---- device helpers ----------------------------------------------------------------

__device__ __forceinline__ float ldcg(const float *p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }

// wait until counter >= target (thread 0); false after `limit` polls
__device__ bool wait_count(const unsigned *ctr, unsigned target, unsigned limit) {
    for (unsigned it = 0; it < limit; ++it) {
        const unsigned v = *reinterpret_cast<const volatile unsigned *>(ctr);
        if (v >= target) {
            __threadfence();
            return true;
        }
        __nanosleep(64);
    }
    return false;
}

// Shift decomposition of one line as in the single-run sweeps (reading R2:
// s = c (dt / h) and its integer split in FP64, so the integer part is exact),
// with the CSL weight polynomials evaluated in FP32 at nu: the FP64 pipe of
// this GPU is narrow and every tile recomputes its lines' shifts.
__device__ __forceinline__ LineShift<float> ens_shift(double speed, double dth, const EnsParams &P) {
    const double sv = __dmul_rn(speed, dth);  // dth = dt / h, one division per tile
    double n = round(sv);
    const double z = __dadd_rn(sv, -n);
    const float nu = (float)fabs(z);
    LineShift<float> sh;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        float acc = 0.f;
        for (int j = P.wp.nterm - 1; j >= 0; --j) acc = fmaf(acc, nu, P.wpf[j][k]);
        sh.w[k] = acc;
    }
    n = fmin(fmax(n, -1.0e9), 1.0e9);
    sh.nu = nu;
    sh.n = (int)n;
    sh.sigma = z < 0.0 ? -1 : 1;
    return sh;
}

// The drift shifts of every run for the step's dt (one entry per velocity
// cell of each drift axis; the same decomposition as a tile would make of
// its lines), computed once per dt outside the step: drift tiles read them
// instead of spending the narrow FP64 pipe on every line of every tile.
__global__ void k_ens_drift_table(const RunDesc *__restrict__ runs, LineShift<float> *__restrict__ tab,
                                  EnsParams P) {
    const RunDesc &r = runs[blockIdx.x];
    for (int axis = 0; axis < r.dims; ++axis) {
        const double dth = P.dt / r.hx[axis];  // drifts move by the full dt
        const long long base = r.dsh_off + (axis ? r.nv[0] : 0);
        for (int j = threadIdx.x; j < r.nv[axis]; j += blockDim.x)
            tab[base + j] = ens_shift(vp_core::cell_centre(r.vlo[axis], r.hv[axis], j), dth, P);
    }
}

template <int ORDER, bool PER, bool FLAT>
__device__ void tile_cols(float *pool, const RunDesc &r, const StageDesc &s, int tile,
                          const double *acc_pool, const LineShift<float> *dsh, const EnsParams &P, float *sm) {
    // zero-inflow lines get VP_GHOST zero rows on each side (direct walks)
    constexpr int GP = PER ? 0 : VP_GHOST;
    const int L = s.L;
    const int W = s.tw;
    const long long tpo = (s.inner + W - 1) / W;
    const long long o = tile / tpo;
    const long long c0 = (tile % tpo) * W;
    const int wc = (int)((s.inner - c0) < W ? (s.inner - c0) : W);
    float *base = pool + r.f_off + o * L * s.inner + c0;
    float *data = sm + GP * W;  // row 0
    // a kick tile holds one spatial point: its shift, made once (thread 0,
    // while the tile is staged) and shared; drift tiles read the table
    __shared__ LineShift<float> s_sh;
    if (threadIdx.x == 0 && s.kick) {
        const double dt = s.half ? 0.5 * P.dt : P.dt;
        const unsigned cls = (unsigned)(o / s.cdiv);
        s_sh = ens_shift(ldcg(acc_pool + r.acc_off + (long long)s.axis * r.NX + cls), dt / r.hv[s.axis], P);
    }
    for (int c = threadIdx.x; c < GP * W; c += blockDim.x) {
        sm[c] = 0.f;
        data[L * W + c] = 0.f;
    }
    // staging: where every row of the tile is whole and 16-byte aligned, all
    // of it in flight at once as 16-byte cp.async.cg copies (L2, as the
    // L1-bypass loads: earlier stages of this launch wrote it); otherwise
    // four rows per thread in flight, (row, column) advanced incrementally
    if (wc == W && W % 4 == 0 && s.inner % 4 == 0 && (reinterpret_cast<uintptr_t>(base) & 15) == 0) {
        const int wv = W >> 2;
        const int dr = blockDim.x / wv, dc = blockDim.x - dr * wv;
        int row = threadIdx.x / wv, cv = threadIdx.x - row * wv;
        while (row < L) {
            vp_tma::cp_async16(data + row * W + 4 * cv, base + (long long)row * s.inner + 4 * cv);
            row += dr;
            cv += dc;
            if (cv >= wv) {
                cv -= wv;
                ++row;
            }
        }
        vp_tma::cp_async_wait_all();
    } else {
        const int dr = blockDim.x / W, dc = blockDim.x - dr * W;
        int row = threadIdx.x / W, cc = threadIdx.x - row * W;
        for (int e = threadIdx.x; e < L * W; e += 4 * blockDim.x) {
            float v[4];
            int rr[4], cq[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                rr[u] = row;
                cq[u] = cc;
                v[u] = (e + u * (int)blockDim.x < L * W && cc < wc) ? ldcg(base + (long long)row * s.inner + cc) : 0.f;
                row += dr;
                cc += dc;
                if (cc >= W) {
                    cc -= W;
                    ++row;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e + u * (int)blockDim.x < L * W) data[rr[u] * W + cq[u]] = v[u];
        }
    }
    __syncthreads();
    const int nseg = blockDim.x / W;
    const int cc = threadIdx.x % W, seg = threadIdx.x / W;
    if (cc < wc && seg < nseg) {
        const unsigned cls = s.cls_from_inner ? (unsigned)(((c0 + cc) / s.cdiv) % s.cmod) : (unsigned)(o / s.cdiv);
        const LineShift<float> sh = s.kick ? s_sh : dsh[r.dsh_off + (s.axis ? r.nv[0] : 0) + cls];
        const int r0 = seg * L / nseg, r1 = (seg + 1) * L / nseg;
        const int i0 = sh.sigma > 0 ? r0 : r1 - 1;
        struct St {
            float *p;
            long long step;
            __device__ void operator()(int, float v) {
                *p = v;
                p += step;
            }
        } st{base + cc + (long long)i0 * s.inner, (long long)sh.sigma * s.inner};
        vp_core::walk<float, ORDER, PER, true, PER ? 1 : VP_GHOST, false, FLAT>(data + cc, W, L, sh, r0, r1,
                                                                                (float)P.alpha,
                                                                    P.mp, P.pp, st);
    }
}

template <int ORDER, bool FLAT>
__device__ void tile_rows(float *pool, const RunDesc &r, const StageDesc &s, int tile,
                          const double *acc_pool, const EnsParams &P, float *sm) {
    constexpr int GP = VP_GHOST;  // velocity lines: zero inflow
    const int L = s.L;
    const int R = s.tw;
    const int Pp = (L + 2 * GP) | 1, Q = L | 1;
    float *in = sm, *out = sm + R * Pp;
    const long long l0 = (long long)tile * R;
    const int nl = (int)((s.outer - l0) < R ? (s.outer - l0) : R);
    float *base = pool + r.f_off + l0 * L;
    // lines of one spatial point (a 2D run's v2 kick): one shift, made once by
    // thread 0 while the tile is staged; otherwise one per line
    const long long cfirst = l0 / s.cdiv;
    const bool uniform = cfirst == (l0 + nl - 1) / s.cdiv;
    __shared__ double s_dth;
    __shared__ LineShift<float> s_sh;
    if (threadIdx.x == 0) {
        s_dth = (s.half ? 0.5 * P.dt : P.dt) / r.hv[s.axis];
        if (uniform) s_sh = ens_shift(ldcg(acc_pool + r.acc_off + (long long)s.axis * r.NX + cfirst), s_dth, P);
    }
    for (int k = threadIdx.x; k < nl * GP; k += blockDim.x) {
        const int ln = k / GP, g = k - ln * GP;
        in[ln * Pp + g] = 0.f;
        in[ln * Pp + GP + L + g] = 0.f;
    }
    const int tot = nl * L;
    const int dr = blockDim.x / L, dp = blockDim.x - dr * L;
    // whole rows of 16-byte pieces (f_off is 128-byte aligned): 16-byte loads and stores
    const bool vec = (L & 3) == 0 && (reinterpret_cast<uintptr_t>(base) & 15) == 0;
    if (vec) {
        const int st4 = 4 * (int)blockDim.x;
        const int vr = st4 / L, vp = st4 - vr * L;
        int row = (4 * (int)threadIdx.x) / L, pos = 4 * (int)threadIdx.x - row * L;
        for (int e = 4 * (int)threadIdx.x; e < tot; e += st4) {
            const float4 v = __ldcg(reinterpret_cast<const float4 *>(base + e));
            float *d = in + row * Pp + GP + pos;
            d[0] = v.x;
            d[1] = v.y;
            d[2] = v.z;
            d[3] = v.w;
            row += vr;
            pos += vp;
            if (pos >= L) {
                pos -= L;
                ++row;
            }
        }
    } else {
        int row = threadIdx.x / L, pos = threadIdx.x - row * L;
        for (int e = threadIdx.x; e < tot; e += 4 * blockDim.x) {
            float v[4];
            int at[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int eu = e + u * (int)blockDim.x;
                at[u] = row * Pp + GP + pos;
                v[u] = eu < tot ? ldcg(base + eu) : 0.f;
                row += dr;
                pos += dp;
                if (pos >= L) {
                    pos -= L;
                    ++row;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e + u * (int)blockDim.x < tot) in[at[u]] = v[u];
        }
    }
    __syncthreads();
    const int nseg = blockDim.x / R;
    const int line = threadIdx.x % R, seg = threadIdx.x / R;
    if (line < nl && seg < nseg) {
        const unsigned cls = (unsigned)((l0 + line) / s.cdiv);
        const LineShift<float> sh =
            uniform ? s_sh : ens_shift(ldcg(acc_pool + r.acc_off + (long long)s.axis * r.NX + cls), s_dth, P);
        const int r0 = seg * L / nseg, r1 = (seg + 1) * L / nseg;
        const int i0 = sh.sigma > 0 ? r0 : r1 - 1;
        struct St {
            float *p;
            int step;
            __device__ void operator()(int, float v) {
                *p = v;
                p += step;
            }
        } st{out + line * Q + i0, sh.sigma};
        vp_core::walk<float, ORDER, false, true, GP, false, FLAT>(in + line * Pp + GP, 1, L, sh, r0, r1,
                                                                  (float)P.alpha, P.mp,
                                                     P.pp, st);
    }
    __syncthreads();
    if (vec) {
        const int st4 = 4 * (int)blockDim.x;
        const int vr = st4 / L, vp = st4 - vr * L;
        int row = (4 * (int)threadIdx.x) / L, pos = 4 * (int)threadIdx.x - row * L;
        for (int e = 4 * (int)threadIdx.x; e < tot; e += st4) {
            const float *src = out + row * Q + pos;
            *reinterpret_cast<float4 *>(base + e) = make_float4(src[0], src[1], src[2], src[3]);
            row += vr;
            pos += vp;
            if (pos >= L) {
                pos -= L;
                ++row;
            }
        }
    } else {
        int row = threadIdx.x / L, pos = threadIdx.x - row * L;
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            base[e] = out[row * Q + pos];
            row += dr;
            pos += dp;
            if (pos >= L) {
                pos -= L;
                ++row;
            }
        }
    }
}

__device__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// density of spatial points [x0, x1): one warp per point, compensated float
// sums per lane combined in double
__device__ void density_points(const float *pool, const RunDesc &r, long long x0, long long x1,
                               double *rho_pool) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double dV = r.dims == 1 ? r.hv[0] : r.hv[0] * r.hv[1];
    for (long long x = x0 + warp; x < x1; x += nw) {
        const float *p = pool + r.f_off + x * r.NV;
        float s = 0.f, e = 0.f;
        for (long long v = lane; v < r.NV; v += 32) {
            const float y = ldcg(p + v);
            const float t = s + y;
            const float bp = t - s;
            e += (s - (t - bp)) + (y - bp);
            s = t;
        }
        const double tot = warp_sum_d((double)s + (double)e);
        if (lane == 0) rho_pool[r.rho_off + x] = tot * dV;
    }
}

// batched in-place radix-2 FFT of a row-major [n0][n1] (or [n0]) complex
// array in shared memory along `axis`; sign -1 forward, +1 inverse (no 1/n)
// tw[j] = (cos, sin)(2 pi j / 256), j < 128: the twiddles of every power-of-two
// length up to 256 (length len uses every (256 / len)-th entry)
constexpr int kTwN = 256;

// runs with at most this many spatial points transform in shared memory;
// larger ones in their slice of a global scratch array (L2-resident), so the
// kernel's shared memory is sized by the sweep tiles alone
constexpr long long kSmemFftMax = 1024;

// element access of the transform array: shared memory, or the global scratch
// through L2 (other SMs used it in earlier launches)
template <bool GLOBAL>
__device__ __forceinline__ double2 ld2(const double2 *p) {
    if constexpr (GLOBAL) return __ldcg(p);
    else return *p;
}
template <bool GLOBAL>
__device__ __forceinline__ void st2(double2 *p, double2 v) {
    if constexpr (GLOBAL) __stcg(p, v);
    else *p = v;
}

template <bool GLOBAL>
__device__ void smem_fft(double2 *a, int dims, int n0, int n1, int axis, int sign, const double2 *__restrict__ tw) {
    const int n = axis == 0 ? n0 : n1;
    const int lines = dims == 1 ? 1 : (axis == 0 ? n1 : n0);
    const int stride = (dims == 1 || axis == 1) ? 1 : n1;   // element stride along the axis
    const int lstride = (dims == 1) ? 0 : (axis == 0 ? 1 : n1);  // stride between lines
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    // bit-reversal permutation
    for (int t = threadIdx.x; t < lines * n; t += blockDim.x) {
        const int l = t / n, j = t - l * n;
        const int rj = logn ? (int)(__brev((unsigned)j) >> (32 - logn)) : 0;
        if (j < rj) {
            double2 *pa = a + l * lstride + j * stride, *pb = a + l * lstride + rj * stride;
            const double2 tmp = ld2<GLOBAL>(pa);
            st2<GLOBAL>(pa, ld2<GLOBAL>(pb));
            st2<GLOBAL>(pb, tmp);
        }
    }
    __syncthreads();
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len >> 1;
        for (int t = threadIdx.x; t < lines * (n / 2); t += blockDim.x) {
            const int l = t / (n / 2), b = t - l * (n / 2);
            const int grp = b / half, k = b - grp * half;
            const int i0 = grp * len + k, i1 = i0 + half;
            const double2 twk = tw[k * (kTwN / len)];
            const double cs = twk.x, sn = sign < 0 ? -twk.y : twk.y;
            double2 *pu = a + l * lstride + i0 * stride, *pv = a + l * lstride + i1 * stride;
            const double2 u = ld2<GLOBAL>(pu), v = ld2<GLOBAL>(pv);
            const double2 tw = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
            st2<GLOBAL>(pu, make_double2(u.x + tw.x, u.y + tw.y));
            st2<GLOBAL>(pv, make_double2(u.x - tw.x, u.y - tw.y));
        }
        __syncthreads();
    }
}

// periodic Poisson + FDA force of one run, all in one CTA (NX <= 4096); the
// transform array a in shared memory or (GLOBAL) the run's global scratch
template <bool GLOBAL>
__device__ void poisson_run(const RunDesc &r, const double *rho_pool, double *acc_pool, double2 *a,
                            const double2 *__restrict__ tw, const double *__restrict__ green) {
    const int D = r.dims;
    const int n0 = r.nx[0], n1 = D == 2 ? r.nx[1] : 1;
    const long long NX = r.NX;
    for (long long x = threadIdx.x; x < NX; x += blockDim.x)
        st2<GLOBAL>(a + x, make_double2(ldcg(rho_pool + r.rho_off + x) - r.rho_bg, 0.0));
    __syncthreads();
    for (int ax = 0; ax < D; ++ax) smem_fft<GLOBAL>(a, D, n0, n1, ax, -1, tw);
    // S / lambda(k) / NX of the run, tabulated at creation (0 at k = 0)
    for (long long x = threadIdx.x; x < NX; x += blockDim.x) {
        const double sc = green[r.rho_off + x];
        const double2 ax = ld2<GLOBAL>(a + x);
        st2<GLOBAL>(a + x, make_double2(ax.x * sc, ax.y * sc));
    }
    __syncthreads();
    for (int ax = 0; ax < D; ++ax) smem_fft<GLOBAL>(a, D, n0, n1, ax, +1, tw);
    // a = -grad phi by the 2/4/6-point FDA (Eqs. C9-C11)
    double c1 = 1.0, c2 = 0.0, c3 = 0.0, den = 2.0;
    if (r.pois_order == 4) {
        c1 = 8.0;
        c2 = -1.0;
        den = 12.0;
    } else if (r.pois_order == 6) {
        c1 = 45.0;
        c2 = -9.0;
        c3 = 1.0;
        den = 60.0;
    }
    const double sc0 = -1.0 / (den * r.hx[0]), sc1 = D == 2 ? -1.0 / (den * r.hx[1]) : 0.0;
    for (long long x = threadIdx.x; x < NX; x += blockDim.x) {
        const int i0 = (int)(D == 2 ? x / n1 : x);
        const int i1 = (int)(D == 2 ? x % n1 : 0);
        for (int d = 0; d < D; ++d) {
            // power-of-two axes: periodic neighbours by masking
            auto at = [&](int off) -> double {
                int j0 = i0, j1 = i1;
                if (d == 0) j0 = (i0 + off) & (n0 - 1);
                else j1 = (i1 + off) & (n1 - 1);
                return ld2<GLOBAL>(a + j0 * n1 + j1).x;
            };
            const double g = c1 * (at(1) - at(-1)) + c2 * (at(2) - at(-2)) + c3 * (at(3) - at(-3));
            acc_pool[r.acc_off + (long long)d * NX + x] = g * (d == 0 ? sc0 : sc1);
        }
    }
}

template <int ORDER, bool FLAT>
__global__ void __launch_bounds__(kThreads, 6) k_ensemble(float *__restrict__ pool,
                                                       const RunDesc *__restrict__ runs,
                                                       const EnsItem *__restrict__ items, int nitems,
                                                       unsigned *__restrict__ ctr, double *acc_pool,
                                                       double *rho_pool, EnsParams P,
                                                       int *__restrict__ status, const double2 *__restrict__ tw,
                                                       const double *__restrict__ green, double2 *fftbuf,
                                                       const LineShift<float> *__restrict__ dsh) {
    extern __shared__ __align__(16) unsigned char ens_smem[];
    __shared__ int s_item;
    __shared__ int s_ok;
    unsigned *head = ctr;
    unsigned *done = ctr + 1;
    if (threadIdx.x == 0) s_item = (int)atomicAdd(head, 1u);
    __syncthreads();
    int met_run = -1, met_stage = -1;  // thread 0: the last dependency seen met (counters only grow)
    while (true) {
        const int it = s_item;
        if (it >= nitems) break;
        const EnsItem e = items[it];
        const RunDesc &r = runs[e.run];
        const StageDesc &s = r.st[e.stage];
        if (threadIdx.x == 0) {
            s_ok = 1;
            if (e.stage > 0 && (e.run != met_run || e.stage != met_stage)) {
                const StageDesc &prev = r.st[e.stage - 1];
                if (!wait_count(done + prev.done_slot, (unsigned)prev.tiles, P.wait_limit)) {
                    atomicExch(status, VP_ETIMEOUT);
                    s_ok = 0;
                } else {
                    met_run = e.run;
                    met_stage = e.stage;
                }
            }
        }
        __syncthreads();
        if (!s_ok) return;
        // every thread has read s_item: the next item is popped now (by a thread
        // of the second warp), its latency hidden behind this item's work; the
        // barrier that ends this item publishes it
        if (threadIdx.x == 32) s_item = (int)atomicAdd(head, 1u);
        if (s.kind == ST_COLS) {
            if (s.periodic)
                tile_cols<ORDER, true, FLAT>(pool, r, s, e.tile, acc_pool, dsh, P,
                                             reinterpret_cast<float *>(ens_smem));
            else
                tile_cols<ORDER, false, FLAT>(pool, r, s, e.tile, acc_pool, dsh, P,
                                              reinterpret_cast<float *>(ens_smem));
        } else if (s.kind == ST_ROWS) {
            tile_rows<ORDER, FLAT>(pool, r, s, e.tile, acc_pool, P, reinterpret_cast<float *>(ens_smem));
        } else if (s.kind == ST_MOMENT) {
            const long long x0 = (long long)e.tile * P.xpt;
            const long long x1 = x0 + P.xpt < r.NX ? x0 + P.xpt : r.NX;
            density_points(pool, r, x0, x1, rho_pool);
        } else {
            if (r.dims == 1) {  // the 1D density is small enough to fuse here
                density_points(pool, r, 0, r.NX, rho_pool);
                __threadfence_block();
                __syncthreads();
            }
            if (r.NX <= kSmemFftMax)
                poisson_run<false>(r, rho_pool, acc_pool, reinterpret_cast<double2 *>(ens_smem), tw, green);
            else
                poisson_run<true>(r, rho_pool, acc_pool, fftbuf + r.rho_off, tw, green);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(done + s.done_slot, 1u);
    }
}

size_t smem_need(const std::vector<RunDesc> &runs) {
    size_t need = 0;
    for (const RunDesc &r : runs) {
        for (int k = 0; k < r.nstage; ++k) {
            const StageDesc &s = r.st[k];
            size_t b = 0;
            if (s.kind == ST_COLS) {
                b = (size_t)(s.L + (s.periodic ? 0 : 2 * VP_GHOST)) * s.tw * sizeof(float);
            } else if (s.kind == ST_ROWS) {
                b = (size_t)s.tw * (((s.L + 2 * VP_GHOST) | 1) + (s.L | 1)) * sizeof(float);
            } else if (s.kind == ST_POISSON) {
                b = r.NX <= kSmemFftMax ? (size_t)r.NX * sizeof(double2) : 0;
            }
            need = b > need ? b : need;
        }
    }
    return need;
}

}  // namespace

// ---- host side --------------------------------------------------------------------

struct vp_ens {
    std::vector<RunDesc> runs;
    std::vector<EnsItem> items_step, items_field;
    cudaStream_t stream;
    int device, sm_count;
    float *pool;
    long long pool_cells;
    double *d_acc, *d_rho;
    double2 *d_tw;     // FFT twiddles (kTwN / 2 entries)
    double *d_green;   // per run: S / lambda(k) / NX at every Fourier mode (rho layout)
    double2 *d_fft;    // per run: transform scratch of runs too large for shared memory (rho layout)
    LineShift<float> *d_dsh;  // drift shifts of every run for dsh_dt (see k_ens_drift_table)
    long long dsh_total;
    double dsh_dt;
    int dsh_valid;
    long long acc_total, rho_total;
    RunDesc *d_runs;
    EnsItem *d_items_step, *d_items_field;
    unsigned *d_ctr;
    int nslots;
    int *d_status;
    EnsParams P;
    int ctas_per_sm;
    int flat;          // 1: the walkers vote on flat stencils (and skip them), 0: no vote
    size_t smem;
    int tuned;
    cudaGraphExec_t graph;
    double graph_dt;
    int graph_valid;
    long long launches;
    char err[256];
};

static int ens_fail(vp_ens *e, int code, const char *msg) {
    if (e) snprintf(e->err, sizeof(e->err), "%s", msg);
    return code;
}

// stage lists of one run
static int build_stages(RunDesc &r, int W, int R, int xpt, int &slot) {
    const int D = r.dims;
    auto cols = [&](int kick, int axis, int half, long long outer, int L, long long inner, int per,
                    int from_inner, long long cdiv, long long cmod) {
        StageDesc s{};
        s.kind = ST_COLS;
        s.kick = kick;
        s.axis = axis;
        s.half = half;
        s.outer = outer;
        s.L = L;
        s.inner = inner;
        s.periodic = per;
        s.cls_from_inner = from_inner;
        s.cdiv = cdiv;
        s.cmod = cmod;
        // tile width: the requested W, halved until the staged tile fits kTileBytes
        int w = W;
        while (w > 8 && (size_t)(L + (per ? 0 : 2 * VP_GHOST)) * w * sizeof(float) > kTileBytes) w /= 2;
        if (inner < w) w = (int)inner;
        s.tw = w;
        s.tiles = (int)(outer * ((inner + w - 1) / w));
        return s;
    };
    auto rows = [&](int axis, long long outer, int L, long long cdiv) {
        StageDesc s{};
        s.kind = ST_ROWS;
        s.kick = 1;
        s.axis = axis;
        s.half = 1;
        s.outer = outer;
        s.L = L;
        s.inner = 1;
        s.cdiv = cdiv;
        s.cmod = 1;
        int rr = R;
        while (rr > 8 && (size_t)rr * (((L + 2 * VP_GHOST) | 1) + (L | 1)) * sizeof(float) > kTileBytes) rr /= 2;
        s.tw = rr;
        s.tiles = (int)((outer + rr - 1) / rr);
        return s;
    };
    int k = 0;
    if (D == 1) {
        r.st[k++] = rows(0, r.NX, r.nv[0], 1);
        r.st[k++] = cols(0, 0, 0, 1, r.nx[0], r.NV, 1, 1, 1, r.nv[0]);
        StageDesc p{};
        p.kind = ST_POISSON;
        p.tiles = 1;
        r.st[k++] = p;
        r.st[k++] = rows(0, r.NX, r.nv[0], 1);
    } else {
        // kick v1 (strided over v2), kick v2 (contiguous)
        r.st[k++] = cols(1, 0, 1, r.NX, r.nv[0], r.nv[1], 0, 0, 1, 1);
        r.st[k++] = rows(1, r.NX * r.nv[0], r.nv[1], r.nv[0]);
        // drift x2 then x1 (Eq. 55 order)
        r.st[k++] = cols(0, 1, 0, r.nx[0], r.nx[1], r.NV, 1, 1, 1, r.nv[1]);
        r.st[k++] = cols(0, 0, 0, 1, r.nx[0], (long long)r.nx[1] * r.NV, 1, 1, r.nv[1], r.nv[0]);
        StageDesc m{};
        m.kind = ST_MOMENT;
        m.tiles = (int)((r.NX + xpt - 1) / xpt);
        r.st[k++] = m;
        StageDesc p{};
        p.kind = ST_POISSON;
        p.tiles = 1;
        r.st[k++] = p;
        r.st[k++] = cols(1, 0, 1, r.NX, r.nv[0], r.nv[1], 0, 0, 1, 1);
        r.st[k++] = rows(1, r.NX * r.nv[0], r.nv[1], r.nv[0]);
    }
    r.nstage = k;
    for (int i = 0; i < k; ++i) r.st[i].done_slot = slot++;
    return VP_OK;
}

static void build_items(vp_ens *e) {
    e->items_step.clear();
    e->items_field.clear();
    int maxst = 0;
    for (const RunDesc &r : e->runs) maxst = r.nstage > maxst ? r.nstage : maxst;
    for (int st = 0; st < maxst; ++st)
        for (int ri = 0; ri < (int)e->runs.size(); ++ri) {
            const RunDesc &r = e->runs[ri];
            if (st >= r.nstage) continue;
            for (int t = 0; t < r.st[st].tiles; ++t) e->items_step.push_back(EnsItem{ri, st, t, 0});
        }
    // field-only list: the density (2D) and Poisson stages, as stages 0/1 of a
    // separate pass (their waits refer to the previous stage of the same list)
    for (int ri = 0; ri < (int)e->runs.size(); ++ri) {
        const RunDesc &r = e->runs[ri];
        for (int st = 0; st < r.nstage; ++st)
            if (r.st[st].kind == ST_MOMENT || r.st[st].kind == ST_POISSON)
                for (int t = 0; t < r.st[st].tiles; ++t) e->items_field.push_back(EnsItem{ri, st, t, 0});
    }
}

static int upload_plan(vp_ens *e) {
    cudaFree(e->d_runs);
    cudaFree(e->d_items_step);
    cudaFree(e->d_items_field);
    e->d_runs = nullptr;
    e->d_items_step = e->d_items_field = nullptr;
    if (cudaMalloc(&e->d_runs, sizeof(RunDesc) * e->runs.size()) != cudaSuccess ||
        cudaMalloc(&e->d_items_step, sizeof(EnsItem) * e->items_step.size()) != cudaSuccess ||
        cudaMalloc(&e->d_items_field, sizeof(EnsItem) * (e->items_field.size() + 1)) != cudaSuccess)
        return ens_fail(e, VP_ENOMEM, "plan allocation failed");
    if (cudaMemcpy(e->d_runs, e->runs.data(), sizeof(RunDesc) * e->runs.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(e->d_items_step, e->items_step.data(), sizeof(EnsItem) * e->items_step.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e->d_items_field, e->items_field.data(), sizeof(EnsItem) * e->items_field.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return ens_fail(e, VP_ECUDA, "plan upload failed");
    return VP_OK;
}

// the field pass waits on stage - 1 of the full list; give it its own view in
// which the density stage (2D) precedes Poisson and nothing precedes density
// the drift shift table for dt (before a step graph is captured; never inside one)
static int ensure_drift_table(vp_ens *e, double dt) {
    if (e->dsh_valid && e->dsh_dt == dt) return VP_OK;
    EnsParams P = e->P;
    P.dt = dt;
    k_ens_drift_table<<<(unsigned)e->runs.size(), 128, 0, e->stream>>>(e->d_runs, e->d_dsh, P);
    e->launches++;
    const cudaError_t er = cudaGetLastError();
    if (er != cudaSuccess) return ens_fail(e, VP_ECUDA, cudaGetErrorString(er));
    e->dsh_valid = 1;
    e->dsh_dt = dt;
    return VP_OK;
}

// the persistent kernel of the ensemble's order and flat-vote choice
static const void *ens_kernel(int order, int flat) {
    if (order == 7) return flat ? (const void *)k_ensemble<7, true> : (const void *)k_ensemble<7, false>;
    return flat ? (const void *)k_ensemble<5, true> : (const void *)k_ensemble<5, false>;
}

static void launch_k(vp_ens *e, const EnsItem *items, int nitems, const EnsParams &P) {
    const int grid = e->ctas_per_sm * e->sm_count;
#define VP_ENS_LAUNCH(O, F)                                                                                 \
    k_ensemble<O, F><<<grid, kThreads, e->smem, e->stream>>>(e->pool, e->d_runs, items, nitems, e->d_ctr,   \
                                                             e->d_acc, e->d_rho, P, e->d_status, e->d_tw,   \
                                                             e->d_green, e->d_fft, e->d_dsh)
    if (e->P.order == 7) {
        if (e->flat) VP_ENS_LAUNCH(7, true);
        else VP_ENS_LAUNCH(7, false);
    } else {
        if (e->flat) VP_ENS_LAUNCH(5, true);
        else VP_ENS_LAUNCH(5, false);
    }
#undef VP_ENS_LAUNCH
}

static int launch_pass(vp_ens *e, const EnsItem *items, int nitems, double dt) {
    EnsParams P = e->P;
    P.dt = dt;
    if (cudaMemsetAsync(e->d_ctr, 0, sizeof(unsigned) * (e->nslots + 1), e->stream) != cudaSuccess)
        return ens_fail(e, VP_ECUDA, "counter reset failed");
    launch_k(e, items, nitems, P);
    e->launches++;
    const cudaError_t er = cudaGetLastError();
    if (er != cudaSuccess) return ens_fail(e, VP_ECUDA, cudaGetErrorString(er));
    return VP_OK;
}

extern "C" {

int vp_ensemble_create(const vp_run_desc *runs, int nruns, int order, void *cuda_stream, vp_ens **out) {
    if (!out) return VP_EINVAL;
    *out = nullptr;
    if (!runs || nruns < 1 || (order != 5 && order != 7)) return VP_EINVAL;
    vp_ens *e = new (std::nothrow) vp_ens();
    if (!e) return VP_ENOMEM;
    e->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&e->device);
    cudaDeviceGetAttribute(&e->sm_count, cudaDevAttrMultiProcessorCount, e->device);
    e->P.alpha = 4.0;
    e->P.mp = 1;
    e->P.pp = 1;
    e->P.order = order;
    e->P.W = 64;
    e->P.wait_limit = 1u << 24;
    e->P.R = 32;
    e->P.xpt = 8;
    e->P.wp = vp_csl_weight_polys(order);
    for (int j = 0; j < 7; ++j)
        for (int k = 0; k < 7; ++k) e->P.wpf[j][k] = (float)e->P.wp.c[j][k];
    long long off = 0, aoff = 0, roff = 0, soff = 0;
    int slot = 0;
    for (int i = 0; i < nruns; ++i) {
        const vp_run_desc &d = runs[i];
        RunDesc r{};
        if (d.dims < 1 || d.dims > 2) {
            delete e;
            return VP_EINVAL;
        }
        r.dims = d.dims;
        r.NX = r.NV = 1;
        for (int k = 0; k < d.dims; ++k) {
            if (d.nx[k] < 1 || d.nv[k] < 1 || d.nv[k] > 4096 || d.nx[k] > 256 ||
                (d.nx[k] & (d.nx[k] - 1)) != 0 || !(d.xhi[k] > d.xlo[k]) || !(d.vhi[k] > d.vlo[k])) {
                delete e;
                return VP_EINVAL;  // power-of-two spatial axes up to 256 (one-CTA FFT)
            }
            r.nx[k] = d.nx[k];
            r.nv[k] = d.nv[k];
            r.xlo[k] = d.xlo[k];
            r.vlo[k] = d.vlo[k];
            r.hx[k] = (d.xhi[k] - d.xlo[k]) / d.nx[k];
            r.hv[k] = (d.vhi[k] - d.vlo[k]) / d.nv[k];
            r.NX *= d.nx[k];
            r.NV *= d.nv[k];
        }
        if (r.NX > 4096) {
            delete e;
            return VP_EINVAL;
        }
        r.f_off = off;
        r.acc_off = aoff;
        r.rho_off = roff;
        r.dsh_off = soff;
        r.coupling = d.coupling;
        r.rho_bg = d.rho_bg;
        r.pois_order = d.pois_order == 2 || d.pois_order == 4 ? d.pois_order : 6;
        off += ((r.NX * r.NV + 31) / 32) * 32;  // 128-byte aligned runs
        aoff += r.dims * r.NX;
        roff += r.NX;
        soff += r.nv[0] + (r.dims > 1 ? r.nv[1] : 0);
        e->runs.push_back(r);
    }
    e->pool_cells = off;
    e->acc_total = aoff;
    e->rho_total = roff;
    e->dsh_total = soff;
    for (RunDesc &r : e->runs) build_stages(r, e->P.W, e->P.R, e->P.xpt, slot);
    e->nslots = slot;
    build_items(e);
    if (cudaMalloc(&e->d_acc, sizeof(double) * aoff) != cudaSuccess ||
        cudaMalloc(&e->d_rho, sizeof(double) * roff) != cudaSuccess ||
        cudaMalloc(&e->d_fft, sizeof(double2) * roff) != cudaSuccess ||
        cudaMalloc(&e->d_dsh, sizeof(LineShift<float>) * soff) != cudaSuccess ||
        cudaMalloc(&e->d_ctr, sizeof(unsigned) * (slot + 1)) != cudaSuccess ||
        cudaMalloc(&e->d_status, sizeof(int)) != cudaSuccess) {
        vp_ensemble_destroy(e);
        return VP_ENOMEM;
    }
    cudaMemset(e->d_acc, 0, sizeof(double) * aoff);
    cudaMemset(e->d_status, 0, sizeof(int));
    {
        // FFT twiddles and every run's Green factors S / lambda(k) / NX (the
        // eigenvalues of the 2/4/6-point discrete Laplacians, Eqs. C1, C5, C6)
        std::vector<double2> tw(kTwN / 2);
        const double two_pi = 6.283185307179586476925286766559;
        for (int j = 0; j < kTwN / 2; ++j) tw[j] = make_double2(std::cos(two_pi * j / kTwN), std::sin(two_pi * j / kTwN));
        std::vector<double> green((size_t)roff, 0.0);
        auto lap = [](int order, double theta) {
            double b1 = 1.0, b2 = 0.0, b3 = 0.0, den = 1.0;
            if (order == 4) {
                b1 = 16.0;
                b2 = -1.0;
                den = 12.0;
            } else if (order == 6) {
                b1 = 270.0;
                b2 = -27.0;
                b3 = 2.0;
                den = 180.0;
            }
            const double s1 = std::sin(0.5 * theta), s2 = std::sin(theta), s3 = std::sin(1.5 * theta);
            return -4.0 * (b1 * s1 * s1 + b2 * s2 * s2 + b3 * s3 * s3) / den;
        };
        for (const RunDesc &r : e->runs) {
            const int n0 = r.nx[0], n1 = r.dims == 2 ? r.nx[1] : 1;
            for (long long x = 0; x < r.NX; ++x) {
                const int k0 = (int)(x / n1), k1 = (int)(x % n1);
                double lam = lap(r.pois_order, two_pi * k0 / n0) / (r.hx[0] * r.hx[0]);
                if (r.dims == 2) lam += lap(r.pois_order, two_pi * k1 / n1) / (r.hx[1] * r.hx[1]);
                green[(size_t)(r.rho_off + x)] = (k0 == 0 && k1 == 0) ? 0.0 : r.coupling / lam / (double)r.NX;
            }
        }
        if (cudaMalloc(&e->d_tw, sizeof(double2) * tw.size()) != cudaSuccess ||
            cudaMalloc(&e->d_green, sizeof(double) * green.size()) != cudaSuccess ||
            cudaMemcpy(e->d_tw, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(e->d_green, green.data(), sizeof(double) * green.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            vp_ensemble_destroy(e);
            return VP_ENOMEM;
        }
    }
    int rc = upload_plan(e);
    if (rc) {
        vp_ensemble_destroy(e);
        return rc;
    }
    e->smem = smem_need(e->runs);
    for (int o = 5; o <= 7; o += 2)
        for (int fl = 0; fl < 2; ++fl)
            cudaFuncSetAttribute(ens_kernel(o, fl), cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    e->flat = 1;
    int per = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ens_kernel(order, e->flat), kThreads, e->smem);
    e->ctas_per_sm = per < 1 ? 1 : per;
    *out = e;
    return VP_OK;
}

void vp_ensemble_destroy(vp_ens *e) {
    if (!e) return;
    cudaStreamSynchronize(e->stream);
    cudaFree(e->d_acc);
    cudaFree(e->d_rho);
    cudaFree(e->d_fft);
    cudaFree(e->d_dsh);
    cudaFree(e->d_tw);
    cudaFree(e->d_green);
    cudaFree(e->d_ctr);
    cudaFree(e->d_status);
    cudaFree(e->d_runs);
    cudaFree(e->d_items_step);
    cudaFree(e->d_items_field);
    if (e->graph_valid) cudaGraphExecDestroy(e->graph);
    delete e;
}

const char *vp_ensemble_last_error(const vp_ens *e) { return e ? e->err : "null ensemble"; }

long long vp_ensemble_num_cells(const vp_ens *e) { return e ? e->pool_cells : 0; }

int vp_ensemble_run_layout(const vp_ens *e, int run, long long *f_offset, long long *acc_offset) {
    if (!e || run < 0 || run >= (int)e->runs.size()) return VP_EINVAL;
    if (f_offset) *f_offset = e->runs[run].f_off;
    if (acc_offset) *acc_offset = e->runs[run].acc_off;
    return VP_OK;
}

int vp_ensemble_bind(vp_ens *e, float *pool_dev) {
    if (!e || !pool_dev || (reinterpret_cast<uintptr_t>(pool_dev) & 127)) return VP_EINVAL;
    e->pool = pool_dev;
    if (e->graph_valid) {
        cudaGraphExecDestroy(e->graph);
        e->graph_valid = 0;
    }
    return VP_OK;
}

int vp_ensemble_accel(const vp_ens *e, const double **accel_dev) {
    if (!e || !accel_dev) return VP_EINVAL;
    *accel_dev = e->d_acc;
    return VP_OK;
}

int vp_ensemble_field(vp_ens *e) {
    if (!e || !e->pool) return VP_EINVAL;
    // the field list holds, per run, (density, Poisson) for 2D and (Poisson) for
    // 1D; the wait of each item refers to stage - 1 of its run in the full
    // plan, which the field pass has not run: run it stage by stage instead
    std::vector<EnsItem> pass;
    for (int phase = 0; phase < 2; ++phase) {
        pass.clear();
        for (const EnsItem &it : e->items_field) {
            const StageDesc &s = e->runs[it.run].st[it.stage];
            if ((phase == 0) == (s.kind == ST_MOMENT)) pass.push_back(it);
        }
        if (pass.empty()) continue;
        if (cudaMemcpy(e->d_items_field, pass.data(), sizeof(EnsItem) * pass.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return ens_fail(e, VP_ECUDA, "field plan upload failed");
        // mark every previous stage complete so the waits pass immediately
        std::vector<unsigned> ctr(e->nslots + 1, 0u);
        for (const RunDesc &r : e->runs)
            for (int k = 0; k < r.nstage; ++k) ctr[1 + r.st[k].done_slot] = (unsigned)r.st[k].tiles;
        for (const EnsItem &it : pass) ctr[1 + e->runs[it.run].st[it.stage].done_slot] = 0;
        if (cudaMemcpyAsync(e->d_ctr, ctr.data(), sizeof(unsigned) * ctr.size(), cudaMemcpyHostToDevice,
                            e->stream) != cudaSuccess)
            return ens_fail(e, VP_ECUDA, "counter upload failed");
        EnsParams P = e->P;
        P.dt = 0.0;
        launch_k(e, e->d_items_field, (int)pass.size(), P);
        e->launches++;
        if (cudaStreamSynchronize(e->stream) != cudaSuccess) return ens_fail(e, VP_ECUDA, "field pass failed");
    }
    return VP_OK;
}

int vp_ensemble_init_run(vp_ens *e, int run, int kind, const double *params, int nparams) {
    if (!e || !e->pool || run < 0 || run >= (int)e->runs.size()) return VP_EINVAL;
    const RunDesc &r = e->runs[run];
    if (kind != VP_IC_LANDAU && kind != VP_IC_TWOSTREAM) return ens_fail(e, VP_EINVAL, "unsupported initial condition");
    vp_grid g{};
    g.dx = g.dv = r.dims;
    for (int k = 0; k < r.dims; ++k) {
        g.nx[k] = r.nx[k];
        g.nv[k] = r.nv[k];
        g.xlo[k] = r.xlo[k];
        g.xhi[k] = r.xlo[k] + r.hx[k] * r.nx[k];
        g.vlo[k] = r.vlo[k];
        g.vhi[k] = r.vlo[k] + r.hv[k] * r.nv[k];
    }
    g.precision = VP_F32;
    const int rc = vp_launch_init_ptr(e->pool + r.f_off, g, kind, params, nparams, e->stream);
    e->launches++;
    return rc ? ens_fail(e, rc, "initial condition launch failed") : VP_OK;
}

int vp_ensemble_set_tiles(vp_ens *e, int W, int R, int ctas_per_sm) {
    if (!e || W < 8 || W > 256 || R < 8 || R > 256 || ctas_per_sm < 0) return VP_EINVAL;
    if (kThreads % W != 0 || kThreads % R != 0) return VP_EINVAL;
    e->P.W = W;
    e->P.R = R;
    int slot = 0;
    for (RunDesc &r : e->runs) build_stages(r, W, R, e->P.xpt, slot);
    build_items(e);
    int rc = upload_plan(e);
    if (rc) return rc;
    e->smem = smem_need(e->runs);
    int per = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ens_kernel(e->P.order, e->flat), kThreads, e->smem);
    per = per < 1 ? 1 : per;
    e->ctas_per_sm = ctas_per_sm > 0 && ctas_per_sm < per ? ctas_per_sm : per;
    if (e->graph_valid) {
        cudaGraphExecDestroy(e->graph);
        e->graph_valid = 0;
    }
    return VP_OK;
}

int vp_ensemble_set_wait_limit(vp_ens *e, long long iterations) {
    if (!e || iterations < 0 || iterations > 0xffffffffLL) return VP_EINVAL;
    e->P.wait_limit = (unsigned)iterations;
    if (e->graph_valid) {  // the limit is a launch parameter baked into the graph
        cudaGraphExecDestroy(e->graph);
        e->graph_valid = 0;
    }
    return VP_OK;
}

int vp_ensemble_set_flat_vote(vp_ens *e, int on) {
    if (!e || on < 0 || on > 1) return VP_EINVAL;
    e->flat = on;
    if (e->graph_valid) {  // the kernel is baked into the graph
        cudaGraphExecDestroy(e->graph);
        e->graph_valid = 0;
    }
    return VP_OK;
}

int vp_ensemble_get_flat_vote(const vp_ens *e, int *on) {
    if (!e || !on) return VP_EINVAL;
    *on = e->flat;
    return VP_OK;
}

int vp_ensemble_get_tiles(const vp_ens *e, int *out3) {
    if (!e || !out3) return VP_EINVAL;
    out3[0] = e->P.W;
    out3[1] = e->P.R;
    out3[2] = e->ctas_per_sm;
    return VP_OK;
}

int vp_ensemble_autotune(vp_ens *e, double dt) {
    if (!e || !e->pool) return VP_EINVAL;
    if (!std::isfinite(dt)) return ens_fail(e, VP_EINVAL, "dt must be finite");
    // time whole steps at the run's dt (the limiters at work, as in the
    // timed steps) from a snapshot of f and the field, restored afterwards:
    // the ensemble's state is unchanged
    float *snap_f = nullptr;
    double *snap_acc = nullptr;
    if (cudaMalloc(&snap_f, sizeof(float) * e->pool_cells) != cudaSuccess ||
        cudaMalloc(&snap_acc, sizeof(double) * e->acc_total) != cudaSuccess) {
        cudaFree(snap_f);
        cudaGetLastError();
        return ens_fail(e, VP_ENOMEM, "no room for the tuning snapshot");
    }
    auto restore = [&]() {
        return cudaMemcpyAsync(e->pool, snap_f, sizeof(float) * e->pool_cells, cudaMemcpyDeviceToDevice,
                               e->stream) == cudaSuccess &&
               cudaMemcpyAsync(e->d_acc, snap_acc, sizeof(double) * e->acc_total, cudaMemcpyDeviceToDevice,
                               e->stream) == cudaSuccess;
    };
    int rc = ensure_drift_table(e, dt);
    if (rc == VP_OK &&
        cudaMemcpyAsync(snap_f, e->pool, sizeof(float) * e->pool_cells, cudaMemcpyDeviceToDevice, e->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(snap_acc, e->d_acc, sizeof(double) * e->acc_total, cudaMemcpyDeviceToDevice, e->stream) !=
            cudaSuccess)
        rc = ens_fail(e, VP_ECUDA, "tuning snapshot failed");
    const int Ws[3] = {32, 64, 128};
    const int Rs[2] = {32, 64};
    float best = 1e30f;
    int bw = e->P.W, br = e->P.R, bc = 0, bf = e->flat;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // the walkers with and without the flat-stencil vote (the same results)
    for (int fl = 1; fl >= 0 && rc == VP_OK; --fl)
    for (int wi = 0; wi < 3 && rc == VP_OK; ++wi)
        for (int ri = 0; ri < 2 && rc == VP_OK; ++ri) {
            e->flat = fl;
            if (vp_ensemble_set_tiles(e, Ws[wi], Rs[ri], 0)) continue;
            const int maxc = e->ctas_per_sm;
            for (int cps = maxc; cps >= 1 && cps >= maxc - 2 && rc == VP_OK; --cps) {
                e->ctas_per_sm = cps;
                float ms = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    cudaEventRecord(a, e->stream);
                    const int lr = launch_pass(e, e->d_items_step, (int)e->items_step.size(), dt);
                    cudaEventRecord(b, e->stream);
                    if (lr || cudaEventSynchronize(b) != cudaSuccess) {
                        rc = ens_fail(e, VP_ECUDA, "autotune pass failed");
                        break;
                    }
                    float m = 0.f;
                    cudaEventElapsedTime(&m, a, b);
                    ms = m < ms ? m : ms;
                    if (!restore()) {
                        rc = ens_fail(e, VP_ECUDA, "tuning restore failed");
                        break;
                    }
                }
                if (rc == VP_OK && ms < best) {
                    best = ms;
                    bw = Ws[wi];
                    br = Rs[ri];
                    bc = cps;
                    bf = fl;
                }
            }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamSynchronize(e->stream);
    cudaFree(snap_f);
    cudaFree(snap_acc);
    e->flat = bf;
    if (rc) return rc;
    e->tuned = 1;
    return vp_ensemble_set_tiles(e, bw, br, bc);
}

int vp_ensemble_step(vp_ens *e, double dt, int nsteps) {
    if (!e || !e->pool || nsteps < 0 || !std::isfinite(dt)) return VP_EINVAL;
    if (nsteps == 0) return VP_OK;
    const int trc = ensure_drift_table(e, dt);
    if (trc) return trc;
    const bool use_graph = e->stream != nullptr && e->stream != cudaStreamLegacy;
    if (use_graph && !(e->graph_valid && e->graph_dt == dt)) {
        if (e->graph_valid) {
            cudaGraphExecDestroy(e->graph);
            e->graph_valid = 0;
        }
        if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return ens_fail(e, VP_ECUDA, "capture failed");
        const long long before = e->launches;
        int rc = launch_pass(e, e->d_items_step, (int)e->items_step.size(), dt);
        cudaGraph_t g;
        const cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
        e->launches = before;
        if (rc) return rc;
        if (ce != cudaSuccess) return ens_fail(e, VP_ECUDA, "capture failed");
        const cudaError_t ie = cudaGraphInstantiate(&e->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return ens_fail(e, VP_ECUDA, "graph instantiate failed");
        e->graph_valid = 1;
        e->graph_dt = dt;
    }
    for (int s = 0; s < nsteps; ++s) {
        if (use_graph) {
            if (cudaGraphLaunch(e->graph, e->stream) != cudaSuccess) return ens_fail(e, VP_ECUDA, "graph launch failed");
            e->launches++;
        } else {
            int rc = launch_pass(e, e->d_items_step, (int)e->items_step.size(), dt);
            if (rc) return rc;
        }
    }
    return VP_OK;
}

int vp_ensemble_sync(vp_ens *e) {
    if (!e) return VP_EINVAL;
    if (cudaStreamSynchronize(e->stream) != cudaSuccess) return ens_fail(e, VP_ECUDA, "stream failed");
    int st = 0;
    cudaMemcpy(&st, e->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (st) {
        cudaMemset(e->d_status, 0, sizeof(int));
        return ens_fail(e, VP_ETIMEOUT, "a bounded wait in the ensemble kernel gave up");
    }
    return VP_OK;
}

long long vp_ensemble_launch_count(const vp_ens *e) { return e ? e->launches : 0; }

}  // extern "C"
