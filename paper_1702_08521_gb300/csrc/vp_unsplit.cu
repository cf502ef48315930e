// vp_unsplit.cu -- unsplit advection in two-dimensional physical space for
// sm_103a (the alternative to directional splitting that Sec. 2.4 discusses
// and Test-1d of Sec. 3.1 compares against):
//
//     f^{n+1} = f^n + (A_1 f^n - f^n) + (A_2 f^n - f^n),
//
// A_d the SL-MPP line update along x_d (Eq. 49 with the MP constraint and the
// PP limiter, exactly what a drift sweep along d makes of f^n).  Both
// increments are formed from the same f^n, so the update cannot run in place
// line by line as the split sweeps do: f^{n+1} goes to a second array (the
// extra storage the paper cites), and a run ping-pongs between the two.
//
// One CTA owns a tile of T1 x1-rows x T2 x2-cells x TV velocity cells.  It
// stages the tile of f^n with a halo of G cells along x1 and x2 in shared
// memory once (cp.async, periodic wrap or zero outside an outflow box), then
//   A. walks every x1 column of the tile with the line walker of the split
//      sweeps (each interface mass computed once) into D = A_1 f^n - f^n,
//      with the PP limiter's theta form at interfaces next to a negative
//      cell (the unsplit step does not keep f >= 0, and there the clamp the
//      split sweeps use is not the theta blend),
//   B. walks every x2 line of the tile the same way and completes
//      D <- f^n + (D + (A_2 f^n - f^n)),
//   C. writes D out with coalesced stores.
// So f^n is read from HBM once (plus the halo, mostly from L2) and f^{n+1}
// written once per step, where the split step reads and writes f once per
// direction.  G = 4 covers the MP7 stencil for shifts below half a cell (the
// unsplit method's regime, CFL < 0.1 in the paper); G = 8 allows integer
// shifts up to 4 cells.
#include <cmath>

#include "vp_internal.cuh"
#include "vp_sweep_core.cuh"
#include "vp_tma.cuh"

namespace {

using vp_core::walk;

constexpr int kThreads = 256;

struct UnsplitGeo {
    int n1, n2, NV;     // cells along x1 and x2; velocity cells per spatial point
    int T1, T2, TV;     // tile: x1 rows, x2 cells, velocity cells
    int P;              // staged row pitch in elements (TV x odd)
    int DP;             // result row pitch in elements (TV x odd)
    int tiles2, tilesv; // tiles along x2 and along v
    int nsegA, nsegB;   // walk segments per x1 column / per x2 line
    int vs0, nv0, vs1, nv1;  // line class: x1 columns (v / vs0) % nv0, x2 lines nv0 + (v / vs1) % nv1
    int periodic;
    FastDiv fd_sw, fd_tv;  // staged elements per row, TV
};

// 4- or 8-byte asynchronous global -> shared copy (completes at cp_async_wait_all)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(vp_tma::saddr(smem)), "l"(gmem),
                 "n"((int)sizeof(T))
                 : "memory");
}

__device__ __forceinline__ int wrap(int x, int n) {
    if (x >= 0 && x < n) return x;
    x %= n;
    return x < 0 ? x + n : x;
}

// phase A: D[i] = A_1 f^n - f^n at row i of a column (c: the column's f^n)
template <typename T>
struct StoreA {
    T *d;
    const T *c;
    int dp, p;
    __device__ __forceinline__ void operator()(int i, T a) { d[i * dp] = a - c[i * p]; }
};

// phase B: D[j] <- f^n + (D[j] + (A_2 f^n - f^n)) at cell j of an x2 line
template <typename T>
struct StoreB {
    T *d;
    const T *c;
    int tv;
    __device__ __forceinline__ void operator()(int j, T a) {
        const T fc = c[j * tv];
        d[j * tv] = fc + (d[j * tv] + (a - fc));
    }
};

template <typename T, int ORDER, bool FULL, int G>
__global__ void __launch_bounds__(kThreads) k_unsplit2(const T *__restrict__ fin, T *__restrict__ fout,
                                                       const LineShift<T> *__restrict__ tab, UnsplitGeo u,
                                                       LimParams lp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);     // (T1 + 2G) rows x P: f^n with its halo
    T *D = sm + (size_t)(u.T1 + 2 * G) * u.P;  // T1 rows x DP: the increments, then f^{n+1}
    unsigned b = blockIdx.x;
    const int tvi = (int)(b % (unsigned)u.tilesv);
    b /= (unsigned)u.tilesv;
    const int t2 = (int)(b % (unsigned)u.tiles2);
    const int t1 = (int)(b / (unsigned)u.tiles2);
    const int r0 = t1 * u.T1, j0 = t2 * u.T2, v0 = tvi * u.TV;

    // stage rows r0 - G .. r0 + T1 + G - 1, x2 cells j0 - G .. j0 + T2 + G - 1,
    // velocities v0 .. v0 + TV - 1 (a ragged velocity tile stages zeros)
    {
        const int SW = (u.T2 + 2 * G) * u.TV, SR = u.T1 + 2 * G;
        const int dr = (int)fdiv(kThreads, u.fd_sw), dq = kThreads - dr * SW;
        int rr = (int)fdiv(threadIdx.x, u.fd_sw), q = threadIdx.x - rr * SW;
        for (; rr < SR;) {
            const int jj = (int)fdiv((unsigned)q, u.fd_tv), tv = q - jj * u.TV;
            int x1 = r0 - G + rr, x2 = j0 - G + jj;
            const int v = v0 + tv;
            bool ok = v < u.NV;
            if (u.periodic) {
                x1 = wrap(x1, u.n1);
                x2 = wrap(x2, u.n2);
            } else {
                ok = ok && x1 >= 0 && x1 < u.n1 && x2 >= 0 && x2 < u.n2;
            }
            T *dst = sm + rr * u.P + q;
            if (ok)
                cp_async_elem(dst, fin + ((long long)x1 * u.n2 + x2) * u.NV + v);
            else
                *dst = T(0);
            rr += dr;
            q += dq;
            if (q >= SW) {
                q -= SW;
                ++rr;
            }
        }
        vp_tma::cp_async_wait_all();
    }
    __syncthreads();

    const T alpha = (T)lp.alpha;
    // A: x1 columns
    {
        const int cols = u.T2 * u.TV, items = cols * u.nsegA;
        for (int it = threadIdx.x; it < items; it += kThreads) {
            const int seg = it / cols, col = it - seg * cols;
            const int jj = col / u.TV, tv = col - jj * u.TV;
            const int v = min(v0 + tv, u.NV - 1);
            const LineShift<T> sh = tab[(v / u.vs0) % u.nv0];
            const int ra = seg * u.T1 / u.nsegA, rb = (seg + 1) * u.T1 / u.nsegA;
            const T *c0 = sm + G * u.P + (jj + G) * u.TV + tv;
            walk<T, ORDER, false, FULL, G, true>(c0, u.P, u.T1, sh, ra, rb, alpha, lp.mp, lp.pp,
                                           StoreA<T>{D + col, c0, u.DP, u.P});
        }
    }
    __syncthreads();
    // B: x2 lines
    {
        const int lines = u.T1 * u.TV, items = lines * u.nsegB;
        for (int it = threadIdx.x; it < items; it += kThreads) {
            const int seg = it / lines, l = it - seg * lines;
            const int r = l / u.TV, tv = l - r * u.TV;
            const int v = min(v0 + tv, u.NV - 1);
            const LineShift<T> sh = tab[u.nv0 + (v / u.vs1) % u.nv1];
            const int ja = seg * u.T2 / u.nsegB, jb = (seg + 1) * u.T2 / u.nsegB;
            const T *l0 = sm + (r + G) * u.P + G * u.TV + tv;
            walk<T, ORDER, false, FULL, G, true>(l0, u.TV, u.T2, sh, ja, jb, alpha, lp.mp, lp.pp,
                                           StoreB<T>{D + r * u.DP + tv, l0, u.TV});
        }
    }
    __syncthreads();
    // C: f^{n+1} out
    {
        const int W = u.T2 * u.TV;
        const int dr = kThreads / W, dq = kThreads - dr * W;
        int r = threadIdx.x / W, q = threadIdx.x - r * W;
        for (; r < u.T1;) {
            const int jj = (int)fdiv((unsigned)q, u.fd_tv), tv = q - jj * u.TV;
            const int x1 = r0 + r, x2 = j0 + jj, v = v0 + tv;
            if (x1 < u.n1 && x2 < u.n2 && v < u.NV) fout[((long long)x1 * u.n2 + x2) * u.NV + v] = D[r * u.DP + q];
            r += dr;
            q += dq;
            if (q >= W) {
                q -= W;
                ++r;
            }
        }
    }
}

// shift decomposition of every drift line class of both axes: entries
// 0 .. nv0 - 1 for x1 (velocity index along v_1), nv0 .. nv0 + nv1 - 1 for x2
struct DriftAxes {
    double lo[2], dvel[2], h[2];
    int nv0, nv1;
};

template <typename T>
__global__ void k_drift_tables(LineShift<T> *__restrict__ tab, DriftAxes ax, double dt, WPoly wp) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ax.nv0 + ax.nv1) return;
    const int d = e < ax.nv0 ? 0 : 1;
    const int k = d ? e - ax.nv0 : e;
    tab[e] = vp_core::make_shift<T>(vp_core::cell_centre(ax.lo[d], ax.dvel[d], k), dt, ax.h[d], wp);
}

template <typename T>
size_t unsplit_smem(const UnsplitGeo &u, int G) {
    return (size_t)((u.T1 + 2 * G) * u.P + u.T1 * u.DP) * sizeof(T);
}

// tile shape: the largest share of useful cells among the staged ones within
// a shared-memory budget, at least 1024 cells per tile
template <typename T>
UnsplitGeo plan(const vp_ctx *c, int G) {
    const vp_grid &g = c->g;
    UnsplitGeo u{};
    u.n1 = g.nx[0];
    u.n2 = g.nx[1];
    u.NV = (int)c->NV;
    u.periodic = g.xbc == VP_BC_PERIODIC;
    u.nv0 = g.nv[0];
    u.nv1 = g.nv[1];
    u.vs0 = g.nv[1];
    u.vs1 = 1;
    // velocity cells per tile: up to a warp's worth, fewer where even the
    // smallest tile's halo would not fit
    double best = -1.0;
    const int T1s[4] = {8, 16, 32, 64}, T2s[5] = {8, 16, 32, 64, 128};
    for (int TV = u.NV < 32 ? u.NV : 32; best < 0.0 && TV >= 1; TV /= 2)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 5; ++b) {
                UnsplitGeo t = u;
                t.TV = TV;
                t.T1 = T1s[a];
                t.T2 = T2s[b];
                t.P = t.TV * ((t.T2 + 2 * G) | 1);
                t.DP = t.TV * (t.T2 | 1);
                if (unsplit_smem<T>(t, G) > 64 * 1024) continue;
                const double eff = (double)t.T1 * t.T2 / ((double)(t.T1 + 2 * G) * (t.T2 + 2 * G));
                const bool big = (long long)t.T1 * t.T2 * t.TV >= 1024;
                const double score = eff + (big ? 1.0 : 0.0);
                if (score > best) {
                    best = score;
                    u = t;
                }
            }
    auto segs = [](int cells, int len) {
        int s = (kThreads + cells - 1) / cells;
        while (s > 1 && len / s < 8) --s;
        return s < 1 ? 1 : s;
    };
    u.nsegA = segs(u.T2 * u.TV, u.T1);
    u.nsegB = segs(u.T1 * u.TV, u.T2);
    u.tiles2 = (u.n2 + u.T2 - 1) / u.T2;
    u.tilesv = (u.NV + u.TV - 1) / u.TV;
    u.fd_sw = make_fastdiv((unsigned)((u.T2 + 2 * G) * u.TV));
    u.fd_tv = make_fastdiv((unsigned)u.TV);
    return u;
}

template <typename T, int ORDER, bool FULL, int G>
void set_attr_one() {
    cudaFuncSetAttribute(k_unsplit2<T, ORDER, FULL, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
}

template <typename T>
int run_t(vp_ctx *c, double dt, int nsteps, void *scratch, int G) {
    static bool attrs = false;
    if (!attrs) {
        set_attr_one<T, 5, false, 4>();
        set_attr_one<T, 5, false, 8>();
        set_attr_one<T, 5, true, 4>();
        set_attr_one<T, 5, true, 8>();
        set_attr_one<T, 7, false, 4>();
        set_attr_one<T, 7, false, 8>();
        set_attr_one<T, 7, true, 4>();
        set_attr_one<T, 7, true, 8>();
        attrs = true;
    }
    const vp_grid &g = c->g;
    DriftAxes ax{};
    for (int d = 0; d < 2; ++d) {
        ax.lo[d] = g.vlo[d];
        ax.dvel[d] = (g.vhi[d] - g.vlo[d]) / g.nv[d];
        ax.h[d] = (g.xhi[d] - g.xlo[d]) / g.nx[d];
    }
    ax.nv0 = g.nv[0];
    ax.nv1 = g.nv[1];
    LineShift<T> *tab = static_cast<LineShift<T> *>(c->d_shift);
    const int ne = ax.nv0 + ax.nv1;
    k_drift_tables<T><<<(ne + 127) / 128, 128, 0, c->stream>>>(tab, ax, dt, c->wp);
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    const UnsplitGeo u = plan<T>(c, G);
    const long long tiles = (long long)((u.n1 + u.T1 - 1) / u.T1) * u.tiles2 * u.tilesv;
    if (tiles >= (1LL << 31)) return vp_fail(c, VP_ENOTSUP, "unsplit step has too many tiles");
    const size_t smem = unsplit_smem<T>(u, G);
    const LimParams lp{g.alpha, g.mp, g.pp};
    const bool full = g.mp && g.pp;
    T *a = static_cast<T *>(c->f), *b = static_cast<T *>(scratch);
    for (int s = 0; s < nsteps; ++s) {
#define VP_LAUNCH(O, F, GG) \
    k_unsplit2<T, O, F, GG><<<(unsigned)tiles, kThreads, smem, c->stream>>>(a, b, tab, u, lp)
        if (g.order == 7) {
            if (full) {
                if (G == 4) VP_LAUNCH(7, true, 4); else VP_LAUNCH(7, true, 8);
            } else {
                if (G == 4) VP_LAUNCH(7, false, 4); else VP_LAUNCH(7, false, 8);
            }
        } else {
            if (full) {
                if (G == 4) VP_LAUNCH(5, true, 4); else VP_LAUNCH(5, true, 8);
            } else {
                if (G == 4) VP_LAUNCH(5, false, 4); else VP_LAUNCH(5, false, 8);
            }
        }
#undef VP_LAUNCH
        c->launches++;
        VP_CUDA_TRY(c, cudaGetLastError());
        T *t = a;
        a = b;
        b = t;
    }
    if (a != c->f) {
        VP_CUDA_TRY(c, cudaMemcpyAsync(c->f, a, (size_t)c->ncell * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
    }
    return VP_OK;
}

}  // namespace

int vp_drift_unsplit(vp_ctx *c, double dt, int nsteps, void *scratch_dev) {
    if (!c) return VP_EINVAL;
    if (!c->f) return vp_fail(c, VP_EINVAL, "no distribution function bound (vp_bind_f)");
    const vp_grid &g = c->g;
    if (g.dx != 2) return vp_fail(c, VP_ENOTSUP, "unsplit advection needs two spatial dimensions");
    if (g.scheme != VP_SCHEME_SL) return vp_fail(c, VP_ENOTSUP, "unsplit advection uses the SL-MPP update");
    if (!std::isfinite(dt)) return vp_fail(c, VP_EINVAL, "dt must be finite");
    if (nsteps < 0) return vp_fail(c, VP_EINVAL, "nsteps must be >= 0");
    if (!scratch_dev) return vp_fail(c, VP_EINVAL, "scratch_dev is NULL");
    const uintptr_t fa = reinterpret_cast<uintptr_t>(c->f), sa = reinterpret_cast<uintptr_t>(scratch_dev);
    const uintptr_t bytes = (uintptr_t)c->ncell * (uintptr_t)c->esize;
    if (sa % 16) return vp_fail(c, VP_EINVAL, "scratch_dev must be 16-byte aligned");
    if (sa < fa + bytes && fa < sa + bytes) return vp_fail(c, VP_EINVAL, "scratch_dev overlaps f");
    // largest whole-cell shift of a line (the extreme velocity centres of each
    // axis, in the arithmetic of the device's shift tables); the halo must
    // cover it and the stencil
    double nmax = 0.0;
    for (int d = 0; d < 2; ++d) {
        const double h = (g.xhi[d] - g.xlo[d]) / g.nx[d];
        const double dvel = (g.vhi[d] - g.vlo[d]) / g.nv[d];
        for (int k : {0, g.nv[d] - 1}) {
            const double s = (g.vlo[d] + ((double)k + 0.5) * dvel) * dt / h;
            if (!(std::fabs(s) < 1e9)) return vp_fail(c, VP_EINVAL, "shift too large");
            nmax = std::fmax(nmax, std::fabs(std::round(s)));
        }
    }
    const int G = nmax == 0.0 ? 4 : (nmax <= 4.0 ? 8 : 0);
    if (!G) return vp_fail(c, VP_ENOTSUP, "unsplit step shifts a line by %.0f whole cells (at most 4 supported)", nmax);
    if (nsteps == 0) return VP_OK;
    if (g.precision == VP_F32) return run_t<float>(c, dt, nsteps, scratch_dev, G);
    return run_t<double>(c, dt, nsteps, scratch_dev, G);
}
