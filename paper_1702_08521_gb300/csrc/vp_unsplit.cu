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

constexpr int kMaxThreads = 256;
constexpr int kMaxSmem = 100 * 1024;

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

// phase A: D = A_1 f^n - f^n along a column (c: the column's f^n), cells in
// walk order (running pointers, steps sigma * pitch)
template <typename T>
struct StoreA {
    T *d;
    const T *c;
    int sd, sc;
    __device__ __forceinline__ void operator()(int, T a) {
        *d = a - *c;
        d += sd;
        c += sc;
    }
};

// phase B: D <- f^n + (D + (A_2 f^n - f^n)) along an x2 line, in walk order
template <typename T>
struct StoreB {
    T *d;
    const T *c;
    int s;
    __device__ __forceinline__ void operator()(int, T a) {
        const T fc = *c;
        *d = fc + (*d + (a - fc));
        d += s;
        c += s;
    }
};

template <typename T, int ORDER, bool FULL, int G>
__global__ void __launch_bounds__(kMaxThreads) k_unsplit2(const T *__restrict__ fin, T *__restrict__ fout,
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
    const int nt = blockDim.x;

    // stage rows r0 - G .. r0 + T1 + G - 1, x2 cells j0 - G .. j0 + T2 + G - 1,
    // velocities v0 .. v0 + TV - 1 (a ragged velocity tile stages zeros)
    const long long rs = (long long)u.n2 * u.NV;  // row stride of f
    const bool allv = u.TV == u.NV;
    if (allv && r0 >= G && r0 + u.T1 + G <= u.n1 && j0 >= G && j0 + u.T2 + G <= u.n2) {
        // interior tile with every velocity: each staged row is one contiguous
        // run of f^n, no wrap and no zero fill
        const int SW = (u.T2 + 2 * G) * u.TV, SR = u.T1 + 2 * G;
        const int dr = (int)fdiv((unsigned)nt, u.fd_sw), dq = nt - dr * SW;
        int rr = (int)fdiv(threadIdx.x, u.fd_sw), q = threadIdx.x - rr * SW;
        const T *gp = fin + (long long)(r0 - G) * rs + (long long)(j0 - G) * u.NV + rr * rs + q;
        T *sp = sm + rr * u.P + q;
        const long long gstep = dr * rs + dq, gwrap = rs - SW;
        const int sstep = dr * u.P + dq, swrap = u.P - SW;
        for (; rr < SR;) {
            cp_async_elem(sp, gp);
            rr += dr;
            q += dq;
            gp += gstep;
            sp += sstep;
            if (q >= SW) {
                q -= SW;
                ++rr;
                gp += gwrap;
                sp += swrap;
            }
        }
        vp_tma::cp_async_wait_all();
    } else {
        const int SW = (u.T2 + 2 * G) * u.TV, SR = u.T1 + 2 * G;
        const int dr = (int)fdiv((unsigned)nt, u.fd_sw), dq = nt - dr * SW;
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
        for (int it = threadIdx.x; it < items; it += nt) {
            const int seg = it / cols, col = it - seg * cols;
            const int jj = col / u.TV, tv = col - jj * u.TV;
            const int v = min(v0 + tv, u.NV - 1);
            const LineShift<T> sh = tab[(v / u.vs0) % u.nv0];
            const int ra = seg * u.T1 / u.nsegA, rb = (seg + 1) * u.T1 / u.nsegA;
            const int i0 = sh.sigma > 0 ? ra : rb - 1;
            const T *c0 = sm + G * u.P + (jj + G) * u.TV + tv;
            walk<T, ORDER, false, FULL, G, true>(
                c0, u.P, u.T1, sh, ra, rb, alpha, lp.mp, lp.pp,
                StoreA<T>{D + col + i0 * u.DP, c0 + i0 * u.P, sh.sigma * u.DP, sh.sigma * u.P});
        }
    }
    __syncthreads();
    // B: x2 lines
    {
        const int lines = u.T1 * u.TV, items = lines * u.nsegB;
        for (int it = threadIdx.x; it < items; it += nt) {
            const int seg = it / lines, l = it - seg * lines;
            const int r = l / u.TV, tv = l - r * u.TV;
            const int v = min(v0 + tv, u.NV - 1);
            const LineShift<T> sh = tab[u.nv0 + (v / u.vs1) % u.nv1];
            const int ja = seg * u.T2 / u.nsegB, jb = (seg + 1) * u.T2 / u.nsegB;
            const int j0w = sh.sigma > 0 ? ja : jb - 1;
            const T *l0 = sm + (r + G) * u.P + G * u.TV + tv;
            walk<T, ORDER, false, FULL, G, true>(
                l0, u.TV, u.T2, sh, ja, jb, alpha, lp.mp, lp.pp,
                StoreB<T>{D + r * u.DP + tv + j0w * u.TV, l0 + j0w * u.TV, sh.sigma * u.TV});
        }
    }
    __syncthreads();
    // C: f^{n+1} out
    if (allv && r0 + u.T1 <= u.n1 && j0 + u.T2 <= u.n2) {
        // whole tile with every velocity: contiguous rows of f^{n+1}
        const int W = u.T2 * u.TV;
        const int dr = nt / W, dq = nt - dr * W;
        int r = threadIdx.x / W, q = threadIdx.x - r * W;
        T *gp = fout + (long long)r0 * rs + (long long)j0 * u.NV + r * rs + q;
        const T *dp = D + r * u.DP + q;
        const long long gstep = dr * rs + dq, gwrap = rs - W;
        const int dstep = dr * u.DP + dq, dwrap = u.DP - W;
        for (; r < u.T1;) {
            *gp = *dp;
            r += dr;
            q += dq;
            gp += gstep;
            dp += dstep;
            if (q >= W) {
                q -= W;
                ++r;
                gp += gwrap;
                dp += dwrap;
            }
        }
    } else {
        const int W = u.T2 * u.TV;
        const int dr = nt / W, dq = nt - dr * W;
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

// launch geometry of one tile shape
template <typename T>
UnsplitGeo make_geo(const vp_ctx *c, int G, const UnsplitTune &t) {
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
    u.T1 = t.T1;
    u.T2 = t.T2;
    u.TV = t.TV;
    u.P = u.TV * ((u.T2 + 2 * G) | 1);
    u.DP = u.TV * (u.T2 | 1);
    // walk segments: enough work items for every thread, at least 8 cells each
    auto segs = [&](int lines, int len) {
        int s = (t.threads + lines - 1) / lines;
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

// velocity cells per tile: up to a warp's worth, fewer where even the
// smallest tile's halo would not fit the shared-memory budget
template <typename T>
int tile_tv(const vp_ctx *c, int G) {
    int TV = c->NV < 32 ? (int)c->NV : 32;
    while (TV > 1) {
        UnsplitTune t{1, 8, 8, TV, 128};
        if (unsplit_smem<T>(make_geo<T>(c, G, t), G) <= (size_t)kMaxSmem) break;
        TV /= 2;
    }
    return TV;
}

// candidate tile shapes: T1, T2 in 16 .. 128 (8 .. 32 for wide velocity
// tiles), 128 or 256 threads, within the shared-memory budget; the default is
// the one with the largest share of useful cells among the staged ones (at
// least 1024 cells, 256 threads)
template <typename T>
int candidates(const vp_ctx *c, int G, UnsplitTune *out, int cap, UnsplitTune *dflt) {
    const int TV = tile_tv<T>(c, G);
    const int lo = TV >= 8 ? 8 : 16, hi = TV >= 8 ? 32 : 128;
    int n = 0;
    double best = -1.0;
    *dflt = UnsplitTune{1, 8, 8, TV, 256};
    for (int T1 = lo; T1 <= hi; T1 *= 2)
        for (int T2 = lo; T2 <= hi; T2 *= 2)
            for (int th = 128; th <= 256; th *= 2) {
                const UnsplitTune t{1, T1, T2, TV, th};
                const UnsplitGeo u = make_geo<T>(c, G, t);
                if (unsplit_smem<T>(u, G) > (size_t)kMaxSmem) continue;
                if ((long long)T1 * T2 * TV < th) continue;  // a cell per thread at least
                if (n < cap) out[n++] = t;
                const double eff = (double)T1 * T2 / ((double)(T1 + 2 * G) * (T2 + 2 * G));
                const double score = eff + ((long long)T1 * T2 * TV >= 1024 ? 1.0 : 0.0) +
                                     (unsplit_smem<T>(u, G) <= 64 * 1024 ? 1.0 : 0.0);
                if (th == 256 && score > best) {
                    best = score;
                    *dflt = t;
                }
            }
    return n;
}

template <typename T, int ORDER, bool FULL, int G>
void set_attr_one() {
    cudaFuncSetAttribute(k_unsplit2<T, ORDER, FULL, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
}

template <typename T>
void set_attrs() {
    static bool done = false;
    if (done) return;
    set_attr_one<T, 5, false, 4>();
    set_attr_one<T, 5, false, 8>();
    set_attr_one<T, 5, true, 4>();
    set_attr_one<T, 5, true, 8>();
    set_attr_one<T, 7, false, 4>();
    set_attr_one<T, 7, false, 8>();
    set_attr_one<T, 7, true, 4>();
    set_attr_one<T, 7, true, 8>();
    done = true;
}

// one step a -> b with tile shape t
template <typename T>
int launch(vp_ctx *c, const T *a, T *b, int G, const UnsplitTune &t) {
    const vp_grid &g = c->g;
    const UnsplitGeo u = make_geo<T>(c, G, t);
    const long long tiles = (long long)((u.n1 + u.T1 - 1) / u.T1) * u.tiles2 * u.tilesv;
    if (tiles >= (1LL << 31)) return vp_fail(c, VP_ENOTSUP, "unsplit step has too many tiles");
    const size_t smem = unsplit_smem<T>(u, G);
    const LimParams lp{g.alpha, g.mp, g.pp};
    const bool full = g.mp && g.pp;
    const LineShift<T> *tab = static_cast<const LineShift<T> *>(c->d_shift);
#define VP_LAUNCH(O, F, GG) \
    k_unsplit2<T, O, F, GG><<<(unsigned)tiles, t.threads, smem, c->stream>>>(a, b, tab, u, lp)
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
    return VP_OK;
}

// Autotuner: time every candidate tile shape on the bound f (f -> scratch,
// which the call may overwrite; f is left unchanged) and keep the fastest.
// Once per halo width, never inside a stream capture.
template <typename T>
int tune(vp_ctx *c, int G, T *scratch) {
    constexpr int kCap = 48;
    UnsplitTune cand[kCap], best;
    const int nc = candidates<T>(c, G, cand, kCap, &best);
    cudaEvent_t e0, e1;
    VP_CUDA_TRY(c, cudaEventCreate(&e0));
    VP_CUDA_TRY(c, cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int rc = VP_OK;
    for (int i = 0; i < nc && rc == VP_OK; ++i) {
        float ms = 1e30f;
        for (int rep = 0; rep < 2 && rc == VP_OK; ++rep) {
            cudaEventRecord(e0, c->stream);
            rc = launch<T>(c, static_cast<const T *>(c->f), scratch, G, cand[i]);
            cudaEventRecord(e1, c->stream);
            if (rc) break;
            const cudaError_t se = cudaEventSynchronize(e1);
            if (se != cudaSuccess) {
                rc = vp_fail(c, VP_ECUDA, "unsplit candidate failed: %s", cudaGetErrorString(se));
                break;
            }
            float m = 0.f;
            cudaEventElapsedTime(&m, e0, e1);
            ms = m < ms ? m : ms;
        }
        if (rc == VP_OK && ms < best_ms) {
            best_ms = ms;
            best = cand[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    c->utune[G == 8] = best;
    c->utune[G == 8].valid = 1;
    return VP_OK;
}

template <typename T>
int run_t(vp_ctx *c, double dt, int nsteps, void *scratch, int G) {
    set_attrs<T>();
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
    T *a = static_cast<T *>(c->f), *b = static_cast<T *>(scratch);
    UnsplitTune t = c->utune[G == 8];
    if (!t.valid) {
        if (c->opt_autotune && !vp_capturing(c)) {
            const int rc = tune<T>(c, G, b);
            if (rc) return rc;
            t = c->utune[G == 8];
        } else {
            UnsplitTune cand[1];
            candidates<T>(c, G, cand, 0, &t);
        }
    }
    for (int s = 0; s < nsteps; ++s) {
        const int rc = launch<T>(c, a, b, G, t);
        if (rc) return rc;
        T *x = a;
        a = b;
        b = x;
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
