// vp_field.cu -- velocity moment, FFT Poisson solver with the 2nd/4th/6th-
// order Green functions (periodic) or doubling-up (isolated), FDA force,
// diagnostics reductions and analytic initial conditions, all on the device.
//
// Precision: f is read as float or double; every sum over velocity space is
// carried in double precision (for float input, a compensated float sum per
// thread -- Knuth's two-sum -- whose value and error term are combined in
// double, then double across threads).  Fourier transforms, Green functions
// and forces are double precision throughout.
#include <cmath>
#include <mutex>

#include "vp_internal.cuh"

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    __syncthreads();
    return v;  // valid in thread 0
}

// ---- density moment ----------------------------------------------------------

struct CSum {
    float s, e;
    __device__ void add(float x) {
        const float t = s + x;
        const float bp = t - s;
        e += (s - (t - bp)) + (x - bp);
        s = t;
    }
};

__device__ __forceinline__ double thread_sum(const float *p, long long n) {
    CSum cs{0.f, 0.f};
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0 && (n & 3) == 0) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
        for (long long i = threadIdx.x; i < n / 4; i += blockDim.x) {
            const float4 v = q[i];
            cs.add(v.x);
            cs.add(v.y);
            cs.add(v.z);
            cs.add(v.w);
        }
    } else {
        for (long long i = threadIdx.x; i < n; i += blockDim.x) cs.add(p[i]);
    }
    return (double)cs.s + (double)cs.e;
}

__device__ __forceinline__ double thread_sum(const double *p, long long n) {
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
    return s;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_moment(const T *__restrict__ f, long long NV, double dV,
                                                   double *__restrict__ rho) {
    __shared__ double sh[32];
    const double s = block_sum(thread_sum(f + (long long)blockIdx.x * NV, NV), sh);
    if (threadIdx.x == 0) rho[blockIdx.x] = s * dV;
}

// ---- Fourier transform along one axis of a row-major complex array ----------
// One CTA per line; power-of-two lengths use an in-shared-memory radix-2
// decimation-in-time transform, other lengths a direct sum.  sign = -1 is the
// forward transform sum_j q_j exp(-i k j 2 pi / n) (Eq. C4), +1 the inverse
// without 1/n.

__global__ void k_fft_axis(double2 *__restrict__ a, long long inner, int n, int sign) {
    extern __shared__ double2 sbuf[];
    double2 *x = sbuf;
    double2 *y = sbuf + n;
    const long long line = blockIdx.x;
    const long long o = line / inner, c = line % inner;
    double2 *base = a + o * (long long)n * inner + c;
    const bool pow2 = (n & (n - 1)) == 0;
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        int dst = j;
        if (pow2 && n > 1) dst = (int)(__brev((unsigned)j) >> (32 - logn));
        x[dst] = base[(long long)j * inner];
    }
    __syncthreads();
    if (pow2) {
        for (int len = 2; len <= n; len <<= 1) {
            const int half = len >> 1;
            for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
                const int grp = t / half, k = t - grp * half;
                const int i0 = grp * len + k, i1 = i0 + half;
                double sn, cs;
                sincospi((double)sign * 2.0 * (double)k / (double)len, &sn, &cs);
                const double2 u = x[i0], v = x[i1];
                const double2 tw = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
                x[i0] = make_double2(u.x + tw.x, u.y + tw.y);
                x[i1] = make_double2(u.x - tw.x, u.y - tw.y);
            }
            __syncthreads();
        }
        for (int j = threadIdx.x; j < n; j += blockDim.x) base[(long long)j * inner] = x[j];
    } else {
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            double sr = 0.0, si = 0.0;
            for (int j = 0; j < n; ++j) {
                const long long m = ((long long)j * k) % n;
                double sn, cs;
                sincospi((double)sign * 2.0 * (double)m / (double)n, &sn, &cs);
                const double2 v = x[j];
                sr += v.x * cs - v.y * sn;
                si += v.x * sn + v.y * cs;
            }
            y[k] = make_double2(sr, si);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) base[(long long)j * inner] = y[j];
    }
}

// scatter rho - rho_bg into the (possibly padded) complex grid, zero elsewhere
__global__ void k_load_rho(double2 *__restrict__ a, const double *__restrict__ rho, double bg,
                           long long MT, int3 nbox, int3 m, int dims) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= MT) return;
    long long r = t;
    int idx[3] = {0, 0, 0};
    const int md[3] = {m.x, m.y, m.z};
    const int nb[3] = {nbox.x, nbox.y, nbox.z};
    for (int d = dims - 1; d >= 0; --d) {
        idx[d] = (int)(r % md[d]);
        r /= md[d];
    }
    bool in = true;
    long long lin = 0;
    for (int d = 0; d < dims; ++d) {
        in = in && idx[d] < nb[d];
        lin = lin * nb[d] + idx[d];
    }
    a[t] = make_double2(in ? rho[lin] - bg : 0.0, 0.0);
}

__global__ void k_mul_real(double2 *__restrict__ a, const double *__restrict__ g, long long n) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double s = g[t];
    a[t] = make_double2(a[t].x * s, a[t].y * s);
}

__global__ void k_mul_cplx(double2 *__restrict__ a, const double2 *__restrict__ g, long long n,
                           double scale) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double2 u = a[t], v = g[t];
    a[t] = make_double2((u.x * v.x - u.y * v.y) * scale, (u.x * v.y + u.y * v.x) * scale);
}

// phi (box) and accel = -grad phi by the 2/4/6-point FDA (Eqs. C9-C11),
// reading the potential of the m-periodic grid (m = box for periodic,
// m = 2 box for doubling-up) with cyclic indices.
struct Fda {
    double c[4];  // c[k] multiplies (phi_{i+k} - phi_{i-k}), k = 1..3
    double den;
};

__global__ void k_force(const double2 *__restrict__ a, double scale, double *__restrict__ phi,
                        double *__restrict__ acc, long long NX, int3 nbox, int3 m, int dims,
                        double3 h, Fda fd, int npts) {
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= NX) return;
    const int nb[3] = {nbox.x, nbox.y, nbox.z};
    const int md[3] = {m.x, m.y, m.z};
    const double hh[3] = {h.x, h.y, h.z};
    int idx[3] = {0, 0, 0};
    long long r = x;
    for (int d = dims - 1; d >= 0; --d) {
        idx[d] = (int)(r % nb[d]);
        r /= nb[d];
    }
    auto at = [&](int axis, int off) -> double {
        long long lin = 0;
        for (int d = 0; d < dims; ++d) {
            int j = idx[d];
            if (d == axis) {
                j = (j + off) % md[d];
                if (j < 0) j += md[d];
            }
            lin = lin * md[d] + j;
        }
        return a[lin].x * scale;
    };
    if (phi) phi[x] = at(0, 0);
    for (int d = 0; d < dims; ++d) {
        double g = 0.0;
        for (int k = 1; k <= npts; ++k) g += fd.c[k] * (at(d, k) - at(d, -k));
        acc[(long long)d * NX + x] = -g / (fd.den * hh[d]);
    }
}

// ---- diagnostics -----------------------------------------------------------

struct VGrid {
    double lo[3], h[3];
    int n[3];
    int dv;
};

template <typename T>
__global__ void __launch_bounds__(kBlock) k_diag_part(const T *__restrict__ f, long long NV,
                                                      VGrid vg, double *__restrict__ part,
                                                      int *__restrict__ bad) {
    __shared__ double sh[32];
    __shared__ double smin[32], smax[32];
    const T *p = f + (long long)blockIdx.x * NV;
    double m0 = 0, m2 = 0, l1 = 0, l2 = 0, mn = INFINITY, mx = -INFINITY;
    int nonfinite = 0;
    for (long long v = threadIdx.x; v < NV; v += blockDim.x) {
        const double val = (double)p[v];
        long long r = v;
        double v2 = 0.0;
        for (int d = vg.dv - 1; d >= 0; --d) {
            const double vc = vg.lo[d] + ((double)(r % vg.n[d]) + 0.5) * vg.h[d];
            r /= vg.n[d];
            v2 += vc * vc;
        }
        if (!isfinite(val)) nonfinite = 1;
        m0 += val;
        m2 += 0.5 * val * v2;
        l1 += fabs(val);
        l2 += val * val;
        mn = fmin(mn, val);
        mx = fmax(mx, val);
    }
    if (nonfinite) atomicExch(bad, 1);
    m0 = block_sum(m0, sh);
    m2 = block_sum(m2, sh);
    l1 = block_sum(l1, sh);
    l2 = block_sum(l2, sh);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        smin[w] = mn;
        smax[w] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x + 31) / 32; ++k) {
            mn = fmin(mn, smin[k]);
            mx = fmax(mx, smax[k]);
        }
        double *q = part + (long long)blockIdx.x * 6;
        q[0] = m0;
        q[1] = m2;
        q[2] = l1;
        q[3] = l2;
        q[4] = mn;
        q[5] = mx;
    }
}

__global__ void __launch_bounds__(kBlock) k_diag_final(const double *__restrict__ part,
                                                       const double *__restrict__ rho,
                                                       const double *__restrict__ phi,
                                                       const double *__restrict__ acc, long long NX,
                                                       int dims, int n1, long long rest, int mode,
                                                       double bg, double dX, double dV,
                                                       double *__restrict__ out) {
    __shared__ double sh[32];
    __shared__ double smin[32], smax[32];
    double m0 = 0, m2 = 0, l1 = 0, l2 = 0, mn = INFINITY, mx = -INFINITY, fe = 0, pe = 0, cr = 0,
           ci = 0;
    for (long long x = threadIdx.x; x < NX; x += blockDim.x) {
        const double *q = part + x * 6;
        m0 += q[0];
        m2 += q[1];
        l1 += q[2];
        l2 += q[3];
        mn = fmin(mn, q[4]);
        mx = fmax(mx, q[5]);
        for (int d = 0; d < dims; ++d) fe += 0.5 * acc[d * NX + x] * acc[d * NX + x];
        pe += 0.5 * (rho[x] - bg) * phi[x];
        const long long j1 = x / rest;
        double sn, cs;
        sincospi(-2.0 * (double)((mode * j1) % n1) / (double)n1, &sn, &cs);
        cr += acc[x] * cs;
        ci += acc[x] * sn;
    }
    m0 = block_sum(m0, sh);
    m2 = block_sum(m2, sh);
    l1 = block_sum(l1, sh);
    l2 = block_sum(l2, sh);
    fe = block_sum(fe, sh);
    pe = block_sum(pe, sh);
    cr = block_sum(cr, sh);
    ci = block_sum(ci, sh);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        smin[w] = mn;
        smax[w] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x + 31) / 32; ++k) {
            mn = fmin(mn, smin[k]);
            mx = fmax(mx, smax[k]);
        }
        out[0] = m0 * dX * dV;
        out[1] = m2 * dX * dV;
        out[2] = fe * dX;
        out[3] = pe * dX;
        out[4] = mn;
        out[5] = mx;
        out[6] = 2.0 / (double)NX * sqrt(cr * cr + ci * ci);
        out[7] = l1 * dX * dV;
        out[8] = l2 * dX * dV;
    }
}

// ---- initial conditions ------------------------------------------------------

struct IcArgs {
    int kind, dims;
    int nx[3], nv[3];
    double xlo[3], hx[3], vlo[3], hv[3], xc[3];
    double p[8];
    long long NV;
};

template <typename T>
__global__ void k_init(T *__restrict__ f, long long ncell, IcArgs a) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell) return;
    long long xi = t / a.NV, vi = t % a.NV;
    double xs[3] = {0, 0, 0}, vs[3] = {0, 0, 0};
    for (int d = a.dims - 1; d >= 0; --d) {
        xs[d] = a.xlo[d] + ((double)(xi % a.nx[d]) + 0.5) * a.hx[d];
        xi /= a.nx[d];
        vs[d] = a.vlo[d] + ((double)(vi % a.nv[d]) + 0.5) * a.hv[d];
        vi /= a.nv[d];
    }
    const double kPi = 3.141592653589793238462643383279502884;
    double val = 0.0;
    if (a.kind == VP_IC_LANDAU) {
        const double alpha = a.p[0], sig = a.p[4], amp = a.p[5];
        double sp = 1.0, g = 1.0;
        for (int d = 0; d < a.dims; ++d) {
            sp += alpha * cos(a.p[1 + d] * xs[d]);
            g *= exp(-vs[d] * vs[d] / (2.0 * sig * sig)) / sqrt(2.0 * kPi * sig * sig);
        }
        val = amp * sp * g;
    } else if (a.kind == VP_IC_TWOSTREAM) {
        double v2 = 0.0;
        for (int d = 0; d < a.dims; ++d) v2 += vs[d] * vs[d];
        val = vs[0] * vs[0] * exp(-0.5 * v2) / pow(2.0 * kPi, 0.5 * a.dims) *
              (1.0 + a.p[0] * cos(a.p[1] * xs[0]));
    } else if (a.kind == VP_IC_PLUMMER) {
        const double G = a.p[0], M = a.p[1], b = a.p[2];
        double r2 = 0.0, v2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            r2 += (xs[d] - a.xc[d]) * (xs[d] - a.xc[d]);
            v2 += vs[d] * vs[d];
        }
        const double E = 0.5 * v2 - G * M / sqrt(r2 + b * b);
        // isotropic Plummer model: F(E) = 24 sqrt(2) a^2 / (7 pi^3 G^5 M^4) (-E)^(7/2)
        val = E < 0.0 ? 24.0 * sqrt(2.0) * b * b / (7.0 * kPi * kPi * kPi * pow(G, 5.0) * pow(M, 4.0)) *
                            pow(-E, 3.5)
                      : 0.0;
    } else if (a.kind == VP_IC_SPHERE) {
        // uniform sphere of mass M and radius 2R about the box centre with a
        // Maxwellian of sigma^2 = G M / (20 R) (Eq. 77, Sec. 3.4)
        const double G = a.p[0], M = a.p[1], R = a.p[2];
        const double rho0 = M / (4.0 * kPi * (8.0 * R * R * R) / 3.0);
        const double s2 = G * M / (20.0 * R);
        double r2 = 0.0, v2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            r2 += (xs[d] - a.xc[d]) * (xs[d] - a.xc[d]);
            v2 += vs[d] * vs[d];
        }
        val = r2 < 4.0 * R * R ? rho0 * exp(-v2 / (2.0 * s2)) / pow(2.0 * kPi * s2, 1.5) : 0.0;
    } else {
        const int shape = (int)a.p[0];
        if (shape == 0) {
            val = 1.0;
            for (int d = 0; d < a.dims; ++d)
                if (!(xs[d] >= 0.25 && xs[d] <= 0.75)) val = 0.0;
        } else if (shape == 1) {
            val = 1.0;
            for (int d = 0; d < a.dims; ++d) val += sin(2.0 * kPi * xs[d]) / a.dims;
        } else {
            for (int d = 0; d < a.dims; ++d) {
                const double s = sin(4.0 * kPi * xs[d]);
                val += s * s * s * s;
            }
        }
    }
    f[t] = (T)val;
}

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

int fft_all_axes(vp_ctx *c, double2 *buf, const int *m, int dims, int sign) {
    long long total = 1;
    for (int d = 0; d < dims; ++d) total *= m[d];
    for (int a = 0; a < dims; ++a) {
        long long inner = 1;
        for (int d = a + 1; d < dims; ++d) inner *= m[d];
        const long long lines = total / m[a];
        const size_t smem = 2 * (size_t)m[a] * sizeof(double2);
        int th = m[a] / 2 < 32 ? 32 : (m[a] / 2 > 256 ? 256 : m[a] / 2);
        k_fft_axis<<<(unsigned)lines, th, smem, c->stream>>>(buf, inner, m[a], sign);
        c->launches++;
    }
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

Fda fda_coeffs(int order) {
    // central differences of Eqs. (C9)-(C11): sum_k c_k (phi_{i+k} - phi_{i-k}) / (den h)
    Fda f{};
    if (order == 2) {
        f.c[1] = 1.0;
        f.den = 2.0;
    } else if (order == 4) {
        f.c[1] = 8.0;
        f.c[2] = -1.0;
        f.den = 12.0;
    } else {
        f.c[1] = 45.0;
        f.c[2] = -9.0;
        f.c[3] = 1.0;
        f.den = 60.0;
    }
    return f;
}

}  // namespace

// ---- setup: Green functions -----------------------------------------------------

// Eigenvalue of the periodic discrete Laplacian stencil (Eqs. C1, C5, C6)
// for theta = k h, written from its coefficients: with the symmetric stencil
// (b_0, b_1, b_2, b_3) / den the eigenvalue is -(4/den) sum_m b_m sin^2(m theta / 2).
static double stencil_eig(int order, double theta) {
    double b[4] = {0, 0, 0, 0}, den = 1.0;
    if (order == 2) {
        b[1] = 1.0;
    } else if (order == 4) {
        b[1] = 16.0;
        b[2] = -1.0;
        den = 12.0;
    } else {
        b[1] = 270.0;
        b[2] = -27.0;
        b[3] = 2.0;
        den = 180.0;
    }
    double s = 0.0;
    for (int mm = 1; mm <= 3; ++mm) {
        const double q = sin(0.5 * mm * theta);
        s += b[mm] * q * q;
    }
    return -4.0 * s / den;
}

// mean of 1/r over a cube of side 1 about its centre: 24 pyramids with apex
// at the centre give 3 * int_0^1 int_0^1 (1 + u^2 + v^2)^(-1/2) du dv, here by
// composite Gauss-Legendre quadrature (the integrand is smooth).
static double cube_inv_r_mean() {
    const double xg[5] = {-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831,
                          0.9061798459386640};
    const double wg[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889,
                          0.4786286704993665, 0.2369268850561891};
    const int nsub = 40;
    double s = 0.0;
    for (int a = 0; a < nsub; ++a)
        for (int i = 0; i < 5; ++i) {
            const double u = (a + 0.5 * (xg[i] + 1.0)) / nsub;
            for (int b2 = 0; b2 < nsub; ++b2)
                for (int j = 0; j < 5; ++j) {
                    const double v = (b2 + 0.5 * (xg[j] + 1.0)) / nsub;
                    s += wg[i] * wg[j] / sqrt(1.0 + u * u + v * v);
                }
        }
    return 3.0 * s / (4.0 * nsub * nsub);
}

int vp_field_setup(vp_ctx *c) {
    const vp_grid &g = c->g;
    VP_CUDA_TRY(c, cudaFuncSetAttribute(k_fft_axis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        2 * 4096 * (int)sizeof(double2)));
    const int D = g.dx;
    if (g.poisson == VP_POIS_PERIODIC) {
        c->MT = c->NX;
        for (int d = 0; d < 3; ++d) c->m[d] = d < D ? g.nx[d] : 1;
        double *h_g = (double *)malloc(sizeof(double) * c->NX);
        if (!h_g) return vp_fail(c, VP_ENOMEM, "host allocation failed");
        for (long long x = 0; x < c->NX; ++x) {
            long long r = x;
            int allzero = 1;
            double lam = 0.0;
            for (int d = D - 1; d >= 0; --d) {
                const long long nk = r % g.nx[d];
                r /= g.nx[d];
                if (nk) allzero = 0;
                const double h = (g.xhi[d] - g.xlo[d]) / g.nx[d];
                lam += stencil_eig(g.pois_order, 2.0 * M_PI * (double)nk / (double)g.nx[d]) / (h * h);
            }
            // phi_hat = S rho_hat / lambda; the inverse transform's 1/NX is folded in
            h_g[x] = allzero ? 0.0 : g.coupling / lam / (double)c->NX;
        }
        VP_CUDA_TRY(c, cudaMalloc(&c->d_green, sizeof(double) * c->NX));
        VP_CUDA_TRY(c, cudaMemcpy(c->d_green, h_g, sizeof(double) * c->NX, cudaMemcpyHostToDevice));
        free(h_g);
        VP_CUDA_TRY(c, cudaMalloc(&c->d_fft, sizeof(double2) * c->MT));
        return VP_OK;
    }
    // isolated: doubling-up with the real-space kernel -(S / 4 pi) dV / r
    const double h = (g.xhi[0] - g.xlo[0]) / g.nx[0];
    for (int d = 0; d < 3; ++d) c->m[d] = 2 * g.nx[d];
    c->MT = (long long)c->m[0] * c->m[1] * c->m[2];
    double2 *h_k = (double2 *)malloc(sizeof(double2) * c->MT);
    if (!h_k) return vp_fail(c, VP_ENOMEM, "host allocation failed");
    const double self = cube_inv_r_mean() / h;
    const double pref = -(g.coupling / (4.0 * M_PI)) * h * h * h;
    for (int a = 0; a < c->m[0]; ++a)
        for (int b = 0; b < c->m[1]; ++b)
            for (int cc = 0; cc < c->m[2]; ++cc) {
                const int ia = a < c->m[0] - a ? a : c->m[0] - a;
                const int ib = b < c->m[1] - b ? b : c->m[1] - b;
                const int ic = cc < c->m[2] - cc ? cc : c->m[2] - cc;
                const double r = h * sqrt((double)ia * ia + (double)ib * ib + (double)ic * ic);
                const double inv = (ia == 0 && ib == 0 && ic == 0) ? self : 1.0 / r;
                h_k[((long long)a * c->m[1] + b) * c->m[2] + cc] = make_double2(pref * inv, 0.0);
            }
    VP_CUDA_TRY(c, cudaMalloc(&c->d_ghat, sizeof(double2) * c->MT));
    VP_CUDA_TRY(c, cudaMalloc(&c->d_fft, sizeof(double2) * c->MT));
    VP_CUDA_TRY(c, cudaMemcpy(c->d_ghat, h_k, sizeof(double2) * c->MT, cudaMemcpyHostToDevice));
    free(h_k);
    int rc = fft_all_axes(c, c->d_ghat, c->m, 3, -1);
    if (rc) return rc;
    VP_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return VP_OK;
}

// ---- launchers ---------------------------------------------------------------

int vp_launch_moment(vp_ctx *c, double *rho) {
    double dV = 1.0;
    for (int d = 0; d < c->g.dv; ++d) dV *= (c->g.vhi[d] - c->g.vlo[d]) / c->g.nv[d];
    if (c->g.precision == VP_F32)
        k_moment<float><<<(unsigned)c->NX, kBlock, 0, c->stream>>>(static_cast<const float *>(c->f),
                                                                   c->NV, dV, rho);
    else
        k_moment<double><<<(unsigned)c->NX, kBlock, 0, c->stream>>>(static_cast<const double *>(c->f),
                                                                    c->NV, dV, rho);
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

int vp_launch_poisson(vp_ctx *c, const double *rho, double *phi, double *acc) {
    const vp_grid &g = c->g;
    const int D = g.dx;
    const int3 nbox = make_int3(g.nx[0], D > 1 ? g.nx[1] : 1, D > 2 ? g.nx[2] : 1);
    const int3 m = make_int3(c->m[0], c->m[1], c->m[2]);
    k_load_rho<<<nblk(c->MT, kBlock), kBlock, 0, c->stream>>>(c->d_fft, rho, g.rho_bg, c->MT, nbox, m, D);
    c->launches++;
    int rc = fft_all_axes(c, c->d_fft, c->m, D, -1);
    if (rc) return rc;
    double scale = 1.0;
    if (g.poisson == VP_POIS_PERIODIC) {
        k_mul_real<<<nblk(c->MT, kBlock), kBlock, 0, c->stream>>>(c->d_fft, c->d_green, c->MT);
    } else {
        k_mul_cplx<<<nblk(c->MT, kBlock), kBlock, 0, c->stream>>>(c->d_fft, c->d_ghat, c->MT,
                                                                   1.0 / (double)c->MT);
    }
    c->launches++;
    rc = fft_all_axes(c, c->d_fft, c->m, D, +1);
    if (rc) return rc;
    double3 h = make_double3((g.xhi[0] - g.xlo[0]) / g.nx[0],
                             D > 1 ? (g.xhi[1] - g.xlo[1]) / g.nx[1] : 1.0,
                             D > 2 ? (g.xhi[2] - g.xlo[2]) / g.nx[2] : 1.0);
    k_force<<<nblk(c->NX, kBlock), kBlock, 0, c->stream>>>(c->d_fft, scale, phi, acc, c->NX, nbox, m, D,
                                                           h, fda_coeffs(g.pois_order),
                                                           g.pois_order / 2);
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

int vp_launch_diag(vp_ctx *c, int mode, double *out_dev) {
    const vp_grid &g = c->g;
    int rc = vp_launch_moment(c, c->d_rho);
    if (rc) return rc;
    rc = vp_launch_poisson(c, c->d_rho, c->d_phi, c->d_acc);
    if (rc) return rc;
    VGrid vg{};
    vg.dv = g.dv;
    for (int d = 0; d < g.dv; ++d) {
        vg.lo[d] = g.vlo[d];
        vg.h[d] = (g.vhi[d] - g.vlo[d]) / g.nv[d];
        vg.n[d] = g.nv[d];
    }
    if (g.precision == VP_F32)
        k_diag_part<float><<<(unsigned)c->NX, kBlock, 0, c->stream>>>(static_cast<const float *>(c->f),
                                                                      c->NV, vg, c->d_part, c->d_flag);
    else
        k_diag_part<double><<<(unsigned)c->NX, kBlock, 0, c->stream>>>(
            static_cast<const double *>(c->f), c->NV, vg, c->d_part, c->d_flag);
    c->launches++;
    double dX = 1.0, dV = 1.0;
    for (int d = 0; d < g.dx; ++d) dX *= (g.xhi[d] - g.xlo[d]) / g.nx[d];
    for (int d = 0; d < g.dv; ++d) dV *= (g.vhi[d] - g.vlo[d]) / g.nv[d];
    long long rest = c->NX / g.nx[0];
    k_diag_final<<<1, kBlock, 0, c->stream>>>(c->d_part, c->d_rho, c->d_phi, c->d_acc, c->NX, g.dx,
                                              g.nx[0], rest, mode, g.rho_bg, dX, dV, out_dev);
    c->launches++;
    VP_CUDA_TRY(c, cudaGetLastError());
    return VP_OK;
}

int vp_launch_init_ptr(void *f, const vp_grid &g, int kind, const double *p, int np, cudaStream_t st) {
    IcArgs a{};
    a.kind = kind;
    a.dims = g.dx;
    a.NV = 1;
    long long NX = 1;
    for (int d = 0; d < g.dx; ++d) {
        a.nx[d] = g.nx[d];
        a.nv[d] = g.nv[d];
        a.xlo[d] = g.xlo[d];
        a.vlo[d] = g.vlo[d];
        a.hx[d] = (g.xhi[d] - g.xlo[d]) / g.nx[d];
        a.hv[d] = (g.vhi[d] - g.vlo[d]) / g.nv[d];
        a.xc[d] = 0.5 * (g.xlo[d] + g.xhi[d]);
        a.NV *= g.nv[d];
        NX *= g.nx[d];
    }
    for (int i = 0; i < np && i < 8; ++i) a.p[i] = p[i];
    const long long ncell = NX * a.NV;
    if (g.precision == VP_F32)
        k_init<float><<<nblk(ncell, kBlock), kBlock, 0, st>>>(static_cast<float *>(f), ncell, a);
    else
        k_init<double><<<nblk(ncell, kBlock), kBlock, 0, st>>>(static_cast<double *>(f), ncell, a);
    return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ECUDA;
}

int vp_launch_init(vp_ctx *c, int kind, const double *p, int np) {
    const int rc = vp_launch_init_ptr(c->f, c->g, kind, p, np, c->stream);
    c->launches++;
    if (rc) return vp_fail(c, rc, "initial condition launch failed");
    return VP_OK;
}

// ---- allocation-free periodic Poisson solve ------------------------------------
// vp_poisson_periodic_noalloc: the periodic solve of vp_poisson_solve for
// callers that must not allocate device memory.  Its complex FFT work array is
// this file-scope device array (VP_NOALLOC_MAX_POINTS complex doubles, 4 MiB,
// held by every device that loads the library until the process exits); the
// Green function is evaluated on the fly instead of read from a table.  The
// array is shared by all calls: calls that overlap on the GPU race on it.

static __device__ __align__(256) double2 g_noalloc_fft[VP_NOALLOC_MAX_POINTS];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
double2 *g_noalloc_dev_ptr[kNoallocMaxDevices];

__device__ double noalloc_stencil_eig(int order, double theta) {
    // eigenvalue of the symmetric discrete Laplacian stencil (b_0..b_3)/den
    // (Eqs. C1, C5, C6) times h^2: -(4/den) sum_m b_m sin^2(m theta / 2)
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
    const double s1 = sin(0.5 * theta), s2 = sin(theta), s3 = sin(1.5 * theta);
    return -4.0 * (b1 * s1 * s1 + b2 * s2 * s2 + b3 * s3 * s3) / den;
}

// multiply every Fourier mode by S / lambda(k) / NX (k = 0 -> 0)
__global__ void k_green_onfly(double2 *__restrict__ a, long long NX, int dims, int3 n, double3 h,
                              int order, double S) {
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= NX) return;
    const int nn[3] = {n.x, n.y, n.z};
    const double hh[3] = {h.x, h.y, h.z};
    long long r = x;
    bool allzero = true;
    double lam = 0.0;
    for (int d = dims - 1; d >= 0; --d) {
        const long long k = r % nn[d];
        r /= nn[d];
        if (k) allzero = false;
        lam += noalloc_stencil_eig(order, 2.0 * 3.141592653589793238462643383279502884 * (double)k / (double)nn[d]) /
               (hh[d] * hh[d]);
    }
    const double sc = allzero ? 0.0 : S / lam / (double)NX;
    a[x] = make_double2(a[x].x * sc, a[x].y * sc);
}

}  // namespace

extern "C" int vp_poisson_periodic_noalloc(const vp_grid *g, void *cuda_stream, const double *rho_dev,
                                           double *phi_dev, double *accel_dev) {
    if (!g || !rho_dev || !accel_dev) return VP_EINVAL;
    if (g->dx < 1 || g->dx > 3 || g->poisson != VP_POIS_PERIODIC) return VP_EINVAL;
    if (g->pois_order != 2 && g->pois_order != 4 && g->pois_order != 6) return VP_EINVAL;
    if (!std::isfinite(g->coupling) || !std::isfinite(g->rho_bg)) return VP_EINVAL;
    const int D = g->dx;
    long long NX = 1;
    for (int d = 0; d < D; ++d) {
        if (g->nx[d] < 1 || g->nx[d] > 4096) return VP_EINVAL;
        if (!(g->xhi[d] > g->xlo[d]) || !std::isfinite(g->xhi[d]) || !std::isfinite(g->xlo[d]))
            return VP_EINVAL;
        NX *= g->nx[d];
    }
    if (NX > VP_NOALLOC_MAX_POINTS) return VP_EINVAL;
    // an error left by earlier work would be indistinguishable from ours at
    // the end: report it (and leave it pending) before launching anything
    if (cudaPeekAtLastError() != cudaSuccess) return VP_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return VP_ECUDA;
    double2 *buf = nullptr;
    {
        // once per device, with that device current: the device address of the
        // static array (its name in host code is only a host-side stand-in)
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_dev_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_fft) != cudaSuccess || !p) return VP_ECUDA;
            if (cudaFuncSetAttribute(k_fft_axis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     2 * 4096 * (int)sizeof(double2)) != cudaSuccess)
                return VP_ECUDA;
            g_noalloc_dev_ptr[dev] = static_cast<double2 *>(p);
        }
        buf = g_noalloc_dev_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int3 nb = make_int3(g->nx[0], D > 1 ? g->nx[1] : 1, D > 2 ? g->nx[2] : 1);
    const int m[3] = {nb.x, nb.y, nb.z};
    // every element of the work array that is read is written first: no clearing needed
    k_load_rho<<<nblk(NX, kBlock), kBlock, 0, st>>>(buf, rho_dev, g->rho_bg, NX, nb, nb, D);
    for (int pass = 0; pass < 2; ++pass) {
        for (int a = 0; a < D; ++a) {
            long long inner = 1;
            for (int d = a + 1; d < D; ++d) inner *= m[d];
            const size_t smem = 2 * (size_t)m[a] * sizeof(double2);
            const int th = m[a] / 2 < 32 ? 32 : (m[a] / 2 > 256 ? 256 : m[a] / 2);
            k_fft_axis<<<(unsigned)(NX / m[a]), th, smem, st>>>(buf, inner, m[a], pass == 0 ? -1 : +1);
        }
        if (pass == 0) {
            const double3 h = make_double3((g->xhi[0] - g->xlo[0]) / g->nx[0],
                                           D > 1 ? (g->xhi[1] - g->xlo[1]) / g->nx[1] : 1.0,
                                           D > 2 ? (g->xhi[2] - g->xlo[2]) / g->nx[2] : 1.0);
            k_green_onfly<<<nblk(NX, kBlock), kBlock, 0, st>>>(buf, NX, D, nb, h, g->pois_order, g->coupling);
        }
    }
    const double3 h = make_double3((g->xhi[0] - g->xlo[0]) / g->nx[0],
                                   D > 1 ? (g->xhi[1] - g->xlo[1]) / g->nx[1] : 1.0,
                                   D > 2 ? (g->xhi[2] - g->xlo[2]) / g->nx[2] : 1.0);
    k_force<<<nblk(NX, kBlock), kBlock, 0, st>>>(buf, 1.0, phi_dev, accel_dev, NX, nb, nb, D, h,
                                                 fda_coeffs(g->pois_order), g->pois_order / 2);
    return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ECUDA;
}
