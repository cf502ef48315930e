// vp_sweep_core.cuh -- per-interface arithmetic of the SL-MPP5/7 sweep and
// the line walker shared by every sweep kernel (strided, contiguous, TMA,
// ensemble).
#pragma once

#include "vp_internal.cuh"

namespace vp_core {

// ---- limiter arithmetic (Appendix A and Sec. 2.1.1) -------------------------

// Every product that meets a sum is written either as fma() or as a
// round-to-nearest multiply (mul_rn), never left to contraction: the walk
// step is compiled in several instances (unrolled and remainder loops, the
// first interface of a segment), and a contraction the compiler takes in one
// instance but not another would make a cell's last bit depend on where the
// tile and segment boundaries fall, i.e. on the autotuner's choice.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// ---- two lines at once ---------------------------------------------------------
//
// P2 holds one value of each of two lines that a thread walks in lockstep.
// Additions, multiplications and fused multiply-adds are the packed FP32
// pair instructions of sm_100+ (one issue slot for both lines, each half
// rounded exactly as the scalar instruction would round it); min, max and
// comparisons are per half.  Every line therefore gets bit for bit the
// result of the one-line walk, whichever of the two walks runs it.
// the scalar overloads stay visible next to the pair overloads below
using ::fma;
using ::fmax;
using ::fmin;

struct P2 {
    float2 v;
    P2() = default;
    __device__ __forceinline__ explicit P2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ P2(float2 x) : v(x) {}
};
__device__ __forceinline__ P2 operator+(P2 a, P2 b) { return P2(__fadd2_rn(a.v, b.v)); }
// a - b as a + (-1) b: the product is exact, so this rounds as the subtraction
__device__ __forceinline__ P2 operator-(P2 a, P2 b) { return P2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ P2 operator-(P2 a) { return P2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ P2 operator*(P2 a, P2 b) { return P2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ P2 fma(P2 a, P2 b, P2 c) { return P2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ P2 fmin(P2 a, P2 b) { return P2(make_float2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y))); }
__device__ __forceinline__ P2 fmax(P2 a, P2 b) { return P2(make_float2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y))); }
// both lines equal (the flat-stencil test asks it of both lines of a pair)
__device__ __forceinline__ bool operator==(P2 a, P2 b) { return a.v.x == b.v.x && a.v.y == b.v.y; }

// shift decompositions of a pair of lines walked together (equal n and sigma)
struct LineShiftP2 {
    P2 w[7];
    P2 nu;
    int n;
    int sigma;
};
__device__ __forceinline__ LineShiftP2 pair_shift(const LineShift<float> &a, const LineShift<float> &b) {
    LineShiftP2 s;
#pragma unroll
    for (int k = 0; k < 7; ++k) s.w[k] = P2(make_float2(a.w[k], b.w[k]));
    s.nu = P2(make_float2(a.nu, b.nu));
    s.n = a.n;
    s.sigma = a.sigma;
    return s;
}

// whether the walker tests for warp-wide flat stencils (and then skips the
// interpolant and the bounds); the result is the same either way
template <typename T>
struct FlatSkip {
    static constexpr bool on = true;
};
template <>
struct FlatSkip<P2> {
    static constexpr bool on = true;
};

// 4/3 in the arithmetic's precision
template <typename T>
__device__ __forceinline__ T c43() { return T(4) / T(3); }
template <>
__device__ __forceinline__ P2 c43<P2>() { return P2(4.0f / 3.0f); }

// minmod of four: min if all > 0, max if all < 0, else 0 (= max(min,0) + min(max,0))
template <typename T>
__device__ __forceinline__ T mm4(T a, T b, T c, T d) {
    const T mn = fmin(fmin(a, b), fmin(c, d));
    const T mx = fmax(fmax(a, b), fmax(c, d));
    return fmax(mn, T(0)) + fmin(mx, T(0));
}

// min / max of three (the three-input PTX form for FP32; measured here at the
// throughput of two two-input operations)
__device__ __forceinline__ float min3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float max3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ double min3(double a, double b, double c) { return fmin(fmin(a, b), c); }
__device__ __forceinline__ double max3(double a, double b, double c) { return fmax(fmax(a, b), c); }
__device__ __forceinline__ P2 min3(P2 a, P2 b, P2 c) {
    return P2(make_float2(min3(a.v.x, b.v.x, c.v.x), min3(a.v.y, b.v.y, c.v.y)));
}
__device__ __forceinline__ P2 max3(P2 a, P2 b, P2 c) {
    return P2(make_float2(max3(a.v.x, b.v.x, c.v.x), max3(a.v.y, b.v.y, c.v.y)));
}

// curvature d_j = u_{j-1} - 2 u_j + u_{j+1} (App. A)
template <typename T>
__device__ __forceinline__ T curv(T um, T u, T up) {
    return fma(T(-2), u, um + up);
}

// d^{M4} between cells with curvatures x and y (App. A):
// minmod(4x - y, 4y - x, x, y).  With m = min(x, y) and M = max(x, y) the
// least of the four is min(m, 4m - M) and the greatest max(M, 4M - m); the
// minmod is the least if it is > 0, the greatest if it is < 0, else 0: the
// clamp of 0 into [least, greatest].
template <typename T>
__device__ __forceinline__ T dm4(T x, T y) {
    const T m = fmin(x, y), M = fmax(x, y);
    const T mn = fmin(m, fma(T(4), m, -M));
    const T mx = fmax(M, fma(T(4), M, -m));
    return fmin(fmax(T(0), mn), mx);
}

// The MP constraint as one clamp.  Steps 4-7 give phi_MP = median(phi, f_min,
// f_max); step 3 keeps phi when it lies strictly between u0 and f^MP, and
// that interval lies inside [f_min, f_max] (f_min <= u0; when the minmod of
// step 2 is positive f_max >= min(u1, f_UL) = f^MP, and the mirror case), so
// there the clamp returns phi as well.  Hence the constraint equals the clamp
// of phi into [f_min, f_max] for every phi.  m4m / m4p are d^{M4} at the
// upwind / downwind face of the upwind cell u0.
template <typename T>
__device__ __forceinline__ void mp_lohi_carried(T um1, T u0, T u1, T alpha, T m4m, T m4p, T &lo, T &hi) {
    const T back = u0 - um1;
    const T ful = fma(alpha, back, u0);
    const T fmd = fma(T(0.5), u0 + u1, T(-0.5) * m4p);
    const T flc = fma(c43<T>(), m4m, fma(T(0.5), back, u0));
    lo = fmax(min3(u0, u1, fmd), min3(u0, ful, flc));
    hi = fmin(max3(u0, u1, fmd), max3(u0, ful, flc));
}
template <typename T>
__device__ __forceinline__ T mp_clamp(T phi, T um1, T u0, T u1, T alpha, T m4m, T m4p) {
    T lo, hi;
    mp_lohi_carried(um1, u0, u1, alpha, m4m, m4p, lo, hi);
    return fmin(fmax(phi, lo), hi);
}

// Steps 4-6 of the MP constraint: the bounds [f_min, f_max].  Both intervals
// of step 6 contain u0, so f_min <= u0 <= f_max exactly.
template <typename T>
__device__ __forceinline__ void mp_lohi(T um2, T um1, T u0, T u1, T u2, T alpha, T &lo, T &hi) {
    const T back = u0 - um1;
    const T dm = um2 + u0 - T(2) * um1;  // curvature at the upwind neighbour
    const T dc = um1 + u1 - T(2) * u0;   // at the upwind cell
    const T dp = u0 + u2 - T(2) * u1;    // at the downwind cell
    const T m4p = mm4(T(4) * dc - dp, T(4) * dp - dc, dc, dp);
    const T m4m = mm4(T(4) * dm - dc, T(4) * dc - dm, dm, dc);
    const T ful = fma(alpha, back, u0);
    const T fmd = fma(T(0.5), u0 + u1, T(-0.5) * m4p);
    const T flc = fma(T(4) / T(3), m4m, fma(T(0.5), back, u0));
    lo = fmax(fmin(fmin(u0, u1), fmd), fmin(fmin(u0, ful), flc));
    hi = fmin(fmax(fmax(u0, u1), fmd), fmax(fmax(u0, ful), flc));
}

// Steps 4-7 (taken only when step 3 rejects phi): the median of step 7 is
// the clamp into [f_min, f_max].
template <typename T>
__device__ __forceinline__ T mp_bounds(T phi, T um2, T um1, T u0, T u1, T u2, T alpha) {
    T lo, hi;
    mp_lohi(um2, um1, u0, u1, u2, alpha, lo, hi);
    return fmin(fmax(phi, lo), hi);
}

// MP constraint of phi at the interface between u0 (upwind) and u1.
// Step 3 accepts phi iff it lies strictly between u0 and f* = u0 + minmod(p, q),
// p = u1 - u0, q = alpha (u0 - u_{-1}); with a = phi - u0 that is: a strictly
// between 0 and p and strictly between 0 and q, i.e. (p - a) a > 0 and
// (q - a) a > 0 -- products on the FMA pipe instead of min/max chains.  A phi
// this test rejects goes to steps 4-7 directly: the interval [u0, f*] lies
// inside [f_min, f_max] (f_min <= u0; f_max >= min(u1, f_UL) >= f* when the
// minmod is positive, and the mirror case), so a phi that step 3 would have
// accepted but whose product underflowed comes back unchanged from the clamp.
template <typename T>
__device__ __forceinline__ T mp_limit(T phi, T um2, T um1, T u0, T u1, T u2, T alpha) {
    const T a = phi - u0;
    const T p = u1 - u0;
    const T q = mul_rn(alpha, u0 - um1);
    if ((p - a) * a > T(0) && (q - a) * a > T(0)) return phi;
    return mp_bounds(phi, um2, um1, u0, u1, u2, alpha);
}

// Half of a cell, rounded towards minus infinity: the most mass one interface
// may take out of a non-negative cell so that two of them leave it >= 0.
__device__ __forceinline__ float half_rd(float u) { return __fmul_rd(u, 0.5f); }
__device__ __forceinline__ double half_rd(double u) { return __dmul_rd(u, 0.5); }
__device__ __forceinline__ P2 half_rd(P2 u) { return P2(__fmul2_rd(u.v, make_float2(0.5f, 0.5f))); }
__device__ __forceinline__ P2 mul_rn(P2 a, P2 b) { return P2(__fmul2_rn(a.v, b.v)); }

// PP limiter (Sec. 2.1.1, Eqs. 15-23) on the mass M = nu Phi that an interface
// carries from its upwind cell u0 into u1.  For u0, u1 >= 0 and 0 < nu <= 1/2
// the theta blend returns Phi unless one half of the Euler update goes
// negative; then U+ < 0 gives theta+ (Phi - u0) = (1 - 2 nu) u0 / (2 nu), i.e.
// exactly the flux u0 / (2 nu) that empties the upwind half, and U- < 0 the
// flux -u1 / (2 nu) (both cannot bind at once).  So the limiter is the clamp
// of M into [-u1 / 2, u0 / 2], with h0, h1 the rounded-down halves of u0, u1.
// A cell then loses at most h through each of its two interfaces, and
// (u - M_out) + M_in >= 0 holds after rounding, subnormals included.
template <typename T>
__device__ __forceinline__ T pp_clamp(T M, T h0, T h1) {
    return fmin(fmax(M, -h1), h0);
}

// The PP limiter in its theta form (Eqs. 15-23), as the mass nu Phi^, for an
// interface next to a negative cell, where the clamp above is not the theta
// blend (the unsplit step can leave cells below zero).  A binding theta is
// scaled by (1 - 8 eps) and clamped to [0, 1]; a non-positive denominator
// gives theta = 0, the upwind flux.  Kept out of line so that the rare call
// stays a branch rather than work predicated into every interface.
template <typename T>
__device__ __noinline__ T pp_theta_mass(T phibar, T u0, T u1, T nu) {
    const T tn = T(2) * nu;
    const T up = u0 - tn * phibar, up_up = u0 - tn * u0;
    const T um = u1 + tn * phibar, um_up = u1 + tn * u0;
    T thp = T(1), thm = T(1);
    bool binds = false;
    if (up < T(0)) {
        const T den = up_up - up;
        thp = den > T(0) ? up_up / den : T(0);
        binds = true;
    }
    if (um < T(0)) {
        const T den = um_up - um;
        thm = den > T(0) ? um_up / den : T(0);
        binds = true;
    }
    T th = fmin(thp, thm);
    if (binds) th *= T(1) - T(8) * (sizeof(T) == 4 ? T(5.9604644775390625e-8) : T(1.1102230246251565e-16));
    th = fmin(fmax(th, T(0)), T(1));
    return nu * (th * phibar + (T(1) - th) * u0);
}

// Interface mass on the upwind-ordered stencil (u0 = upwind cell): the CSL
// flux, the MP constraint, times nu, then the PP limiter.  FULL: MP and PP
// both on, so the runtime switches drop out of the loop.
template <typename T, int ORDER, bool FULL>
__device__ __forceinline__ T flux(const LineShift<T> &sh, T um3, T um2, T um1, T u0, T u1, T u2, T u3,
                                  T alpha, int mp, int pp) {
    T phi;
    if ((FULL || mp) && um1 == u0 && u0 == u1) {
        // flat around the interface: every MP bound collapses onto u0, whatever
        // the interpolated value (App. A steps 2-7), so skip computing it
        phi = u0;
    } else {
        if (ORDER == 7) {
            phi = sh.w[0] * um3;
            phi = fma(sh.w[1], um2, phi);
        } else {
            phi = sh.w[1] * um2;
        }
        phi = fma(sh.w[2], um1, phi);
        phi = fma(sh.w[3], u0, phi);
        phi = fma(sh.w[4], u1, phi);
        phi = fma(sh.w[5], u2, phi);
        if (ORDER == 7) phi = fma(sh.w[6], u3, phi);
        if (FULL || mp) phi = mp_limit(phi, um2, um1, u0, u1, u2, alpha);
    }
    T M = mul_rn(sh.nu, phi);
    if (FULL || pp) M = pp_clamp(M, half_rd(u0), half_rd(u1));
    return M;
}

// The CSL interpolant and, for the line walker, the MP constraint as a clamp
// (no branch) with d^{M4} at both faces of u0 passed in.
template <typename T, int ORDER, bool FULL, typename SH>
__device__ __forceinline__ T flux_walk(const SH &sh, T um3, T um2, T um1, T u0, T u1, T u2, T u3,
                                       T alpha, int mp, T m4m, T m4p) {
    T phi;
    if (ORDER == 7) {
        phi = sh.w[0] * um3;
        phi = fma(sh.w[1], um2, phi);
    } else {
        phi = sh.w[1] * um2;
    }
    phi = fma(sh.w[2], um1, phi);
    phi = fma(sh.w[3], u0, phi);
    phi = fma(sh.w[4], u1, phi);
    phi = fma(sh.w[5], u2, phi);
    if (ORDER == 7) phi = fma(sh.w[6], u3, phi);
    if (FULL || mp) phi = mp_clamp(phi, um1, u0, u1, alpha, m4m, m4p);
    return phi;
}

// ---- line walker ---------------------------------------------------------------
//
// Advance cells [r0, r1) of one line staged in shared memory; row r of the
// line is at sm0[r * ss].  Zero-inflow lines have GP >= 1 zero rows on each
// side (rows -GP..-1 and L..L+GP-1); periodic lines wrap.
// The walk goes upwind -> downwind so that each interface mass is computed
// once; the 8-cell stencil window rotates through registers (unrolled by 8).
// The curvature of the upwind cell, d^{M4} at its upwind face and the
// rounded-down half of the cell carry over from one interface to the next, so
// each interface adds one curvature, one d^{M4} and one half.  Where every
// active lane of a warp sits on a flat stencil (u_{-1} = u_0 = u_1) the
// constrained flux is u_0 exactly (all MP bounds collapse onto u_0, d^{M4} at
// the downwind face is 0) and the warp skips the interpolant and the bounds.
// The update is the flux form of Eq. 49 in masses, f' = (u - M_out) + M_in.
// store(i, v) writes the new value of cell i.  NEG: interfaces next to a
// negative cell take the PP limiter's theta form (pp_theta_mass) instead of
// the clamp (scalar T only).  FLAT = false leaves the flat-stencil vote out
// (the same results; for data that is nowhere flat the vote only costs).

template <typename T, int ORDER, bool PERIODIC, bool FULL, int GP, bool NEG = false, bool FLAT = true,
          typename Store, typename SH>
__device__ __forceinline__ void walk(const T *__restrict__ sm0, int ss, int L, const SH &sh,
                                     int r0, int r1, T alpha, int mp, int pp, Store store) {
    if (r0 >= r1) return;
    const int sg = sh.sigma;
    const T nu = sh.nu;
    int i = sg > 0 ? r0 : r1 - 1;
    const int cnt = r1 - r0;
    // Source row of load k (k = 0, 1, ...) is p0 + k sg; load k feeds step
    // k - 8 of the walk.
    int p0;
    if (PERIODIC) {
        const int n = sh.n % L;
        p0 = (i - n - 4 * sg) % L;
        if (p0 < 0) p0 += L;
    } else {
        p0 = i - sh.n - 4 * sg;
    }
    // Zero-inflow lines read rows outside the staged extent [-GP, L + GP) as
    // the zero row at its edge; periodic lines wrap.
    auto row = [&](int q) -> const T * {
        if (PERIODIC) {
            q %= L;
            if (q < 0) q += L;
        } else {
            q = min(max(q, -GP), L + GP - 1);
        }
        return sm0 + q * ss;
    };
    const T *src = sm0;
    int inc = 0;
    T w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = *row(p0 + k * sg);
    // incoming mass of the first cell: upwind cell i - sg, stencil w[0..6]
    T dc = T(0), m4m = T(0);  // curvature at the next upwind cell, d^{M4} at its upwind face
    T m4p = T(0);
    if (FULL || mp) {
        const T dm = curv(w[1], w[2], w[3]);
        dc = curv(w[2], w[3], w[4]);
        const T dp = curv(w[3], w[4], w[5]);
        m4m = dm4(dm, dc);
        m4p = dm4(dc, dp);
    }
    // hc: rounded-down half of the cell the walk is on (the upwind cell of its
    // outgoing interface)
    T hc = (FULL || pp) ? half_rd(w[4]) : T(0);
    const T phi0 = flux_walk<T, ORDER, FULL>(sh, w[0], w[1], w[2], w[3], w[4], w[5], w[6], alpha, mp, m4m, m4p);
    T fin = mul_rn(nu, phi0);
    if (FULL || pp) {
        if constexpr (NEG) {
            if (w[3] < T(0) || w[4] < T(0))
                fin = pp_theta_mass(phi0, w[3], w[4], nu);
            else
                fin = pp_clamp(fin, half_rd(w[3]), hc);
        } else {
            fin = pp_clamp(fin, half_rd(w[3]), hc);
        }
    }
    if (FULL || mp) {
        dc = curv(w[3], w[4], w[5]);
        m4m = m4p;
    }

    // one cell with the window rotated by K (u_k at w[(K + 4 + k) & 7]): the
    // outgoing mass, then f' = (u - M_out) + M_in; the next value enters from
    // *src, which then moves by inc
#define VP_WALK_STEP(K)                                                                           \
    {                                                                                             \
        const T u0_ = w[(K + 4) & 7], u1_ = w[(K + 5) & 7];                                       \
        T phi;                                                                                    \
        if (FULL || mp) {                                                                         \
            const T dp = curv(u0_, u1_, w[(K + 6) & 7]);                                          \
            if (FLAT && FlatSkip<T>::on &&                                                        \
                __all_sync(__activemask(), w[(K + 3) & 7] == u0_ && u0_ == u1_)) {                \
                phi = u0_;                                                                        \
                m4m = T(0);                                                                       \
            } else {                                                                              \
                m4p = dm4(dc, dp);                                                                \
                phi = flux_walk<T, ORDER, FULL>(sh, w[(K + 1) & 7], w[(K + 2) & 7],               \
                                                w[(K + 3) & 7], u0_, u1_, w[(K + 6) & 7],         \
                                                w[(K + 7) & 7], alpha, mp, m4m, m4p);             \
                m4m = m4p;                                                                        \
            }                                                                                     \
            dc = dp;                                                                              \
        } else {                                                                                  \
            phi = flux_walk<T, ORDER, FULL>(sh, w[(K + 1) & 7], w[(K + 2) & 7], w[(K + 3) & 7],   \
                                            u0_, u1_, w[(K + 6) & 7], w[(K + 7) & 7], alpha, mp,  \
                                            T(0), T(0));                                          \
        }                                                                                         \
        T fout = mul_rn(nu, phi);                                                                 \
        if (FULL || pp) {                                                                         \
            const T hn = half_rd(u1_);                                                            \
            if constexpr (NEG) {                                                                  \
                if (u0_ < T(0) || u1_ < T(0))                                                     \
                    fout = pp_theta_mass(phi, u0_, u1_, nu);                                      \
                else                                                                              \
                    fout = pp_clamp(fout, hc, hn);                                                \
            } else {                                                                              \
                fout = pp_clamp(fout, hc, hn);                                                    \
            }                                                                                     \
            hc = hn;                                                                              \
        }                                                                                         \
        store(i, (u0_ - fout) + fin);                                                             \
        fin = fout;                                                                               \
        i += sg;                                                                                  \
        w[K & 7] = *src;                                                                          \
        src += inc;                                                                               \
    }

    // The walk runs in chunks over which the load pointer moves uniformly:
    // inside the staged extent it steps one row per cell; beyond it, it stays
    // on the edge row (zero).  A zero-inflow line whose shift keeps every load
    // inside the extent (|n| <= GP - 4) is a single chunk.
    int t = 0;
    while (t < cnt) {
        const int q = p0 + (t + 8) * sg;  // row of the next load
        int end;
        if (PERIODIC) {
            const int qq = ((q % L) + L) % L;
            src = sm0 + qq * ss;
            inc = sg * ss;
            end = t + (sg > 0 ? L - qq : qq + 1);  // loads before the wrap
        } else if (q < -GP || q > L + GP - 1) {
            src = row(q);
            inc = 0;
            const int back = sg > 0 ? -GP - q : q - (L + GP - 1);  // loads until the extent
            end = back > 0 ? t + back : cnt;
        } else {
            src = sm0 + q * ss;
            inc = sg * ss;
            end = t + (sg > 0 ? L + GP - q : q + GP + 1);  // loads through the far edge
        }
        if (end > cnt) end = cnt;
#pragma unroll 1
        for (; t + 8 <= end; t += 8) {
            VP_WALK_STEP(0)
            VP_WALK_STEP(1)
            VP_WALK_STEP(2)
            VP_WALK_STEP(3)
            VP_WALK_STEP(4)
            VP_WALK_STEP(5)
            VP_WALK_STEP(6)
            VP_WALK_STEP(7)
        }
#pragma unroll 1
        for (; t < end; ++t) {
            VP_WALK_STEP(0)
            // restore the canonical order (u_-4 in w[0])
            const T w0 = w[0];
#pragma unroll
            for (int kk = 0; kk < 7; ++kk) w[kk] = w[kk + 1];
            w[7] = w0;
        }
    }
#undef VP_WALK_STEP
}

// Shift decomposition of one line, in double precision so that the integer
// part is exact (reading R2): s = c dt / h, n = nearest integer (halves away
// from zero), zeta = s - n, nu = |zeta|, sigma = sign(zeta); the CSL weights
// are the weight polynomials evaluated at nu.
template <typename T>
__device__ __forceinline__ LineShift<T> make_shift(double speed, double dt, double h, const WPoly &wp) {
    const double s = __ddiv_rn(__dmul_rn(speed, dt), h);
    double n = round(s);
    const double z = __dadd_rn(s, -n);
    const double nu = fabs(z);
    LineShift<T> sh;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        double acc = 0.0;
        for (int j = wp.nterm - 1; j >= 0; --j) acc = fma(acc, nu, wp.c[j][k]);
        sh.w[k] = (T)acc;
    }
    // shifts beyond a billion cells only happen with absurd inputs; clamp so
    // the integer conversion stays defined (a zero-inflow line is empty anyway)
    n = fmin(fmax(n, -1.0e9), 1.0e9);
    sh.nu = (T)nu;
    sh.n = (int)n;
    sh.sigma = z < 0.0 ? -1 : 1;
    return sh;
}

// velocity of cell j of an axis: lo + (j + 1/2) dv, rounded step by step
__device__ __forceinline__ double cell_centre(double lo, double dvel, int j) {
    return __dadd_rn(lo, __dmul_rn((double)j + 0.5, dvel));
}

__device__ __forceinline__ unsigned line_class(const SweepGeo &g, unsigned o, unsigned c) {
    return g.cls_from_inner ? fmod_u(fdiv(c, g.fd_cdiv), g.fd_cmod) : fdiv(o, g.fd_cdiv);
}

}  // namespace vp_core
