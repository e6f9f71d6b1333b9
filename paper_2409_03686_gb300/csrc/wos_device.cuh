// wos_device.cuh -- device-side building blocks of the walk-on-ellipsoids
// (WoE) operator build: Philox4x32-10, the uniform-direction maps, the
// distance to dD and the boundary-element map pi (paper App. A).
//
// The functions are __host__ __device__ so the host-side point check runs the
// very code the walk kernel runs.
//
// Paper: Cimpean, Grecu & Marin, arXiv:2409.03686.
//   Sec. 4.2, Eq. (wos chain):  X_{n+1} = X_n + dist(X_n, dD) K^{1/2} U_n,
//       lambda_max(K) = 1;  Eq. (N epsilon x): stop when dist <= eps.
//   Sec. 5.1, Rem. (wos algorithm)(ii): any Lipschitz lower bound of the
//       distance may replace it; the distances here are exact for points of D.
//   App. A, Ex. A.3 / Eq. (voronoi weights extended): the element of a
//       stopped point is the cell holding its projection pi(x), ties to the
//       lowest index; Ex. A.2: extrinsic Voronoi cells (nearest site).
// Philox4x32-10: Salmon, Moraes, Dror & Shaw, SC'11.
#pragma once

#include <cstdint>
#include <cmath>

#ifdef __CUDACC__
#define WOS_HD __host__ __device__ __forceinline__
#else
#define WOS_HD inline
#endif

namespace wos {

constexpr int kMaxVerts = 64;
constexpr int kMaxHoles = 16;
constexpr int kMaxPlanes = 8;  // faces of a mapped polytope

enum OuterKind : int32_t { kSphere = 1, kBox = 2, kPolygon = 3 };

// ---------------------------------------------------------------------------
// scalar helpers that resolve to the device intrinsics or the host libm
// ---------------------------------------------------------------------------
// FP32 square root: on the device the SFU approximation (sqrt.approx.f32,
// no slow path; exact at 0 and inf): the distances it feeds only need to sit
// far inside the eps-shell, which FP32 rounding already limits.
WOS_HD float w_sqrt(float x)
{
#ifdef __CUDA_ARCH__
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return sqrtf(x);
#endif
}
WOS_HD double w_sqrt(double x) { return sqrt(x); }
// Division: FP32 from the SFU reciprocal (__fdividef, 2 ulp for divisors of
// normal size), FP64 IEEE.
WOS_HD float w_div(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
WOS_HD double w_div(double a, double b) { return a / b; }
WOS_HD float w_floor(float x) { return floorf(x); }
WOS_HD double w_floor(double x) { return floor(x); }
WOS_HD float w_atan2(float y, float x) { return atan2f(y, x); }
WOS_HD double w_atan2(double y, double x) { return atan2(y, x); }
WOS_HD float w_fabs(float x) { return fabsf(x); }
WOS_HD double w_fabs(double x) { return fabs(x); }
template <typename Real> WOS_HD Real w_min(Real a, Real b) { return b < a ? b : a; }
template <typename Real> WOS_HD Real w_max(Real a, Real b) { return b > a ? b : a; }

template <typename Real> struct Consts;
template <> struct Consts<float> {
    static constexpr float inv_2pi = 0.15915494309189535f;
};
template <> struct Consts<double> {
    static constexpr double inv_2pi = 0.15915494309189533577;
};

// ---------------------------------------------------------------------------
// Domain and partition as the kernel sees them (Real = walk precision)
// ---------------------------------------------------------------------------
template <typename Real> struct Geom {
    int32_t dim;
    int32_t outer_kind;
    int32_t n_vert;
    int32_t n_holes;
    int32_t M_tot;
    int32_t vn;              // extrinsic Voronoi sites (0 = cells below)
    const Real *vsites;      // device, vn x dim
    // candidate grid of the sites (null vcell = scan every site): cell
    // (ix, iy, iz) = ((iz g1 + iy) g0 + ix) keeps sites vcand[vcell[c] ..
    // vcell[c + 1]) in ascending order
    const int32_t *vcell;
    const int32_t *vcand;
    int32_t vg[3];
    Real vlo[3];
    Real vinv_h;
    Real c[3];               // sphere / box centre
    Real R;                  // sphere radius
    Real h[3];               // box half-extents
    // polygon: vertex, edge vector, 1 / |edge|^2
    Real vx[kMaxVerts], vy[kMaxVerts], ex[kMaxVerts], ey[kMaxVerts];
    Real il2[kMaxVerts];
    Real hc[kMaxHoles][3], hr[kMaxHoles];
    // one concentric hole (annulus, shell): the walk distance
    // min(R - rho, rho - r_1) = ahalf - |rho - amid|, amid = (R + r_1) / 2,
    // ahalf = (R - r_1) / 2 (each rounded once from double)
    Real amid, ahalf;
    // partition of the outer component
    int32_t outer_m;         // circle arcs
    Real outer_t0;           // theta0 / (2 pi)
    int32_t edge_m[kMaxVerts], edge_off[kMaxVerts]; // polygon / 2-D box sides
    int32_t nb, ns;          // sphere bands x sectors
    int32_t n1, n2;          // 3-D box cells per face
    // partition of the holes
    int32_t hole_m[kMaxHoles], hole_off[kMaxHoles];
    int32_t hole_nb[kMaxHoles], hole_ns[kMaxHoles];
    Real hole_t0[kMaxHoles]; // theta0 / (2 pi)
    // mapped walks: the polytope S^{-1} D, dist(y) = min_f (pd[f] - pn[f] . y)
    int32_t mapped;
    int32_t np;
    Real pn[kMaxPlanes][3], pd[kMaxPlanes];
    Real mS[9], mSinv[9];    // S and S^{-1}, row-major DIM x DIM
    Real qmu2;               // mapped disc / ball: lambda_min(S)^2
};

// Index of the cell of t in [0, 1) split into m equal cells (clamped).
template <typename Real> WOS_HD int32_t cell_of(Real t, int32_t m)
{
    if (!(t > Real(0)))
        return 0;
    Real f = w_floor(t * Real(m));
    return f >= Real(m) ? m - 1 : int32_t(f);
}

// Arc index of the direction (vx, vy) on a circle of m arcs from t0 * 2 pi.
template <typename Real>
WOS_HD int32_t circle_cell(Real vx, Real vy, int32_t m, Real t0)
{
    Real t = w_atan2(vy, vx) * Consts<Real>::inv_2pi - t0;
    t -= w_floor(t);
    return cell_of(t, m);
}

// Equal-area patch of the direction v on a sphere (nb z-bands x ns sectors).
template <typename Real>
WOS_HD int32_t sphere_cell(Real vx, Real vy, Real vz, int32_t nb, int32_t ns)
{
    Real r = w_sqrt(vx * vx + vy * vy + vz * vz);
    Real z = vz / r;
    int32_t band = cell_of((z + Real(1)) * Real(0.5), nb);
    Real t = w_atan2(vy, vx) * Consts<Real>::inv_2pi;
    t -= w_floor(t);
    return band * ns + cell_of(t, ns);
}

// --- outer components -------------------------------------------------------
template <typename Real, int DIM>
WOS_HD Real sphere_dist(const Geom<Real> &g, const Real *x)
{
    Real s = Real(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        Real d = x[a] - g.c[a];
        s += d * d;
    }
    return g.R - w_sqrt(s);
}

// Distance to the box boundary; *side = side / face in element order
// (2-D: bottom, right, top, left; 3-D: -x, -y, -z, +x, +y, +z), lowest on ties.
template <typename Real, int DIM>
WOS_HD Real box_dist(const Geom<Real> &g, const Real *x, int32_t *side)
{
    Real rel[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
        rel[a] = x[a] - g.c[a];
    Real best;
    int32_t bf;
    if (DIM == 2) {
        Real d0 = g.h[1] + rel[1];  // bottom
        Real d1 = g.h[0] - rel[0];  // right
        Real d2 = g.h[1] - rel[1];  // top
        Real d3 = g.h[0] + rel[0];  // left
        best = d0; bf = 0;
        if (d1 < best) { best = d1; bf = 1; }
        if (d2 < best) { best = d2; bf = 2; }
        if (d3 < best) { best = d3; bf = 3; }
    } else {
        best = g.h[0] + rel[0];
        bf = 0;
#pragma unroll
        for (int f = 1; f < 2 * DIM; ++f) {
            int ax = f % DIM;
            Real df = (f < DIM) ? (g.h[ax] + rel[ax]) : (g.h[ax] - rel[ax]);
            if (df < best) { best = df; bf = f; }
        }
    }
    if (side)
        *side = bf;
    return best;
}

// Fast box distance for the walk (the value only).
template <typename Real, int DIM>
WOS_HD Real box_dist_value(const Geom<Real> &g, const Real *x)
{
    Real best = g.h[0] - w_fabs(x[0] - g.c[0]);
#pragma unroll
    for (int a = 1; a < DIM; ++a)
        best = w_min(best, g.h[a] - w_fabs(x[a] - g.c[a]));
    return best;
}

// Squared distance to edge e and the foot parameter; clamped feet are
// measured to the vertex itself so that the two edges sharing a vertex give
// identical values and the lowest edge index wins the tie.
template <typename Real>
WOS_HD Real edge_dist2(const Geom<Real> &g, int e, Real x, Real y, Real *t_out)
{
    Real px = x - g.vx[e], py = y - g.vy[e];
    Real ex = g.ex[e], ey = g.ey[e];
    Real t = (px * ex + py * ey) * g.il2[e];
    if (t <= Real(0)) {
        *t_out = Real(0);
        return px * px + py * py;
    }
    if (t >= Real(1)) {
        int e1 = (e + 1 == g.n_vert) ? 0 : e + 1;
        Real qx = x - g.vx[e1], qy = y - g.vy[e1];
        *t_out = Real(1);
        return qx * qx + qy * qy;
    }
    Real cr = px * ey - py * ex;
    *t_out = t;
    return cr * cr * g.il2[e];
}

template <typename Real>
WOS_HD Real polygon_dist(const Geom<Real> &g, const Real *x, int32_t *edge,
                         Real *tpar)
{
    Real best = Real(INFINITY), bt = Real(0);
    int32_t be = 0;
    for (int e = 0; e < g.n_vert; ++e) {
        Real t;
        Real d2 = edge_dist2(g, e, x[0], x[1], &t);
        if (d2 < best) {
            best = d2;
            be = e;
            bt = t;
        }
    }
    if (edge) *edge = be;
    if (tpar) *tpar = bt;
    return w_sqrt(best);
}

template <typename Real, int DIM>
WOS_HD Real hole_dist(const Geom<Real> &g, int hidx, const Real *x)
{
    Real s = Real(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        Real d = x[a] - g.hc[hidx][a];
        s += d * d;
    }
    return w_sqrt(s) - g.hr[hidx];
}

template <typename Real, int DIM>
WOS_HD Real outer_dist(const Geom<Real> &g, const Real *x)
{
    if (g.outer_kind == kSphere)
        return sphere_dist<Real, DIM>(g, x);
    if (g.outer_kind == kBox)
        return box_dist_value<Real, DIM>(g, x);
    return polygon_dist<Real>(g, x, nullptr, nullptr);
}

// dist(x, dD) for any domain (outer body minus holes).
template <typename Real, int DIM>
WOS_HD Real domain_dist(const Geom<Real> &g, const Real *x)
{
    Real r = outer_dist<Real, DIM>(g, x);
    for (int hidx = 0; hidx < g.n_holes; ++hidx)
        r = w_min(r, hole_dist<Real, DIM>(g, hidx, x));
    return r;
}

// Cell of pi(x) on an outer sphere (circle arcs / z-band x sector patches).
template <typename Real, int DIM>
WOS_HD int32_t outer_sphere_cell(const Geom<Real> &g, const Real *x)
{
    Real v0 = x[0] - g.c[0], v1 = x[1] - g.c[1];
    if (DIM == 2)
        return circle_cell(v0, v1, g.outer_m, g.outer_t0);
    return sphere_cell(v0, v1, x[DIM - 1] - g.c[DIM - 1], g.nb, g.ns);
}

// Cell of pi(x) on a box: nearest side / face, then its cell.
template <typename Real, int DIM>
WOS_HD int32_t outer_box_cell(const Geom<Real> &g, const Real *x)
{
    Real v[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int a = 0; a < DIM; ++a)
        v[a] = x[a] - g.c[a];
    int32_t f;
    box_dist<Real, DIM>(g, x, &f);
    if (DIM == 2) {
        Real t;
        if (f == 0) t = (v[0] + g.h[0]) / (Real(2) * g.h[0]);
        else if (f == 1) t = (v[1] + g.h[1]) / (Real(2) * g.h[1]);
        else if (f == 2) t = (g.h[0] - v[0]) / (Real(2) * g.h[0]);
        else t = (g.h[1] - v[1]) / (Real(2) * g.h[1]);
        return g.edge_off[f] + cell_of(t, g.edge_m[f]);
    }
    int ax = f % 3;
    int b0 = ax == 0 ? 1 : 0;
    int b1 = ax == 2 ? 1 : 2;
    Real t0 = (v[b0] + g.h[b0]) / (Real(2) * g.h[b0]);
    Real t1 = (v[b1] + g.h[b1]) / (Real(2) * g.h[b1]);
    return f * g.n1 * g.n2 + cell_of(t0, g.n1) * g.n2 + cell_of(t1, g.n2);
}

// Element of the outer component holding pi(x).
template <typename Real, int DIM>
WOS_HD int32_t outer_cell(const Geom<Real> &g, const Real *x)
{
    if (g.outer_kind == kSphere)
        return outer_sphere_cell<Real, DIM>(g, x);
    if (g.outer_kind == kBox)
        return outer_box_cell<Real, DIM>(g, x);
    int32_t e;
    Real t;
    polygon_dist<Real>(g, x, &e, &t);
    return g.edge_off[e] + cell_of(t, g.edge_m[e]);
}

// Cell of pi(x) on hole `comp`.
template <typename Real, int DIM>
WOS_HD int32_t hole_cell(const Geom<Real> &g, int comp, const Real *x)
{
    Real vx = x[0] - g.hc[comp][0], vy = x[1] - g.hc[comp][1];
    if (DIM == 2)
        return g.hole_off[comp] + circle_cell(vx, vy, g.hole_m[comp], g.hole_t0[comp]);
    Real vz = x[DIM - 1] - g.hc[comp][DIM - 1];
    return g.hole_off[comp] + sphere_cell(vx, vy, vz, g.hole_nb[comp], g.hole_ns[comp]);
}

// Sphere with holes: nearest component (outer first, lowest hole on ties).
template <typename Real, int DIM>
WOS_HD int32_t sphere_holes_cell(const Geom<Real> &g, const Real *x)
{
    Real best = sphere_dist<Real, DIM>(g, x);
    int32_t comp = -1;
    for (int hidx = 0; hidx < g.n_holes; ++hidx) {
        Real rh = hole_dist<Real, DIM>(g, hidx, x);
        if (rh < best) {
            best = rh;
            comp = hidx;
        }
    }
    return comp < 0 ? outer_sphere_cell<Real, DIM>(g, x) : hole_cell<Real, DIM>(g, comp, x);
}

// The element j of a stopped point: extrinsic Voronoi site, or the cell of
// the nearest boundary component (outer first, then holes; lowest on ties).
template <typename Real, int DIM>
WOS_HD int32_t classify(const Geom<Real> &g, const Real *x)
{
    if (g.vn > 0) {
        int32_t lo = 0, hi = g.vn;
        const int32_t *cand = nullptr;
        if (g.vcell) {  // candidate list of the grid cell of x, if x is inside the grid
            int32_t c = 0;
            bool inside = true;
#pragma unroll
            for (int a = DIM - 1; a >= 0; --a) {
                const Real t = (x[a] - g.vlo[a]) * g.vinv_h;
                const int32_t q = int32_t(floor(t));
                inside = inside && t >= Real(0) && q < g.vg[a];
                c = c * g.vg[a] + q;
            }
            if (inside) {
                lo = g.vcell[c];
                hi = g.vcell[c + 1];
                cand = g.vcand;
            }
        }
        Real best = Real(INFINITY);
        int32_t bj = 0;
        for (int32_t q = lo; q < hi; ++q) {
            const int32_t j = cand ? cand[q] : q;
            Real s = Real(0);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                Real d = x[a] - g.vsites[j * DIM + a];
                s += d * d;
            }
            if (s < best) {
                best = s;
                bj = j;
            }
        }
        return bj;
    }
    if (g.n_holes == 0)
        return outer_cell<Real, DIM>(g, x);
    Real best = outer_dist<Real, DIM>(g, x);
    int32_t comp = -1;
    for (int hidx = 0; hidx < g.n_holes; ++hidx) {
        Real rh = hole_dist<Real, DIM>(g, hidx, x);
        if (rh < best) {
            best = rh;
            comp = hidx;
        }
    }
    return comp < 0 ? outer_cell<Real, DIM>(g, x) : hole_cell<Real, DIM>(g, comp, x);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 with a precomputed key schedule rk[2r], rk[2r+1] (round r).
// ---------------------------------------------------------------------------
WOS_HD void philox_round_keys(uint64_t seed, uint32_t *rk)
{
    uint32_t k0 = uint32_t(seed), k1 = uint32_t(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0;
        rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

#ifdef __CUDACC__
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1,
                                              uint32_t c2, uint32_t c3,
                                              const uint32_t *rk, uint32_t *out)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        uint32_t lo0 = 0xD2511F53u * c0;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        uint32_t lo1 = 0xCD9E8D57u * c2;
        c0 = hi1 ^ c1 ^ rk[2 * r];
        c1 = lo1;
        c2 = hi0 ^ c3 ^ rk[2 * r + 1];
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Uniform on [0, 1): 23 bits of one word (FP32 walks) or 53 bits of two
// words (FP64 walks).  The FP32 uniform is built from the bits, not by a
// conversion: 1 + (w >> 9) 2^-23 has exponent 0 and those 23 bits as its
// mantissa, so subtracting 1 leaves (w >> 9) 2^-23 exactly (a logic op and
// an add on the FMA pipe instead of an I2F on the conversion unit).
template <typename Real> struct Uniform;
template <> struct Uniform<float> {
    static constexpr int kWords = 1;
    __device__ __forceinline__ static float get(const uint32_t *w)
    {
        return __uint_as_float(0x3f800000u | (w[0] >> 9)) - 1.0f;
    }
};
template <> struct Uniform<double> {
    static constexpr int kWords = 2;
    __device__ __forceinline__ static double get(const uint32_t *w)
    {
        uint64_t m = (uint64_t(w[0]) << 21) | uint64_t(w[1] >> 11);
        return double(m) * 0x1p-53;
    }
};

// sin(pi x), cos(pi x) for x = 2u in [0, 2): FP32 walks use the SFU sine and
// cosine on the angle pi (x - 1) in [-pi, pi) -- the range of their
// documented absolute error bound (2^-21.41) -- and flip both signs.
__device__ __forceinline__ void w_sincospi(float x, float *s, float *c)
{
    float ss, cc;
    __sincosf(3.14159265358979f * (x - 1.0f), &ss, &cc);
    *s = -ss;
    *c = -cc;
}
__device__ __forceinline__ void w_sincospi(double x, double *s, double *c) { sincospi(x, s, c); }

// FP32 2-D walks take five 23-bit uniforms from one Philox block: step j of
// the block reads bits 23j .. 23j + 22 of the 128-bit number w0 + 2^32 w1 +
// 2^64 w2 + 2^96 w3 (bits 115..127 are unused), one funnel shift each.
constexpr int kPacked2dSteps = 5;
__device__ __forceinline__ uint32_t window23(const uint32_t *w, int j)
{
    switch (j) {  // j is a constant once the step loop is unrolled
    case 0: return w[0];
    case 1: return __funnelshift_r(w[0], w[1], 23);
    case 2: return __funnelshift_r(w[1], w[2], 14);
    case 3: return __funnelshift_r(w[2], w[3], 5);
    default: return __funnelshift_r(w[2], w[3], 28);
    }
}

// U uniform on S^{d-1}: d = 2 (cos 2 pi u, sin 2 pi u); d = 3 Archimedes:
// z = 1 - 2 u1, (s cos 2 pi u2, s sin 2 pi u2, z), s = sqrt(1 - z^2).
template <typename Real, int DIM>
__device__ __forceinline__ void direction(const uint32_t *w, Real *U)
{
    if (DIM == 2) {
        Real s, c;
        if constexpr (sizeof(Real) == 4) {
            // w[0] holds the step's 23-bit window in its low bits: one logic
            // op builds f = 2 + window 2^-22 = 2 + 2u in [2, 4); the angle
            // pi (2u - 1) = pi f - 3 pi is one FMA, rounded once and inside
            // [-pi, pi]; with the float constants each angle is within
            // 4.5e-7 rad of the exact one (an offset, a stretch of 3e-8
            // relative and the rounding; checked over every window on the
            // host), below the SFU sine's own error.  Then the SFU path of
            // w_sincospi
            const float f = __uint_as_float(0x40000000u | (w[0] & 0x7fffffu));
            float ss, cc;
            __sincosf(fmaf(f, 3.14159265358979f, -9.42477796076938f), &ss, &cc);
            s = -ss;
            c = -cc;
        } else {
            Real u = Uniform<Real>::get(w);
            w_sincospi(Real(2) * u, &s, &c);
        }
        U[0] = c;
        U[1] = s;
    } else if constexpr (sizeof(Real) == 4) {
        // f_j = 1 + u_j in [1, 2) from the bits (one logic op each); z = 3 -
        // 2 f_1 is 1 - 2 u_1 exactly (a multiple of 2^-22 in (-1, 1]), and the
        // angle pi (2 u_2 - 1) = 2 pi f_2 - 3 pi is one FMA (float constants
        // and rounding: within 4.5e-7 rad), inside [-pi, pi] for the SFU path
        // of w_sincospi
        const float f1 = __uint_as_float(0x3f800000u | (w[0] >> 9));
        const float f2 = __uint_as_float(0x3f800000u | (w[1] >> 9));
        const float z = fmaf(-2.0f, f1, 3.0f);
        const float s2 = fmaf(-z, z, 1.0f);
        const float sr = w_sqrt(s2 > 0.0f ? s2 : 0.0f);
        float ss, cc;
        __sincosf(fmaf(f2, 6.28318530717959f, -9.42477796076938f), &ss, &cc);
        U[0] = -sr * cc;
        U[1] = -sr * ss;
        U[2] = z;
    } else {
        Real u1 = Uniform<Real>::get(w);
        Real u2 = Uniform<Real>::get(w + Uniform<Real>::kWords);
        Real z = Real(1) - Real(2) * u1;
        Real s2 = Real(1) - z * z;
        Real sr = w_sqrt(s2 > Real(0) ? s2 : Real(0));
        Real s, c;
        w_sincospi(Real(2) * u2, &s, &c);
        U[0] = sr * c;
        U[1] = sr * s;
        U[2] = z;
    }
}
#endif

}  // namespace wos
