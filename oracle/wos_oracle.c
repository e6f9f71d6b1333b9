/*
 * wos_oracle.c -- plain, slow, FP64 CPU oracle of the walk-on-ellipsoids
 * (WoE) Monte Carlo build of the direct operator, and of the one-sided
 * Jacobi SVD used on it.
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the
 * benchmark's CPU-baseline leg are the only callers.  The CUDA library shares
 * no code, header, table or helper with this file; each side implements the
 * published definitions on its own.
 *
 * What it follows (Cimpean, Grecu & Marin, arXiv:2409.03686):
 *   Sec. 4.1, Eq. (Y) / (harmonicmeasure): mu_x is the exit law of
 *       Y_t = K^{1/2} B_t + x.
 *   Sec. 4.2, Eq. (wos chain): X_{n+1} = X_n + dist(X_n, dD) K^{1/2} U_n,
 *       U_n uniform on S^{d-1}, with lambda_max(K) = 1 (K is rescaled,
 *       which does not change mu_x).
 *   Sec. 4.2, Eq. (N epsilon x): N_eps = min{n : dist(X_n, dD) <= eps}.
 *   Sec. 4.3, Eq. (WoE_matrix_MC) and the Voronoi remark after it:
 *       [A]_ij = #{k : X^{i,k}_{N_eps} in cell j} / N.
 *   Sec. 5.1, Algorithm MC-REM; Rem. (wos algorithm)(i) for the step cap.
 *   App. A, Ex. A.3 (intrinsic Voronoi cells through the projection pi,
 *       ties to the lowest index) and Ex. A.2 (extrinsic Voronoi cells).
 * Random numbers: Philox4x32-10 as published by Salmon, Moraes, Dror & Shaw,
 *   "Parallel random numbers: as easy as 1, 2, 3", SC'11.
 * SVD: one-sided (Hestenes) Jacobi in cyclic-by-rows order with the relative
 *   off-diagonal test of Demmel & Veselic, SIAM J. Matrix Anal. Appl. 13
 *   (1992).
 *
 * Chain specification shared (as a specification, not as code) with the GPU:
 *   key     = (seed & 0xffffffff, seed >> 32)
 *   counter = (b, walk & 0xffffffff, walk >> 32, stream), walk = i*N + k
 *   FP32 2-D walks (wpu = 1, d = 2): G = 5 steps per Philox block, step j
 *   of the block takes u = ((B >> 23 j) mod 2^23) 2^-23 from the 128-bit
 *   B = w0 + 2^32 w1 + 2^64 w2 + 2^96 w3.  Otherwise a step uses
 *   wps = (d == 2 ? 1 : 2) * wpu words, wpu = 1 (23-bit uniforms
 *   u = (w >> 9) 2^-23) or 2 (53-bit u = (w0 2^21 + (w1 >> 11)) 2^-53), and
 *   G = 4 / wps.  Philox block b serves steps b*G .. b*G+G-1.
 *   d = 2: U = (cos 2 pi u, sin 2 pi u)
 *   d = 3: z = 1 - 2 u1, phi = 2 pi u2, U = (s cos phi, s sin phi, z),
 *          s = sqrt(1 - z^2).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include "wos_oracle.h"

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11).                               */
/* ------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        mulhilo32(M0, c0, &hi0, &lo0);
        mulhilo32(M1, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Steps served by one Philox block (see the chain specification above). */
static int steps_per_block(int d, int wpu)
{
    return (d == 2 && wpu == 1) ? 5 : 4 / ((d == 2 ? 1 : 2) * wpu);
}

/* The 23-bit window j (bits 23 j .. 23 j + 22) of the 128-bit block, as a
 * uniform on [0, 1). */
static double window23_uniform(const uint32_t *w, int j)
{
    const int off = 23 * j, q = off / 32, r = off % 32;
    uint64_t pair = (uint64_t)w[q];
    if (q + 1 < 4)
        pair |= (uint64_t)w[q + 1] << 32;
    return (double)((pair >> r) & 0x7FFFFFu) * 0x1p-23;
}

/* Uniform on [0, 1) from one word (23 bits) or two words (53 bits). */
static double uniform_from_words(const uint32_t *w, int wpu)
{
    if (wpu == 1)
        return (double)(w[0] >> 9) * 0x1p-23;
    uint64_t m = ((uint64_t)w[0] << 21) | (uint64_t)(w[1] >> 11);
    return (double)m * 0x1p-53;
}

/* ------------------------------------------------------------------ */
/* Geometry: distance to the boundary and the exit element.            */
/* ------------------------------------------------------------------ */
static double norm_d(const double *v, int d)
{
    double s = 0.0;
    for (int a = 0; a < d; ++a)
        s += v[a] * v[a];
    return sqrt(s);
}

/* Squared distance from p to segment [a, b] and the foot parameter t.
 * Clamped feet are measured to the vertex itself, so the two edges that
 * share a vertex produce bit-identical values there and the lowest-index
 * rule decides the tie. */
static double seg_dist2(const double *p, const double *a, const double *b,
                        double *t_out)
{
    double ex = b[0] - a[0], ey = b[1] - a[1];
    double px = p[0] - a[0], py = p[1] - a[1];
    double L2 = ex * ex + ey * ey;
    double t = (px * ex + py * ey) / L2;
    if (t <= 0.0) {
        *t_out = 0.0;
        return px * px + py * py;
    }
    if (t >= 1.0) {
        double qx = p[0] - b[0], qy = p[1] - b[1];
        *t_out = 1.0;
        return qx * qx + qy * qy;
    }
    double cr = px * ey - py * ex;
    *t_out = t;
    return cr * cr / L2;
}

/* Distance from x to the outer boundary component (signed: > 0 inside). */
static double outer_dist(const orc_domain *D, const double *x, int *edge,
                         double *tpar)
{
    int d = D->dim;
    if (D->outer_kind == ORC_OUTER_SPHERE) {
        double v[3];
        for (int a = 0; a < d; ++a)
            v[a] = x[a] - D->center[a];
        return D->radius - norm_d(v, d);
    }
    if (D->outer_kind == ORC_OUTER_BOX) {
        /* 2-D: sides in element order bottom, right, top, left (the polygon
         * whose first vertex is the corner c - h).  3-D: faces -x, -y, -z,
         * +x, +y, +z.  Strict < keeps the lowest index on ties. */
        double best = INFINITY;
        int bf = 0;
        for (int f = 0; f < 2 * d; ++f) {
            int ax;
            double df;
            if (d == 2) {
                static const int axis2[4] = {1, 0, 1, 0};
                static const int low2[4] = {1, 0, 0, 1};
                ax = axis2[f];
                double rel = x[ax] - D->center[ax];
                df = low2[f] ? (D->half[ax] + rel) : (D->half[ax] - rel);
            } else {
                ax = f % d;
                double rel = x[ax] - D->center[ax];
                df = (f < d) ? (D->half[ax] + rel) : (D->half[ax] - rel);
            }
            if (df < best) {
                best = df;
                bf = f;
            }
        }
        if (edge)
            *edge = bf;
        return best;
    }
    /* polygon (2-D only): min over edges, vertices listed counter-clockwise */
    double best = INFINITY, bt = 0.0;
    int be = 0;
    int n = D->n_vertices;
    for (int e = 0; e < n; ++e) {
        const double *a = &D->vertices[2 * e];
        const double *b = &D->vertices[2 * ((e + 1) % n)];
        double t;
        double d2 = seg_dist2(x, a, b, &t);
        if (d2 < best) {
            best = d2;
            be = e;
            bt = t;
        }
    }
    if (edge)
        *edge = be;
    if (tpar)
        *tpar = bt;
    return sqrt(best);
}

static double hole_dist(const orc_domain *D, int h, const double *x)
{
    double v[3];
    for (int a = 0; a < D->dim; ++a)
        v[a] = x[a] - D->hole_center[h][a];
    return norm_d(v, D->dim) - D->hole_radius[h];
}

double orc_dist(const orc_domain *D, const double *x)
{
    double r = outer_dist(D, x, NULL, NULL);
    for (int h = 0; h < D->n_holes; ++h) {
        double rh = hole_dist(D, h, x);
        if (rh < r)
            r = rh;
    }
    return r;
}

static int clamp_cell(double t, int m)
{
    if (!(t > 0.0))
        return 0;
    double f = floor(t * (double)m);
    if (f >= (double)m)
        return m - 1;
    return (int)f;
}

/* Arc index of direction v on a circle split into m arcs from theta0. */
static int circle_cell(const double *v, int m, double theta0)
{
    double th = atan2(v[1], v[0]);
    double t = (th - theta0) / (2.0 * M_PI);
    t -= floor(t);
    return clamp_cell(t, m);
}

/* Equal-area patch of direction v on a sphere: nb z-bands x ns sectors. */
static int sphere_cell(const double *v, int nb, int ns)
{
    double r = norm_d(v, 3);
    double z = v[2] / r;
    int band = clamp_cell((z + 1.0) * 0.5, nb);
    double ph = atan2(v[1], v[0]);
    double t = ph / (2.0 * M_PI);
    t -= floor(t);
    int sec = clamp_cell(t, ns);
    return band * ns + sec;
}

int orc_outer_elements(const orc_domain *D)
{
    if (D->outer_kind == ORC_OUTER_SPHERE)
        return D->dim == 2 ? D->outer_m : D->outer_nb * D->outer_ns;
    if (D->outer_kind == ORC_OUTER_BOX && D->dim == 3)
        return 6 * D->face_n1 * D->face_n2;
    int ne = (D->outer_kind == ORC_OUTER_BOX) ? 4 : D->n_vertices;
    int s = 0;
    for (int e = 0; e < ne; ++e)
        s += D->edge_m[e];
    return s;
}

int orc_hole_elements(const orc_domain *D, int h)
{
    return D->dim == 2 ? D->hole_m[h] : D->hole_nb[h] * D->hole_ns[h];
}

int orc_num_elements(const orc_domain *D)
{
    if (D->voronoi_n > 0)
        return D->voronoi_n;
    int s = orc_outer_elements(D);
    for (int h = 0; h < D->n_holes; ++h)
        s += orc_hole_elements(D, h);
    return s;
}

/* Element of the outer component whose cell holds pi(x). */
static int outer_cell(const orc_domain *D, const double *x)
{
    int d = D->dim;
    double v[3];
    for (int a = 0; a < d; ++a)
        v[a] = x[a] - D->center[a];
    if (D->outer_kind == ORC_OUTER_SPHERE)
        return d == 2 ? circle_cell(v, D->outer_m, D->outer_theta0)
                      : sphere_cell(v, D->outer_nb, D->outer_ns);
    if (D->outer_kind == ORC_OUTER_BOX) {
        int f;
        outer_dist(D, x, &f, NULL);
        if (d == 2) {
            /* f is the side index in element order: bottom, right, top, left */
            double hx = D->half[0], hy = D->half[1];
            double t;
            if (f == 0) t = (v[0] + hx) / (2.0 * hx);
            else if (f == 1) t = (v[1] + hy) / (2.0 * hy);
            else if (f == 2) t = (hx - v[0]) / (2.0 * hx);
            else t = (hy - v[1]) / (2.0 * hy);
            int off = 0;
            for (int k = 0; k < f; ++k)
                off += D->edge_m[k];
            return off + clamp_cell(t, D->edge_m[f]);
        }
        /* 3-D faces -x,-y,-z,+x,+y,+z; cells over the two other axes in
         * increasing axis order. */
        int ax = f % 3;
        int b0 = ax == 0 ? 1 : 0;
        int b1 = ax == 2 ? 1 : 2;
        double t0 = (v[b0] + D->half[b0]) / (2.0 * D->half[b0]);
        double t1 = (v[b1] + D->half[b1]) / (2.0 * D->half[b1]);
        int p = clamp_cell(t0, D->face_n1);
        int q = clamp_cell(t1, D->face_n2);
        return f * D->face_n1 * D->face_n2 + p * D->face_n2 + q;
    }
    int e;
    double t;
    outer_dist(D, x, &e, &t);
    int off = 0;
    for (int k = 0; k < e; ++k)
        off += D->edge_m[k];
    return off + clamp_cell(t, D->edge_m[e]);
}

int orc_classify(const orc_domain *D, const double *x)
{
    int d = D->dim;
    if (D->voronoi_n > 0) {
        /* App. A, Ex. A.2: nearest site, ties to the lowest index. */
        double best = INFINITY;
        int bj = 0;
        for (int j = 0; j < D->voronoi_n; ++j) {
            double s = 0.0;
            for (int a = 0; a < d; ++a) {
                double dv = x[a] - D->voronoi_sites[j * d + a];
                s += dv * dv;
            }
            if (s < best) {
                best = s;
                bj = j;
            }
        }
        return bj;
    }
    /* Nearest component (outer first, then holes in order; ties lowest). */
    double best = outer_dist(D, x, NULL, NULL);
    int comp = -1;
    for (int h = 0; h < D->n_holes; ++h) {
        double rh = hole_dist(D, h, x);
        if (rh < best) {
            best = rh;
            comp = h;
        }
    }
    if (comp < 0)
        return outer_cell(D, x);
    int off = orc_outer_elements(D);
    for (int h = 0; h < comp; ++h)
        off += orc_hole_elements(D, h);
    double v[3];
    for (int a = 0; a < d; ++a)
        v[a] = x[a] - D->hole_center[comp][a];
    if (d == 2)
        return off + circle_cell(v, D->hole_m[comp], D->hole_theta0[comp]);
    return off + sphere_cell(v, D->hole_nb[comp], D->hole_ns[comp]);
}

/* ------------------------------------------------------------------ */
/* One walk of the chain (Eq. wos chain) stopped at N_eps.             */
/* ------------------------------------------------------------------ */
/* The mapped chain (a reading of Sec. 4.2 with the exact distance): in
 * y = S^{-1} x the diffusion of div(K grad) is a Brownian motion in the
 * polytope S^{-1} D, and the walk is walk-on-spheres there,
 * Y_{n+1} = Y_n + dist_y(Y_n) U_n, stopped at dist_y <= eps; the exit point
 * S Y is classified in x. */
static int orc_walk_mapped(const orc_instance *I, const double *x0, uint64_t walk,
                           double *x_exit, uint32_t *nsteps)
{
    const int d = I->dom.dim;
    const int wpu = I->words_per_uniform;
    const int wps = (d == 2 ? 1 : 2) * wpu;
    const int G = steps_per_block(d, wpu);
    const int packed = d == 2 && wpu == 1;
    const uint32_t key[2] = {(uint32_t)I->seed, (uint32_t)(I->seed >> 32)};
    double Y[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b)
            Y[a] += I->Sinv[a * d + b] * x0[b];
    uint32_t words[4] = {0, 0, 0, 0};
    for (uint32_t n = 0;; ++n) {
        double r = INFINITY;
        for (int f = 0; f < I->n_planes; ++f) {
            double s = I->plane_d[f];
            for (int a = 0; a < d; ++a)
                s -= I->plane_n[f][a] * Y[a];
            r = fmin(r, s);
        }
        if (r <= I->eps || n >= I->step_cap) {
            double X[3] = {0.0, 0.0, 0.0};
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b)
                    X[a] += I->S[a * d + b] * Y[b];
            for (int a = 0; a < d; ++a)
                x_exit[a] = X[a];
            *nsteps = n;
            return r <= I->eps ? orc_classify(&I->dom, X) : -1;
        }
        if (n % (uint32_t)G == 0) {
            uint32_t ctr[4] = {n / (uint32_t)G, (uint32_t)walk,
                               (uint32_t)(walk >> 32), I->stream};
            orc_philox4x32_10(ctr, key, words);
        }
        const uint32_t *w = words + (packed ? 0u : (n % (uint32_t)G) * (uint32_t)wps);
        if (d == 2) {
            double u = packed ? window23_uniform(words, (int)(n % (uint32_t)G))
                              : uniform_from_words(w, wpu);
            Y[0] += r * cos(2.0 * M_PI * u);
            Y[1] += r * sin(2.0 * M_PI * u);
        } else {
            double u1 = uniform_from_words(w, wpu);
            double u2 = uniform_from_words(w + wpu, wpu);
            double z = 1.0 - 2.0 * u1;
            double sr = sqrt(fmax(0.0, 1.0 - z * z));
            Y[0] += r * sr * cos(2.0 * M_PI * u2);
            Y[1] += r * sr * sin(2.0 * M_PI * u2);
            Y[2] += r * z;
        }
    }
}

/* The mapped chain on a disc / ball D minus disc / ball holes (mapped = 2).
 * Its step from X is the largest ellipsoid X + rho S B(0, 1) inside D, whose
 * radius is rho = dist_y(S^{-1} X, S^{-1} dD) in y = S^{-1} x (where the
 * diffusion of div(K grad) is a Brownian motion, Sec. 4.2); that distance to
 * an ellipse / ellipsoid is replaced by a lower bound, component by
 * component.  With v = X - c and w = S v (S symmetric, lambda_max(S) = 1):
 *   outer |x - c| <= R:  along y + s u, |S(y + s u) - c|^2 - R^2 <=
 *     (rho^2 - R^2) + 2 s |w| + s^2, negative for s below the root
 *     s_out = (R^2 - rho^2) / (|w| + sqrt(|w|^2 + R^2 - rho^2));
 *   hole |x - c_h| >= r:  |S(y + s u) - c_h|^2 - r^2 >= F - 2 s |w| +
 *     s^2 mu^2 (F = rho^2 - r^2, mu = lambda_min(S)), positive below the
 *     smaller root s_h = F / (|w| + sqrt(|w|^2 - mu^2 F)); also
 *     dist_y >= dist_x = rho - r (y -> S y does not expand distances), so
 *     the hole gives max(s_h, rho - r).
 * Both bounds equal the distance to first order at the boundary, and with
 * S = I they are R - rho and rho - r exactly; s_out >= R - rho because
 * |w| <= rho.  The radius is the smallest bound (<= 0 outside D).  The walk
 * stops when it is <= eps, and then dist_x <= eps. */
double orc_quadric_radius(const orc_instance *I, const double *x)
{
    const orc_domain *D = &I->dom;
    const int d = D->dim;
    double v[3] = {0.0, 0.0, 0.0}, rho2 = 0.0, w2 = 0.0;
    for (int a = 0; a < d; ++a) {
        v[a] = x[a] - D->center[a];
        rho2 += v[a] * v[a];
    }
    for (int a = 0; a < d; ++a) {
        double wa = 0.0;
        for (int b = 0; b < d; ++b)
            wa += I->S[a * d + b] * v[b];
        w2 += wa * wa;
    }
    const double F0 = D->radius * D->radius - rho2;
    if (F0 <= 0.0)
        return 0.0;
    double r = F0 / (sqrt(w2) + sqrt(w2 + F0));
    for (int h = 0; h < D->n_holes; ++h) {
        rho2 = 0.0;
        w2 = 0.0;
        for (int a = 0; a < d; ++a) {
            v[a] = x[a] - D->hole_center[h][a];
            rho2 += v[a] * v[a];
        }
        for (int a = 0; a < d; ++a) {
            double wa = 0.0;
            for (int b = 0; b < d; ++b)
                wa += I->S[a * d + b] * v[b];
            w2 += wa * wa;
        }
        const double rh = D->hole_radius[h];
        const double F = rho2 - rh * rh;
        if (F <= 0.0)
            return 0.0;
        double sh = F / (sqrt(w2) + sqrt(fmax(0.0, w2 - I->mu2 * F)));
        sh = fmax(sh, sqrt(rho2) - rh);
        r = fmin(r, sh);
    }
    return r;
}

int orc_walk(const orc_instance *I, const double *x0, uint64_t walk,
             double *x_exit, uint32_t *nsteps)
{
    if (I->mapped == 1)
        return orc_walk_mapped(I, x0, walk, x_exit, nsteps);
    const int d = I->dom.dim;
    const int wpu = I->words_per_uniform;
    const int wps = (d == 2 ? 1 : 2) * wpu;
    const int G = steps_per_block(d, wpu);
    const int packed = d == 2 && wpu == 1;
    const uint32_t key[2] = {(uint32_t)I->seed, (uint32_t)(I->seed >> 32)};
    double X[3] = {x0[0], x0[1], d == 3 ? x0[2] : 0.0};
    uint32_t words[4] = {0, 0, 0, 0};
    for (uint32_t n = 0;; ++n) {
        double r = I->mapped == 2 ? orc_quadric_radius(I, X) : orc_dist(&I->dom, X);
        if (r <= I->eps || n >= I->step_cap) {
            for (int a = 0; a < d; ++a)
                x_exit[a] = X[a];
            *nsteps = n;
            return r <= I->eps ? orc_classify(&I->dom, X) : -1;
        }
        if (n % (uint32_t)G == 0) {
            uint32_t ctr[4] = {n / (uint32_t)G, (uint32_t)walk,
                               (uint32_t)(walk >> 32), I->stream};
            orc_philox4x32_10(ctr, key, words);
        }
        const uint32_t *w = words + (packed ? 0u : (n % (uint32_t)G) * (uint32_t)wps);
        double U[3];
        if (d == 2) {
            double u = packed ? window23_uniform(words, (int)(n % (uint32_t)G))
                              : uniform_from_words(w, wpu);
            U[0] = cos(2.0 * M_PI * u);
            U[1] = sin(2.0 * M_PI * u);
            U[2] = 0.0;
        } else {
            double u1 = uniform_from_words(w, wpu);
            double u2 = uniform_from_words(w + wpu, wpu);
            double z = 1.0 - 2.0 * u1;
            double s = sqrt(fmax(0.0, 1.0 - z * z));
            U[0] = s * cos(2.0 * M_PI * u2);
            U[1] = s * sin(2.0 * M_PI * u2);
            U[2] = z;
        }
        double step[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b)
                step[a] += I->S[a * d + b] * U[b];
        for (int a = 0; a < d; ++a)
            X[a] += r * step[a];
    }
}

int orc_walk_batch(const orc_instance *I, const double *x0,
                   const uint64_t *walks, int64_t n, double *x_exit,
                   int32_t *elem, uint32_t *nsteps)
{
    const int d = I->dom.dim;
    for (int64_t q = 0; q < n; ++q)
        elem[q] = orc_walk(I, x0 + q * d, walks[q], x_exit + q * d,
                           nsteps + q);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Algorithm MC-REM: counts C[i][j] over walks k in [k0, k1).          */
/* Points are shared out to plain POSIX threads.                       */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_instance *I;
    const double *points;
    int32_t M_D;
    uint32_t k0, k1;
    uint32_t *counts;
    uint32_t *unterminated;
    int32_t M;
    int32_t next; /* shared point cursor */
    uint64_t steps;
    pthread_mutex_t mu;
} build_job;

static void *build_worker(void *arg)
{
    build_job *J = (build_job *)arg;
    const int d = J->I->dom.dim;
    uint64_t my_steps = 0;
    for (;;) {
        int i = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (i >= J->M_D)
            break;
        uint32_t *row = J->counts + (size_t)i * (size_t)J->M;
        for (uint32_t k = J->k0; k < J->k1; ++k) {
            uint64_t walk = (uint64_t)i * (uint64_t)J->I->N + k;
            double xe[3];
            uint32_t ns;
            int j = orc_walk(J->I, J->points + (size_t)i * d, walk, xe, &ns);
            my_steps += ns;
            if (j >= 0)
                row[j] += 1u;
            else
                J->unterminated[i] += 1u;
        }
    }
    pthread_mutex_lock(&J->mu);
    J->steps += my_steps;
    pthread_mutex_unlock(&J->mu);
    return NULL;
}

int orc_build_counts(const orc_instance *I, const double *points, int32_t M_D,
                     uint32_t k0, uint32_t k1, uint32_t *counts,
                     uint32_t *unterminated, uint64_t *total_steps,
                     int32_t nthreads)
{
    if (k1 < k0 || k1 > I->N)
        return 1;
    build_job J;
    J.I = I;
    J.points = points;
    J.M_D = M_D;
    J.k0 = k0;
    J.k1 = k1;
    J.counts = counts;
    J.unterminated = unterminated;
    J.M = orc_num_elements(&I->dom);
    J.next = 0;
    J.steps = 0;
    pthread_mutex_init(&J.mu, NULL);
    if (nthreads <= 0)
        nthreads = (int32_t)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1)
        nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t)
        pthread_create(&th[t], NULL, build_worker, &J);
    for (int t = 0; t < nthreads; ++t)
        pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
    if (total_steps)
        *total_steps = J.steps;
    return 0;
}

/* ------------------------------------------------------------------ */
/* One-sided Jacobi SVD (Hestenes), cyclic-by-rows.                    */
/* B is m x n row-major.  Returns U (m x k), s (k), V (n x k), k =     */
/* min(m, n), singular values descending, each V column signed so its  */
/* largest-magnitude entry is positive.  0 = converged.                */
/* ------------------------------------------------------------------ */
static int jacobi_cols(int m, int n, double *W /* m x n col-major */,
                       double *V /* n x n col-major */, double tol,
                       int max_sweeps, int *sweeps_out)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            V[(size_t)j * n + i] = (i == j) ? 1.0 : 0.0;
    int sweep;
    for (sweep = 1; sweep <= max_sweeps; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double *wp = W + (size_t)p * m, *wq = W + (size_t)q * m;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int i = 0; i < m; ++i) {
                    alpha += wp[i] * wp[i];
                    beta += wq[i] * wq[i];
                    gamma += wp[i] * wq[i];
                }
                if (alpha == 0.0 || beta == 0.0)
                    continue;
                if (fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta))
                    continue;
                rotated = 1;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) /
                           (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = c * t;
                for (int i = 0; i < m; ++i) {
                    double a = wp[i], b = wq[i];
                    wp[i] = c * a - s * b;
                    wq[i] = s * a + c * b;
                }
                double *vp = V + (size_t)p * n, *vq = V + (size_t)q * n;
                for (int i = 0; i < n; ++i) {
                    double a = vp[i], b = vq[i];
                    vp[i] = c * a - s * b;
                    vq[i] = s * a + c * b;
                }
            }
        }
        if (!rotated)
            break;
    }
    if (sweeps_out)
        *sweeps_out = sweep > max_sweeps ? max_sweeps : sweep;
    return sweep > max_sweeps ? 1 : 0;
}

int orc_jacobi_svd(int32_t m, int32_t n, const double *B, double *U,
                   double *S, double *V, int32_t *sweeps)
{
    /* Work on the orientation with more rows than columns. */
    int tr = m < n;
    int mm = tr ? n : m, nn = tr ? m : n;
    double *W = (double *)malloc(sizeof(double) * (size_t)mm * nn);
    double *Vw = (double *)malloc(sizeof(double) * (size_t)nn * nn);
    double *sv = (double *)malloc(sizeof(double) * (size_t)nn);
    int *ord = (int *)malloc(sizeof(int) * (size_t)nn);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            double b = B[(size_t)i * n + j];
            if (!tr)
                W[(size_t)j * mm + i] = b; /* column j of B */
            else
                W[(size_t)i * mm + j] = b; /* column i of B^T */
        }
    int rc = jacobi_cols(mm, nn, W, Vw, 1e-15, 80, sweeps);
    for (int j = 0; j < nn; ++j) {
        double s = 0.0;
        for (int i = 0; i < mm; ++i)
            s += W[(size_t)j * mm + i] * W[(size_t)j * mm + i];
        sv[j] = sqrt(s);
        ord[j] = j;
    }
    /* insertion sort, descending */
    for (int a = 1; a < nn; ++a) {
        int key = ord[a];
        int b = a - 1;
        while (b >= 0 && sv[ord[b]] < sv[key]) {
            ord[b + 1] = ord[b];
            --b;
        }
        ord[b + 1] = key;
    }
    int k = nn;
    for (int c = 0; c < k; ++c) {
        int j = ord[c];
        double s = sv[j];
        /* left vectors of the worked matrix are W_j / s_j, right are V_j */
        double *wl = W + (size_t)j * mm;
        double *wr = Vw + (size_t)j * nn;
        /* sign: largest-magnitude entry of the B-side right vector > 0 */
        const double *rv = tr ? wl : wr;
        int rn = tr ? mm : nn;
        double big = 0.0, sign = 1.0;
        for (int i = 0; i < rn; ++i) {
            double a = fabs(rv[i]) * (tr ? (s > 0 ? 1.0 / s : 0.0) : 1.0);
            if (a > big) {
                big = a;
                sign = rv[i] >= 0.0 ? 1.0 : -1.0;
            }
        }
        S[c] = s;
        for (int i = 0; i < mm; ++i) {
            double u = s > 0.0 ? sign * wl[i] / s : 0.0;
            if (!tr)
                U[(size_t)i * k + c] = u;
            else
                V[(size_t)i * k + c] = u;
        }
        for (int i = 0; i < nn; ++i) {
            double v = sign * wr[i];
            if (!tr)
                V[(size_t)i * k + c] = v;
            else
                U[(size_t)i * k + c] = v;
        }
    }
    free(W);
    free(Vw);
    free(sv);
    free(ord);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Instance set-up: K_s = K / lambda_max(K), S = K_s^{1/2} (Sec. 4.2). */
/* Returns 0, or 1 when K is not symmetric positive definite.          */
/* ------------------------------------------------------------------ */
int orc_setup_S(int32_t d, const double *K, double *S, double *lam_max)
{
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b)
            if (fabs(K[a * d + b] - K[b * d + a]) >
                1e-12 * (fabs(K[a * d + b]) + fabs(K[b * d + a]) + 1e-300))
                return 1;
    double U[9], s[3], V[9];
    int32_t sw;
    orc_jacobi_svd(d, d, K, U, s, V, &sw);
    /* For symmetric K, K = V diag(s) V^T with positive eigenvalues exactly
     * when the Rayleigh quotients v^T K v are all positive. */
    double lam[3];
    for (int c = 0; c < d; ++c) {
        double q = 0.0;
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b)
                q += V[a * d + c] * K[a * d + b] * V[b * d + c];
        lam[c] = q;
    }
    double lmax = s[0];
    for (int c = 0; c < d; ++c)
        if (!(lam[c] > 1e-12 * lmax))
            return 1;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double acc = 0.0;
            for (int c = 0; c < d; ++c)
                acc += V[a * d + c] * sqrt(s[c] / lmax) * V[b * d + c];
            S[a * d + b] = acc;
        }
    if (lam_max)
        *lam_max = lmax;
    return 0;
}
