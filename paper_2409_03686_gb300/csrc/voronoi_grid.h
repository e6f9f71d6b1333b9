// voronoi_grid.h -- host-side candidate grid for the extrinsic Voronoi cells
// of App. A, Ex. A.2 (the element of a stopped point is its nearest site,
// the lowest index on ties).
//
// A uniform grid covers the domain and the sites.  Cell C with centre c and
// half-diagonal h_C keeps every site s whose box distance to C is at most
// r_C = min_s' |c - s'| + h_C: for any x in C the nearest site s* satisfies
// dist(s*, C) <= |x - s*| <= |x - s'| <= |c - s'| + h_C, so s* (and every
// site tied with it) is a candidate.  r_C is inflated by a relative 1e-6 so
// that a point the walk's own rounding puts just outside its cell, and a
// site the walk precision finds nearest, are still covered: the scan of a
// cell's candidates (ascending index, strict <) returns what a scan of all
// sites in the same precision returns.  Points outside the grid scan all
// sites.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "wos.h"

namespace wos {

struct VoronoiGrid {
    int32_t g[3] = {1, 1, 1};   // cells per axis (unused axes 1)
    double lo[3] = {0, 0, 0};   // origin
    double h = 1.0;             // cell size
    std::vector<int32_t> start; // ncell + 1 offsets into cand
    std::vector<int32_t> cand;  // candidate sites per cell, ascending
};

inline void voronoi_bbox(const wos_domain &d, const wos_partition &p, double *lo, double *hi)
{
    const int dim = d.dim;
    for (int a = 0; a < 3; ++a) {
        lo[a] = 0.0;
        hi[a] = 0.0;
    }
    for (int a = 0; a < dim; ++a) {
        if (d.outer_kind == WOS_OUTER_SPHERE) {
            lo[a] = d.center[a] - d.radius;
            hi[a] = d.center[a] + d.radius;
        } else if (d.outer_kind == WOS_OUTER_BOX) {
            lo[a] = d.center[a] - d.half[a];
            hi[a] = d.center[a] + d.half[a];
        } else {
            lo[a] = hi[a] = d.vertices[a];
            for (int v = 1; v < d.n_vertices; ++v) {
                lo[a] = std::min(lo[a], d.vertices[2 * v + a]);
                hi[a] = std::max(hi[a], d.vertices[2 * v + a]);
            }
        }
        for (int s = 0; s < p.voronoi_n; ++s) {
            lo[a] = std::min(lo[a], p.voronoi_sites[size_t(s) * dim + a]);
            hi[a] = std::max(hi[a], p.voronoi_sites[size_t(s) * dim + a]);
        }
    }
}

// Builds the grid; false when the sites are too few for a grid to pay.
inline bool build_voronoi_grid(const wos_domain &d, const wos_partition &p, VoronoiGrid *G)
{
    const int dim = d.dim, n = p.voronoi_n;
    if (n < 32)
        return false;
    double lo[3], hi[3], ext = 0.0;
    voronoi_bbox(d, p, lo, hi);
    for (int a = 0; a < dim; ++a)
        ext = std::max(ext, hi[a] - lo[a]);
    const double pad = 1e-3 * ext;
    const int gmax = dim == 2 ? std::min(256, std::max(4, int(std::lround(std::sqrt(4.0 * n)))))
                              : std::min(64, std::max(4, int(std::lround(std::cbrt(8.0 * n)))));
    const double h = (ext + 2 * pad) / gmax;
    size_t ncell = 1;
    for (int a = 0; a < 3; ++a) {
        if (a < dim) {
            G->lo[a] = lo[a] - pad;
            G->g[a] = std::max(1, int(std::ceil((hi[a] - lo[a] + 2 * pad) / h)));
        } else {
            G->lo[a] = 0.0;
            G->g[a] = 1;
        }
        ncell *= size_t(G->g[a]);
    }
    G->h = h;
    const double *S = p.voronoi_sites;
    auto cell_index = [&](const double *x, int *c) {
        for (int a = 0; a < 3; ++a) {
            c[a] = a < dim ? int(std::floor((x[a] - G->lo[a]) / h)) : 0;
            c[a] = std::min(std::max(c[a], 0), G->g[a] - 1);
        }
    };
    // sites bucketed by cell (CSR, ascending site index within a bucket)
    std::vector<int32_t> bstart(ncell + 1, 0), bsite(n);
    std::vector<int32_t> scell(n);
    for (int s = 0; s < n; ++s) {
        int c[3];
        cell_index(S + size_t(s) * dim, c);
        scell[s] = (c[2] * G->g[1] + c[1]) * G->g[0] + c[0];
        ++bstart[scell[s] + 1];
    }
    for (size_t q = 0; q < ncell; ++q)
        bstart[q + 1] += bstart[q];
    {
        std::vector<int32_t> fill(bstart.begin(), bstart.end() - 1);
        for (int s = 0; s < n; ++s)
            bsite[fill[scell[s]]++] = s;
    }
    const int gz = G->g[2], gy = G->g[1], gx = G->g[0];
    const double half_diag = 0.5 * h * std::sqrt(double(dim));
    auto visit_ring = [&](int cx, int cy, int cz, int r, auto &&fn) {
        for (int z = std::max(0, cz - r); z <= std::min(gz - 1, cz + r); ++z)
            for (int y = std::max(0, cy - r); y <= std::min(gy - 1, cy + r); ++y)
                for (int x = std::max(0, cx - r); x <= std::min(gx - 1, cx + r); ++x) {
                    int cheb = std::max({std::abs(z - cz), std::abs(y - cy), std::abs(x - cx)});
                    if (cheb != r)
                        continue;
                    size_t q = (size_t(z) * gy + y) * gx + x;
                    for (int32_t b = bstart[q]; b < bstart[q + 1]; ++b)
                        fn(bsite[b]);
                }
    };
    const int rmax = std::max({gx, gy, gz});
    G->start.assign(ncell + 1, 0);
    G->cand.clear();
    std::vector<int32_t> tmp;
    for (int cz = 0; cz < gz; ++cz)
        for (int cy = 0; cy < gy; ++cy)
            for (int cx = 0; cx < gx; ++cx) {
                const int ci[3] = {cx, cy, cz};
                double c[3], blo[3], bhi[3];
                for (int a = 0; a < 3; ++a) {
                    blo[a] = G->lo[a] + ci[a] * h;
                    bhi[a] = blo[a] + h;
                    c[a] = blo[a] + 0.5 * h;
                }
                // nearest-site distance from the centre (ring search: a site
                // in ring r' is at least (r' - 1/2) h from the centre)
                double best = INFINITY;
                for (int r = 0; r <= rmax; ++r) {
                    visit_ring(cx, cy, cz, r, [&](int s) {
                        double q2 = 0.0;
                        for (int a = 0; a < dim; ++a) {
                            double t = c[a] - S[size_t(s) * dim + a];
                            q2 += t * t;
                        }
                        best = std::min(best, std::sqrt(q2));
                    });
                    if (best <= (r + 0.5) * h)
                        break;
                }
                const double rc = (best + half_diag) * (1.0 + 1e-6) + 1e-6 * ext;
                const int rings = int(std::floor(rc / h)) + 1;
                tmp.clear();
                for (int r = 0; r <= std::min(rings, rmax); ++r)
                    visit_ring(cx, cy, cz, r, [&](int s) {
                        double q2 = 0.0;
                        for (int a = 0; a < dim; ++a) {
                            double v = S[size_t(s) * dim + a];
                            double t = v < blo[a] ? blo[a] - v : (v > bhi[a] ? v - bhi[a] : 0.0);
                            q2 += t * t;
                        }
                        if (std::sqrt(q2) <= rc)
                            tmp.push_back(s);
                    });
                std::sort(tmp.begin(), tmp.end());
                const size_t q = (size_t(cz) * gy + cy) * gx + cx;
                G->cand.insert(G->cand.end(), tmp.begin(), tmp.end());
                G->start[q + 1] = int32_t(G->cand.size());
            }
    return true;
}

}  // namespace wos
