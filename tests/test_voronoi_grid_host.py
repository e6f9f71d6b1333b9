"""Host logic of the extrinsic-Voronoi candidate grid (App. A, Ex. A.2):
for random points in and around the domain, the nearest site found by
scanning the candidates of the point's grid cell (ascending index, strict <)
equals the brute-force nearest site with the lowest index on ties, in FP32
and in FP64, for Bauer-spiral sites on a shell and sites on two circles."""
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <vector>
#include "voronoi_grid.h"

template <typename Real>
int nearest_all(const double *S, int n, int dim, const Real *x) {
    Real best = Real(INFINITY); int bj = 0;
    for (int j = 0; j < n; ++j) {
        Real s = 0;
        for (int a = 0; a < dim; ++a) { Real d = x[a] - Real(S[j * dim + a]); s += d * d; }
        if (s < best) { best = s; bj = j; }
    }
    return bj;
}

template <typename Real>
int nearest_grid(const wos::VoronoiGrid &G, const double *S, int n, int dim, const Real *x) {
    int c = 0; bool inside = true;
    Real inv_h = Real(1.0 / G.h);
    for (int a = dim - 1; a >= 0; --a) {
        Real t = (x[a] - Real(G.lo[a])) * inv_h;
        int q = int(std::floor(t));
        inside = inside && t >= Real(0) && q < G.g[a];
        c = c * G.g[a] + q;
    }
    if (!inside) return nearest_all(S, n, dim, x);
    Real best = Real(INFINITY); int bj = 0;
    for (int q = G.start[c]; q < G.start[c + 1]; ++q) {
        int j = G.cand[q];
        Real s = 0;
        for (int a = 0; a < dim; ++a) { Real d = x[a] - Real(S[j * dim + a]); s += d * d; }
        if (s < best) { best = s; bj = j; }
    }
    return bj;
}

int main(int argc, char **argv) {
    // stdin: dim n_sites n_points, outer kind (0 sphere, 1 box), centre, radius/half, sites, points
    int dim, n, m, kind;
    if (scanf("%d %d %d %d", &dim, &n, &m, &kind) != 4) return 2;
    wos_domain d = {};
    d.dim = dim;
    d.outer_kind = kind == 0 ? WOS_OUTER_SPHERE : WOS_OUTER_BOX;
    for (int a = 0; a < 3; ++a) if (scanf("%lf", &d.center[a]) != 1) return 2;
    if (scanf("%lf", &d.radius) != 1) return 2;
    for (int a = 0; a < 3; ++a) d.half[a] = d.radius;
    std::vector<double> S(size_t(n) * dim), X(size_t(m) * dim);
    for (auto &v : S) if (scanf("%lf", &v) != 1) return 2;
    for (auto &v : X) if (scanf("%lf", &v) != 1) return 2;
    wos_partition p = {};
    p.voronoi_n = n;
    p.voronoi_sites = S.data();
    wos::VoronoiGrid G;
    if (!wos::build_voronoi_grid(d, p, &G)) { printf("nogrid\n"); return 0; }
    long bad32 = 0, bad64 = 0;
    for (int i = 0; i < m; ++i) {
        float xf[3]; double xd[3];
        for (int a = 0; a < dim; ++a) { xd[a] = X[i * dim + a]; xf[a] = float(xd[a]); }
        bad32 += nearest_grid<float>(G, S.data(), n, dim, xf) != nearest_all<float>(S.data(), n, dim, xf);
        bad64 += nearest_grid<double>(G, S.data(), n, dim, xd) != nearest_all<double>(S.data(), n, dim, xd);
    }
    printf("%ld %ld %zu %zu\n", bad32, bad64, G.start.size() - 1, G.cand.size());
    return 0;
}
"""


def _bauer(n, R, c):
    k = np.arange(1, n + 1)
    phi = np.arccos(1 - (2 * k - 1) / n)
    th = np.sqrt(n * np.pi) * phi
    return np.asarray(c)[None, :] + R * np.stack(
        [np.sin(phi) * np.cos(th), np.sin(phi) * np.sin(th), np.cos(phi)], 1)


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("vgrid")
    src = d / "vgrid.cpp"
    src.write_text(DRIVER)
    exe = d / "vgrid"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", str(ROOT / "include"),
                    "-I", str(ROOT / "paper_2409_03686_gb300" / "csrc"), str(src), "-o",
                    str(exe)], check=True)
    return exe


def _run(exe, dim, sites, pts, kind=0, center=(0, 0, 0), radius=1.0):
    lines = [f"{dim} {len(sites)} {len(pts)} {kind}", " ".join(map(str, center)), str(radius)]
    lines += [" ".join(repr(float(v)) for v in s) for s in sites]
    lines += [" ".join(repr(float(v)) for v in x) for x in pts]
    out = subprocess.run([str(exe)], input="\n".join(lines), capture_output=True, text=True,
                         check=True).stdout.split()
    return [int(v) for v in out]


def test_shell_bauer_sites(driver):
    rng = np.random.default_rng(3)
    sites = np.concatenate([_bauer(1000, 1.0, (0, 0, 0)), _bauer(100, 0.5, (0.3, 0, 0))])
    # points near both spheres (where walks stop), inside the ball and outside it
    u = rng.standard_normal((6000, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    near = np.concatenate([u[:3000] * (1 - 1e-4 * rng.random((3000, 1))),
                           np.array([0.3, 0, 0]) + 0.5 * u[3000:] * (1 + 1e-4 * rng.random((3000, 1)))])
    far = rng.uniform(-1.2, 1.2, (2000, 3))
    bad32, bad64, ncell, ncand = _run(driver, 3, sites, np.concatenate([near, far]))
    assert bad32 == 0 and bad64 == 0
    assert ncand < 40 * ncell  # the lists are short


def test_circle_sites_with_exact_ties(driver):
    rng = np.random.default_rng(4)
    th = 2 * np.pi * np.arange(400) / 400
    sites = np.concatenate([np.stack([np.cos(th), np.sin(th)], 1),
                            0.2 * np.stack([np.cos(th[:50] * 8), np.sin(th[:50] * 8)], 1)
                            + np.array([0.5, 0.0])])
    sites = np.concatenate([sites, sites[:10]])  # duplicated sites: exact ties
    mids = 0.5 * (sites[:-11] + sites[1:-10])    # equidistant from two sites
    pts = np.concatenate([mids, rng.uniform(-1.1, 1.1, (4000, 2))])
    bad32, bad64, ncell, ncand = _run(driver, 2, sites, pts)
    assert bad32 == 0 and bad64 == 0
