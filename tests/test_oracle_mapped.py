"""Pins of the oracle's mapped chain (walk-on-spheres in y = S^{-1} x with
the exact distance to the polytope S^{-1} D; boxes and convex polygons):

* the face-plane distance min_f (d_f - n_f . y) equals the brute-force
  distance to densely sampled, mapped boundary points;
* the mapped chain and the paper's chain (Euclidean distance, ellipsoid
  steps, Sec. 4.2) sample the same elliptic measure: two-sample chi-square
  per row of their counts (Bonferroni over rows);
* the martingale identity E[u(X_tau)] = u(x) holds for K-harmonic cubics;
* for anisotropic K the mapped chain needs far fewer steps;
* domains it does not cover are rejected.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2409_03686_gb300 import workloads as W
from test_oracle_pins import _harmonic_check

K_RAND3 = W.random_spd(np.random.default_rng(6), 3, 0.5, 4.0)
HEXAGON = tuple((0.9 * math.cos(t), 0.6 * math.sin(t))
                for t in np.linspace(0, 2 * math.pi, 7)[:-1] + 0.3)


def _hexagon(N=2000, K=None):
    dom = W.Domain(dim=2, outer="polygon", vertices=HEXAGON)
    part = W.Partition(edge_m=(8,) * 6)
    part.gamma1 = (np.arange(48) >= 24).astype(np.uint8)
    pts = np.random.default_rng(3).uniform(-0.3, 0.3, (6, 2))
    return W.Instance("hexagon", dom, part, W.K_CONFIG2 if K is None else K, pts, N=N,
                      eps=1e-5, seed=5)


CASES = {
    "square": lambda: W.square_config(N=2000, grid=4),
    "cube_diag": lambda: W.cube_config(N=1000, n_points=8, n_face=4),
    "cube_rand": lambda: W.cube_config(N=1000, n_points=8, n_face=4, K=K_RAND3),
    "hexagon": lambda: _hexagon(),
}


def _boundary_samples(inst, n=80):
    dom = inst.domain
    if dom.outer == "polygon":
        v = np.asarray(dom.vertices)
        t = (np.arange(n) + 0.5) / n
        return np.concatenate([v[e] + t[:, None] * (v[(e + 1) % len(v)] - v[e])
                               for e in range(len(v))])
    d = dom.dim
    c, h = np.asarray(dom.center[:d]), np.asarray(dom.half[:d])
    out = []
    g = np.linspace(-1, 1, n)
    for a in range(d):
        for sgn in (-1, 1):
            if d == 2:
                p = np.zeros((n, 2))
                p[:, a] = sgn
                p[:, 1 - a] = g
            else:
                b0, b1 = [x for x in range(3) if x != a]
                G0, G1 = np.meshgrid(g, g)
                p = np.zeros((n * n, 3))
                p[:, a] = sgn
                p[:, b0] = G0.ravel()
                p[:, b1] = G1.ravel()
            out.append(c + p * h)
    return np.concatenate(out)


@pytest.mark.parametrize("name", list(CASES))
def test_plane_distance_against_brute_force(name):
    inst = CASES[name]()
    S, _ = O.setup_S(inst.K)
    Sinv = np.linalg.inv(S)
    pn, pd = O.mapped_planes(inst.domain, S)
    yb = _boundary_samples(inst) @ Sinv.T
    rng = np.random.default_rng(2)
    x = inst.points[:6] + 0.05 * rng.standard_normal((6, inst.dim))
    for y in x @ Sinv.T:
        dist = np.min(pd - pn @ y)
        brute = np.min(np.linalg.norm(yb - y, axis=1))
        spacing = 2.5 * np.max(np.linalg.norm(np.diff(yb[:80], axis=0), axis=1))
        assert dist <= brute + 1e-12
        assert dist >= brute - spacing


@pytest.mark.parametrize("name", ["square", "cube_rand", "hexagon"])
def test_mapped_and_paper_chains_sample_the_same_measure(name):
    inst = CASES[name]().replace(N=40_000)
    inst = inst.replace(points=inst.points[:4])
    Ca, _, sa = O.build_counts(inst)
    Cb, _, sb = O.build_counts(inst.replace(mapped=True, seed=inst.seed + 1))
    groups = 12
    M = Ca.shape[1]
    edges = np.linspace(0, M, groups + 1).astype(int)
    pvals = []
    for i in range(Ca.shape[0]):
        a = np.add.reduceat(Ca[i].astype(float), edges[:-1])
        b = np.add.reduceat(Cb[i].astype(float), edges[:-1])
        keep = (a + b) > 0
        chi2 = np.sum((a[keep] - b[keep]) ** 2 / (a[keep] + b[keep]))
        pvals.append(stats.chi2.sf(chi2, keep.sum() - 1))
    assert min(pvals) > 1e-3 / len(pvals), pvals


def test_mapped_martingale_on_k_harmonic_cubics():
    for K in (W.K_CONFIG2, np.array([[1.0, -0.6], [-0.6, 0.5]])):
        u = W.k_harmonic_cubic(K)
        sq = W.square_config(N=4000, grid=3, K=K).replace(mapped=True, eps=1e-4)
        _harmonic_check(sq, u, 4000)
        hx = _hexagon(K=K).replace(mapped=True, eps=1e-4)
        _harmonic_check(hx, u, 4000)
    for K in (W.K_DIAG124, K_RAND3):
        u = W.k_harmonic_cubic(K)
        cb = W.cube_config(N=3000, n_points=4, K=K).replace(mapped=True)
        _harmonic_check(cb, u, 3000)


def test_mapped_chain_needs_fewer_steps_for_anisotropic_k():
    for inst in (CASES["square"](), CASES["cube_diag"]()):
        _, _, sa = O.build_counts(inst)
        _, _, sb = O.build_counts(inst.replace(mapped=True))
        assert sb < 0.6 * sa, (inst.name, sa, sb)


def test_unsupported_domains_are_rejected():
    S = np.eye(2)
    with pytest.raises(ValueError):
        O.mapped_planes(W.lshape_config().domain, S)      # not convex
    with pytest.raises(ValueError):
        O.mapped_planes(W.annulus_config().domain, S)     # sphere with a hole
    with pytest.raises(ValueError):
        O.mapped_planes(W.square_hole_config().domain, S)  # hole


# ---------------------------------------------------------------------------
# The mapped chain on discs / balls minus holes: the step radius is the
# quadric lower bound of dist_y (oracle/wos_oracle.c, orc_quadric_radius).
# ---------------------------------------------------------------------------
def _curved(name):
    return {
        "annulus": lambda: W.annulus_config(N=3000, grid=4),
        "ball_diag": lambda: W.ball_config(N=1500, n_points=8, nb=4, ns=6),
        "ball_rand": lambda: W.ball_config(N=1500, n_points=8, nb=4, ns=6, K=K_RAND3),
        "shell_shifted": lambda: W.shell_config(N=1500, shift=0.3, n_points=8, nb=4, ns=6,
                                                K=K_RAND3),
        "perforated": lambda: W.perforated_disc_config(N=3000, eps=1e-5, m_outer=20, m_hole=4,
                                                       n_points=8).replace(K=W.K_CONFIG2),
    }[name]()


def _curved_boundary(dom, n):
    """Dense samples of dD (outer circle / sphere and the holes)."""
    d = dom.dim
    comps = [(np.asarray(dom.center[:d]), dom.radius)] + [
        (np.asarray(c[:d]), r) for c, r in dom.holes]
    out = []
    for c, r in comps:
        if d == 2:
            t = np.linspace(0, 2 * math.pi, n, endpoint=False)
            out.append(c + r * np.stack([np.cos(t), np.sin(t)], 1))
        else:
            k = np.arange(n) + 0.5          # Fibonacci sphere
            z = 1 - 2 * k / n
            phi = math.pi * (1 + 5 ** 0.5) * k
            s = np.sqrt(1 - z * z)
            out.append(c + r * np.stack([s * np.cos(phi), s * np.sin(phi), z], 1))
    return np.concatenate(out)


@pytest.mark.parametrize("name", ["annulus", "ball_diag", "ball_rand", "shell_shifted",
                                  "perforated"])
def test_quadric_radius_is_a_tight_lower_bound_of_dist_y(name):
    """dist_x <= radius <= dist_y (brute force over dense samples of the
    mapped boundary), and at points 1e-3 from dD the radius is within 2 % of
    dist_y (first-order exact at the boundary)."""
    inst = _curved(name)
    S, _ = O.setup_S(inst.K)
    Sinv = np.linalg.inv(S)
    yb = _curved_boundary(inst.domain, 400_000 if inst.dim == 2 else 300_000) @ Sinv.T
    rng = np.random.default_rng(7)
    x = inst.points[:6] + 0.02 * rng.standard_normal((6, inst.dim))
    dx = O.dist(inst.domain, inst.partition, x)
    ok = dx > 0
    x, dx = x[ok], dx[ok]
    rad = O.mapped_radius(inst, x)
    brute = np.array([np.min(np.linalg.norm(yb - y, axis=1)) for y in x @ Sinv.T])
    assert np.all(rad >= dx - 1e-15)
    assert np.all(rad <= brute + 1e-12), (rad, brute)
    # near the outer boundary: move points to 1e-3 from it along the radius
    c = np.asarray(inst.domain.center[:inst.dim])
    v = x - c
    near = c + v / np.linalg.norm(v, axis=1)[:, None] * (inst.domain.radius - 1e-3)
    rn = O.mapped_radius(inst, near)
    bn = np.array([_refined_dist_y(inst, Sinv, yb, y) for y in near @ Sinv.T])
    assert np.all(rn <= bn + 1e-12)
    assert np.all(rn >= 0.98 * bn), rn / bn


def _refined_dist_y(inst, Sinv, yb, y):
    """dist_y to the mapped outer boundary: the nearest dense sample, then a
    local minimisation over the circle's angle / the sphere's two angles."""
    from scipy import optimize
    d = inst.dim
    c, R = np.asarray(inst.domain.center[:d]), inst.domain.radius
    if d == 2:
        f = lambda t: np.linalg.norm(y - Sinv @ (c + R * np.array([np.cos(t[0]), np.sin(t[0])])))
    else:
        f = lambda t: np.linalg.norm(y - Sinv @ (c + R * np.array(
            [np.sin(t[0]) * np.cos(t[1]), np.sin(t[0]) * np.sin(t[1]), np.cos(t[0])])))
    xb = yb @ np.linalg.inv(Sinv).T - c
    q = np.argmin(np.linalg.norm(yb - y, axis=1))
    v = xb[q] / np.linalg.norm(xb[q])
    t0 = [math.atan2(v[1], v[0])] if d == 2 else [math.acos(np.clip(v[2], -1, 1)),
                                                   math.atan2(v[1], v[0])]
    res = optimize.minimize(f, t0, method="Nelder-Mead",
                            options=dict(xatol=1e-12, fatol=1e-15, maxiter=20000))
    return min(res.fun, f(t0))


def test_quadric_radius_is_the_distance_for_isotropic_k():
    """With K = I the bounds are R - rho and rho - r exactly."""
    for inst in (W.annulus_config(N=10, grid=4, K=np.eye(2)),
                 W.shell_config(N=10, shift=0.3, n_points=8, nb=4, ns=6)):
        x = inst.points
        np.testing.assert_allclose(O.mapped_radius(inst, x),
                                   O.dist(inst.domain, inst.partition, x), rtol=1e-14)


@pytest.mark.parametrize("name", ["annulus", "ball_rand", "shell_shifted"])
def test_quadric_chain_samples_the_paper_chains_measure(name):
    inst = _curved(name).replace(N=40_000)
    inst = inst.replace(points=inst.points[:4])
    Ca, _, _ = O.build_counts(inst)
    Cb, _, _ = O.build_counts(inst.replace(mapped=True, seed=inst.seed + 1))
    groups = 12
    edges = np.linspace(0, Ca.shape[1], groups + 1).astype(int)
    pvals = []
    for i in range(Ca.shape[0]):
        a = np.add.reduceat(Ca[i].astype(float), edges[:-1])
        b = np.add.reduceat(Cb[i].astype(float), edges[:-1])
        keep = (a + b) > 0
        chi2 = np.sum((a[keep] - b[keep]) ** 2 / (a[keep] + b[keep]))
        pvals.append(stats.chi2.sf(chi2, keep.sum() - 1))
    assert min(pvals) > 1e-3 / len(pvals), pvals


def test_quadric_chain_martingale_and_fewer_steps():
    """E[u(X_tau)] = u(x) for K-harmonic cubics; and far fewer steps than the
    paper's chain for anisotropic K (the annulus and the ball of the
    benchmark configurations)."""
    for name in ("annulus", "ball_rand", "shell_shifted"):
        inst = _curved(name)
        _harmonic_check(inst.replace(mapped=True, eps=1e-4), W.k_harmonic_cubic(inst.K),
                        inst.N)
    for name in ("annulus", "ball_diag"):
        inst = _curved(name)
        _, _, sa = O.build_counts(inst)
        _, _, sb = O.build_counts(inst.replace(mapped=True))
        assert sb < 0.7 * sa, (name, sa, sb)
