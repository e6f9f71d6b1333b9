"""Closed-form elliptic (harmonic) measures used to pin the oracle.

TEST INFRASTRUCTURE ONLY.  These are textbook potential-theory formulas, not
the Monte Carlo method; they are what the walks must reproduce.

* Disc (K = I): the Poisson kernel of the ball stated in the paper's Sec. 1,
  d mu_x / d sigma = (1 - |x|^2) / (sigma(dB) |x - y|^d).  In 2-D its
  antiderivative in the boundary angle is continuous:
  H(psi) = psi + 2 atan(rho sin psi / (1 - rho cos psi)), psi = theta - phi,
  so an arc [alpha, beta] has measure (H(beta - phi) - H(alpha - phi)) / 2 pi.
* Ball (K = I, d = 3): the same kernel integrated over a z-band x phi-sector
  patch by tensor Gauss-Legendre (area element dz dphi on the unit sphere).
* Concentric annulus / shell (K = I): mu_x(inner) = ln r / ln a in 2-D and
  (1/r - 1) / (1/a - 1) in 3-D (harmonic in r, 1 / 0 on the circles / spheres);
  per-arc measures of the annulus from the Fourier series of the Dirichlet
  problem (the paper's Sec. 1 remark that the annulus needs an infinite sum).
* Unit square and a x b rectangle (K = I): harmonic measure of one side by
  the sine series of separation of variables; a box's face by the double
  sine series.
"""
from __future__ import annotations

import math

import numpy as np


def disc_arc_measure(x, alpha, beta, center=(0.0, 0.0), R=1.0):
    """mu_x([alpha, beta]) on the circle |y - c| = R (2-D, K = I)."""
    x = np.asarray(x, float) - np.asarray(center[:2], float)
    rho = math.hypot(x[0], x[1]) / R
    phi = math.atan2(x[1], x[0])

    def H(psi):
        return psi + 2.0 * math.atan(rho * math.sin(psi) / (1.0 - rho * math.cos(psi)))
    return (H(beta - phi) - H(alpha - phi)) / (2.0 * math.pi)


def disc_row(x, m, theta0=0.0, center=(0.0, 0.0), R=1.0):
    edges = theta0 + 2 * math.pi * np.arange(m + 1) / m
    return np.array([disc_arc_measure(x, edges[j], edges[j + 1], center, R)
                     for j in range(m)])


def ball_patch_row(x, nb, ns, n_gl: int = 24):
    """mu_x of every z-band x phi-sector patch of the unit sphere (K = I),
    patch index band * ns + sector, band 0 at the south pole."""
    x = np.asarray(x, float)
    g, w = np.polynomial.legendre.leggauss(n_gl)
    out = np.zeros(nb * ns)
    r2 = float(x @ x)
    for b in range(nb):
        z0, z1 = -1 + 2 * b / nb, -1 + 2 * (b + 1) / nb
        zs = 0.5 * (z1 - z0) * g + 0.5 * (z1 + z0)
        wz = 0.5 * (z1 - z0) * w
        for s in range(ns):
            p0, p1 = 2 * math.pi * s / ns, 2 * math.pi * (s + 1) / ns
            ps = 0.5 * (p1 - p0) * g + 0.5 * (p1 + p0)
            wp = 0.5 * (p1 - p0) * w
            Z, P = np.meshgrid(zs, ps, indexing="ij")
            sr = np.sqrt(1 - Z ** 2)
            y = np.stack([sr * np.cos(P), sr * np.sin(P), Z], -1)
            dist3 = np.linalg.norm(y - x, axis=-1) ** 3
            kern = (1 - r2) / (4 * math.pi * dist3)
            out[b * ns + s] = float(np.einsum("i,j,ij->", wz, wp, kern))
    return out


def annulus_inner_total(r, a):
    """mu_x(inner circle |y| = a) for the annulus a < |x| < 1, K = I."""
    return math.log(r) / math.log(a)


def shell_inner_total(r, a):
    """mu_x(inner sphere |y| = a) for the shell a < |x| < 1, K = I."""
    return (1.0 / r - 1.0) / (1.0 / a - 1.0)


def annulus_arc_measures(x, a, m_outer, m_inner, theta0_outer=0.0,
                         theta0_inner=0.0, n_terms: int = 4000):
    """Per-arc harmonic measures on the concentric annulus a < |x| < 1 (K=I).

    u solves the Dirichlet problem with data 1_arc on one circle and 0 on the
    other: radial parts (r^n - r^-n) / (a^n - a^-n) for inner data and
    (r^n - a^{2n} r^-n) / (1 - a^{2n}) for outer data, and ln r / ln a,
    1 - ln r / ln a for n = 0."""
    x = np.asarray(x, float)
    r = math.hypot(x[0], x[1])
    th = math.atan2(x[1], x[0])
    n = np.arange(1, n_terms + 1, dtype=float)
    # radial factors computed in a form that cannot overflow
    with np.errstate(over="ignore", under="ignore"):
        inner_f = (a / r) ** n * (1 - (r * r) ** n) / (1 - (a * a) ** n)
        outer_f = r ** n * (1 - (a * a / (r * r)) ** n) / (1 - (a * a) ** n)

    def arcs(m, th0, radial, mean):
        e = th0 + 2 * math.pi * np.arange(m + 1) / m
        res = np.empty(m)
        for j in range(m):
            al, be = e[j], e[j + 1]
            an = (np.sin(n * be) - np.sin(n * al)) / (n * math.pi)
            bn = (np.cos(n * al) - np.cos(n * be)) / (n * math.pi)
            res[j] = mean * (be - al) / (2 * math.pi) + float(
                np.sum(radial * (an * np.cos(n * th) + bn * np.sin(n * th))))
        return res
    p_in = math.log(r) / math.log(a)
    return np.concatenate([arcs(m_outer, theta0_outer, outer_f, 1 - p_in),
                           arcs(m_inner, theta0_inner, inner_f, p_in)])


def rectangle_side_measure(x, y, a: float, b: float, n_terms: int = 4001):
    """Harmonic measure (K = I) of the bottom side of the rectangle [0,a] x
    [0,b] seen from (x, y): separation of variables for Laplace's equation
    with data 1 on y = 0 and 0 on the other sides, sum over odd n of
    4/(n pi) sin(n pi x / a) sinh(n pi (b - y) / a) / sinh(n pi b / a)
    (the sinh ratio written with decaying exponentials)."""
    n = np.arange(1, n_terms + 1, 2, dtype=float)
    k = n * math.pi / a
    ratio = np.exp(-k * y) * (1 - np.exp(-2 * k * (b - y))) / (1 - np.exp(-2 * k * b))
    return float(np.sum(4 / (n * math.pi) * np.sin(k * x) * ratio))


def box_face_measure(u, v, w, a: float, b: float, c: float, n_terms: int = 401,
                     cell=None):
    """Harmonic measure (K = I) of the face w = 0 of the box [0,a] x [0,b] x
    [0,c], or of its sub-rectangle cell = (u0, u1, v0, v1), seen from the
    point with in-face coordinates (u, v) and distance w from that face: the
    double sine series of separation of variables, sum over m, n of
    A_m B_n sin(m pi u / a) sin(n pi v / b) sinh(g (c - w)) / sinh(g c),
    g = pi sqrt((m/a)^2 + (n/b)^2), A_m = 2/(m pi) (cos(m pi u0 / a) -
    cos(m pi u1 / a)) the sine coefficients of the cell's indicator (4/(m pi)
    for odd m and 0 for even m on the whole face), B_n likewise."""
    u0, u1, v0, v1 = cell if cell is not None else (0.0, a, 0.0, b)
    m = np.arange(1, n_terms + 1, dtype=float)[:, None]
    n = np.arange(1, n_terms + 1, dtype=float)[None, :]
    A = 2 / (m * math.pi) * (np.cos(m * math.pi * u0 / a) - np.cos(m * math.pi * u1 / a))
    B = 2 / (n * math.pi) * (np.cos(n * math.pi * v0 / b) - np.cos(n * math.pi * v1 / b))
    g = math.pi * np.sqrt((m / a) ** 2 + (n / b) ** 2)
    ratio = np.exp(-g * w) * (1 - np.exp(-2 * g * (c - w))) / (1 - np.exp(-2 * g * c))
    terms = A * B * np.sin(m * math.pi * u / a) * np.sin(n * math.pi * v / b) * ratio
    return float(terms.sum())


def square_side_measure(x, y, n_terms: int = 2001):
    """Harmonic measure (K = I) of the bottom side of the unit square [0,1]^2
    seen from (x, y): sum over odd n of 4/(n pi) sin(n pi x) sinh(n pi (1-y))
    / sinh(n pi)."""
    n = np.arange(1, n_terms + 1, 2, dtype=float)
    ratio = np.exp(-n * math.pi * y) * (1 - np.exp(-2 * n * math.pi * (1 - y))) / (
        1 - np.exp(-2 * n * math.pi))
    return float(np.sum(4 / (n * math.pi) * np.sin(n * math.pi * x) * ratio))
