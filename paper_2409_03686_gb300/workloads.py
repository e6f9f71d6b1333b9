"""Seeded synthetic workloads shaped like the paper's experiments.

This module only *describes* inputs: domains, boundary partitions, the
conductivity K, observation points and synthetic measurements.  It holds none
of the method's arithmetic (no distance, walk, classification, tally or SVD).
Both the CUDA path and the CPU oracle take their inputs from here, so the two
sides see identical data.

Geometry conventions (the element order is part of the interface):

* ``Domain`` is an outer body (``sphere`` = disc in 2-D / ball in 3-D, ``box``
  or ``polygon``) minus disjoint holes (discs / balls).  Boundary components are
  ordered outer first, then the holes in the given order.
* circle: ``m`` arcs counter-clockwise from ``theta0``; arc j covers
  [theta0 + 2 pi j / m, theta0 + 2 pi (j+1) / m).
* polygon: vertices counter-clockwise; edge e runs v_e -> v_{e+1}, split in
  ``edge_m[e]`` equal cells.  A 2-D box is the polygon whose first vertex is
  the corner (c - h): edges bottom, right, top, left.
* sphere: ``nb`` equal-height z-bands (equal area, Archimedes) from the south
  pole, times ``ns`` equal phi-sectors from phi = 0; cell = band * ns + sector.
* 3-D box: faces -x, -y, -z, +x, +y, +z, each an ``n1 x n2`` grid over its two
  other axes in increasing axis order.

The six configurations follow the paper's Sec. 5.2-5.3 examples and the
benchmark configurations; the readings taken where the text leaves a detail
open are listed in the design notes.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Domain:
    dim: int
    outer: str  # "sphere" | "box" | "polygon"
    center: tuple = (0.0, 0.0, 0.0)
    radius: float = 1.0
    half: tuple = (1.0, 1.0, 1.0)
    vertices: tuple = ()  # polygon: ((x, y), ...) counter-clockwise
    holes: tuple = ()  # ((centre tuple, radius), ...)


@dataclass
class Partition:
    outer_m: int = 0
    outer_theta0: float = 0.0
    edge_m: tuple = ()
    outer_nb: int = 0
    outer_ns: int = 0
    face_n1: int = 0
    face_n2: int = 0
    hole_m: tuple = ()
    hole_theta0: tuple = ()
    hole_nb: tuple = ()
    hole_ns: tuple = ()
    voronoi_sites: np.ndarray | None = None  # App. A, Ex. A.2 sites
    gamma1: np.ndarray | None = None  # uint8 per element: 1 = Gamma_1


@dataclass
class Instance:
    name: str
    domain: Domain
    partition: Partition
    K: np.ndarray
    points: np.ndarray  # M_D x d, float64
    N: int
    eps: float
    seed: int
    stream: int = 0
    fp64: bool = False
    step_cap: int = 1_000_000
    nu: np.ndarray | None = None  # default 1/sqrt(M_D) (Sec. 5.2)
    mapped: bool = False  # walk-on-spheres in y = S^{-1} x (boxes, convex polygons)

    @property
    def dim(self) -> int:
        return self.domain.dim

    @property
    def M_D(self) -> int:
        return int(self.points.shape[0])

    @property
    def M_tot(self) -> int:
        return element_count(self.domain, self.partition)

    def nu_vec(self) -> np.ndarray:
        if self.nu is not None:
            return np.asarray(self.nu, dtype=np.float64)
        return np.full(self.M_D, 1.0 / math.sqrt(self.M_D))

    def replace(self, **kw) -> "Instance":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------
# partition bookkeeping (description only)
# ----------------------------------------------------------------------------
def _outer_count(dom: Domain, part: Partition) -> int:
    if dom.outer == "sphere":
        return part.outer_m if dom.dim == 2 else part.outer_nb * part.outer_ns
    if dom.outer == "box" and dom.dim == 3:
        return 6 * part.face_n1 * part.face_n2
    return int(sum(part.edge_m))


def _hole_count(dom: Domain, part: Partition, h: int) -> int:
    if dom.dim == 2:
        return int(part.hole_m[h])
    return int(part.hole_nb[h] * part.hole_ns[h])


def element_count(dom: Domain, part: Partition) -> int:
    if part.voronoi_sites is not None:
        return int(len(part.voronoi_sites))
    return _outer_count(dom, part) + sum(
        _hole_count(dom, part, h) for h in range(len(dom.holes)))


def box_polygon(center, half) -> tuple:
    cx, cy = center[0], center[1]
    hx, hy = half[0], half[1]
    return ((cx - hx, cy - hy), (cx + hx, cy - hy), (cx + hx, cy + hy),
            (cx - hx, cy + hy))


def element_centres(dom: Domain, part: Partition) -> np.ndarray:
    """Representative point x_j of every element (midpoint of its cell), used
    only to lay out labels and boundary data."""
    if part.voronoi_sites is not None:
        return np.asarray(part.voronoi_sites, dtype=np.float64)
    d = dom.dim
    out = []

    def circle(c, r, m, th0):
        t = th0 + 2 * np.pi * (np.arange(m) + 0.5) / m
        return np.stack([c[0] + r * np.cos(t), c[1] + r * np.sin(t)], 1)

    def sphere(c, r, nb, ns):
        z = -1 + 2 * (np.arange(nb) + 0.5) / nb
        ph = 2 * np.pi * (np.arange(ns) + 0.5) / ns
        Z, P = np.meshgrid(z, ph, indexing="ij")
        s = np.sqrt(1 - Z ** 2)
        pts = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
        return np.asarray(c[:3]) + r * pts

    def polygon(verts, em):
        res = []
        n = len(verts)
        for e in range(n):
            a = np.asarray(verts[e], float)
            b = np.asarray(verts[(e + 1) % n], float)
            t = (np.arange(em[e]) + 0.5) / em[e]
            res.append(a[None] + t[:, None] * (b - a)[None])
        return np.concatenate(res, 0)

    if dom.outer == "sphere":
        if d == 2:
            out.append(circle(dom.center, dom.radius, part.outer_m,
                              part.outer_theta0))
        else:
            out.append(sphere(dom.center, dom.radius, part.outer_nb,
                              part.outer_ns))
    elif dom.outer == "box" and d == 2:
        out.append(polygon(box_polygon(dom.center, dom.half), part.edge_m))
    elif dom.outer == "box":
        c = np.asarray(dom.center[:3], float)
        h = np.asarray(dom.half[:3], float)
        n1, n2 = part.face_n1, part.face_n2
        for f in range(6):
            ax = f % 3
            b0 = 1 if ax == 0 else 0
            b1 = 1 if ax == 2 else 2
            t0 = -1 + 2 * (np.arange(n1) + 0.5) / n1
            t1 = -1 + 2 * (np.arange(n2) + 0.5) / n2
            T0, T1 = np.meshgrid(t0, t1, indexing="ij")
            p = np.zeros((n1, n2, 3))
            p[..., ax] = (-1 if f < 3 else 1) * h[ax]
            p[..., b0] = T0 * h[b0]
            p[..., b1] = T1 * h[b1]
            out.append(c + p.reshape(-1, 3))
    else:
        out.append(polygon(dom.vertices, part.edge_m))
    for h, (hc, hr) in enumerate(dom.holes):
        if d == 2:
            out.append(circle(hc, hr, part.hole_m[h], part.hole_theta0[h]))
        else:
            out.append(sphere(hc, hr, part.hole_nb[h], part.hole_ns[h]))
    return np.concatenate(out, 0)


def element_component(dom: Domain, part: Partition) -> np.ndarray:
    """Boundary component (0 = outer, 1 + h = hole h) of every element."""
    n0 = _outer_count(dom, part)
    comp = [np.zeros(n0, np.int32)]
    for h in range(len(dom.holes)):
        comp.append(np.full(_hole_count(dom, part, h), h + 1, np.int32))
    return np.concatenate(comp)


# ----------------------------------------------------------------------------
# conductivities and synthetic exact solutions
# ----------------------------------------------------------------------------
def random_spd(rng: np.random.Generator, d: int, lo: float, hi: float
               ) -> np.ndarray:
    """Haar rotation (QR of a Gaussian matrix, sign-fixed) times eigenvalues
    log-uniform in [lo, hi]."""
    Q, R = np.linalg.qr(rng.standard_normal((d, d)))
    Q = Q * np.sign(np.diag(R))[None, :]
    lam = np.exp(rng.uniform(math.log(lo), math.log(hi), d))
    return (Q * lam[None, :]) @ Q.T


def k_harmonic_cubic(K: np.ndarray):
    """A polynomial u with div(K grad u) = 0.

    2-D: the cubic of the paper's Eq. (2D-sol4), whose coefficients are fixed
    by K: u = a x^3 - x^2 y + x y^2 - b y^3, a = (2 K12 - K22) / (3 K11),
    b = (2 K12 - K11) / (3 K22).
    3-D: h(K^{-1/2} x) with h the harmonic polynomial of Eq. (3D-sol1).
    """
    K = np.asarray(K, dtype=np.float64)
    if K.shape == (2, 2):
        a = (2 * K[0, 1] - K[1, 1]) / (3 * K[0, 0])
        b = (2 * K[0, 1] - K[0, 0]) / (3 * K[1, 1])

        def u(x):
            x = np.asarray(x, dtype=np.float64)
            X, Y = x[..., 0], x[..., 1]
            return a * X ** 3 - X ** 2 * Y + X * Y ** 2 - b * Y ** 3
        return u
    w, Vm = np.linalg.eigh(K)
    Kmh = (Vm / np.sqrt(w)[None, :]) @ Vm.T

    def u(x):
        y = np.asarray(x, dtype=np.float64) @ Kmh.T
        return y[..., 0] * y[..., 1] + y[..., 1] ** 2 - y[..., 2] ** 2
    return u


@dataclass
class Measurements:
    uD: np.ndarray  # at the observation points (noisy)
    u0: np.ndarray  # on the Gamma_0 elements (exact)
    g: np.ndarray  # exact values on the Gamma_1 elements (for reference)


def measurements(inst: Instance, noise: float = 0.0, seed: int = 3
                 ) -> Measurements:
    """Synthetic data from a K-harmonic cubic: u^D = u(x_i) (+ noise
    p * ||u^D||_inf * z, z ~ N(0, 1)), u^0 = u at the Gamma_0 element
    points."""
    u = k_harmonic_cubic(inst.K)
    xc = element_centres(inst.domain, inst.partition)
    g1 = inst.partition.gamma1.astype(bool)
    uD = u(inst.points)
    if noise > 0:
        rng = np.random.default_rng(seed)
        uD = uD + noise * np.max(np.abs(uD)) * rng.standard_normal(uD.shape)
    return Measurements(uD=uD, u0=u(xc[~g1]), g=u(xc[g1]))


# ----------------------------------------------------------------------------
# point sets
# ----------------------------------------------------------------------------
def _inside(dom: Domain, x: np.ndarray, margin: float = 0.0) -> np.ndarray:
    """Membership test used only for rejection sampling of input points."""
    c = np.asarray(dom.center[: dom.dim])
    if dom.outer == "sphere":
        ok = np.linalg.norm(x - c, axis=-1) < dom.radius - margin
    elif dom.outer == "box":
        h = np.asarray(dom.half[: dom.dim])
        ok = np.all(np.abs(x - c) < h - margin, axis=-1)
    else:  # polygon: crossing number (points far from edges only)
        v = np.asarray(dom.vertices, float)
        ok = np.zeros(len(x), bool)
        for e in range(len(v)):
            a, b = v[e], v[(e + 1) % len(v)]
            cond = (a[1] > x[:, 1]) != (b[1] > x[:, 1])
            xint = a[0] + (x[:, 1] - a[1]) * (b[0] - a[0]) / (b[1] - a[1] + 1e-300)
            ok ^= cond & (x[:, 0] < xint)
    for hc, hr in dom.holes:
        ok &= np.linalg.norm(x - np.asarray(hc[: dom.dim]), axis=-1) > hr + margin
    return ok


def uniform_points(dom: Domain, n: int, rng: np.random.Generator,
                   lo, hi, margin: float = 0.0) -> np.ndarray:
    pts = []
    need = n
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    while need > 0:
        x = rng.uniform(lo, hi, size=(4 * need + 16, dom.dim))
        x = x[_inside(dom, x, margin)]
        pts.append(x[:need])
        need -= len(pts[-1])
    return np.concatenate(pts, 0)


def circle_points(center, r, n, theta0=0.0) -> np.ndarray:
    t = theta0 + 2 * np.pi * np.arange(n) / n
    return np.stack([center[0] + r * np.cos(t), center[1] + r * np.sin(t)], 1)


def bauer_spiral(n: int, R: float = 1.0, center=(0.0, 0.0, 0.0)
                 ) -> np.ndarray:
    """n points on the Bauer spherical spiral (paper, Sec. 5.3):
    phi_k = arccos(1 - (2k - 1)/n), theta_k = sqrt(n pi) phi_k."""
    k = np.arange(1, n + 1)
    phi = np.arccos(1 - (2 * k - 1) / n)
    th = np.sqrt(n * np.pi) * phi
    p = np.stack([np.sin(phi) * np.cos(th), np.sin(phi) * np.sin(th),
                  np.cos(phi)], 1)
    return np.asarray(center, float)[None, :] + R * p


# ----------------------------------------------------------------------------
# the configurations
# ----------------------------------------------------------------------------
def disc_config(N: int = 10_000, eps: float = 1e-4, seed: int = 0,
                fp64: bool = True) -> Instance:
    """Unit disc, K = I, 32 equal arcs from theta = 0 (arcs 0-15 = upper half
    = Gamma_0, arcs 16-31 = Gamma_1), 32 points on radius 0.5 at 2 pi k / 32."""
    dom = Domain(dim=2, outer="sphere", center=(0.0, 0.0, 0.0), radius=1.0)
    g1 = np.zeros(32, np.uint8)
    g1[16:] = 1
    part = Partition(outer_m=32, outer_theta0=0.0, gamma1=g1)
    return Instance("disc-32", dom, part, np.eye(2), circle_points((0, 0), 0.5, 32),
                    N=N, eps=eps, seed=seed, fp64=fp64)


K_CONFIG2 = np.array([[1.0, 0.5], [0.5, 2.0]])


def _jittered_grid(rng, n, lo, hi):
    cell = (hi - lo) / n
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    base = np.stack([lo + (i + 0.5) * cell, lo + (j + 0.5) * cell], -1)
    jit = rng.uniform(-0.25, 0.25, size=base.shape) * cell
    return (base + jit).reshape(-1, 2)


def square_config(N: int = 100_000, eps: float = 1e-5, seed: int = 1,
                  geom_seed: int = 2, n_side: int = 64, grid: int = 16,
                  K: np.ndarray | None = None) -> Instance:
    """Square [-1/2, 1/2]^2, 4 x n_side elements counter-clockwise from the
    corner (-1/2, -1/2); Gamma_1 = elements whose midpoint has polar angle in
    [pi, 2 pi); grid x grid jittered points over [-0.45, 0.45]^2."""
    dom = Domain(dim=2, outer="box", center=(0.0, 0.0, 0.0), half=(0.5, 0.5, 0.0))
    part = Partition(edge_m=(n_side,) * 4)
    xc = element_centres(dom, part)
    part.gamma1 = (np.arctan2(xc[:, 1], xc[:, 0]) < 0).astype(np.uint8)
    rng = np.random.default_rng(geom_seed)
    pts = _jittered_grid(rng, grid, -0.45, 0.45)
    return Instance("square-256", dom, part, K_CONFIG2 if K is None else K,
                    pts, N=N, eps=eps, seed=seed)


def annulus_config(N: int = 100_000, eps: float = 1e-5, seed: int = 1,
                   geom_seed: int = 2, m_each: int = 128, grid: int = 16,
                   r_in: float = 0.5, K: np.ndarray | None = None) -> Instance:
    """Annulus r in [r_in, 1]: m_each arcs on the outer circle (Gamma_0) and
    m_each on the inner circle (Gamma_1, as in Ex. 5.2); polar jittered grid
    over r in [r_in + 0.05, 0.95]."""
    dom = Domain(dim=2, outer="sphere", center=(0.0, 0.0, 0.0), radius=1.0,
                 holes=(((0.0, 0.0, 0.0), r_in),))
    g1 = np.concatenate([np.zeros(m_each, np.uint8), np.ones(m_each, np.uint8)])
    part = Partition(outer_m=m_each, outer_theta0=0.0, hole_m=(m_each,),
                     hole_theta0=(0.0,), gamma1=g1)
    rng = np.random.default_rng(geom_seed)
    i, j = np.meshgrid(np.arange(grid), np.arange(grid), indexing="ij")
    rl, rh = r_in + 0.05, 0.95
    dr, dt = (rh - rl) / grid, 2 * np.pi / grid
    r = rl + (i + 0.5 + rng.uniform(-0.25, 0.25, i.shape)) * dr
    t = (j + 0.5 + rng.uniform(-0.25, 0.25, j.shape)) * dt
    pts = np.stack([r * np.cos(t), r * np.sin(t)], -1).reshape(-1, 2)
    return Instance("annulus-256", dom, part, K_CONFIG2 if K is None else K,
                    pts, N=N, eps=eps, seed=seed)


K_DIAG124 = np.diag([1.0, 2.0, 4.0])


def ball_config(N: int = 100_000, eps: float = 1e-4, K: np.ndarray | None = None,
                seed: int = 4, geom_seed: int = 5, n_points: int = 1024,
                nb: int = 32, ns: int = 48) -> Instance:
    """Unit ball, nb x ns equal-area patches, Gamma_1 = z < 0; points uniform
    in the ball of radius 1/2."""
    dom = Domain(dim=3, outer="sphere", center=(0.0, 0.0, 0.0), radius=1.0)
    g1 = np.zeros(nb * ns, np.uint8)
    g1[: (nb // 2) * ns] = 1
    part = Partition(outer_nb=nb, outer_ns=ns, gamma1=g1)
    rng = np.random.default_rng(geom_seed)
    inner = Domain(dim=3, outer="sphere", radius=0.5)
    pts = uniform_points(inner, n_points, rng, [-0.5] * 3, [0.5] * 3)
    return Instance(f"ball-{nb * ns}", dom, part,
                    K_DIAG124 if K is None else K, pts, N=N, eps=eps, seed=seed)


def cube_config(N: int = 100_000, eps: float = 1e-4, K: np.ndarray | None = None,
                seed: int = 4, geom_seed: int = 5, n_points: int = 1024,
                n_face: int = 16) -> Instance:
    """Cube [-1, 1]^3, 6 x n_face x n_face cells, Gamma_1 = faces -x, -y, -z;
    points uniform in [-1/2, 1/2]^3."""
    dom = Domain(dim=3, outer="box", center=(0.0, 0.0, 0.0), half=(1.0, 1.0, 1.0))
    m = 6 * n_face * n_face
    g1 = np.zeros(m, np.uint8)
    g1[: 3 * n_face * n_face] = 1
    part = Partition(face_n1=n_face, face_n2=n_face, gamma1=g1)
    rng = np.random.default_rng(geom_seed)
    pts = rng.uniform(-0.5, 0.5, size=(n_points, 3))
    return Instance(f"cube-{m}", dom, part, K_DIAG124 if K is None else K, pts,
                    N=N, eps=eps, seed=seed)


def config3_instances(N: int = 100_000, n_points: int = 1024) -> list:
    rng = np.random.default_rng(6)
    Krand = random_spd(rng, 3, 0.5, 4.0)
    return [ball_config(N=N, n_points=n_points),
            ball_config(N=N, n_points=n_points, K=Krand),
            cube_config(N=N, n_points=n_points),
            cube_config(N=N, n_points=n_points, K=Krand)]


L_SHAPE = ((-1.0, -1.0), (0.0, -1.0), (0.0, 0.0), (1.0, 0.0), (1.0, 1.0),
           (-1.0, 1.0))


def lshape_config(N: int = 100_000, eps: float = 1e-4, m_total: int = 256,
                  n_points: int = 256, seed: int = 7, geom_seed: int = 7,
                  K: np.ndarray | None = None) -> Instance:
    """L-shape [-1, 1]^2 minus [0, 1] x [-1, 0] (re-entrant corner at the
    origin); elements per edge in proportion to edge length; Gamma_1 = the
    two edges at the re-entrant corner."""
    v = np.asarray(L_SHAPE)
    lens = np.linalg.norm(np.roll(v, -1, 0) - v, axis=1)
    em = np.maximum(1, np.round(m_total * lens / lens.sum()).astype(int))
    em[-1] += m_total - em.sum()
    dom = Domain(dim=2, outer="polygon", vertices=L_SHAPE)
    g1 = np.zeros(int(em.sum()), np.uint8)
    g1[em[0]: em[0] + em[1] + em[2]] = 1
    part = Partition(edge_m=tuple(int(e) for e in em), gamma1=g1)
    rng = np.random.default_rng(geom_seed)
    pts = uniform_points(dom, n_points, rng, [-0.9, -0.9], [0.9, 0.9], margin=0.05)
    return Instance(f"lshape-{m_total}", dom, part,
                    np.eye(2) if K is None else K, pts, N=N, eps=eps, seed=seed)


def perforated_disc_config(N: int = 1_000_000, eps: float = 1e-10,
                           m_outer: int = 500, m_hole: int = 100,
                           n_points: int = 100, seed: int = 11,
                           fp64: bool = True) -> Instance:
    """Ex. 5.4 (and the Sec. 1 illustration): unit disc minus five discs of
    radius 0.2 centred at 0.5 (cos theta_l, sin theta_l), theta_l = 2 (l-1) pi/5;
    Gamma_0 = outer circle, Gamma_1 = the five small circles; the points are
    n_points equally spaced on the circle at distance 0.05 from Gamma_0."""
    holes = tuple(((0.5 * math.cos(2 * l * math.pi / 5),
                    0.5 * math.sin(2 * l * math.pi / 5), 0.0), 0.2)
                  for l in range(5))
    dom = Domain(dim=2, outer="sphere", radius=1.0, holes=holes)
    g1 = np.concatenate([np.zeros(m_outer, np.uint8), np.ones(5 * m_hole, np.uint8)])
    part = Partition(outer_m=m_outer, hole_m=(m_hole,) * 5, hole_theta0=(0.0,) * 5,
                     gamma1=g1)
    pts = circle_points((0, 0), 0.95, n_points)
    return Instance("perforated-disc", dom, part, np.eye(2), pts, N=N, eps=eps,
                    seed=seed, fp64=fp64)


def square_perimeter_points(half: float, n: int) -> np.ndarray:
    """n points equally spaced along the perimeter of the square of
    half-side `half` centred at the origin, counter-clockwise from
    (-half, -half)."""
    t = 8.0 * half * (np.arange(n) + 0.5) / n
    out = np.zeros((n, 2))
    for q, s in enumerate(t):
        side, u = int(s // (2 * half)), s % (2 * half) - half
        out[q] = [(u, -half), (half, u), (-u, half), (-half, -u)][side]
    return out


def square_hole_config(example: int = 1, N: int = 1_000_000, eps: float = 1e-7,
                       m_edge: int = 100, m_hole: int = 50, n_points: int = 40,
                       seed: int = 13, fp64: bool = True) -> Instance:
    """Ex. 5.1 / 5.5: the square (-1, 1)^2 minus the disc of radius 0.2 at
    (0.5, 0); m_edge cells per side (counter-clockwise from (-1, -1)) and
    m_hole arcs.  Ex. 5.1: Gamma_0 = the square, Gamma_1 = the circle, points
    on {dist(x, Gamma_0) = 0.05} (the square of half-side 0.95).  Ex. 5.5:
    Gamma_0 empty, Gamma_1 = both boundaries, points on the circle of radius
    0.3 about (-0.5, 0.5)."""
    dom = Domain(dim=2, outer="box", half=(1.0, 1.0, 0.0),
                 holes=(((0.5, 0.0, 0.0), 0.2),))
    part = Partition(edge_m=(m_edge,) * 4, hole_m=(m_hole,), hole_theta0=(0.0,))
    if example == 1:
        part.gamma1 = np.concatenate([np.zeros(4 * m_edge, np.uint8),
                                      np.ones(m_hole, np.uint8)])
        pts = square_perimeter_points(0.95, n_points)
    elif example == 5:
        part.gamma1 = np.ones(4 * m_edge + m_hole, np.uint8)
        pts = circle_points((-0.5, 0.5), 0.3, n_points)
    else:
        raise ValueError("Ex. 5.1 or 5.5")
    return Instance(f"square-hole-ex{example}", dom, part, np.eye(2), pts, N=N, eps=eps,
                    seed=seed, fp64=fp64)


def shell_config(N: int = 100_000, eps: float = 1e-4, shift: float = 0.0,
                 nb: int = 16, ns: int = 24, n_points: int = 100, seed: int = 12,
                 K: np.ndarray | None = None, voronoi: tuple | None = None,
                 fp64: bool = False) -> Instance:
    """Ex. 5.6 / 5.7: unit ball minus the ball of radius 0.5 centred at
    (shift, 0, 0); Gamma_1 = inner sphere; points on the Bauer spiral of the
    sphere at distance 0.05 from Gamma_0.  Elements: nb x ns bands x sectors
    on each sphere, or with voronoi = (M_0, M_1) the paper's extrinsic
    Voronoi cells of M_0 Bauer-spiral sites on the outer sphere and M_1 on the
    inner one (Sec. 5.3; Ex. 5.6 / 5.7 use (1000, 100))."""
    dom = Domain(dim=3, outer="sphere", radius=1.0,
                 holes=(((shift, 0.0, 0.0), 0.5),))
    if voronoi is None:
        g1 = np.concatenate([np.zeros(nb * ns, np.uint8), np.ones(nb * ns, np.uint8)])
        part = Partition(outer_nb=nb, outer_ns=ns, hole_nb=(nb,), hole_ns=(ns,),
                         gamma1=g1)
    else:
        m0, m1 = voronoi
        sites = np.concatenate([bauer_spiral(m0, 1.0), bauer_spiral(m1, 0.5, (shift, 0, 0))])
        part = Partition(voronoi_sites=sites,
                         gamma1=np.concatenate([np.zeros(m0, np.uint8), np.ones(m1, np.uint8)]))
    return Instance("shell" if voronoi is None else "shell-voronoi", dom, part,
                    np.eye(3) if K is None else K, bauer_spiral(n_points, 0.95), N=N,
                    eps=eps, seed=seed, fp64=fp64)


def annulus_voronoi_config(N: int = 1_000_000, eps: float = 1e-10, m0: int = 500,
                           m1: int = 100, n_points: int = 100, r_in: float = 0.5,
                           seed: int = 14, fp64: bool = True) -> Instance:
    """Ex. 5.2 / 5.3 with the paper's element choice: the annulus
    r in [r_in, 1], extrinsic Voronoi cells of m0 equally spaced points on the
    outer circle (Gamma_0) and m1 on the inner circle (Gamma_1); points on the
    circle at distance 0.05 from Gamma_0."""
    dom = Domain(dim=2, outer="sphere", radius=1.0, holes=(((0.0, 0.0, 0.0), r_in),))
    sites = np.concatenate([circle_points((0, 0), 1.0, m0), circle_points((0, 0), r_in, m1)])
    part = Partition(voronoi_sites=sites,
                     gamma1=np.concatenate([np.zeros(m0, np.uint8), np.ones(m1, np.uint8)]))
    return Instance("annulus-voronoi", dom, part, np.eye(2), circle_points((0, 0), 0.95, n_points),
                    N=N, eps=eps, seed=seed, fp64=fp64)


def mixed_batch(n_instances: int = 64, seed: int = 7, m_lo: int = 64,
                m_hi: int = 2048, n_lo: float = 1e4, n_hi: float = 1e6,
                scale: float = 1.0) -> list:
    """Batch of instances drawn from disc, annulus, square, L-shape, ball and
    box with log-uniform element / point counts and walks per point, eps in
    {1e-3, 1e-4, 1e-5} and random SPD K of condition number <= 10.

    ``scale`` multiplies the walks per point (for reduced test sizes)."""
    rng = np.random.default_rng(seed)
    kinds = ["disc", "annulus", "square", "lshape", "ball", "box"]
    out = []
    for q in range(n_instances):
        kind = kinds[q % len(kinds)]
        M = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        MD = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        N = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))) * scale))
        N = max(N, 1)
        eps = float(rng.choice([1e-3, 1e-4, 1e-5]))
        d = 3 if kind in ("ball", "box") else 2
        K = random_spd(rng, d, 1.0, 10.0)  # eigenvalues in [1, 10]: kappa <= 10
        gs = int(rng.integers(1 << 30))
        if kind == "disc":
            dom = Domain(dim=2, outer="sphere", radius=1.0)
            g1 = (np.arange(M) >= M // 2).astype(np.uint8)
            part = Partition(outer_m=M, gamma1=g1)
            pts = uniform_points(dom, MD, np.random.default_rng(gs), [-.7] * 2, [.7] * 2,
                                 margin=0.3)
        elif kind == "annulus":
            mo = max(M // 2, 1)
            mi = max(M - mo, 1)
            dom = Domain(dim=2, outer="sphere", radius=1.0,
                         holes=(((0.0, 0.0, 0.0), 0.5),))
            g1 = np.concatenate([np.zeros(mo, np.uint8), np.ones(mi, np.uint8)])
            part = Partition(outer_m=mo, hole_m=(mi,), hole_theta0=(0.0,), gamma1=g1)
            pts = uniform_points(dom, MD, np.random.default_rng(gs), [-.95] * 2, [.95] * 2,
                                 margin=0.05)
        elif kind == "square":
            side = max(M // 4, 1)
            dom = Domain(dim=2, outer="box", half=(0.5, 0.5, 0.0))
            part = Partition(edge_m=(side,) * 4)
            xc = element_centres(dom, part)
            part.gamma1 = (np.arctan2(xc[:, 1], xc[:, 0]) < 0).astype(np.uint8)
            pts = np.random.default_rng(gs).uniform(-0.45, 0.45, (MD, 2))
        elif kind == "lshape":
            inst = lshape_config(N=N, eps=eps, m_total=max(M, 6), n_points=MD,
                                 seed=seed, geom_seed=gs, K=K)
            out.append(inst.replace(name=f"b{q}-lshape", stream=q))
            continue
        elif kind == "ball":
            nb = max(2, int(round(math.sqrt(M / 2))))
            ns = max(1, M // nb)
            dom = Domain(dim=3, outer="sphere", radius=1.0)
            g1 = np.zeros(nb * ns, np.uint8)
            g1[: (nb // 2) * ns] = 1
            part = Partition(outer_nb=nb, outer_ns=ns, gamma1=g1)
            inner = Domain(dim=3, outer="sphere", radius=0.5)
            pts = uniform_points(inner, MD, np.random.default_rng(gs), [-.5] * 3, [.5] * 3)
        else:
            nf = max(1, int(round(math.sqrt(M / 6))))
            dom = Domain(dim=3, outer="box", half=(1.0, 1.0, 1.0))
            g1 = np.zeros(6 * nf * nf, np.uint8)
            g1[: 3 * nf * nf] = 1
            part = Partition(face_n1=nf, face_n2=nf, gamma1=g1)
            pts = np.random.default_rng(gs).uniform(-0.5, 0.5, (MD, 3))
        out.append(Instance(f"b{q}-{kind}", dom, part, K, pts, N=N, eps=eps,
                            seed=seed, stream=q))
    return out


@dataclass
class Request:
    """One request of a served stream: an instance, its measurement noise
    level and its arrival offset in units of the mean inter-arrival time."""
    index: int
    arrival: float
    inst: Instance
    noise: float


def serve_stream(n_requests: int = 10_000, seed: int = 11, first: int | None = None,
                 N: int = 100_000, m_lo: int = 256, m_hi: int = 1024) -> list:
    """Poisson-arrival stream over the 3-D mix of the ball / cube workloads
    (1536 boundary patches, K = diag(1, 2, 4) or a random SPD K with
    eigenvalues log-uniform in [0.5, 4]): per request a domain, a K, a point
    count log-uniform in [m_lo, m_hi] (points uniform in the inner half), eps
    in {1e-3, 1e-4}, noise uniform in [0.1, 5] % and an exponential
    inter-arrival gap of mean 1.  Request q draws from its own generator
    (seed, q), so a prefix ``first`` of the stream is the same requests as
    the whole stream's first ones; its walks use stream id q."""
    n = n_requests if first is None else min(first, n_requests)
    gaps = np.random.default_rng(seed).exponential(1.0, n_requests)[:n]
    arrival = np.cumsum(gaps) - gaps[0]
    out = []
    for q in range(n):
        rng = np.random.default_rng([seed, q])
        cube = bool(rng.integers(2))
        K = K_DIAG124 if rng.integers(2) == 0 else random_spd(rng, 3, 0.5, 4.0)
        MD = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        eps = float(rng.choice([1e-3, 1e-4]))
        noise = float(rng.uniform(0.001, 0.05))
        gs = int(rng.integers(1 << 30))
        inst = (cube_config if cube else ball_config)(N=N, eps=eps, K=K, seed=seed,
                                                      geom_seed=gs, n_points=MD)
        out.append(Request(q, float(arrival[q]),
                           inst.replace(name=f"r{q}-{inst.name}", stream=q), noise))
    return out


def synthetic_counts(M_D: int, M_tot: int, N: int, seed: int = 0,
                     width: float = 0.05) -> np.ndarray:
    """Seeded multinomial count matrix shaped like an operator: row i draws N
    samples from a smooth periodic bump centred at i / M_D (for SVD tests at
    sizes the oracle walker would take too long to build)."""
    rng = np.random.default_rng(seed)
    t = np.arange(M_tot) / M_tot
    C = np.empty((M_D, M_tot), np.uint32)
    for i in range(M_D):
        dc = np.abs(t - (i + 0.5) / M_D)
        dc = np.minimum(dc, 1 - dc)
        p = 1.0 / (dc ** 2 + width ** 2)
        p /= p.sum()
        C[i] = rng.multinomial(N, p)
    return C
