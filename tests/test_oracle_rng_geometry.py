"""Pins of the oracle's Philox, chain layout, distance and classification.

Everything here runs on the CPU (-m "not gpu")."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_03686_gb300 import workloads as W


# ---------------------------------------------------------------------------
# Philox4x32-10: known-answer values published with the Random123 library
# (Salmon, Moraes, Dror & Shaw, SC'11).
# ---------------------------------------------------------------------------
KAT = [
    ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
    ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2,
     [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
    ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
]


@pytest.mark.parametrize("ctr,key,expect", KAT)
def test_philox_known_answers(ctr, key, expect):
    assert O.philox(ctr, key) == expect


def test_philox_uniformity_and_independence():
    # 23-bit uniforms (the FP32 walks' map) from 4 * 20000 words: chi^2 over
    # 64 bins, and lag-1 correlation between consecutive counters.
    words = []
    for b in range(20000):
        words.extend(O.philox([b, 7, 0, 0], [123, 456]))
    w = np.array(words, dtype=np.uint64)
    u = (w >> np.uint64(9)).astype(np.float64) * 2.0 ** -23
    # and the five 23-bit windows of each 128-bit block (FP32 2-D walks)
    blocks = np.array(words, dtype=object).reshape(-1, 4)
    big = [int(b[0]) | (int(b[1]) << 32) | (int(b[2]) << 64) | (int(b[3]) << 96) for b in blocks]
    win = np.array([(v >> (23 * j)) & 0x7FFFFF for v in big for j in range(5)],
                   dtype=np.float64) * 2.0 ** -23
    hw, _ = np.histogram(win, bins=64, range=(0, 1))
    ew = len(win) / 64
    assert float(((hw - ew) ** 2 / ew).sum()) < 63 + 6 * math.sqrt(2 * 63)
    cw = np.corrcoef(win[:-1], win[1:])[0, 1]  # neighbouring windows of a block
    assert abs(cw) < 6 / math.sqrt(len(win))
    assert u.min() >= 0.0 and u.max() < 1.0
    h, _ = np.histogram(u, bins=64, range=(0, 1))
    e = len(u) / 64
    chi2 = float(((h - e) ** 2 / e).sum())
    assert chi2 < 63 + 6 * math.sqrt(2 * 63)  # ~6 sigma of chi^2_63
    c = np.corrcoef(u[:-4], u[4:])[0, 1]
    assert abs(c) < 6 / math.sqrt(len(u))


def _first_step_by_hand(inst, i, k):
    """X_1 of walk (i, k) recomputed from the counter layout
    (block 0, walk lo, walk hi, stream), key (seed lo, seed hi)."""
    S, _ = O.setup_S(inst.K)
    wid = i * inst.N + k
    words = O.philox([0, wid & 0xFFFFFFFF, wid >> 32, inst.stream],
                     [inst.seed & 0xFFFFFFFF, inst.seed >> 32])
    x0 = inst.points[i]
    r = O.dist(inst.domain, inst.partition, x0)[0]
    if inst.dim == 2:
        if inst.fp64:
            u = ((words[0] << 21) | (words[1] >> 11)) * 2.0 ** -53
        else:  # step 0 of the block: bits 0..22 of the 128-bit block
            u = (words[0] & 0x7FFFFF) * 2.0 ** -23
        U = np.array([math.cos(2 * math.pi * u), math.sin(2 * math.pi * u)])
    else:
        if inst.fp64:
            u1 = ((words[0] << 21) | (words[1] >> 11)) * 2.0 ** -53
            u2 = ((words[2] << 21) | (words[3] >> 11)) * 2.0 ** -53
        else:
            u1 = (words[0] >> 9) * 2.0 ** -23
            u2 = (words[1] >> 9) * 2.0 ** -23
        z = 1 - 2 * u1
        s = math.sqrt(1 - z * z)
        U = np.array([s * math.cos(2 * math.pi * u2), s * math.sin(2 * math.pi * u2), z])
    return x0 + r * (S @ U)


@pytest.mark.parametrize("make", [
    lambda: W.disc_config(N=1000, fp64=True),
    lambda: W.square_config(N=1000),
    lambda: W.ball_config(N=1000, n_points=8),
    lambda: W.ball_config(N=1000, n_points=8).replace(fp64=True),
])
def test_chain_counter_layout(make):
    inst = make().replace(step_cap=1, seed=0x1234567890AB, stream=5)
    for i, k in [(0, 0), (1, 17), (3, 999)]:
        xe, el, ns = O.walks(inst, [i], [k])
        assert el[0] == -1 and ns[0] == 1  # stopped by the cap after one move
        np.testing.assert_allclose(xe[0], _first_step_by_hand(inst, i, k),
                                   rtol=0, atol=1e-15)


def _steps_by_hand(inst, i, k, n_steps):
    """X_n of a FP32 2-D walk (i, k) recomputed step by step: step n takes
    Philox block n // 5 and its 23-bit window n % 5 (bits 23 j .. 23 j + 22
    of the 128-bit block)."""
    S, _ = O.setup_S(inst.K)
    wid = i * inst.N + k
    x = np.array(inst.points[i], dtype=np.float64)
    for n in range(n_steps):
        words = O.philox([n // 5, wid & 0xFFFFFFFF, wid >> 32, inst.stream],
                         [inst.seed & 0xFFFFFFFF, inst.seed >> 32])
        big = words[0] | (words[1] << 32) | (words[2] << 64) | (words[3] << 96)
        u = ((big >> (23 * (n % 5))) & 0x7FFFFF) * 2.0 ** -23
        r = O.dist(inst.domain, inst.partition, x)[0]
        x = x + r * (S @ np.array([math.cos(2 * math.pi * u), math.sin(2 * math.pi * u)]))
    return x


def test_packed_windows_of_fp32_2d_walks():
    """Every window of a block and the move to the next block: the oracle's
    walk stopped by a cap of 1..7 steps equals the chain recomputed by hand
    (square, FP32 walks, anisotropic K)."""
    inst = W.square_config(N=1000, eps=1e-9).replace(seed=0x1234567890AB, stream=5)
    for cap in range(1, 8):
        ic = inst.replace(step_cap=cap)
        for i, k in [(0, 0), (2, 31)]:
            xe, el, ns = O.walks(ic, [i], [k])
            if ns[0] < cap:  # stopped inside the eps shell first
                continue
            np.testing.assert_allclose(xe[0], _steps_by_hand(ic, i, k, cap), rtol=0,
                                       atol=1e-14)


def test_setup_S_is_normalised_square_root():
    rng = np.random.default_rng(0)
    for d in (2, 3):
        for _ in range(5):
            K = W.random_spd(rng, d, 0.3, 7.0)
            S, lam = O.setup_S(K)
            assert lam == pytest.approx(np.linalg.eigvalsh(K).max(), rel=1e-13)
            np.testing.assert_allclose(S @ S, K / lam, atol=1e-14)
            np.testing.assert_allclose(S, S.T, atol=1e-15)
            assert np.linalg.eigvalsh(S).max() == pytest.approx(1.0, abs=1e-14)
            assert np.linalg.eigvalsh(S).min() > 0
            S2, _ = O.setup_S(3.7 * K)  # scaling K does not change the chain
            np.testing.assert_allclose(S2, S, atol=1e-14)
    with pytest.raises(ValueError):
        O.setup_S(np.array([[1.0, 2.0], [2.0, 1.0]]))  # indefinite
    with pytest.raises(ValueError):
        O.setup_S(np.array([[1.0, 0.5], [0.1, 1.0]]))  # not symmetric


# ---------------------------------------------------------------------------
# Distance and classification against brute force over dense boundary samples
# ---------------------------------------------------------------------------
def _boundary_samples(dom, part, n_per=4000):
    """Dense boundary samples with the element each belongs to, built from
    the partition description (parametric, independent of the oracle)."""
    pts, lab = [], []
    off = 0
    d = dom.dim

    def circle(c, r, m, th0, off):
        t = th0 + 2 * np.pi * (np.arange(n_per * m) + 0.5) / (n_per * m)
        p = np.stack([c[0] + r * np.cos(t), c[1] + r * np.sin(t)], 1)
        return p, off + np.arange(n_per * m) // n_per

    def sphere(c, r, nb, ns, off):
        k = 24
        z = -1 + 2 * (np.arange(nb * k) + 0.5) / (nb * k)
        ph = 2 * np.pi * (np.arange(ns * k) + 0.5) / (ns * k)
        Z, P = np.meshgrid(z, ph, indexing="ij")
        s = np.sqrt(1 - Z ** 2)
        p = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
        B, Sx = np.meshgrid(np.arange(nb * k) // k, np.arange(ns * k) // k, indexing="ij")
        return np.asarray(c[:3]) + r * p, off + (B * ns + Sx).ravel()

    def poly(verts, em, off):
        P, L = [], []
        n = len(verts)
        for e in range(n):
            a, b = np.asarray(verts[e], float), np.asarray(verts[(e + 1) % n], float)
            t = (np.arange(n_per * em[e]) + 0.5) / (n_per * em[e])
            P.append(a + t[:, None] * (b - a))
            L.append(off + np.arange(n_per * em[e]) // n_per)
            off += em[e]
        return np.concatenate(P), np.concatenate(L)

    if dom.outer == "sphere":
        p, l = (circle(dom.center, dom.radius, part.outer_m, part.outer_theta0, off)
                if d == 2 else sphere(dom.center, dom.radius, part.outer_nb, part.outer_ns, off))
    elif dom.outer == "polygon":
        p, l = poly(dom.vertices, part.edge_m, off)
    elif d == 2:
        p, l = poly(W.box_polygon(dom.center, dom.half), part.edge_m, off)
    else:
        k = 24
        P, L = [], []
        n1, n2 = part.face_n1, part.face_n2
        for f in range(6):
            ax = f % 3
            b0 = 1 if ax == 0 else 0
            b1 = 1 if ax == 2 else 2
            t0 = -1 + 2 * (np.arange(n1 * k) + 0.5) / (n1 * k)
            t1 = -1 + 2 * (np.arange(n2 * k) + 0.5) / (n2 * k)
            T0, T1 = np.meshgrid(t0, t1, indexing="ij")
            q = np.zeros(T0.shape + (3,))
            q[..., ax] = (-1 if f < 3 else 1) * dom.half[ax]
            q[..., b0] = T0 * dom.half[b0]
            q[..., b1] = T1 * dom.half[b1]
            I0, I1 = np.meshgrid(np.arange(n1 * k) // k, np.arange(n2 * k) // k, indexing="ij")
            P.append(q.reshape(-1, 3))
            L.append((off + f * n1 * n2 + I0 * n2 + I1).ravel())
        p, l = np.concatenate(P), np.concatenate(L)
    pts.append(p)
    lab.append(l)
    off = int(l.max()) + 1
    for h, (c, r) in enumerate(dom.holes):
        if d == 2:
            p, l = circle(c, r, part.hole_m[h], part.hole_theta0[h], off)
        else:
            p, l = sphere(c, r, part.hole_nb[h], part.hole_ns[h], off)
        pts.append(p)
        lab.append(l)
        off = int(l.max()) + 1
    return np.concatenate(pts), np.concatenate(lab)


GEOMS = {
    "disc": lambda: W.disc_config(),
    "annulus": lambda: W.annulus_config(m_each=16),
    "square": lambda: W.square_config(n_side=8),
    "lshape": lambda: W.lshape_config(m_total=24),
    "perforated": lambda: W.perforated_disc_config(m_outer=20, m_hole=8),
    "ball": lambda: W.ball_config(nb=4, ns=6, n_points=4),
    "cube": lambda: W.cube_config(n_face=3, n_points=4),
    "shell": lambda: W.shell_config(nb=4, ns=6, shift=0.3),
    "square_hole": lambda: W.square_hole_config(m_edge=6, m_hole=8),
}


@pytest.mark.parametrize("name", list(GEOMS))
def test_distance_and_cell_against_brute_force(name):
    inst = GEOMS[name]()
    dom, part = inst.domain, inst.partition
    bp, bl = _boundary_samples(dom, part, n_per=600 if dom.dim == 2 else 1)
    assert bl.max() + 1 == O.num_elements(dom, part) == W.element_count(dom, part)
    rng = np.random.default_rng(1)
    lo = np.asarray(dom.center[: dom.dim]) - 1.0
    pts = W.uniform_points(dom, 300, rng, lo, lo + 2.0, margin=1e-3)
    pts = np.concatenate([pts, inst.points[:20]])
    dv = O.dist(dom, part, pts)
    # brute force: distance to the nearest boundary sample (an upper bound
    # within the sample spacing of the true distance)
    spacing = 2 * np.pi / (600 * 8) if dom.dim == 2 else 0.2
    for q in range(len(pts)):
        dd = np.linalg.norm(bp - pts[q], axis=1)
        assert dv[q] <= dd.min() + 1e-12
        assert dv[q] >= dd.min() - spacing
    # classification near the boundary: points pushed a little inside from a
    # boundary sample that is well inside its cell
    idx = rng.choice(len(bp), 400, replace=False)
    near = []
    labs = []
    for q in idx:
        y = bp[q]
        for dirv in rng.standard_normal((8, dom.dim)):
            x = y + 2e-7 * dirv / np.linalg.norm(dirv)
            if O.dist(dom, part, x)[0] >= 0:
                near.append(x)
                labs.append(bl[q])
                break
    near = np.array(near)
    cl = O.classify(dom, part, near)
    dd = np.array([np.linalg.norm(bp - x, axis=1).min() for x in near])
    # nearest-sample element must match wherever the sample is unambiguous
    nearest_lab = np.array([bl[np.argmin(np.linalg.norm(bp - x, axis=1))] for x in near])
    agree = (cl == nearest_lab)
    assert agree.mean() > 0.97, (name, agree.mean())
    assert (dd < 1e-3).all()


def test_lowest_index_tie_break():
    # square: the point on the diagonal near corner (-1/2,-1/2) is at equal
    # distance from edge 0 (bottom) and edge 3 (left): lowest index -> bottom,
    # first cell (element 0).  Polygon vertex ties: the shared vertex gives
    # the lower edge's cell.
    inst = W.square_config(n_side=8)
    x = np.array([[-0.5 + 1e-3, -0.5 + 1e-3]])
    assert O.classify(inst.domain, inst.partition, x)[0] == 0
    L = W.lshape_config(m_total=24)
    em = L.partition.edge_m
    # the re-entrant corner (0, 0) is vertex 2, shared by edges 1 and 2; points
    # whose nearest boundary point is the corner go to the last cell of edge 1
    x = np.array([[1e-4, -1e-4]]) * -1.0  # (-1e-4, 1e-4): nearest point = corner
    got = O.classify(L.domain, L.partition, x)[0]
    assert got == em[0] + em[1] - 1
    # circle arc boundaries: theta exactly on an arc edge goes to the arc
    # that starts there
    D = W.disc_config()
    t = 2 * np.pi * 5 / 32
    x = np.array([[0.9999 * math.cos(t), 0.9999 * math.sin(t)]])
    assert O.classify(D.domain, D.partition, x)[0] in (4, 5)


def test_element_measures_sum_to_boundary_measure():
    cases = [
        (W.disc_config(), 2 * math.pi),
        (W.annulus_config(m_each=16), 2 * math.pi * 1.5),
        (W.square_config(n_side=8), 4.0),
        (W.lshape_config(m_total=24), 8.0),
        (W.ball_config(nb=4, ns=6, n_points=4), 4 * math.pi),
        (W.cube_config(n_face=3, n_points=4), 24.0),
        (W.shell_config(nb=4, ns=6), 4 * math.pi * 1.25),
    ]
    for inst, total in cases:
        m = O.element_measures(inst.domain, inst.partition)
        assert len(m) == inst.M_tot
        assert m.sum() == pytest.approx(total, rel=1e-13)


# ---------------------------------------------------------------------------
# sigma(omega_j) element by element (Eq. (boundary_weights): the surface
# measure of each cell), on shapes whose sides differ, so that an axis or
# edge mix-up in the oracle changes a value; the expected numbers are worked
# by hand from the cell definitions of the partition descriptor.
# ---------------------------------------------------------------------------
def test_element_measures_cuboid_by_hand():
    """Box with half-extents (1/2, 1, 2), 2 x 4 cells per face over the two
    other axes in increasing order: face -x cells are (2/2) x (4/4) = 1,
    face -y (1/2) x (4/4) = 1/2, face -z (1/2) x (2/4) = 1/4; +x, +y, +z
    repeat them."""
    dom = W.Domain(dim=3, outer="box", center=(0.1, -0.2, 0.3), half=(0.5, 1.0, 2.0))
    part = W.Partition(face_n1=2, face_n2=4)
    m = O.element_measures(dom, part)
    per_face = [1.0, 0.5, 0.25, 1.0, 0.5, 0.25]
    np.testing.assert_allclose(m, np.repeat(per_face, 8), rtol=1e-15)


def test_element_measures_rectangle_and_lshape_by_hand():
    """2-D box (1/2, 2) with 2, 4, 2, 4 cells on the bottom, right, top, left
    edges: cell lengths 1/2, 1, 1/2, 1.  The L-shape's edges (lengths 1, 1,
    1, 1, 2, 2 counter-clockwise from (-1, -1)) with 1, 2, 4, 1, 2, 8 cells:
    1, 1/2, 1/4, 1, 1, 1/4."""
    dom = W.Domain(dim=2, outer="box", center=(0.3, 0.0, 0.0), half=(0.5, 2.0, 1.0))
    m = O.element_measures(dom, W.Partition(edge_m=(2, 4, 2, 4)))
    np.testing.assert_allclose(m, [0.5] * 2 + [1.0] * 4 + [0.5] * 2 + [1.0] * 4,
                               rtol=1e-15)
    L = W.Domain(dim=2, outer="polygon", vertices=W.L_SHAPE)
    em = (1, 2, 4, 1, 2, 8)
    m = O.element_measures(L, W.Partition(edge_m=em))
    want = np.repeat([1.0, 0.5, 0.25, 1.0, 1.0, 0.25], em)
    np.testing.assert_allclose(m, want, rtol=1e-15)


def test_element_measures_sphere_patch_and_holes_by_quadrature():
    """A z-band x phi-sector patch of a sphere of radius 1.5 (4 bands, 6
    sectors) against the surface integral R^2 sin(theta) dtheta dphi done by
    scipy's adaptive quadrature; circle arcs of a hole against R dtheta."""
    from scipy import integrate
    R = 1.5
    dom = W.Domain(dim=3, outer="sphere", radius=R,
                   holes=(((0.2, 0.0, 0.1), 0.3),))
    part = W.Partition(outer_nb=4, outer_ns=6, hole_nb=(2,), hole_ns=(3,))
    m = O.element_measures(dom, part)
    assert len(m) == 24 + 6
    # band 1 spans z in [-R/2, 0]: theta from acos(0) to acos(-1/2)
    th0, th1 = math.acos(0.0), math.acos(-0.5)
    area, _ = integrate.dblquad(lambda th, ph: R * R * math.sin(th),
                                2 * math.pi * 2 / 6, 2 * math.pi * 3 / 6, th0, th1,
                                epsabs=1e-14, epsrel=1e-13)
    np.testing.assert_allclose(m[1 * 6 + 2], area, rtol=1e-12)
    np.testing.assert_allclose(m[:24], area, rtol=1e-12)
    # hole: 2 bands x 3 sectors of the sphere of radius 0.3
    harea, _ = integrate.dblquad(lambda th, ph: 0.09 * math.sin(th),
                                 0.0, 2 * math.pi / 3, 0.0, math.pi / 2,
                                 epsabs=1e-15, epsrel=1e-13)
    np.testing.assert_allclose(m[24:], harea, rtol=1e-12)
    disc = W.Domain(dim=2, outer="sphere", radius=2.0, holes=(((0.5, 0.0, 0.0), 0.25),))
    m2 = O.element_measures(disc, W.Partition(outer_m=5, hole_m=(3,)))
    arc, _ = integrate.quad(lambda t: 2.0, 0.0, 2 * math.pi / 5)
    harc, _ = integrate.quad(lambda t: 0.25, 0.0, 2 * math.pi / 3)
    np.testing.assert_allclose(m2, [arc] * 5 + [harc] * 3, rtol=1e-14)
