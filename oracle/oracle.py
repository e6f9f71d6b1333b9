"""Python front of the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline / reference leg are the only callers.  Nothing here imports the
CUDA library, and the CUDA library never imports this.

The walk, distance, classification, Philox and Jacobi arithmetic is the plain
C in ``wos_oracle.c``.  This file adds marshalling plus the small FP64 steps
the paper writes as matrix algebra:

* element measures sigma(omega_j) (Sec. 3.1, Eq. (boundary_weights));
* the scaled operator B = diag(nu) A_{Gamma_1} diag(sigma)^{-1/2}
  (Sec. 4.3, Eq. (A_r_MC)), with A = C / N (Eq. (WoE_matrix_MC));
* the r-TSVD reconstruction u_{Gamma_1} = diag(sigma)^{-1/2} V_r Sigma_r^{-1}
  U_r^T diag(nu) b with b = u^D - A_{Gamma_0} u^0 (Sec. 2, Eq. (u1r);
  Sec. 4.3, Eq. (u_omega_M1_r_MC A); Rem. (b and u0 simulations)), optionally
  with the Tikhonov filter sigma / (sigma^2 + alpha) in place of 1 / sigma;
* the fitted interior values u^D_hat = A_{Gamma_1} u_{Gamma_1} + A_{Gamma_0} u^0
  (Sec. 5.2, item (iv));
* the spectral diagnostics of Sec. 5.2 items (i)-(iv): eigenvalues of
  Lambda^nu (Eq. (Lambda_tilde_nu)), the eigenfunction estimators
  (Eq. (eigenfunctions_MC)), the averaged density estimator (Eq. (rho omega1
  MC) averaged over the poles) and the TSVD solutions and fitted interior
  data for every truncation r.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_LIB_PATH = _HERE / "_lib" / "liboracle.so"
MAX_VERTS = 64
MAX_HOLES = 16


def build(force: bool = False) -> Path:
    """Compile the C oracle with gcc (seconds)."""
    src = [_HERE / "wos_oracle.c"]
    hdr = _HERE / "wos_oracle.h"
    if (not force and _LIB_PATH.exists() and all(
            _LIB_PATH.stat().st_mtime >= p.stat().st_mtime for p in src + [hdr])):
        return _LIB_PATH
    _LIB_PATH.parent.mkdir(exist_ok=True)
    tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
           "-o", str(tmp)] + [str(s) for s in src] + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB_PATH))
        L.orc_dist.restype = ctypes.c_double
        L.orc_quadric_radius.restype = ctypes.c_double
        _lib = L
    return _lib


class OrcDomain(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("outer_kind", ctypes.c_int32),
        ("center", ctypes.c_double * 3),
        ("radius", ctypes.c_double),
        ("half", ctypes.c_double * 3),
        ("n_vertices", ctypes.c_int32),
        ("vertices", ctypes.c_double * (2 * MAX_VERTS)),
        ("n_holes", ctypes.c_int32),
        ("hole_center", (ctypes.c_double * 3) * MAX_HOLES),
        ("hole_radius", ctypes.c_double * MAX_HOLES),
        ("outer_m", ctypes.c_int32),
        ("outer_theta0", ctypes.c_double),
        ("edge_m", ctypes.c_int32 * MAX_VERTS),
        ("outer_nb", ctypes.c_int32),
        ("outer_ns", ctypes.c_int32),
        ("face_n1", ctypes.c_int32),
        ("face_n2", ctypes.c_int32),
        ("hole_m", ctypes.c_int32 * MAX_HOLES),
        ("hole_theta0", ctypes.c_double * MAX_HOLES),
        ("hole_nb", ctypes.c_int32 * MAX_HOLES),
        ("hole_ns", ctypes.c_int32 * MAX_HOLES),
        ("voronoi_n", ctypes.c_int32),
        ("voronoi_sites", ctypes.POINTER(ctypes.c_double)),
    ]


class OrcInstance(ctypes.Structure):
    _fields_ = [
        ("dom", OrcDomain),
        ("S", ctypes.c_double * 9),
        ("eps", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("stream", ctypes.c_uint32),
        ("N", ctypes.c_uint32),
        ("step_cap", ctypes.c_uint32),
        ("words_per_uniform", ctypes.c_int32),
        ("mapped", ctypes.c_int32),
        ("n_planes", ctypes.c_int32),
        ("plane_n", (ctypes.c_double * 3) * 64),
        ("plane_d", ctypes.c_double * 64),
        ("Sinv", ctypes.c_double * 9),
        ("mu2", ctypes.c_double),
    ]


_KIND = {"sphere": 1, "box": 2, "polygon": 3}


def make_domain(dom, part):
    """Marshal a workloads Domain / Partition into the oracle's struct.
    Returns (struct, keep-alive list)."""
    D = OrcDomain()
    keep = []
    D.dim = dom.dim
    D.outer_kind = _KIND[dom.outer]
    for a in range(3):
        D.center[a] = float(dom.center[a]) if a < len(dom.center) else 0.0
        D.half[a] = float(dom.half[a]) if a < len(dom.half) else 0.0
    D.radius = float(dom.radius)
    if dom.outer == "polygon":
        assert len(dom.vertices) <= MAX_VERTS
        D.n_vertices = len(dom.vertices)
        for e, (x, y) in enumerate(dom.vertices):
            D.vertices[2 * e] = x
            D.vertices[2 * e + 1] = y
    assert len(dom.holes) <= MAX_HOLES
    D.n_holes = len(dom.holes)
    for h, (c, r) in enumerate(dom.holes):
        for a in range(3):
            D.hole_center[h][a] = float(c[a]) if a < len(c) else 0.0
        D.hole_radius[h] = r
    D.outer_m = part.outer_m
    D.outer_theta0 = part.outer_theta0
    for e, m in enumerate(part.edge_m):
        D.edge_m[e] = m
    D.outer_nb, D.outer_ns = part.outer_nb, part.outer_ns
    D.face_n1, D.face_n2 = part.face_n1, part.face_n2
    for h in range(len(dom.holes)):
        if part.voronoi_sites is not None:
            break  # Voronoi sites replace the per-component cells
        if dom.dim == 2:
            D.hole_m[h] = part.hole_m[h]
            D.hole_theta0[h] = part.hole_theta0[h]
        else:
            D.hole_nb[h] = part.hole_nb[h]
            D.hole_ns[h] = part.hole_ns[h]
    if part.voronoi_sites is not None:
        sites = np.ascontiguousarray(part.voronoi_sites, dtype=np.float64)
        keep.append(sites)
        D.voronoi_n = sites.shape[0]
        D.voronoi_sites = sites.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return D, keep


def setup_S(K):
    """K_s = K / lambda_max, S = K_s^{1/2} (Sec. 4.2).  Raises on non-SPD."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    d = K.shape[0]
    S = np.zeros(9)
    lam = ctypes.c_double()
    rc = lib().orc_setup_S(d, K.ctypes.data_as(ctypes.c_void_p),
                           S.ctypes.data_as(ctypes.c_void_p), ctypes.byref(lam))
    if rc != 0:
        raise ValueError("K is not symmetric positive definite")
    return S[: d * d].reshape(d, d).copy(), lam.value


def mapped_planes(dom, S):
    """Faces of the polytope S^{-1} D (D a box or a convex polygon without
    holes): unit outward normals n_f and offsets d_f in y = S^{-1} x, so that
    dist(y, boundary) = min_f (d_f - n_f . y) inside.  A face a.x = c of D
    becomes (S a).y = c, S symmetric."""
    d = dom.dim
    if dom.holes:
        raise ValueError("mapped walks: domains without holes only")
    faces = []  # (a, c): a.x <= c inside
    if dom.outer == "box":
        for a in range(d):
            for sgn in (-1.0, 1.0):
                n = np.zeros(d)
                n[a] = sgn
                faces.append((n, sgn * dom.center[a] + dom.half[a]))
    elif dom.outer == "polygon" and d == 2:
        v = np.asarray(dom.vertices, dtype=np.float64)
        for e in range(len(v)):
            t = v[(e + 1) % len(v)] - v[e]
            t2 = v[(e + 2) % len(v)] - v[(e + 1) % len(v)]
            if t[0] * t2[1] - t[1] * t2[0] <= 0:
                raise ValueError("mapped walks: convex counter-clockwise polygons only")
            n = np.array([t[1], -t[0]]) / np.hypot(t[0], t[1])
            faces.append((n, float(n @ v[e])))
    else:
        raise ValueError("mapped walks: boxes and convex polygons only")
    out_n, out_d = [], []
    for a, c in faces:
        m = S @ a
        L = np.linalg.norm(m)
        out_n.append(m / L)
        out_d.append(c / L)
    return np.array(out_n), np.array(out_d)


def make_instance(inst, words_per_uniform: int | None = None):
    D, keep = make_domain(inst.domain, inst.partition)
    I = OrcInstance()
    I.dom = D
    S, _ = setup_S(inst.K)
    for q, v in enumerate(S.ravel()):
        I.S[q] = v
    I.eps = inst.eps
    I.seed = inst.seed
    I.stream = inst.stream
    I.N = inst.N
    I.step_cap = inst.step_cap
    if words_per_uniform is None:
        words_per_uniform = 2 if inst.fp64 else 1
    I.words_per_uniform = words_per_uniform
    if getattr(inst, "mapped", False) and inst.domain.outer == "sphere":
        # disc / ball minus holes: the quadric lower bound of dist_y
        I.mapped = 2
        I.mu2 = float(np.linalg.eigvalsh(S)[0]) ** 2
    elif getattr(inst, "mapped", False):
        pn, pd = mapped_planes(inst.domain, S)
        I.mapped = 1
        I.n_planes = len(pd)
        for f in range(len(pd)):
            for a in range(inst.dim):
                I.plane_n[f][a] = pn[f, a]
            I.plane_d[f] = pd[f]
        Sinv = np.linalg.inv(S)
        for q, v in enumerate(Sinv.ravel()):
            I.Sinv[q] = v
    return I, keep


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key):
    C = (ctypes.c_uint32 * 4)(*[int(c) & 0xFFFFFFFF for c in ctr])
    Kk = (ctypes.c_uint32 * 2)(*[int(k) & 0xFFFFFFFF for k in key])
    O = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(C, Kk, O)
    return [int(o) for o in O]


def dist(dom, part, X):
    D, keep = make_domain(dom, part)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, dom.dim)
    L = lib()
    out = np.empty(len(X))
    for q in range(len(X)):
        out[q] = L.orc_dist(ctypes.byref(D), _p(X[q]))
    return out


def mapped_radius(inst, X):
    """Step radius of the mapped chain on a disc / ball minus holes (the
    quadric lower bound of dist_y, Sec. 4.2 in y = S^{-1} x) at points X."""
    I, keep = make_instance(inst.replace(mapped=True))
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, inst.dim)
    L = lib()
    return np.array([L.orc_quadric_radius(ctypes.byref(I), _p(X[q]))
                     for q in range(len(X))])


def classify(dom, part, X):
    D, keep = make_domain(dom, part)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, dom.dim)
    L = lib()
    return np.array([L.orc_classify(ctypes.byref(D), _p(X[q]))
                     for q in range(len(X))], dtype=np.int32)


def num_elements(dom, part) -> int:
    D, keep = make_domain(dom, part)
    return int(lib().orc_num_elements(ctypes.byref(D)))


def walks(inst, point_index, k, words_per_uniform=None):
    """Run the walks (i, k) one by one; returns exit points, exit elements
    (-1 = stopped by the step cap) and step counts N_eps."""
    I, keep = make_instance(inst, words_per_uniform)
    point_index = np.asarray(point_index, dtype=np.int64).ravel()
    k = np.asarray(k, dtype=np.int64).ravel()
    n = len(point_index)
    x0 = np.ascontiguousarray(inst.points[point_index], dtype=np.float64)
    wid = (point_index.astype(np.uint64) * np.uint64(inst.N) + k.astype(np.uint64))
    wid = np.ascontiguousarray(wid, dtype=np.uint64)
    xe = np.empty_like(x0)
    el = np.empty(n, np.int32)
    ns = np.empty(n, np.uint32)
    lib().orc_walk_batch(ctypes.byref(I), _p(x0), _p(wid), ctypes.c_int64(n),
                         _p(xe), _p(el), _p(ns))
    return xe, el, ns


def build_counts(inst, k0: int = 0, k1: int | None = None, nthreads: int = 0,
                 rows=None, words_per_uniform=None):
    """Algorithm MC-REM: C[i][j] = #walks k in [k0, k1) from point i that stop
    in element j.  ``rows`` restricts the build to a subset of points (the
    walk ids still use the full point index)."""
    I, keep = make_instance(inst, words_per_uniform)
    k1 = inst.N if k1 is None else k1
    M = num_elements(inst.domain, inst.partition)
    if rows is None:
        pts = np.ascontiguousarray(inst.points, dtype=np.float64)
        counts = np.zeros((inst.M_D, M), np.uint32)
        unterm = np.zeros(inst.M_D, np.uint32)
        steps = ctypes.c_uint64()
        rc = lib().orc_build_counts(ctypes.byref(I), _p(pts), inst.M_D,
                                    ctypes.c_uint32(k0), ctypes.c_uint32(k1),
                                    _p(counts), _p(unterm), ctypes.byref(steps),
                                    nthreads)
        assert rc == 0
        return counts, unterm, int(steps.value)
    rows = np.asarray(rows, dtype=np.int64)
    counts = np.zeros((len(rows), M), np.uint32)
    unterm = np.zeros(len(rows), np.uint32)
    total = 0
    for q, i in enumerate(rows):
        ks = np.arange(k0, k1)
        xe, el, ns = walks(inst, np.full(len(ks), i), ks, words_per_uniform)
        ok = el >= 0
        np.add.at(counts[q], el[ok], 1)
        unterm[q] = int((~ok).sum())
        total += int(ns.sum())
    return counts, unterm, total


# ----------------------------------------------------------------------------
# the FP64 post-processing (Sec. 2 and Sec. 4.3)
# ----------------------------------------------------------------------------
def element_measures(dom, part) -> np.ndarray:
    """sigma(omega_j): arc length / edge-cell length / patch area of every
    element (surface measure of the cell, Eq. (boundary_weights))."""
    if part.voronoi_sites is not None:
        return voronoi_measures(dom, part)
    d = dom.dim
    out = []
    if dom.outer == "sphere":
        if d == 2:
            out.append(np.full(part.outer_m, 2 * math.pi * dom.radius / part.outer_m))
        else:
            n = part.outer_nb * part.outer_ns
            out.append(np.full(n, 4 * math.pi * dom.radius ** 2 / n))
    elif dom.outer == "box" and d == 3:
        h = dom.half
        n1, n2 = part.face_n1, part.face_n2
        for f in range(6):
            ax = f % 3
            b0 = 1 if ax == 0 else 0
            b1 = 1 if ax == 2 else 2
            out.append(np.full(n1 * n2, (2 * h[b0] / n1) * (2 * h[b1] / n2)))
    else:
        if dom.outer == "box":
            cx, cy = dom.center[0], dom.center[1]
            hx, hy = dom.half[0], dom.half[1]
            v = [(cx - hx, cy - hy), (cx + hx, cy - hy), (cx + hx, cy + hy),
                 (cx - hx, cy + hy)]
        else:
            v = list(dom.vertices)
        for e in range(len(v)):
            a, b = np.asarray(v[e]), np.asarray(v[(e + 1) % len(v)])
            out.append(np.full(part.edge_m[e], np.linalg.norm(b - a) / part.edge_m[e]))
    for h, (c, r) in enumerate(dom.holes):
        if d == 2:
            out.append(np.full(part.hole_m[h], 2 * math.pi * r / part.hole_m[h]))
        else:
            n = part.hole_nb[h] * part.hole_ns[h]
            out.append(np.full(n, 4 * math.pi * r ** 2 / n))
    return np.concatenate(out)


def voronoi_measures(dom, part) -> np.ndarray:
    """sigma(omega_j) of extrinsic Voronoi cells (App. A, Ex. A.2) whose sites
    lie on circles / spheres of the domain (outer boundary and holes), each
    component's surface shared by its own sites only: the arc between the
    angular bisectors of a site's neighbours (2-D) or the spherical Voronoi
    cell area (3-D, scipy.spatial.SphericalVoronoi).  Sites on a box or
    polygon are not supported."""
    from scipy.spatial import SphericalVoronoi
    sites = np.asarray(part.voronoi_sites, dtype=np.float64)
    d = dom.dim
    comps = []
    if dom.outer == "sphere":
        comps.append((np.asarray(dom.center[:d], float), dom.radius))
    for c, r in dom.holes:
        comps.append((np.asarray(c[:d], float), r))
    if dom.outer != "sphere":
        raise NotImplementedError("Voronoi measures on circles / spheres only")
    out = np.zeros(len(sites))
    owner = np.full(len(sites), -1)
    for q, (c, r) in enumerate(comps):
        on = np.abs(np.linalg.norm(sites - c, axis=1) - r) <= 1e-9 * max(r, 1.0)
        owner[on & (owner < 0)] = q
    if (owner < 0).any():
        raise ValueError("a Voronoi site lies on no circle / sphere of the domain")
    for q, (c, r) in enumerate(comps):
        idx = np.flatnonzero(owner == q)
        if d == 2:
            ang = np.arctan2(sites[idx, 1] - c[1], sites[idx, 0] - c[0])
            order = np.argsort(ang)
            a = ang[order]
            nxt = np.roll(a, -1) - a
            nxt[-1] += 2 * math.pi
            prv = np.roll(nxt, 1)
            out[idx[order]] = r * 0.5 * (nxt + prv)
        else:
            sv = SphericalVoronoi(sites[idx], radius=r, center=c)
            out[idx] = sv.calculate_areas()
    return out


def operator_B(counts, N, gamma1, nu, measures):
    """B = diag(nu) (C[:, Gamma_1] / N) diag(sigma_{Gamma_1})^{-1/2}
    (Eq. (A_r_MC))."""
    g1 = np.asarray(gamma1).astype(bool)
    A1 = np.asarray(counts, dtype=np.float64)[:, g1] / float(N)
    return (np.asarray(nu, float)[:, None] * A1) / np.sqrt(
        np.asarray(measures, float)[g1])[None, :]


def jacobi_svd(B):
    """Thin SVD B = U diag(s) V^T by the C one-sided Jacobi; returns
    (U, s, V, sweeps, converged)."""
    B = np.ascontiguousarray(B, dtype=np.float64)
    m, n = B.shape
    k = min(m, n)
    U = np.zeros((m, k))
    s = np.zeros(k)
    V = np.zeros((n, k))
    sw = ctypes.c_int32()
    rc = lib().orc_jacobi_svd(m, n, _p(B), _p(U), _p(s), _p(V), ctypes.byref(sw))
    return U, s, V, int(sw.value), rc == 0


def reconstruct(U, s, V, r, counts, N, gamma1, nu, measures, uD, u0=None,
                tikhonov: float = 0.0):
    """r-TSVD (or Tikhonov-filtered) Gamma_1 data and fitted interior values.

    Returns (u_gamma1, uD_hat)."""
    g1 = np.asarray(gamma1).astype(bool)
    A = np.asarray(counts, dtype=np.float64) / float(N)
    A1, A0 = A[:, g1], A[:, ~g1]
    uD = np.asarray(uD, dtype=np.float64)
    b = uD.copy()
    if u0 is not None and A0.shape[1] > 0:
        b = b - A0 @ np.asarray(u0, dtype=np.float64)
    q = np.asarray(nu, float) * b
    sr = s[:r]
    if tikhonov > 0:
        filt = sr / (sr * sr + tikhonov)
    else:
        filt = 1.0 / sr
    w = V[:, :r] @ (filt * (U[:, :r].T @ q))
    u1 = w / np.sqrt(np.asarray(measures, float)[g1])
    uhat = A1 @ u1
    if u0 is not None and A0.shape[1] > 0:
        uhat = uhat + A0 @ np.asarray(u0, dtype=np.float64)
    return u1, uhat


def spectral(U, s, V, counts, N, gamma1, nu, measures, uD=None, u0=None, r_max=0):
    """Spectral diagnostics of one operator, from their definitions
    (Sec. 5.2 items (i)-(iv)).

    * lam: the eigenvalues of Lambda^nu = diag(nu) A_1 diag(sigma)^{-1} A_1^T
      diag(nu) (Eq. (Lambda_tilde_nu)), descending, the first k = len(s);
    * eigfun[l, j]: u~_j on Gamma_1 element l = lambda_j^{-1/2} sum_i nu_i
      U[i, j] rho_i(l), with rho_i(l) = A_1[i, l] / sigma_l (Eq. (rho omega1
      MC), (eigenfunctions_MC)) and lambda_j = s_j^2 (Prop. coro:B-Lambda);
    * density[l] = (1 / M_D) sum_i rho_i(l), the averaged estimator the
      paper maps in every example (Sec. 5.2);
    * u_sweep[r - 1] = the r-TSVD solution on Gamma_1 (Eq. (tsvd solution
      simulations)), r = 1..r_max;
    * uD_sweep[r - 1] = A_1 u_sweep[r - 1] + A_0 u^0, the fitted interior data
      of item (iv).
    Returns a dict."""
    g1 = np.asarray(gamma1).astype(bool)
    A = np.asarray(counts, dtype=np.float64) / float(N)
    A1, A0 = A[:, g1], A[:, ~g1]
    sig1 = np.asarray(measures, float)[g1]
    nu = np.asarray(nu, float)
    k = len(s)
    Lam = (nu[:, None] * A1 / sig1[None, :]) @ (A1.T * nu[None, :])
    lam = np.sort(np.linalg.eigvalsh(Lam))[::-1][:k]
    rho = A1 / sig1[None, :]
    eigfun = (rho.T @ (nu[:, None] * U)) / s[None, :]
    density = rho.mean(axis=0)
    out = dict(lam=lam, eigfun=eigfun, density=density)
    if r_max > 0:
        b = np.asarray(uD, dtype=np.float64).copy()
        f0 = np.zeros(A.shape[0])
        if u0 is not None and A0.shape[1] > 0:
            f0 = A0 @ np.asarray(u0, dtype=np.float64)
        b = b - f0
        us, ys = [], []
        for r in range(1, r_max + 1):
            w = V[:, :r] @ ((U[:, :r].T @ (nu * b)) / s[:r])
            u1 = w / np.sqrt(sig1)
            us.append(u1)
            ys.append(A1 @ u1 + f0)
        out["u_sweep"] = np.array(us)
        out["uD_sweep"] = np.array(ys)
    return out
