"""Parity of the CUDA walk kernel (wos_build_operator) with the FP64 oracle.

With the same Philox counters the GPU and the oracle run the same chain, so
exit elements are compared walk by walk: at least 99.9 % must agree (the
rest are knife-edge walks where FP32 rounding differs from FP64), integer
counts must equal the histogram of the GPU's own per-walk trace bit for bit,
and every row must sum to N exactly.  FP64 walks agree with the oracle to
rounding, so their agreement is essentially total."""
import dataclasses
import math

import numpy as np
import pytest
import torch

from gpu_util import ctx, gpu_build, oracle_walks
from oracle import closed_forms as CF
from paper_2409_03686_gb300 import workloads as W
from paper_2409_03686_gb300 import wos
from stats_util import beta_eps, check_band

pytestmark = pytest.mark.gpu


def _hist(trace, M):
    out = np.zeros((trace.shape[0], M), np.int64)
    for i in range(trace.shape[0]):
        t = trace[i]
        out[i] = np.bincount(t[t >= 0], minlength=M)
    return out


def _check_consistent(inst, r):
    tr = r["trace"]
    assert (tr >= -1).all(), "every walk must be traced"
    np.testing.assert_array_equal(r["counts"], _hist(tr, inst.M_tot))
    np.testing.assert_array_equal(r["unterm"], (tr == -1).sum(1))
    assert (r["counts"].sum(1) + r["unterm"] == tr.shape[1]).all()


def test_fp64_walks_match_oracle_walk_by_walk():
    inst = W.disc_config(N=2000, fp64=True)
    r = gpu_build(inst, trace_steps=True)
    _check_consistent(inst, r)
    el, ns, _ = oracle_walks(inst)
    agree = (r["trace"] == el).mean()
    assert agree >= 0.9999, agree
    assert (r["steps"] == ns).mean() >= 0.9999
    assert r["stats"]["walks"] == inst.M_D * inst.N
    assert r["stats"]["steps"] == int(r["steps"].sum())


def _stretched(inst, half):
    """The instance on a box with the given half-extents, points scaled with it."""
    old = np.asarray(inst.domain.half[:inst.dim], float)
    new = np.asarray(half[:inst.dim], float)
    dom = dataclasses.replace(inst.domain, half=tuple(half))
    return inst.replace(domain=dom, points=inst.points * (new / old),
                        name=inst.name + "-stretched")


def _moved(inst, center):
    """The instance with its domain and points moved to the given centre."""
    c = np.asarray(center[:inst.dim], float) - np.asarray(inst.domain.center[:inst.dim], float)
    dom = dataclasses.replace(inst.domain, center=tuple(center))
    return inst.replace(domain=dom, points=inst.points + c, name=inst.name + "-moved")


GEOMS = {
    "disc32": lambda: W.disc_config(N=1000, fp64=False),
    "square": lambda: W.square_config(N=600, grid=8),
    "annulus": lambda: W.annulus_config(N=600, grid=8),
    "lshape": lambda: W.lshape_config(N=600, n_points=40),
    "perforated": lambda: W.perforated_disc_config(N=600, eps=1e-5, fp64=False,
                                                   n_points=40, m_outer=100, m_hole=20),
    "ball": lambda: W.ball_config(N=500, n_points=40),
    "ball_rand_K": lambda: W.config3_instances(N=500, n_points=40)[1],
    "cube": lambda: W.cube_config(N=500, n_points=40),
    # unequal half-extents: the general box kernel (squares and cubes take
    # the equal-extent one)
    "rectangle": lambda: _stretched(W.square_config(N=600, grid=8), (0.5, 0.3, 0.0)),
    "cuboid": lambda: _stretched(W.cube_config(N=500, n_points=40), (1.0, 0.8, 0.6)),
    "square_moved": lambda: _moved(W.square_config(N=600, grid=8), (0.2, -0.1, 0.0)),
    "shell": lambda: W.shell_config(N=500, shift=0.3, n_points=40),
    "shell_concentric": lambda: W.shell_config(N=500, shift=0.0, n_points=40),
    "square_hole": lambda: W.square_hole_config(example=1, N=600, eps=1e-5, fp64=False),
    "square_hole_ex5": lambda: W.square_hole_config(example=5, N=600, eps=1e-5, fp64=False),
    "shell_voronoi": lambda: W.shell_config(N=500, shift=0.3, n_points=40, voronoi=(300, 60)),
    "shell_voronoi64": lambda: W.shell_config(N=300, shift=0.3, n_points=20, voronoi=(300, 60),
                                              fp64=True, eps=1e-8),
    "annulus_voronoi": lambda: W.annulus_voronoi_config(N=600, eps=1e-5, fp64=False,
                                                        n_points=40, m0=200, m1=60),
    "ball64": lambda: W.ball_config(N=300, n_points=20).replace(fp64=True),
    "lshape64": lambda: W.lshape_config(N=300, n_points=20).replace(fp64=True, eps=1e-8),
}


@pytest.mark.parametrize("name", list(GEOMS))
def test_walks_match_oracle(name):
    inst = GEOMS[name]()
    r = gpu_build(inst, trace_steps=True)
    _check_consistent(inst, r)
    el, ns, _ = oracle_walks(inst)
    agree = (r["trace"] == el).mean()
    assert agree >= 0.999, (name, agree)
    # counts differ from the oracle's by at most the disagreeing walks
    Co = _hist(el, inst.M_tot)
    bad = (r["trace"] != el).sum(1)
    assert (np.abs(r["counts"] - Co).sum(1) <= 2 * bad).all()


def test_schedule_does_not_change_results():
    inst = W.square_config(N=1000, grid=6)
    ref = gpu_build(inst, trace=False)["counts"]
    for kw in [dict(tile_walks=64), dict(tile_walks=96, hist_slots=1),
               dict(tile_walks=1000, hist_slots=-1), dict(block_size=64, blocks_per_sm=1),
               dict(block_size=128, tile_walks=32, hist_slots=2)]:
        np.testing.assert_array_equal(gpu_build(inst, trace=False, **kw)["counts"], ref)


@pytest.mark.parametrize("make", [
    lambda: W.square_config(N=2000, grid=6),
    lambda: W.cube_config(N=800, n_points=24),
])
def test_equal_extent_box_kind_matches_box_kind(make):
    """A square / cube walks on the equal-half-extent kernel (distance h -
    max |x_a|); a box whose half-extents differ only in FP64 (by 1e-12, the
    same FP32 values) walks on the general box kernel (min (h_a - |x_a|)).
    The rounding of h - t is monotone in t, so both give the same FP32
    distances and the same walks bit for bit."""
    inst = make()
    half = list(inst.domain.half)
    for a in range(1, inst.dim):
        half[a] += 1e-12
    assert all(np.float32(half[a]) == np.float32(half[0]) for a in range(inst.dim))
    boxed = inst.replace(domain=dataclasses.replace(inst.domain, half=tuple(half)))
    r_eq = gpu_build(inst, trace_steps=True)
    r_box = gpu_build(boxed, trace_steps=True)
    np.testing.assert_array_equal(r_eq["counts"], r_box["counts"])
    np.testing.assert_array_equal(r_eq["trace"], r_box["trace"])
    np.testing.assert_array_equal(r_eq["steps"], r_box["steps"])


@pytest.mark.parametrize("make", [
    lambda: W.square_config(N=1000, grid=6),
    lambda: W.annulus_config(N=800, grid=4),
    lambda: W.ball_config(N=600, n_points=24),
    lambda: W.square_config(N=400, grid=4).replace(fp64=True, eps=1e-8),
    lambda: W.square_config(N=500, grid=4).replace(step_cap=13),
])
def test_group_length_does_not_change_results(make):
    """Walks advance group_blocks Philox blocks per refill; the counter of
    step n is n / (steps per block) whatever the group, so counts, the
    unterminated tallies (with a step cap inside a group) and every exit
    are the same for every group length."""
    inst = make()
    ref = gpu_build(inst, group_blocks=1)
    for nb in (2, 3, 5, 16):
        got = gpu_build(inst, group_blocks=nb)
        np.testing.assert_array_equal(got["counts"], ref["counts"])
        np.testing.assert_array_equal(got["unterm"], ref["unterm"])
        np.testing.assert_array_equal(got["trace"], ref["trace"])


def test_resume_is_bit_identical():
    inst = W.annulus_config(N=1500, grid=4)
    full = gpu_build(inst, trace=False)
    a = gpu_build(inst, trace=False, k0=0, k1=700)
    b = gpu_build(inst, trace=False, k0=700, k1=1500, counts=a["counts_t"],
                  unterminated=a["unterm_t"], accumulate=True)
    np.testing.assert_array_equal(b["counts"], full["counts"])
    np.testing.assert_array_equal(b["unterm"], full["unterm"])


def test_step_cap_leaves_walks_unterminated():
    inst = W.square_config(N=800, grid=4).replace(step_cap=4)
    r = gpu_build(inst, trace_steps=True)
    _check_consistent(inst, r)
    assert r["unterm"].sum() > 0
    assert r["stats"]["unterminated"] == r["unterm"].sum()
    assert r["steps"].max() == 4
    el, ns, _ = oracle_walks(inst)
    assert (r["trace"] == el).mean() >= 0.999


def test_edge_cases():
    # one point, one walk; a ragged tail of tiles
    inst = W.disc_config(N=1, fp64=False).replace(points=np.array([[0.3, -0.2]]))
    r = gpu_build(inst)
    _check_consistent(inst, r)
    inst = W.disc_config(N=33, fp64=False)
    r = gpu_build(inst, tile_walks=32)
    _check_consistent(inst, r)
    el, _, _ = oracle_walks(inst)
    assert (r["trace"] == el).mean() >= 0.99
    # a point already inside the eps-shell stops with N_eps = 0
    inst = W.disc_config(N=64, fp64=False, eps=1e-4).replace(
        points=np.array([[0.99995, 0.0], [0.0, -0.5]]))
    r = gpu_build(inst, trace_steps=True)
    assert (r["steps"][0] == 0).all() and (r["trace"][0] == 0).all()
    # many elements: the shared-memory histogram is replaced by HBM atomics
    # (cells 1e-4 rad wide are below FP32 position resolution: FP64 walks)
    inst = W.disc_config(N=400, fp64=True).replace(
        partition=W.Partition(outer_m=60000, gamma1=np.ones(60000, np.uint8)))
    r = gpu_build(inst)
    assert r["stats"]["hist_slots"] == 0
    _check_consistent(inst, r)
    el, _, _ = oracle_walks(inst)
    assert (r["trace"] == el).mean() >= 0.999


def test_closed_form_disc_fp32():
    inst = W.disc_config(N=100_000, fp64=False)
    r = gpu_build(inst, trace=False)
    A = r["counts"] / inst.N
    P = np.array([CF.disc_row(x, 32) for x in inst.points])
    ok, info = check_band(A, P, inst.N, beta_eps(inst.eps, 0.75 / (2 * math.pi * 0.25)))
    assert ok, info


def test_closed_form_disc_fp32_large_n():
    """The FP32 chain's random-number map (Philox words, 23-bit windows, the
    FMA angle) at N = 1e6 walks per point on config 1's disc: every arc of
    every point within the Bonferroni band of the Poisson kernel, whose
    statistical width is now ten times narrower than at N = 1e5 -- a defect
    of the direction map (a bias of the angle of 1e-3 or a lost window) would
    leave it."""
    inst = W.disc_config(N=1_000_000, fp64=False)
    r = gpu_build(inst, trace=False)
    assert (r["counts"].sum(1) + r["unterm"] == inst.N).all()
    A = r["counts"] / inst.N
    P = np.array([CF.disc_row(x, 32) for x in inst.points])
    ok, info = check_band(A, P, inst.N, beta_eps(inst.eps, 0.75 / (2 * math.pi * 0.25)))
    assert ok, info


def test_closed_form_ball_fp32():
    inst = W.ball_config(N=100_000, n_points=16, nb=4, ns=6, K=np.eye(3))
    r = gpu_build(inst, trace=False)
    A = r["counts"] / inst.N
    P = np.array([CF.ball_patch_row(x, 4, 6) for x in inst.points])
    rmax = np.linalg.norm(inst.points, axis=1).max()
    ok, info = check_band(A, P, inst.N,
                          beta_eps(inst.eps, (1 - rmax ** 2) / (4 * math.pi * (1 - rmax) ** 3)))
    assert ok, info


def test_harmonic_martingale_on_gpu_exit_points():
    # E[u(X_exit)] = u(x) for the K-harmonic cubic (no eps bias)
    inst = W.annulus_config(N=20_000, grid=2)
    r = gpu_build(inst, trace_x=True)
    u = W.k_harmonic_cubic(inst.K)
    vals = u(r["x"])
    z = (vals.mean(1) - u(inst.points)) / (vals.std(1) / math.sqrt(inst.N))
    assert np.abs(z).max() < 4.5, z


@pytest.mark.parametrize("make", [
    W.square_config,
    W.annulus_config,
    lambda: W.config3_instances()[0],   # ball, K = diag(1, 2, 4)
    lambda: W.config3_instances()[3],   # cube, random SPD K
], ids=["square", "annulus", "ball-diag124", "cube-randK"])
def test_full_size_sampled_parity(make):
    """The benchmark instances at full size (2-D: 256 points, N = 1e5, eps =
    1e-5; 3-D: 1024 points, 1536 patches, N = 1e5, eps = 1e-4; FP32) in the
    default launch configuration: every row sums to N exactly, three sampled
    rows are replayed walk by walk by the oracle, and the untraced launch the
    benchmark times gives the traced launch's counts bit for bit."""
    inst = make()
    r = gpu_build(inst)
    _check_consistent(inst, r)
    rows = [0, inst.M_D // 2 + 9, inst.M_D - 1]
    el, _, _ = oracle_walks(inst, rows=rows)
    agree = (r["trace"][rows] == el).mean()
    assert agree >= 0.999, agree
    u = gpu_build(inst, trace=False)
    np.testing.assert_array_equal(u["counts"], r["counts"])
    np.testing.assert_array_equal(u["unterm"], r["unterm"])


def test_point_outside_is_reported_and_runs_no_walk():
    """An observation point outside D (the L-shape's missing quadrant, where
    the unsigned polygon distance stays positive) or on dD: the build runs no
    walk; with statistics it returns WOS_POINT_OUTSIDE, without them it
    returns at once and every row sums to zero.  The no-allocation build
    behaves the same."""
    inst = W.lshape_config(N=5000, m_total=24, n_points=4)
    for bad in ([0.5, -0.5], [1.0, 0.5]):
        pts = inst.points.copy()
        pts[2] = bad
        b = inst.replace(points=pts)
        with pytest.raises(wos.WosError) as e:
            gpu_build(b, trace=False)
        assert e.value.code == 3
        t = torch.as_tensor(pts, dtype=torch.float64, device=torch.device("cuda:0"))
        c, u, st = wos.wos_build_operator(ctx(), b.domain, b.K, t, b.partition, b.N, b.eps,
                                          b.seed, stats=False)
        torch.cuda.synchronize()
        assert st is None and int(c.abs().sum()) == 0 and int(u.abs().sum()) == 0
        c2 = torch.full_like(c, 5)
        with pytest.raises(wos.WosError) as e:
            wos.wos_build_operator_noalloc(ctx(), b.domain, b.K, t, b.partition, b.N,
                                           b.eps, b.seed, c2)
        assert e.value.code == 3
        assert int(c2.abs().sum()) == 0
    # the same points inside D build normally
    r = gpu_build(inst)
    _check_consistent(inst, r)


def test_errors_are_reported():
    inst = W.square_config(N=10, grid=2)
    with pytest.raises(wos.WosError) as e:
        gpu_build(inst.replace(K=np.array([[1.0, 2.0], [2.0, 1.0]])), trace=False)
    assert e.value.code == 2
    with pytest.raises(wos.WosError) as e:
        gpu_build(inst.replace(eps=1e-7), trace=False)
    assert e.value.code == 4
    with pytest.raises(wos.WosError) as e:
        gpu_build(inst, trace=False, k0=5, k1=3)
    assert e.value.code == 1


def _golden(key):
    from pathlib import Path
    for line in open(Path(__file__).resolve().parent / "golden" / "paper_printed_values.txt"):
        if line.strip() and not line.startswith("#"):
            k, v, _ = line.split()
            if k == key:
                return float(v)
    raise KeyError(key)


def test_paper_eps_perforated_disc_fp64():
    """Ex. 5.4 at the paper's eps = 1e-10 with FP64 walks (500 + 5 x 100
    arcs, 100 points on the circle at distance 0.05 from Gamma_0): the
    averaged harmonic measure of Gamma_1 lies within the printed 0.1126 +-
    0.002 (Sec. 1), and the first 2000 walks of three rows are replayed walk
    by walk by the oracle at the same eps."""
    inst = W.perforated_disc_config(N=20_000, eps=1e-10)
    r = gpu_build(inst, trace=False)
    assert (r["counts"].sum(1) + r["unterm"] == inst.N).all()
    assert r["unterm"].sum() == 0
    g1 = inst.partition.gamma1.astype(bool)
    avg = (r["counts"][:, g1].sum(1) / inst.N).mean()
    assert abs(avg - _golden("avg_mu_gamma1_on_dotted_circle")) < 2e-3, avg
    part = gpu_build(inst, k0=0, k1=2000, trace_steps=True)
    rows = [0, 37, 99]
    el, ns, _ = oracle_walks(inst, rows=rows, k0=0, k1=2000)
    agree = (part["trace"][rows] == el).mean()
    assert agree >= 0.999, agree
    assert (part["steps"][rows] == ns).mean() >= 0.999


def test_paper_eps_annulus_fp64():
    """Ex. 5.2's annulus (K = I, extrinsic Voronoi cells of 500 + 100 equally
    spaced sites) at eps = 1e-10 with FP64 walks: the measure of the inner
    circle averaged over the 100 points at radius 0.95 against ln r / ln a =
    0.0740005814 (4 sigma + beta(eps)), and three rows walk by walk against
    the oracle."""
    inst = W.annulus_voronoi_config(N=20_000, eps=1e-10)
    r = gpu_build(inst, trace=False)
    assert (r["counts"].sum(1) + r["unterm"] == inst.N).all()
    g1 = inst.partition.gamma1.astype(bool)
    mu = r["counts"][:, g1].sum(1) / inst.N
    p = math.log(0.95) / math.log(0.5)
    sd = math.sqrt(p * (1 - p) / (inst.N * inst.M_D))
    assert abs(mu.mean() - p) <= 4 * sd + 1e-9, (mu.mean(), p, sd)
    part = gpu_build(inst, k0=0, k1=2000)
    rows = [0, 50, 99]
    el, _, _ = oracle_walks(inst, rows=rows, k0=0, k1=2000)
    assert (part["trace"][rows] == el).mean() >= 0.999
