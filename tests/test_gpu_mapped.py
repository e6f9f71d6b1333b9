"""Mapped walks on the GPU (walk-on-spheres in y = S^{-1} x, exact distance to
the polytope S^{-1} D): exits agree walk by walk with the oracle's mapped
chain, batched equals lone, the chain needs far fewer steps than the paper's
for anisotropic K, and unsupported domains are rejected."""
import numpy as np
import pytest
import torch

from gpu_util import ctx, gpu_build, oracle_walks
from paper_2409_03686_gb300 import workloads as W
from paper_2409_03686_gb300 import wos
from test_oracle_mapped import K_RAND3, _hexagon

pytestmark = pytest.mark.gpu

CASES = {
    "square": lambda: W.square_config(N=600, grid=8),
    "cube_diag": lambda: W.cube_config(N=400, n_points=40),
    "cube_rand": lambda: W.cube_config(N=400, n_points=40, K=K_RAND3),
    "hexagon": lambda: _hexagon(N=600).replace(eps=1e-4),
    "square64": lambda: W.square_config(N=300, grid=4).replace(fp64=True, eps=1e-8),
    "cube64": lambda: W.cube_config(N=200, n_points=16, K=K_RAND3).replace(fp64=True,
                                                                            eps=1e-8),
}


@pytest.mark.parametrize("name", list(CASES))
def test_mapped_walks_match_oracle(name):
    """Exit elements as the oracle's for >= 99.9 % of walks (the FP32 bar of
    reading 12: FP32 rounding against the oracle's FP64 decides knife-edge
    stops); step counts as the oracle's for >= 99.9 % of FP64 walks, and for
    >= 99.5 % of FP32 walks (the same chain: a wrong counter, window or move
    would leave almost none equal; a stop that FP32 and FP64 decide on
    opposite sides of eps changes N_eps without moving the exit element)."""
    inst = CASES[name]().replace(mapped=True)
    r = gpu_build(inst, trace_steps=True)
    assert (r["counts"].sum(1) + r["unterm"] == inst.N).all()
    el, ns, _ = oracle_walks(inst)
    agree = (r["trace"] == el).mean()
    assert agree >= 0.999, (name, agree)
    steps_agree = (r["steps"] == ns).mean()
    assert steps_agree >= (0.999 if inst.fp64 else 0.995), (name, steps_agree)


def test_mapped_batch_equals_lone_builds():
    insts = [CASES["square"]().replace(mapped=True, stream=1, seed=7),
             CASES["cube_rand"]().replace(mapped=True, stream=2, seed=7),
             CASES["hexagon"]().replace(mapped=True, stream=3, seed=7)]
    counts, _, _ = wos.wos_build_operators_batched(ctx(), insts, seed=7)
    torch.cuda.synchronize()
    for q, inst in enumerate(insts):
        lone = gpu_build(inst, trace=False)
        np.testing.assert_array_equal(counts[q].cpu().numpy().astype(np.int64),
                                      lone["counts"], err_msg=inst.name)


def test_mapped_chain_takes_fewer_steps():
    for make in (lambda: W.square_config(N=20_000, grid=8),
                 lambda: W.cube_config(N=5_000, n_points=64)):
        inst = make()
        a = gpu_build(inst, trace=False)["stats"]
        b = gpu_build(inst.replace(mapped=True), trace=False)["stats"]
        assert b["steps"] < 0.6 * a["steps"], (inst.name, a["steps"], b["steps"])


def test_unsupported_domains_are_rejected():
    """Polygons must be convex and polytopes hole-free (discs / balls minus
    holes take the quadric bound instead, tested below)."""
    for inst in (W.lshape_config(N=100, n_points=4),
                 W.square_hole_config(N=100, eps=1e-5, n_points=4, fp64=False)):
        with pytest.raises(wos.WosError) as e:
            gpu_build(inst.replace(mapped=True), trace=False)
        assert e.value.code == 1


# ---------------------------------------------------------------------------
# Mapped walks on discs / balls minus holes (the quadric lower bound of the
# distance in y = S^{-1} x as the radius of the paper's ellipsoid steps)
# ---------------------------------------------------------------------------
QUADRIC = {
    "annulus": lambda: W.annulus_config(N=600, grid=8),
    "ball_diag": lambda: W.ball_config(N=500, n_points=40),
    "ball_rand": lambda: W.config3_instances(N=500, n_points=40)[1],
    "shell_shifted": lambda: W.shell_config(N=500, shift=0.3, n_points=40,
                                            K=W.config3_instances(N=1, n_points=1)[1].K),
    "perforated": lambda: W.perforated_disc_config(N=600, eps=1e-5, fp64=False, n_points=40,
                                                   m_outer=100, m_hole=20).replace(
                                                       K=W.K_CONFIG2),
    "ball_fp64": lambda: W.ball_config(N=300, n_points=20).replace(fp64=True, eps=1e-8),
}


@pytest.mark.parametrize("name", list(QUADRIC))
def test_quadric_mapped_walks_match_oracle(name):
    """Walk by walk against the oracle's mapped chain (the same bound in
    FP64): >= 99.9 % of exit elements equal; counts differ by at most the
    disagreeing walks; far fewer steps than the paper's chain."""
    inst = QUADRIC[name]().replace(mapped=True)
    r = gpu_build(inst, trace_steps=True)
    tr = r["trace"]
    assert (tr >= -1).all()
    assert (r["counts"].sum(1) + r["unterm"] == inst.N).all()
    el, ns, _ = oracle_walks(inst)
    agree = (tr == el).mean()
    assert agree >= 0.999, (name, agree)
    plain = gpu_build(inst.replace(mapped=False), trace=False)
    assert r["stats"]["steps"] < 0.8 * plain["stats"]["steps"], name
