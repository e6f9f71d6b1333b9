"""wos_build_operators_batched: a mixed batch (disc, annulus, square, L-shape,
ball, box; uneven sizes, eps and K) in one launch per dimension gives, for
every instance, the counts of the same instance built alone -- bit for bit,
since every walk's Philox counter carries the instance's stream id -- and
those counts agree walk by walk with the FP64 oracle."""
import numpy as np
import pytest
import torch

from gpu_util import ctx, gpu_build, oracle_walks
from paper_2409_03686_gb300 import workloads as W
from paper_2409_03686_gb300 import wos

pytestmark = pytest.mark.gpu


def _small_batch(n=12):
    return W.mixed_batch(n_instances=n, seed=7, m_lo=16, m_hi=160, n_lo=200, n_hi=3000)


def test_batch_equals_lone_builds():
    insts = _small_batch()
    assert {i.dim for i in insts} == {2, 3}
    counts, unterm, st = wos.wos_build_operators_batched(ctx(), insts, seed=7)
    torch.cuda.synchronize()
    assert st["walks"] == sum(i.M_D * i.N for i in insts)
    for q, inst in enumerate(insts):
        lone = gpu_build(inst, trace=False)
        np.testing.assert_array_equal(counts[q].cpu().numpy().astype(np.int64),
                                      lone["counts"], err_msg=inst.name)
        np.testing.assert_array_equal(unterm[q].cpu().numpy().astype(np.int64), lone["unterm"])


def test_batch_walks_match_oracle():
    insts = _small_batch()
    counts, unterm, st = wos.wos_build_operators_batched(ctx(), insts, seed=7)
    torch.cuda.synchronize()
    for q in (0, 4, 5):  # a disc, a ball and a box
        inst = insts[q]
        rows = [0, inst.M_D - 1]
        el, _, _ = oracle_walks(inst, rows=rows)
        C = counts[q].cpu().numpy().astype(np.int64)[rows]
        Co = np.stack([np.bincount(e[e >= 0], minlength=inst.M_tot) for e in el])
        # the histogram of the oracle's exits differs from the GPU's counts by
        # at most two per disagreeing walk (0.1 % allowed)
        assert np.abs(C - Co).sum() <= 2 * max(1, int(0.001 * el.size)), inst.name


def test_batch_options_and_errors():
    insts = _small_batch(4)
    c1, u1, _ = wos.wos_build_operators_batched(ctx(), insts, seed=7)
    c2, u2, _ = wos.wos_build_operators_batched(
        ctx(), insts, seed=7, opts=wos.make_opts(block_size=128, tile_walks=64, hist_slots=-1))
    torch.cuda.synchronize()
    for a, b in zip(c1, c2):
        assert torch.equal(a, b)
    with pytest.raises(wos.WosError) as e:
        wos.wos_build_operators_batched(ctx(), insts, seed=7, opts=wos.make_opts(k0=1))
    assert e.value.code == 1


def test_autotune_picks_a_config_without_changing_results():
    inst = W.square_config(N=3000, grid=8)
    wos.wos_autotune_reset(ctx())
    ref = gpu_build(inst, trace=False)["counts"]
    t = wos.wos_autotune(ctx(), inst, sample_walks=2_000_000)
    assert t["trials"] >= 6 and t["best_ms"] > 0 and t["best_ms"] <= t["default_ms"]
    assert t["block_size"] in (128, 256) and t["refill_min"] in (1, 4, 8)
    assert t["tiles_per_warp"] in (4, 16, 64) and t["hist_slots"] in (0, -1)
    tuned = gpu_build(inst, trace=False)  # default opts now use the tuned config
    np.testing.assert_array_equal(tuned["counts"], ref)
    assert tuned["stats"]["block"] == t["block_size"]
    wos.wos_autotune_reset(ctx())


def test_batch_with_voronoi_instances_equals_lone_builds():
    """Extrinsic-Voronoi instances (candidate grids in the batch scratch) next
    to cell-partition ones: every instance's counts equal its lone build."""
    insts = [W.shell_config(N=400, shift=0.3, n_points=24, voronoi=(300, 60)).replace(stream=1),
             W.annulus_voronoi_config(N=500, eps=1e-5, fp64=False, n_points=24, m0=200,
                                      m1=60).replace(stream=2),
             W.disc_config(N=500, fp64=False).replace(stream=3),
             W.ball_config(N=300, n_points=24).replace(stream=4)]
    insts = [i.replace(seed=7) for i in insts]
    counts, unterm, st = wos.wos_build_operators_batched(ctx(), insts, seed=7)
    torch.cuda.synchronize()
    for q, inst in enumerate(insts):
        lone = gpu_build(inst, trace=False)
        np.testing.assert_array_equal(counts[q].cpu().numpy().astype(np.int64),
                                      lone["counts"], err_msg=inst.name)
