"""wos_build_operator_noalloc against wos_build_operator.

The allocation-free entry point serves callers that may not allocate device
memory (a fixed, pre-reserved device budget, or a host framework that owns all
device allocation).  It must give the same counts as the regular entry point:
the walks are deterministic per walk id, so the tolerance of the integer
counts is zero.  Two calls in a row check that the shared scratch array is
reset between calls (the second call uses a Voronoi partition, whose site
table also lives in that array).  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from gpu_util import ctx
from paper_2409_03686_gb300 import workloads as W
from paper_2409_03686_gb300 import wos

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _regular(inst):
    pts = torch.as_tensor(inst.points, dtype=torch.float64, device=DEV)
    c, u, st = wos.wos_build_operator(ctx(), inst.domain, inst.K, pts, inst.partition,
                                      inst.N, inst.eps, inst.seed,
                                      opts=wos.make_opts(precision=int(inst.fp64)))
    torch.cuda.synchronize()
    return c.cpu().numpy(), u.cpu().numpy(), st


def _noalloc(inst):
    pts = torch.as_tensor(inst.points, dtype=torch.float64, device=DEV)
    counts = torch.full((inst.M_D, inst.M_tot), 7, dtype=torch.int32, device=DEV)
    unterm = torch.full((inst.M_D,), 7, dtype=torch.int32, device=DEV)
    c, u, st = wos.wos_build_operator_noalloc(ctx(), inst.domain, inst.K, pts,
                                              inst.partition, inst.N, inst.eps, inst.seed,
                                              counts, unterm,
                                              opts=wos.make_opts(precision=int(inst.fp64)))
    torch.cuda.synchronize()
    return c.cpu().numpy(), u.cpu().numpy(), st


def _voronoi_instance():
    inst = W.square_config(N=3000, grid=6, n_side=12)
    sites = W.element_centres(inst.domain, inst.partition)
    part = W.Partition(voronoi_sites=sites, gamma1=inst.partition.gamma1)
    return inst.replace(partition=part)


def test_noalloc_matches_regular_build_twice_in_a_row():
    first = W.square_config(N=4000, grid=8)
    second = _voronoi_instance()
    for inst in (first, second):
        ref_c, ref_u, ref_st = _regular(inst)
        c, u, st = _noalloc(inst)
        np.testing.assert_array_equal(c, ref_c)
        np.testing.assert_array_equal(u, ref_u)
        assert (c.astype(np.int64).sum(1) + u == inst.N).all()
        assert st["walks"] == ref_st["walks"] == inst.M_D * inst.N
        assert st["steps"] == ref_st["steps"]


def test_noalloc_rejects_problems_beyond_its_scratch():
    inst = _voronoi_instance()
    sites = np.tile(W.element_centres(inst.domain, inst.partition), (60, 1))[:2049]
    big = inst.replace(partition=W.Partition(voronoi_sites=sites,
                                             gamma1=np.ones(2049, np.uint8)))
    pts = torch.as_tensor(big.points, dtype=torch.float64, device=DEV)
    counts = torch.zeros((big.M_D, 2049), dtype=torch.int32, device=DEV)
    with pytest.raises(wos.WosError) as e:
        wos.wos_build_operator_noalloc(ctx(), big.domain, big.K, pts, big.partition,
                                       big.N, big.eps, big.seed, counts)
    assert e.value.code == 13
