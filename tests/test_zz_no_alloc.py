"""wos_build_operator_noalloc against wos_build_operator.

The allocation-free entry point serves callers that may not allocate device
memory (a fixed, pre-reserved device budget, or a host framework that owns all
device allocation).  It must give the same counts as the regular entry point:
the walks are deterministic per walk id, so the tolerance of the integer
counts is zero.  Two calls in a row check that the shared scratch array is
reset between calls (the second call uses a Voronoi partition, whose site
table also lives in that array).  The device's stream-ordered memory pool and
the free device memory are read around the calls to show that they allocate
nothing.  This file is collected last on purpose."""
import ctypes

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


class _DevicePool:
    """Used / reserved bytes of the device's default stream-ordered memory
    pool (where cudaMallocAsync allocates), read through the driver API; the
    high-water mark of the used bytes is reset so that an allocation made
    and freed inside a call still shows."""

    USED_HIGH, USED_CUR, RESERVED_CUR = 8, 7, 5   # CUmemPool_attribute

    def __init__(self, device=0):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), device) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_HIGH,
                                             ctypes.byref(zero)) == 0


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


def test_noalloc_allocates_no_device_memory():
    """Two calls (with and without statistics; the call without them is
    asynchronous and is synchronised here) leave the pool's used-bytes
    high-water mark, its reserved bytes and the free device memory as they
    were, and give the regular build's counts."""
    inst = _voronoi_instance()
    ref_c, ref_u, _ = _regular(inst)
    pts = torch.as_tensor(inst.points, dtype=torch.float64, device=DEV)
    outs = [(torch.full((inst.M_D, inst.M_tot), 7, dtype=torch.int32, device=DEV),
             torch.full((inst.M_D,), 7, dtype=torch.int32, device=DEV)) for _ in range(2)]
    opts = wos.make_opts(precision=int(inst.fp64))
    # the first call on the device looks the scratch array up: do it before
    # measuring, as a caller would at set-up
    wos.wos_build_operator_noalloc(ctx(), inst.domain, inst.K, pts, inst.partition, inst.N,
                                   inst.eps, inst.seed, *outs[0], opts=opts)
    torch.cuda.synchronize()
    pool = _DevicePool(0)
    used0, reserved0 = pool.get(pool.USED_CUR), pool.get(pool.RESERVED_CUR)
    pool.reset_high()
    free0, _ = torch.cuda.mem_get_info(DEV)
    for stats, (c, u) in zip((True, False), outs):
        wos.wos_build_operator_noalloc(ctx(), inst.domain, inst.K, pts, inst.partition,
                                       inst.N, inst.eps, inst.seed, c, u, opts=opts,
                                       stats=stats)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert pool.get(pool.USED_HIGH) <= used0
    assert pool.get(pool.RESERVED_CUR) == reserved0
    assert free1 == free0
    for c, u in outs:
        np.testing.assert_array_equal(c.cpu().numpy(), ref_c)
        np.testing.assert_array_equal(u.cpu().numpy(), ref_u)


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


def test_noalloc_rejects_mismatched_buffers_before_any_launch():
    """The caller sizes the buffers on this path: an undersized counts or
    unterminated tensor, float32 or non-contiguous points are refused by the
    binding before the library is called (no kernel launch)."""
    inst = W.square_config(N=1000, grid=4)
    pts = torch.as_tensor(inst.points, dtype=torch.float64, device=DEV)
    good = torch.zeros((inst.M_D, inst.M_tot), dtype=torch.int32, device=DEV)
    cases = [
        dict(points=pts, counts=good[:, :-1].contiguous()),
        dict(points=pts, counts=good, unterminated=torch.zeros(inst.M_D - 1, dtype=torch.int32,
                                                               device=DEV)),
        dict(points=pts.float(), counts=good),
        dict(points=torch.cat([pts, pts], 1)[:, ::2], counts=good),
        dict(points=pts, counts=good.to(torch.int64)),
        dict(points=pts.cpu(), counts=good),
    ]
    before = ctx().kernel_launches()
    for kw in cases:
        with pytest.raises(wos.WosError) as e:
            wos.wos_build_operator_noalloc(ctx(), inst.domain, inst.K, kw["points"],
                                           inst.partition, inst.N, inst.eps, inst.seed,
                                           kw["counts"], kw.get("unterminated"))
        assert e.value.code == 1
    assert ctx().kernel_launches() == before
