"""The C ABI library on the CPU: it loads, exports every symbol the headers
declare, its struct layout matches the binding, and its host-side logic
(K set-up, element counts and measures, point check, FP32 floor, truncation
rule) agrees with the oracle.  No device code runs here."""
import ctypes
import math
import re
import subprocess
from pathlib import Path

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_03686_gb300 import build as B
from paper_2409_03686_gb300 import workloads as W
from paper_2409_03686_gb300 import wos

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    B.build()
    return wos.load()


def _declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = h.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(wos_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "wos_build_operator" in names and "wos_op_svd" in names
    assert "wos_reconstruct" in names
    out = subprocess.run(["nm", "-D", "--defined-only", str(wos.LIB_PATH)],
                         capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_struct_layout_matches_binding(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stddef.h>
#include <stdio.h>
#include "wos.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(wos_domain), sizeof(wos_partition),
         sizeof(wos_opts), sizeof(wos_stats));
  printf("%zu %zu %zu %zu\\n", offsetof(wos_domain, hole_radius),
         offsetof(wos_partition, voronoi_sites), offsetof(wos_opts, kernel_events),
         offsetof(wos_stats, kernel_ms));
  printf("%zu %zu\\n", sizeof(wos_svd_problem), offsetof(wos_svd_problem, V));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(wos_problem), sizeof(wos_request),
         sizeof(wos_queue_opts), sizeof(wos_queue_stats), offsetof(wos_problem, k1),
         offsetof(wos_request, r_used), offsetof(wos_queue_opts, side_streams),
         offsetof(wos_queue_stats, queued));
  printf("%zu %zu %zu %zu\\n", offsetof(wos_opts, group_blocks), sizeof(wos_tuning),
         offsetof(wos_tuning, group_blocks), offsetof(wos_tuning, best_ms));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", str(ROOT / "include"), str(src), "-o", str(exe)],
                   check=True)
    a, b, sp, c, t = subprocess.run([str(exe)], capture_output=True, text=True,
                                    check=True).stdout.split("\n")[:5]
    assert [int(x) for x in t.split()] == [
        wos.WosOpts.group_blocks.offset, ctypes.sizeof(wos.WosTuning),
        wos.WosTuning.group_blocks.offset, wos.WosTuning.best_ms.offset]
    assert [int(x) for x in sp.split()] == [ctypes.sizeof(wos.WosSvdProblem),
                                            wos.WosSvdProblem.V.offset]
    sizes = [int(x) for x in a.split()]
    offs = [int(x) for x in b.split()]
    assert sizes == [ctypes.sizeof(wos.WosDomain), ctypes.sizeof(wos.WosPartition),
                     ctypes.sizeof(wos.WosOpts), ctypes.sizeof(wos.WosStats)]
    assert offs == [wos.WosDomain.hole_radius.offset,
                    wos.WosPartition.voronoi_sites.offset,
                    wos.WosOpts.kernel_events.offset, wos.WosStats.kernel_ms.offset]
    assert [int(x) for x in c.split()] == [
        ctypes.sizeof(wos.WosProblem), ctypes.sizeof(wos.WosRequest),
        ctypes.sizeof(wos.WosQueueOpts), ctypes.sizeof(wos.WosQueueStats),
        wos.WosProblem.k1.offset, wos.WosRequest.r_used.offset,
        wos.WosQueueOpts.side_streams.offset, wos.WosQueueStats.queued.offset]


def test_conductivity_sqrt_matches_oracle(lib):
    rng = np.random.default_rng(4)
    for d in (2, 3):
        for _ in range(10):
            K = W.random_spd(rng, d, 0.2, 9.0)
            np.testing.assert_allclose(wos.wos_conductivity_sqrt(K), O.setup_S(K)[0],
                                       atol=2e-15)
    np.testing.assert_allclose(wos.wos_conductivity_sqrt(W.K_CONFIG2),
                               O.setup_S(W.K_CONFIG2)[0], atol=2e-15)
    with pytest.raises(wos.WosError) as e:
        wos.wos_conductivity_sqrt(np.array([[1.0, 2.0], [2.0, 1.0]]))
    assert e.value.code == 2
    with pytest.raises(wos.WosError):
        wos.wos_conductivity_sqrt(np.array([[1.0, 0.4], [0.0, 1.0]]))


CASES = {
    "disc": lambda: W.disc_config(),
    "annulus": lambda: W.annulus_config(),
    "square": lambda: W.square_config(),
    "lshape": lambda: W.lshape_config(),
    "perforated": lambda: W.perforated_disc_config(),
    "ball": lambda: W.ball_config(n_points=16),
    "cube": lambda: W.cube_config(n_points=16),
    "shell": lambda: W.shell_config(shift=0.3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_elements_measures_points(lib, name):
    inst = CASES[name]()
    n = wos.wos_num_elements(inst.domain, inst.partition)
    assert n == inst.M_tot == O.num_elements(inst.domain, inst.partition)
    np.testing.assert_allclose(wos.wos_element_measures(inst.domain, inst.partition),
                               O.element_measures(inst.domain, inst.partition),
                               rtol=1e-14)
    assert wos.wos_check_points(inst.domain, inst.points) == -1
    bad = inst.points.copy()
    bad[3] = 5.0  # far outside
    assert wos.wos_check_points(inst.domain, bad) == 3
    assert inst.eps >= wos.wos_fp32_eps_floor(inst.domain) or inst.fp64


def test_fp32_floor_and_truncation_rule(lib):
    D = W.disc_config().domain
    assert wos.wos_fp32_eps_floor(D) == pytest.approx(128 * 2.0 ** -24)
    assert wos.wos_fp32_eps_floor(D) < 1e-5
    S = np.array([1.0, 0.5, 0.45, 0.1])
    assert wos.wos_truncation_gap(S, 1)       # 2.0 >= 1.5
    assert not wos.wos_truncation_gap(S, 2)   # 1.11 < 1.5
    assert wos.wos_truncation_gap(S, 3)
    assert wos.wos_truncation_gap(S, 4)


def test_invalid_descriptors_rejected(lib):
    inst = W.lshape_config()
    dom = W.Domain(dim=2, outer="polygon", vertices=tuple(reversed(inst.domain.vertices)))
    assert wos.wos_num_elements(dom, inst.partition) == -1  # clockwise
    part = W.Partition(edge_m=(0, 4, 4, 4))
    sq = W.square_config()
    assert wos.wos_num_elements(sq.domain, part) == -1


def test_no_gpu_means_loud_failure(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(wos.WosError):
        wos.Context(0)


def test_voronoi_partition_with_holes_marshals(lib):
    inst = W.annulus_config(m_each=8)
    sites = W.element_centres(inst.domain, inst.partition)
    part = W.Partition(voronoi_sites=sites, gamma1=inst.partition.gamma1)
    assert wos.wos_num_elements(inst.domain, part) == 16
    assert O.num_elements(inst.domain, part) == 16
    x = np.array([[0.0, 0.99], [0.51, 0.0]])
    np.testing.assert_array_equal(O.classify(inst.domain, part, x),
                                  np.argmin(((sites[None] - x[:, None]) ** 2).sum(-1), 1))


def test_build_wrappers_refuse_host_tensors_before_the_library(lib):
    """Device arrays are checked by the binding before any library call: a
    host (CPU) points tensor would hand the library a host address."""
    import torch

    class FakeCtx:      # never reaches the library: the checks raise first
        h = None
        device = 0

    inst = W.square_config(N=10, grid=2)
    pts = torch.as_tensor(inst.points, dtype=torch.float64)
    counts = torch.zeros((inst.M_D, inst.M_tot), dtype=torch.int32)
    with pytest.raises(wos.WosError) as e:
        wos.wos_build_operator(FakeCtx(), inst.domain, inst.K, pts, inst.partition, inst.N,
                               inst.eps, inst.seed)
    assert e.value.code == 1
    with pytest.raises(wos.WosError) as e:
        wos.wos_build_operator_noalloc(FakeCtx(), inst.domain, inst.K, pts, inst.partition,
                                       inst.N, inst.eps, inst.seed, counts)
    assert e.value.code == 1


@pytest.mark.parametrize("make", [
    lambda: W.shell_config(voronoi=(1000, 100)),             # Ex. 5.6 sizes
    lambda: W.shell_config(voronoi=(300, 40), shift=0.3),    # off-centre hole
    lambda: W.annulus_voronoi_config(m0=500, m1=200),        # Ex. 5.2 / 5.3
], ids=["shell-1000-100", "shell-shifted", "annulus"])
def test_voronoi_cell_measures_match_the_oracle(lib, make):
    """sigma(omega_j) of extrinsic Voronoi cells (App. A, Ex. A.2): the
    library's own construction (half-plane clipping in the central
    projection; arcs between bisectors) against the oracle's (scipy's
    spherical Voronoi diagram; arcs), cell by cell, and their totals against
    the surfaces' measures."""
    inst = make()
    a = wos.wos_element_measures(inst.domain, inst.partition)
    b = O.voronoi_measures(inst.domain, inst.partition)
    np.testing.assert_allclose(a, b, rtol=1e-12)
    d = inst.domain
    if d.dim == 3:
        total = 4 * math.pi * (d.radius ** 2 + sum(r ** 2 for _, r in d.holes))
    else:
        total = 2 * math.pi * (d.radius + sum(r for _, r in d.holes))
    assert a.sum() == pytest.approx(total, rel=1e-13)


def test_voronoi_cell_measures_reject_unsupported_sites(lib):
    """Sites off every circle / sphere of D, or a box domain: no closed
    construction, WOS_INVALID_ARG."""
    inst = W.shell_config(voronoi=(50, 10))
    sites = inst.partition.voronoi_sites.copy()
    sites[3] *= 0.9
    bad = W.Partition(voronoi_sites=sites, gamma1=inst.partition.gamma1)
    with pytest.raises(wos.WosError):
        wos.wos_element_measures(inst.domain, bad)
    sq = W.square_config(n_side=4)
    part = W.Partition(voronoi_sites=W.element_centres(sq.domain, sq.partition),
                       gamma1=sq.partition.gamma1)
    with pytest.raises(wos.WosError):
        wos.wos_element_measures(sq.domain, part)
