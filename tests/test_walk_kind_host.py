"""Host logic of the walk kernel's kind selection (no GPU): which distance
and classifier specialisation a domain gets.  A square or cube (equal
half-extents) takes the equal-extent box kind, any other box the general box
kind, a disc / ball with one hole of the same centre the concentric kind,
any other holes the holes kind, Voronoi partitions and polygons the generic
kernel, mapped walks their own kind.  The driver is compiled with nvcc (the
header holds the kernel template) and calls only the host function."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]

DRIVER = r"""
#include <cstdio>
#include <cstring>
#include "walk_launch.cuh"
using namespace wos;

static wos_domain dom(int dim, int outer) {
    wos_domain d; std::memset(&d, 0, sizeof d);
    d.dim = dim; d.outer_kind = outer; d.radius = 1.0;
    for (int a = 0; a < 3; ++a) d.half[a] = a < dim ? 0.5 : 0.0;
    return d;
}

int main() {
    wos_partition p; std::memset(&p, 0, sizeof p);
    wos_domain sq = dom(2, WOS_OUTER_BOX);
    wos_domain rect = sq; rect.half[1] = 0.3;
    wos_domain near = sq; near.half[1] = 0.5 + 1e-12;  // equal in FP32 only
    wos_domain cube = dom(3, WOS_OUTER_BOX);
    wos_domain cuboid = cube; cuboid.half[2] = 0.6;
    wos_domain flat = dom(2, WOS_OUTER_BOX); flat.half[2] = 7.0;  // unused third extent
    wos_domain disc = dom(2, WOS_OUTER_SPHERE);
    wos_domain ann = disc; ann.n_holes = 1; ann.hole_radius[0] = 0.5;
    wos_domain off = ann; off.hole_center[0][0] = 0.1;
    wos_domain ball = dom(3, WOS_OUTER_SPHERE);
    wos_domain shell = ball; shell.n_holes = 1; shell.hole_radius[0] = 0.5;
    wos_domain holey_sq = sq; holey_sq.n_holes = 1; holey_sq.hole_radius[0] = 0.1;
    wos_domain poly = dom(2, WOS_OUTER_POLYGON);
    wos_partition vor = p; vor.voronoi_n = 10;
    printf("square %d\n", walk_kind(sq, p));
    printf("rectangle %d\n", walk_kind(rect, p));
    printf("near_square %d\n", walk_kind(near, p));
    printf("cube %d\n", walk_kind(cube, p));
    printf("cuboid %d\n", walk_kind(cuboid, p));
    printf("square_unused_z %d\n", walk_kind(flat, p));
    printf("disc %d\n", walk_kind(disc, p));
    printf("annulus %d\n", walk_kind(ann, p));
    printf("offset_hole %d\n", walk_kind(off, p));
    printf("ball %d\n", walk_kind(ball, p));
    printf("shell %d\n", walk_kind(shell, p));
    printf("square_with_hole %d\n", walk_kind(holey_sq, p));
    printf("polygon %d\n", walk_kind(poly, p));
    printf("square_voronoi %d\n", walk_kind(sq, vor));
    printf("disc_voronoi %d\n", walk_kind(disc, vor));
    printf("square_mapped %d\n", walk_kind(sq, p, true));
    printf("kinds %d %d %d %d %d %d %d\n", kGeneric, kSphereOnly, kBoxOnly, kSphereHoles,
           kAnnulus, kMapped, kCubeOnly);
    return 0;
}
"""


@pytest.fixture(scope="module")
def kinds(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not Path(nvcc).exists():
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("walkkind")
    src = d / "kind.cu"
    src.write_text(DRIVER)
    exe = d / "kind"
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", str(ROOT / "include"),
                    "-I", str(ROOT / "paper_2409_03686_gb300" / "csrc"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    rows = dict(line.split(" ", 1) for line in out.strip().splitlines())
    names = ("generic", "sphere", "box", "holes", "annulus", "mapped", "cube")
    code = dict(zip(names, map(int, rows.pop("kinds").split())))
    return {k: next(n for n, c in code.items() if c == int(v)) for k, v in rows.items()}


@pytest.mark.parametrize("name, want", [
    ("square", "cube"), ("cube", "cube"), ("square_unused_z", "cube"),
    ("rectangle", "box"), ("cuboid", "box"), ("near_square", "box"),
    ("disc", "sphere"), ("ball", "sphere"),
    ("annulus", "annulus"), ("shell", "annulus"), ("offset_hole", "holes"),
    ("square_with_hole", "generic"), ("polygon", "generic"),
    ("square_voronoi", "generic"), ("disc_voronoi", "generic"),
    ("square_mapped", "mapped"),
])
def test_walk_kind(kinds, name, want):
    assert kinds[name] == want
