"""Host logic of the cluster SVD kernel's data layout (the round-robin
order of one-sided Jacobi, Sec. 4.3's SVD step): for every column count the
kernel takes, positions map one to one onto (CTA, slot), the move between
rounds sends the column at each position to the position that holds it next
round, a sweep of n_pad - 1 rounds meets every pair of columns exactly once
and returns every column to its start, and the shared memory of the
benchmark shapes fits a CTA.  Compiled with g++ (no GPU)."""
import itertools
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]

DRIVER = r"""
#include <cstdio>
#include <set>
#include <vector>
#include <utility>
#include <algorithm>
#include "svd_cluster_layout.h"

int main() {
    int bad = 0;
    for (int n = 1; n <= kClMaxN; ++n) {
        const int n_pad = std::max(2, n + (n & 1));
        const int CL = std::min(kClMaxCtas, n_pad / 2);
        const ClLayout L = cl_layout(n, n, 0, CL);
        if (L.PP > kClWarps) { printf("PP %d > warps at n=%d\n", L.PP, n); ++bad; }
        // positions <-> (cta, slot): one to one, inside the cluster
        std::set<std::pair<int,int>> seen;
        for (int pos = 0; pos < n_pad; ++pos) {
            int cta, slot;
            cl_where(pos, L, cta, slot);
            if (cta < 0 || cta >= CL || slot < 0 || slot >= 2 * L.PP) { ++bad; continue; }
            if (!seen.insert({cta, slot}).second) { printf("slot reused n=%d\n", n); ++bad; }
        }
        // the move is a permutation that carries each column to its next position
        std::vector<int> hit(n_pad, 0);
        for (int pos = 0; pos < n_pad; ++pos) ++hit[cl_next(pos, n_pad)];
        for (int q = 0; q < n_pad; ++q) if (hit[q] != 1) { printf("move not 1:1 n=%d\n", n); ++bad; break; }
        for (int r = 0; r < n_pad - 1; ++r)
            for (int pos = 0; pos < n_pad; ++pos)
                if (cl_column(cl_next(pos, n_pad), r + 1, n_pad) != cl_column(pos, r, n_pad)) {
                    printf("column lost n=%d r=%d pos=%d\n", n, r, pos); ++bad; r = n_pad; break;
                }
        // a sweep meets every pair once and returns the columns to their start
        std::set<std::pair<int,int>> pairs;
        for (int r = 0; r < n_pad - 1; ++r)
            for (int pr = 0; pr < n_pad / 2; ++pr) {
                int a = cl_column(pr, r, n_pad), b = cl_column(n_pad - 1 - pr, r, n_pad);
                if (!pairs.insert({std::min(a, b), std::max(a, b)}).second) { ++bad; }
            }
        if (int(pairs.size()) != n_pad * (n_pad - 1) / 2) { printf("pairs n=%d\n", n); ++bad; }
        for (int pos = 0; pos < n_pad; ++pos)
            if (cl_column(pos, n_pad - 1, n_pad) != cl_column(pos, 0, n_pad) ||
                cl_column(pos, 0, n_pad) != pos) { ++bad; break; }
    }
    // shared memory of the cluster launches of the benchmark and config shapes
    const int shapes[][3] = {{256, 128, 1}, {128, 96, 1}, {200, 96, 1}, {300, 256, 1},
                             {32, 16, 0}, {30, 20, 0}, {1024, 16, 0}};
    for (auto &s : shapes) {
        const int n_pad = std::max(2, s[1] + (s[1] & 1));
        const ClLayout L = cl_layout(s[0], s[1], s[2], std::min(kClMaxCtas, n_pad / 2));
        printf("%d %d %d %zu\n", s[0], s[1], s[2], L.total);
    }
    printf("bad %d\n", bad);
    return 0;
}
"""


@pytest.fixture(scope="module")
def layout_run(tmp_path_factory):
    d = tmp_path_factory.mktemp("cllayout")
    src = d / "layout.cpp"
    src.write_text(DRIVER)
    exe = d / "layout"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I",
                    str(ROOT / "paper_2409_03686_gb300" / "csrc"), str(src), "-o", str(exe)],
                   check=True)
    return subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout


def test_round_robin_movement_is_consistent(layout_run):
    assert layout_run.strip().splitlines()[-1] == "bad 0", layout_run[-2000:]


def test_benchmark_shapes_fit_one_cta(layout_run):
    sizes = {}
    for line in layout_run.strip().splitlines()[:-1]:
        if line.count(" ") == 3:
            m, n, pre, total = (int(x) for x in line.split())
            sizes[(m, n, pre)] = total
    assert sizes[(256, 128, 1)] < 64 * 1024           # the benchmark operators
    assert all(v <= 227 * 1024 for v in sizes.values())  # the per-CTA opt-in limit
