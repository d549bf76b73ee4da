"""How the persistent launch divides its blocks between the images of a batch
(csrc/wsm_split.h), compiled with the host C++ compiler and checked on
seeded random batches: every image gets at least one block and at least
min(want, floor); the groups are contiguous and never exceed the grid; a
batch that fits gets exactly what it wants; beyond the floors, a larger
demand never gets fewer blocks; and the autotuner's work weights scale the
demand (1024 = 1, 0 = unweighted, never below one block)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1011_0093_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "wsm_split.h"
// stdin: "s <grid> <n> <want_1> .. <want_n>" -> the n+1 group starts;
//        "w <want> <weight>" -> the weighted demand;
//        "g <n> <K> <threads>" -> group_want
int main() {
    char op[4];
    while (std::scanf("%3s", op) == 1) {
        if (op[0] == 's') {
            int grid = 0, n = 0;
            if (std::scanf("%d %d", &grid, &n) != 2 || n < 1 || n > 4096) return 1;
            static int64_t want[4096];
            static int first[4097];
            for (int i = 0; i < n; ++i) {
                long long v = 0;
                if (std::scanf("%lld", &v) != 1) return 1;
                want[i] = v;
            }
            wsm::split_groups(want, n, grid, first);
            for (int i = 0; i <= n; ++i) std::printf("%d ", first[i]);
            std::printf("\n");
        } else if (op[0] == 'w') {
            long long v = 0;
            int w = 0;
            if (std::scanf("%lld %d", &v, &w) != 2) return 1;
            std::printf("%lld\n", (long long)wsm::weighted_want(v, w));
        } else {
            long long n = 0;
            int K = 0, t = 0;
            if (std::scanf("%lld %d %d", &n, &K, &t) != 3) return 1;
            std::printf("%lld\n", (long long)wsm::group_want(n, K, t));
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("split")
    src, exe = d / "driver.cpp", d / "driver"
    src.write_text(DRIVER)
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)])

    def run(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True).stdout
        return [[int(x) for x in line.split()] for line in out.strip().splitlines()]
    return run


def test_splits_of_random_batches(driver):
    rng = np.random.default_rng(1234)
    cases = []
    for _ in range(400):
        n = int(rng.integers(1, 65))
        grid = int(rng.integers(n, 1217))
        want = rng.integers(1, 4000, n) if rng.random() < 0.7 else rng.integers(1, 20, n)
        cases.append((grid, [int(w) for w in want]))
    outs = driver([f"s {g} {len(w)} " + " ".join(map(str, w)) for g, w in cases])
    for (grid, want), first in zip(cases, outs):
        n = len(want)
        assert len(first) == n + 1 and first[0] == 0
        g = np.diff(first)
        assert np.all(g >= 1) and first[-1] <= grid
        if sum(want) <= grid:
            assert g.tolist() == want
            continue
        floor = min(16, max(1, grid // (2 * n)))
        assert np.all(g >= np.minimum(want, floor))
        assert first[-1] >= grid - n            # the rounding loses less than a block each
        above = [i for i in range(n) if want[i] > floor]
        for i in above:
            for j in above:
                if want[i] > want[j]:
                    assert g[i] >= g[j] - 1, (grid, want, g.tolist())


def test_weights_scale_the_demand(driver):
    lines = [f"w {v} {w}" for v, w in [(100, 0), (100, 1024), (100, 2048), (100, 512), (3, 64),
                                       (1, 1), (4000, 16384)]]
    assert [r[0] for r in driver(lines)] == [100, 100, 200, 50, 1, 1, 64000]


def test_a_heavier_image_gets_more_blocks(driver):
    want = [300, 300, 300, 300]
    plain = np.diff(driver([f"s 304 4 {' '.join(map(str, want))}"])[0])
    heavy = [300, 300, 600, 300]                 # the third image weighted 2x
    weighted = np.diff(driver([f"s 304 4 {' '.join(map(str, heavy))}"])[0])
    assert plain.tolist() == [76, 76, 76, 76]
    assert weighted[2] > plain[2] and weighted.sum() == 304


def test_group_want(driver):
    rows = driver(["g 1 256 512", "g 18049 256 512", "g 229024 256 512", "g 100 16 256",
                   "g 0 1 1024"])
    # one color per lane, or one table row per warp, whichever needs more blocks
    assert [r[0] for r in rows] == [16, 36, 448, 2, 1]
