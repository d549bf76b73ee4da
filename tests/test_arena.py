"""The server's device-arena bookkeeping (csrc/wsm_arena.h), compiled with
the host C++ compiler and driven by seeded random sequences of requests and
releases.  After every step the placement is checked against the live
blocks alone: blocks are granule-aligned, inside the arena and disjoint;
each allocation lands at the lowest gap between live blocks that holds it
(first fit over fully merged free ranges) and fails only when no gap does;
the free list is exactly the complement of the live blocks, with no two
ranges adjacent; the used count is the sum of the live blocks."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1011_0093_gb300", "csrc")
G = 256

DRIVER = r"""
#include <cstdio>
#include <cstring>
#include "wsm_arena.h"
// stdin: "c <bytes>" (reset), "a <bytes>", "r <off> <bytes>", "f" (dump the
// free ranges); stdout: one line per command.
int main() {
    wsm::ArenaBook book;
    char op[4];
    while (std::scanf("%3s", op) == 1) {
        unsigned long long x = 0, y = 0;
        if (!std::strcmp(op, "c")) {
            if (std::scanf("%llu", &x) != 1) return 1;
            book.reset(x);
            std::printf("C %zu\n", book.capacity());
        } else if (!std::strcmp(op, "a")) {
            if (std::scanf("%llu", &x) != 1) return 1;
            const size_t off = book.alloc(x);
            if (off == SIZE_MAX) std::printf("A none %zu\n", book.used());
            else std::printf("A %zu %zu\n", off, book.used());
        } else if (!std::strcmp(op, "r")) {
            if (std::scanf("%llu %llu", &x, &y) != 2) return 1;
            book.release(x, y);
            std::printf("R %zu\n", book.used());
        } else {
            std::printf("F");
            for (const auto& kv : book.free_ranges()) std::printf(" %zu:%zu", kv.first, kv.second);
            std::printf("\n");
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("needs a C++ compiler")
    d = tmp_path_factory.mktemp("arena")
    src, exe = d / "arena.cpp", d / "arena"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC, str(src), "-o",
                    str(exe)], check=True)

    def run(commands):
        out = subprocess.run([str(exe)], input="\n".join(commands) + "\n", capture_output=True,
                             text=True, check=True).stdout
        return out.splitlines()
    return run


def up(b):
    return (b + G - 1) // G * G


def gaps(live, cap):
    """Free ranges implied by the live blocks: (offset, size), ascending."""
    out, at = [], 0
    for off, size in sorted(live.items()):
        if off > at:
            out.append((at, off - at))
        at = off + size
    if at < cap:
        out.append((at, cap - at))
    return out


def simulate(driver, seed, cap, steps):
    """Random requests and releases.  The next command depends on earlier
    replies (which block to release), so each step reruns the driver on the
    whole history and reads its last replies."""
    rng = np.random.default_rng(seed)
    history = [f"c {cap}"]
    reply = driver(history)
    cap_r = int(reply[0].split()[1])
    assert cap_r == up(cap)
    live = {}                      # offset -> rounded size
    asked = {}                     # offset -> requested bytes
    n_fail = n_alloc = 0
    for _ in range(steps):
        if live and rng.random() < 0.45:
            off = int(rng.choice(sorted(live)))
            cmd = f"r {off} {asked[off]}"
            history.append(cmd)
            line = driver(history)[-1]
            del live[off], asked[off]
            assert line == f"R {sum(live.values())}"
        else:
            b = int(rng.integers(1, cap_r // 3)) if rng.random() < 0.8 else int(
                rng.integers(1, 2 * G))
            history += [f"a {b}", "f"]
            lines = driver(history)
            a, f = lines[-2].split(), lines[-1].split()[1:]
            fits = [o for o, s in gaps(live, cap_r) if s >= up(b)]
            if a[1] == "none":
                n_fail += 1
                assert not fits, (b, gaps(live, cap_r))
            else:
                n_alloc += 1
                off = int(a[1])
                assert fits and off == fits[0]          # first fit over merged ranges
                assert off % G == 0 and off + up(b) <= cap_r
                for o, s in live.items():
                    assert off + up(b) <= o or o + s <= off
                live[off], asked[off] = up(b), b
            assert int(a[-1]) == sum(live.values())
            ranges = [tuple(map(int, r.split(":"))) for r in f]
            assert ranges == gaps(live, cap_r)          # no two free ranges adjacent
    return n_alloc, n_fail, history, live, asked


@pytest.mark.parametrize("seed,cap", [(1, 64 * G), (2, 1000 * G + 17), (3, 40 * G)])
def test_first_fit_with_merged_free_ranges(driver, seed, cap):
    n_alloc, n_fail, history, live, asked = simulate(driver, seed, cap, 120)
    assert n_alloc > 20 and n_fail > 0
    # releasing everything leaves one free range, the whole arena
    history += [f"r {o} {asked[o]}" for o in sorted(live)] + ["f"]
    out = driver(history)
    assert out[-2] == "R 0"
    assert out[-1] == f"F 0:{up(cap)}"


def test_release_merges_both_neighbours(driver):
    cmds = ["c 4096", "a 256", "a 300", "a 256", "a 1000", "r 0 256", "r 768 256", "f",
            "r 256 300", "f", "a 768", "f"]
    out = driver(cmds)
    assert out[1:5] == ["A 0 256", "A 256 768", "A 768 1024", "A 1024 2048"]
    assert out[7] == "F 0:256 768:256 2048:2048"
    assert out[9] == "F 0:1024 2048:2048"           # merged with the ranges before and after
    assert out[10] == "A 0 1792" and out[11] == "F 768:256 2048:2048"
