"""The serving arena's block placement (csrc/arena.h), compiled on its own with the host C++
compiler and driven through a seeded random sequence of allocations and releases.

A brute-force model keeps the set of allocated intervals. With free blocks fully merged, the
free list must always be the maximal gaps between allocated intervals, and first fit must
return the lowest-offset gap at least as large as the request (-1 if there is none). Every
step of the sequence is checked: each returned offset, and the whole free list after it.
"""
import shutil
import subprocess
import textwrap
from pathlib import Path

import numpy as np
import pytest

CSRC = Path(__file__).resolve().parents[1] / "paper_1711_08095_gb300" / "csrc"

DRIVER = textwrap.dedent("""
    #include <cstdio>
    #include "arena.h"
    // stdin: "z size" (reset), "a bytes" (alloc: prints the offset), "r off bytes" (release);
    // after every command prints the free list as "off:len ..." on one line
    int main() {
        snect::ArenaBlocks A;
        char op;
        long long x, y;
        while (std::scanf(" %c", &op) == 1) {
            if (op == 'z' && std::scanf("%lld", &x) == 1) A.reset(x);
            else if (op == 'a' && std::scanf("%lld", &x) == 1) std::printf("%lld\\n", (long long)A.alloc(x));
            else if (op == 'r' && std::scanf("%lld %lld", &x, &y) == 2) A.release(x, y);
            else return 2;
            for (const auto &b : A.free_blocks) std::printf("%lld:%lld ", (long long)b.first, (long long)b.second);
            std::printf("|\\n");
        }
        return 0;
    }
""")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("arena")
    (d / "drive.cpp").write_text(DRIVER)
    exe = d / "drive"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", str(CSRC), str(d / "drive.cpp"), "-o", str(exe)], check=True)
    return exe


class Model:
    """Allocated intervals of [0, size); the free list is the maximal gaps between them."""

    def __init__(self, size):
        self.size = size
        self.used = {}  # offset -> bytes

    def gaps(self):
        out, pos = [], 0
        for off in sorted(self.used):
            if off > pos:
                out.append((pos, off - pos))
            pos = off + self.used[off]
        if pos < self.size:
            out.append((pos, self.size - pos))
        return out

    def alloc(self, n):
        for off, ln in self.gaps():
            if ln >= n:
                self.used[off] = n
                return off
        return -1

    def release(self, off):
        return self.used.pop(off)


def run(driver, size, ops):
    """ops: the model-driven command list; returns the driver's output lines."""
    text = "z %d\n" % size + "".join(ops)
    r = subprocess.run([str(driver)], input=text, capture_output=True, text=True, check=True)
    return r.stdout.splitlines()


def free_line(gaps):
    return "".join("%d:%d " % g for g in gaps) + "|"


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_first_fit_and_merging_match_the_model(driver, seed):
    rng = np.random.default_rng(seed)
    size = 1 << 16
    m = Model(size)
    ops, expect = [], [free_line(m.gaps())]
    for _ in range(3000):
        if m.used and rng.random() < 0.45:
            off = int(rng.choice(sorted(m.used)))
            n = m.release(off)
            ops.append("r %d %d\n" % (off, n))
        else:
            # mostly 256-byte multiples as the server asks for; sometimes the whole range or more
            n = int(rng.choice([256, 512, 768, 4096, 12288, size, size + 1])) if rng.random() < 0.2 else \
                256 * int(rng.integers(1, 40))
            got = m.alloc(n)
            ops.append("a %d\n" % n)
            expect.append(str(got))
        expect.append(free_line(m.gaps()))
    assert run(driver, size, ops) == expect


def test_each_merge_case(driver):
    """Four 1,024-byte blocks fill the range. Releases then cover each merge: no free
    neighbour, the previous block only, the end of the range, both sides, and the next block
    only. An exact fit takes a whole block, and a request with no room gets -1."""
    ops = ["a 1024\n"] * 4 + [
        "r 0 1024\n",     # no free neighbour
        "r 1024 1024\n",  # merges with the previous
        "r 3072 1024\n",  # last block, its previous still in use
        "r 2048 1024\n",  # merges on both sides
        "a 4096\n",       # exact fit
        "a 256\n",        # no room
        "r 0 4096\n",
        "a 1024\n", "a 1024\n",
        "r 1024 1024\n",  # merges with the next
        "r 0 1024\n",     # and again
    ]
    out = run(driver, 4096, ops)
    allocs = [ln for ln in out if not ln.endswith("|")]
    frees = [ln for ln in out if ln.endswith("|")]
    assert allocs == ["0", "1024", "2048", "3072", "0", "-1", "0", "1024"]
    assert frees == ["0:4096 |",  # reset
                     "1024:3072 |", "2048:2048 |", "3072:1024 |", "|",
                     "0:1024 |", "0:2048 |", "0:2048 3072:1024 |", "0:4096 |",
                     "|", "|", "0:4096 |",
                     "1024:3072 |", "2048:2048 |", "1024:3072 |", "0:4096 |"]
