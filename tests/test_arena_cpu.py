"""Host logic of the serving loop's device arena (csrc/arena.h), on the CPU:
a small C++ driver replays seeded random alloc/release sequences through the
allocator, and every answer is checked against an independent first-fit model
over a list of free intervals, plus the invariants (no overlap, in bounds,
full coalescing once everything is released)."""
import os
import random
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2012_08655_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "arena.h"
int main() {
  fovea::Arena a;
  char op;
  unsigned long long x, y;
  while (std::scanf(" %c", &op) == 1) {
    if (op == 'z') { std::scanf("%llu", &x); a.reset((size_t)x); }
    else if (op == 'a') {
      std::scanf("%llu", &x);
      size_t off = 0;
      if (a.alloc((size_t)x, &off)) std::printf("%llu\n", (unsigned long long)off);
      else std::printf("-\n");
    } else if (op == 'r') { std::scanf("%llu %llu", &x, &y); a.release((size_t)x, (size_t)y); }
    else if (op == 'f') {
      std::printf("F");
      for (auto& kv : a.free_ranges()) std::printf(" %llu:%llu", (unsigned long long)kv.first,
                                                   (unsigned long long)kv.second);
      std::printf("\n");
    }
    std::fflush(stdout);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    d = os.path.join(HERE, "_build", "arena")  # git-ignored build folder inside the tree
    os.makedirs(d, exist_ok=True)
    src = os.path.join(d, "driver.cpp")
    with open(src, "w") as f:
        f.write(DRIVER)
    exe = os.path.join(d, "driver")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, src, "-o", exe], check=True)
    return exe


class FirstFit:
    """Free space as sorted, non-adjacent [start, end) intervals."""

    def __init__(self, size):
        self.free = [[0, size]] if size else []

    def alloc(self, n):
        for i, (s, e) in enumerate(self.free):
            if e - s >= n:
                if e - s == n:
                    del self.free[i]
                else:
                    self.free[i][0] = s + n
                return s
        return None

    def release(self, off, n):
        self.free.append([off, off + n])
        self.free.sort()
        merged = []
        for s, e in self.free:
            if merged and merged[-1][1] == s:
                merged[-1][1] = e
            else:
                merged.append([s, e])
        self.free = merged


def run_script(driver, lines):
    out = subprocess.run([driver], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return out.stdout.split("\n")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_arena_matches_first_fit_model(driver, seed):
    rng = random.Random(seed)
    size = 1 << 20
    model = FirstFit(size)
    live = []       # (offset, length) currently allocated, in the model
    script = [f"z {size}"]
    expect = []     # the model's answer to every 'a'
    for _ in range(2000):
        if live and rng.random() < 0.45:
            off, n = live.pop(rng.randrange(len(live)))
            model.release(off, n)
            script.append(f"r {off} {n}")
        else:
            n = rng.choice([256, 512, 4096, 65536, 200704, rng.randrange(1, 300000)])
            off = model.alloc(n)
            expect.append(off)
            script.append(f"a {n}")
            if off is not None:
                assert 0 <= off and off + n <= size
                assert all(off + n <= o or o + m <= off for o, m in live), "model handed out overlapping ranges"
                live.append((off, n))
    for off, n in live:
        model.release(off, n)
        script.append(f"r {off} {n}")
    script.append("f")
    got = run_script(driver, script)
    answers = [ln for ln in got if ln and not ln.startswith("F")]
    assert len(answers) == len(expect)
    for a, e in zip(answers, expect):
        assert (a == "-") == (e is None)
        if e is not None:
            assert int(a) == e
    granted = [e for e in expect if e is not None]
    assert len(granted) < len(expect), "the sequence never filled the arena (no refusal exercised)"
    assert len(set(granted)) < len(granted), "the sequence never reused a released range"
    final = [ln for ln in got if ln.startswith("F")][0]
    assert final == f"F 0:{size}", "releasing everything did not coalesce the arena back into one range"


def test_arena_exact_fit_reuse_and_refusal(driver):
    lines = ["z 1024", "a 512", "a 512", "a 1", "r 0 512", "a 256", "a 256", "a 1", "r 512 512",
             "r 0 256", "r 256 256", "f"]
    got = [ln for ln in run_script(driver, lines) if ln]
    assert got == ["0", "512", "-", "0", "256", "-", "F 0:1024"]
