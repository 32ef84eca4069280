"""The point-tile rule of the fitness launches (csrc/ptiles.h, host code):
compiled on its own with the host compiler and checked without a GPU.

* every choice lies in [1, the bound the partial sums are sized for], for
  the full point count and every smaller one (a decimated schedule), so a
  launch never finds its workspace too small;
* the choices of the benchmarked workloads on 152 SMs x 3 resident CTAs:
  the 640x480 search (3072 particles over 307 200 points: 19 tiles, four
  exact waves), the paper's schedule (1024 x 1/8: 38, 3072 x 1/16: 19,
  10240 x 1/32: 5 -- two full passes per CTA rather than 7 tiles with a
  third-full second pass), and the single-pose evaluation (one chunk: a tile
  per 1024-point sub-tile);
* the rule's objective: no candidate within 3.5-8.5 waves has fewer
  waves x passes than the choice."""
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_24236_gb300", "csrc")
CAP, SUB = 152 * 3, 1024

HARNESS = r"""
#include <cstdio>
#include "ptiles.h"
int main() {
    long long cap, sub, ne; int chunks;
    while (std::scanf("%lld %lld %d %lld", &cap, &sub, &chunks, &ne) == 4)
        std::printf("%d %d\n", pf::choose_ptiles_for(cap, sub, chunks, ne), pf::ptiles_bound_for(cap, sub, chunks, ne));
    return 0;
}
"""


@pytest.fixture(scope="module")
def rule(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("ptiles")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def ask(cases):
        inp = "".join(f"{CAP} {SUB} {c} {n}\n" for c, n in cases)
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
        return [tuple(int(v) for v in line.split()) for line in out if line.strip()]

    return ask


def test_choices_never_exceed_the_workspace_bound(rule):
    chunks = list(range(1, 41)) + [48, 64, 96, 128, 160, 200, 256, 320, 400, 640, 1024, 2048, 4096]
    full = [307200, 76800, 19200, 4096, 1000, 1]
    cases = []
    for c in chunks:
        for n in full:
            for stride in (1, 2, 3, 5, 8, 13, 16, 32, 64):
                cases.append((c, (n + stride - 1) // stride))
    got = rule(cases)
    bounds = {(c, n): b for (c, n), (_, b) in zip(cases, got) if n in full}
    for (c, n), (t, b) in zip(cases, got):
        assert 1 <= t <= b, (c, n, t, b)
        # the workspace is sized with the full point count of the frame
        full_n = min(f for f in full if f >= n)
        assert t <= bounds[(c, full_n)], (c, n, t, bounds[(c, full_n)])


def test_benchmarked_workloads(rule):
    cases = [(96, 307200), (32, 38400), (96, 19200), (320, 9600), (1, 307200), (1, 38400)]
    got = [t for t, _ in rule(cases)]
    assert got == [19, 38, 19, 5, 300, 38]


def test_choice_minimises_waves_times_passes(rule):
    cases = [(c, n) for c in (24, 32, 64, 96, 128, 160, 320, 512) for n in (9600, 19200, 38400, 76800, 153600, 307200)]
    for (c, n), (t, _) in zip(cases, rule(cases)):
        cands = [u for u in range(1, (n + SUB - 1) // SUB + 1) if 3.5 <= c * u / CAP <= 8.5]
        if not cands:
            continue
        cost = lambda u: math.ceil(c * u / CAP) * ((n + u * SUB - 1) // (u * SUB))
        assert t in cands and cost(t) == min(cost(u) for u in cands), (c, n, t)
