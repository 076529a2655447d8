"""The wavefront's team sizes (csrc/pit_teams.h), compiled with g++ on the host: no GPU.

K teams of Gw CTAs share the grid rows as strips; the SMs they leave over go to the teams nearest
the middle, each with the fewest CTAs whose strips are shorter, within the automatic team size's
cap of one CTA per 256 unknowns. Both the single-problem launch (pit_create) and the batched
solver's wavefront jobs take their sizes from this function.
"""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2406_00878_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "pit_teams.h"
int main() {
    int K, Gw, nx, ny, P, min_local, max_team, fixed;
    while (std::scanf("%d %d %d %d %d %d %d %d", &K, &Gw, &nx, &ny, &P, &min_local, &max_team, &fixed) == 8) {
        int sizes[64];
        const int total = pit_wave_team_sizes(K, Gw, nx, ny, P, min_local, max_team, fixed, sizes);
        std::printf("%d", total);
        for (int t = 0; t < K; ++t) std::printf(" %d", sizes[t]);
        std::printf("\n");
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def team_sizes(tmp_path_factory):
    d = tmp_path_factory.mktemp("teams")
    src, exe = d / "drv.cpp", d / "drv"
    src.write_text(DRIVER)
    subprocess.run(["g++", "-std=c++17", "-O1", f"-I{CSRC}", str(src), "-o", str(exe)], check=True)

    def run(cases):
        text = "".join(" ".join(map(str, c)) + "\n" for c in cases)
        out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
        rows = [list(map(int, line.split())) for line in out if line.strip()]
        return [(r[0], r[1:]) for r in rows]

    return run


def _ceil(a, b):
    return (a + b - 1) // b


def test_the_measured_configurations(team_sizes):
    # (K, Gw, nx, ny, P, min_local, max_team, fixed)
    cases = [
        (5, 29, 256, 256, 152, 256, 256, 0),   # burgers256, FP64: teams 2 and 3 get 8-row strips
        (6, 24, 256, 256, 152, 256, 256, 0),   # burgers256, FP32 level solves
        (6, 24, 64, 256, 152, 256, 256, 0),    # the GPU test of teams of different sizes
        (6, 4, 32, 32, 152, 256, 32, 0),       # heat32: 5 CTAs exceed the cap of one per 256 unknowns
        (5, 29, 256, 256, 152, 256, 256, 29),  # a fixed team size keeps every team equal
        (1, 74, 512, 512, 152, 256, 512, 0),   # one team: nothing to give
    ]
    got = team_sizes(cases)
    assert got[0] == (151, [29, 29, 32, 32, 29])
    assert got[1] == (152, [24, 26, 26, 26, 26, 24])
    assert got[2] == (152, [24, 26, 26, 26, 26, 24])
    assert got[3] == (24, [4] * 6)
    assert got[4] == (145, [29] * 5)
    assert got[5] == (74, [74])


def test_properties_over_many_shapes(team_sizes):
    cases = []
    for nx in (16, 32, 64, 96, 128, 256, 384, 512):
        for ny in (8, 33, 64, 100, 256, 384, 1000):
            for K in (2, 3, 4, 5, 6):
                for rows in (2, 3, 4, 7, 9, 11, 20):
                    Gw = _ceil(ny, rows)
                    for P in (148, 152, 160):
                        if K * Gw <= P:
                            cases.append((K, Gw, nx, ny, P, 256, 160, 0))
    got = team_sizes(cases)
    assert len(got) == len(cases) > 500
    for (K, Gw, nx, ny, P, min_local, max_team, _), (total, sizes) in zip(cases, got):
        assert len(sizes) == K and total == sum(sizes) <= P
        up = [t for t in range(K) if sizes[t] != Gw]
        if not up:
            continue
        G2 = sizes[up[0]]
        rows = _ceil(ny, Gw)
        # one size for every upgraded team: the fewest CTAs whose strips are shorter, within the
        # automatic size's cap of one CTA per min_local unknowns
        assert all(sizes[t] == G2 for t in up) and Gw < G2 <= max_team
        assert _ceil(ny, G2) <= rows - 1 and _ceil(ny, G2 - 1) >= rows
        assert G2 <= _ceil(ny, _ceil(min_local, nx))
        # as many as the spare SMs allow, the teams nearest the middle first
        assert len(up) == K or P - total < G2 - Gw
        dist = sorted(range(K), key=lambda t: (abs(2 * t - K), t))
        assert sorted(up) == sorted(dist[:len(up)])
