"""The bounds-checking build (compiled with PIT_CHECK_BOUNDS, see pit_bounds_status in
include/pit.h): built here, loaded in a fresh process, and run through every kernel
family -- residual, assembly, the level chain (SOR and BiCGStab, several team sizes),
the context-free block solve, the Newton wavefront (one and several teams, deep rows,
FP32 level solves, windows) and the batched launch -- on one node, a ragged tiny grid,
a single column, a single row and multi-strip grids. Every call must match the FP64
oracle and leave the bounds record empty (no array indexed out of range)."""
import json
import os
import subprocess
import sys

import pytest

from paper_2406_00878_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_checking_build_runs_every_kernel_in_range_and_matches_the_oracle():
    path = build.build_check()
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    proc = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_bounds_child.py"), path], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=1800)
    assert proc.returncode == 0, proc.stderr[-4000:]
    rows = [json.loads(line) for line in proc.stdout.splitlines() if line.startswith("{")]
    assert rows and rows[0]["name"] == "loaded" and rows[0]["bounds"] == [1, 0], rows[:1]
    names = [r["name"] for r in rows]
    # every family ran on every tiny shape
    for shape in ("1x1x1", "3x5x2", "1x37x3", "41x1x3"):
        for family in ("residual", "assemble", "block_solve", "noalloc", "solve"):
            assert any(n.startswith(f"{family} {shape}") for n in names), (family, shape)
    assert sum(n.startswith("batch") for n in names) == 4 * 6
    bad_bounds = [r for r in rows if r["bounds"] != [1, 0]]
    assert not bad_bounds, bad_bounds[:5]
    bad = [r for r in rows if not r["err"] <= r["tol"]]
    assert not bad, bad[:5]
