"""The C ABI library builds, loads without a GPU and exports every declared symbol;
argument checks reject bad input before touching CUDA."""
import ctypes
import os
import re

import pytest

from paper_2406_00878_gb300 import build as B
from paper_2406_00878_gb300 import pit

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(pit_\w+)\s*\(", text, flags=re.M))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert {"pit_create", "pit_residual", "pit_newton_step", "pit_solve", "pit_destroy"} <= declared
    assert declared == set(pit.EXPORTS), declared ^ set(pit.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_bounds_checking_build_builds_and_exports_every_declared_symbol():
    # the check build (-DPIT_CHECK_BOUNDS) compiles the same sources; its status query
    # answers NULL arguments before any CUDA call, so it can be called without a GPU
    path = B.build_check()
    assert path.endswith("libpit_check.so") and path != B.LIB
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    lib.pit_bounds_status.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.pit_bounds_status.restype = ctypes.c_int
    assert lib.pit_bounds_status(None, None) == pit.PIT_EINVAL
    lib.pit_status_string.restype = ctypes.c_char_p
    assert lib.pit_status_string(pit.PIT_EBOUNDS) == b"PIT_EBOUNDS"


def test_default_options_and_status_strings():
    o = pit.pit_default_options()
    assert o.newton_max == 30 and o.tol_res == 1e-12 and o.lin_solver == pit.PIT_LIN_AUTO
    assert o.wait_budget > 0 and o.lin_max_iter > 0
    assert pit._status_name(pit.PIT_ETIMEOUT) == "PIT_ETIMEOUT"


@pytest.mark.parametrize("grid,M,dt,params", [
    (pit.pit_grid(0, 4, 0, 1, 0, 1), 3, 0.1, pit.pit_params(0, 1.0, 0.0)),
    (pit.pit_grid(4, 4, 1, 0, 0, 1), 3, 0.1, pit.pit_params(0, 1.0, 0.0)),
    (pit.pit_grid(4, 4, 0, 1, 0, 1), 0, 0.1, pit.pit_params(0, 1.0, 0.0)),
    (pit.pit_grid(4, 4, 0, 1, 0, 1), 3, -0.1, pit.pit_params(0, 1.0, 0.0)),
    (pit.pit_grid(4, 4, 0, 1, 0, 1), 3, float("nan"), pit.pit_params(0, 1.0, 0.0)),
    (pit.pit_grid(4, 4, 0, 1, 0, 1), 3, 0.1, pit.pit_params(2, 1.0, 0.0)),
    (pit.pit_grid(4, 4, 0, 1, 0, 1), 3, 0.1, pit.pit_params(1, -1.0, 0.0)),
    (pit.pit_grid(4, 4, 0, 1, 0, 1), 3, 0.1, pit.pit_params(0, 1.0, -0.5)),
])
def test_create_rejects_invalid_arguments_without_cuda(grid, M, dt, params):
    h = ctypes.c_void_p()
    s = pit.lib().pit_create(ctypes.byref(grid), M, dt, ctypes.byref(params), None, None, ctypes.byref(h))
    assert s == pit.PIT_EINVAL and not h.value


def test_create_rejects_invalid_options_without_cuda():
    for field, value in [("newton_max", -1), ("lin_solver", 7), ("eta_max", 0.0), ("lin_max_iter", 0),
                         ("wait_budget", 0), ("team_ctas", -2)]:
        o = pit.pit_default_options()
        setattr(o, field, value)
        h = ctypes.c_void_p()
        g, p = pit.pit_grid(4, 4, 0, 1, 0, 1), pit.pit_params(0, 1.0, 0.0)
        s = pit.lib().pit_create(ctypes.byref(g), 3, 0.1, ctypes.byref(p), ctypes.byref(o), None, ctypes.byref(h))
        assert s == pit.PIT_EINVAL, field


def test_null_context_calls_return_einval():
    L = pit.lib()
    assert L.pit_residual(None, None, None, None) == pit.PIT_EINVAL
    assert L.pit_solve(None, None, None) == pit.PIT_EINVAL
    assert L.pit_last_error(None) == b"null context"
    L.pit_destroy(None)


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets (a C
    program built against include/pit.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [c for c in vars(pit).values()
               if isinstance(c, type) and issubclass(c, ctypes.Structure) and c.__name__.startswith("pit_")]
    assert {"pit_options", "pit_solve_info", "pit_batch_info", "pit_instance"} <= {c.__name__ for c in structs}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "pit.h"', "int main(void) {"]
    for c in structs:
        lines.append(f'  printf("{c.__name__} size %zu\\n", sizeof({c.__name__}));')
        for f, _ in c._fields_:
            lines.append(f'  printf("{c.__name__} {f} %zu\\n", offsetof({c.__name__}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for c in structs:
        assert c_layout[(c.__name__, "size")] == ctypes.sizeof(c), c.__name__
        for f, _ in c._fields_:
            assert c_layout[(c.__name__, f)] == getattr(c, f).offset, (c.__name__, f)


def test_build_compiles_every_batched_kernel_instance_once():
    """The build compiles the batched-kernel source once per level-solve precision and
    closure (the four closure bits), and every other source once."""
    units = B.units()
    names = [u[2] for u in units]
    assert len(names) == len(set(names))
    bk = [u for u in units if os.path.basename(u[0]) == B.BATCH_KERNELS]
    sets = {(f, c) for f in (0, 1) for c in (1, 2, 4, 8)}
    assert {(int(u[1][0].split("=")[1]), int(u[1][1].split("=")[1])) for u in bk} == sets and len(bk) == 8
    others = sorted(u[0] for u in units if os.path.basename(u[0]) != B.BATCH_KERNELS)
    assert others == sorted(B.sources()) and all(not u[1] for u in units if u not in bk)
