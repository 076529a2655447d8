"""Build libpit.so in-tree with nvcc for GB300 (sm_103a)."""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libpit.so")
# the bounds-checking build (-DPIT_CHECK_BOUNDS): every kernel array access checked
CHECK_LIB = os.path.join(OUT_DIR, "libpit_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


# compiled once per level-solve precision and closure (see that file)
BATCH_KERNELS = "pit_batch_kernels.cu"


def sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cu") and f != BATCH_KERNELS]


def units():
    """(source, extra flags, object tag) of every compilation, the slowest first."""
    out = [(s, [], os.path.basename(s)[:-3]) for s in sources()]
    bk = os.path.join(CSRC, BATCH_KERNELS)
    out[1:1] = [(bk, [f"-DPIT_BK_FP32={f}", f"-DPIT_BK_CLOSURES={c}"], f"bk_{f}_{c}") for c in (1, 2, 4, 8) for f in (0, 1)]
    return out


def _deps():
    deps = sources() + [os.path.join(CSRC, BATCH_KERNELS)]
    deps += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return deps


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpit.so")


def build(force: bool = False, verbose: bool = False, check_bounds: bool = False) -> str:
    """Compile every csrc/*.cu into paper_2406_00878_gb300/_build/libpit.so (skipped when up to date).
    The compilations run in parallel (one nvcc each, at most one per CPU), then one nvcc call links.
    check_bounds: the bounds-checking build, libpit_check.so (see pit_bounds_status)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    lib_path = CHECK_LIB if check_bounds else LIB
    if not force and os.path.exists(lib_path):
        t = os.path.getmtime(lib_path)
        if all(os.path.getmtime(d) <= t for d in _deps()):
            return lib_path
    tag = f"{os.getpid()}{'c' if check_bounds else ''}"
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2", f"-I{INCLUDE}", f"-I{CSRC}"]
    if check_bounds:
        flags.append("-DPIT_CHECK_BOUNDS")
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    jobs = units()
    objs = [os.path.join(OUT_DIR, f"{name}.{tag}.o") for _, _, name in jobs]

    def compile_one(i):
        src, extra, _ = jobs[i]
        return subprocess.run([nvcc(), *flags, *extra, "-c", src, "-o", objs[i]]).returncode

    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as pool:
        codes = list(pool.map(compile_one, range(len(jobs))))
    try:
        for (src, extra, _), c in zip(jobs, codes):
            if c != 0:
                raise subprocess.CalledProcessError(c, f"nvcc -c {src} {' '.join(extra)}")
        tmp = lib_path + f".{tag}.tmp"
        subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, lib_path)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return lib_path


def build_check(force: bool = False) -> str:
    """The bounds-checking build, _build/libpit_check.so."""
    return build(force=force, check_bounds=True)


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, check_bounds="--check-bounds" in sys.argv))
