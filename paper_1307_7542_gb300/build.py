"""Compile the CUDA library (sm_103a) into ``_build/libhub.so`` inside the package.

Every ``.cu`` file under ``csrc/`` is compiled in parallel with nvcc and linked into
one shared library whose exported symbols are the ``extern "C"`` entry points
declared in ``include/hub.h``.
"""
from __future__ import annotations

import glob
import json
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libhub.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


TUNED = os.path.join(PKG, "tuned.json")


def tuned_defines() -> list:
    """Kernel shape knobs chosen by autotune.py on this GPU (tuned.json), as NAME=value."""
    if not os.path.exists(TUNED):
        return []
    with open(TUNED) as f:
        knobs = json.load(f).get("defines", {})
    return [f"{k}={v}" for k, v in sorted(knobs.items())]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + [os.path.join(ROOT, "include", "hub.h")])
    if os.path.exists(TUNED):
        deps.append(TUNED)
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, out: str | None = None, defines=None) -> str:
    """Build libhub.so if any source is newer than it; return its path.  The kernel knobs
    come from tuned.json; `out` and `defines` (-D macros replacing those knobs) build a
    separate copy, as the autotuner does for each candidate."""
    if out is None and not force and not _stale():
        return LIB
    if defines is None:
        defines = tuned_defines()
    lib_path = LIB if out is None else out
    build_dir = BUILD if out is None else os.path.dirname(os.path.abspath(out))
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    srcs = sources()

    tag = os.path.basename(lib_path).replace(".so", "")

    def compile_one(src):
        obj = os.path.join(build_dir, f"{tag}_{os.path.basename(src)[:-3]}.o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *[f"-D{d}" for d in defines], "-I", os.path.join(ROOT, "include"),
               "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib_path + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
