"""Builds the CUDA library libflb.so in-tree for sm_103a (nvcc only, no cmake).

The translation units compile in parallel; the shared library links the CUDA
runtime statically so the only run-time dependency is the driver.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libflb.so")
# the checking build (FLB_BOUNDS_CHECK: bounds-checked kernel accesses), for debugging and its tests
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(BUILD_CHECK, "libflb_check.so")
FORMATS = ["f32", "f64", "f16", "bf16", "bf16sr"]
# per format: the dispatching TU plus one TU per streaming layout, so the kernels compile in parallel
SOURCES = [f"step_{f}{l}.cu" for f in FORMATS for l in ("", "_ab", "_aae", "_aao")] + \
    ["aux.cu", "api.cu", "noalloc.cu", "d2q9.cu", "rng.cu", "host_mem.cu", "sq.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    return files + [os.path.join(INCLUDE, "flb.h"), __file__]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, check: bool = False) -> str:
    """Compiles libflb.so (check=True: the bounds-checked libflb_check.so in
    its own directory) unless it is newer than every source."""
    out_dir, lib = (BUILD_CHECK, LIB_CHECK) if check else (BUILD, LIB)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}", f"-I{CSRC}",
                    "-Xptxas", "-v" if verbose else "-O3"] + (["-DFLB_BOUNDS_CHECK"] if check else []) + (extra or [])
    cc = nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + flags
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stderr}")
        if verbose:
            sys.stderr.write(res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(4, min(len(SOURCES), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, check="--check" in sys.argv))
