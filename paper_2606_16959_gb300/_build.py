"""Compile libhs.so in-tree for sm_103a (nvcc, one process per translation unit)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
SO = os.path.join(OUT_DIR, "libhs.so")
# Index-checking build (-DHS_DEBUG_BOUNDS): a separate library, selected by
# HS_DEBUG_BOUNDS=1 when the package loads.
DEBUG_DIR = os.path.join(HERE, "_build_debug")
ROOT = os.path.dirname(HERE)
HEADERS = (glob.glob(os.path.join(ROOT, "include", "*.h")) + glob.glob(os.path.join(CSRC, "*.h"))
           + glob.glob(os.path.join(CSRC, "*.cuh")))

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    out_dir = DEBUG_DIR if debug else OUT_DIR
    so = os.path.join(out_dir, "libhs.so")
    flags = FLAGS + (["-DHS_DEBUG_BOUNDS"] if debug else [])
    os.makedirs(out_dir, exist_ok=True)
    srcs = sources()
    if not force and not _stale(so, srcs + HEADERS + [__file__]):
        return so
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        if force or _stale(obj, [src] + HEADERS + [__file__]):
            cmd = [nvcc] + ARCH + flags + ["-c", src, "-o", obj]
            if src.endswith(".cu"):
                cmd += ["-Xptxas", "-v"] if verbose else []
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
            if verbose:
                print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = so + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, so)
    return so


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
