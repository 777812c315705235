"""Build libgbfd.so (the CUDA library behind include/gbfd.h) in-tree.

Each translation unit under csrc/ is compiled by nvcc for sm_103a only, in
parallel, then linked into ``_build/libgbfd.so``.  No cmake, no torch
extension machinery: the library exports a plain C ABI.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC_DIR = os.path.join(HERE, "csrc")
INC_DIR = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libgbfd.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + INC_DIR]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def _sources():
    return sorted(glob.glob(os.path.join(SRC_DIR, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(SRC_DIR, "*.cuh")) + [os.path.join(INC_DIR, "gbfd.h")]


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    headers = glob.glob(os.path.join(SRC_DIR, "*.cuh")) + [os.path.join(INC_DIR, "gbfd.h")]
    return any(os.path.getmtime(p) > t for p in [src] + headers)


def _compile(src, verbose_ptxas=False):
    obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, "-c", src, "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{res.stderr}")
    return obj, res.stderr


def build(force=False, verbose_ptxas=False, jobs=None):
    """Compile and link; returns the library path.  Rebuilds only stale objects."""
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = _sources()
    todo = [s for s in srcs if force or verbose_ptxas
            or _stale(os.path.join(OUT_DIR, os.path.basename(s)[:-3] + ".o"), s)]
    logs = {}
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            for src, (obj, err) in zip(todo, ex.map(lambda s: _compile(s, verbose_ptxas), todo)):
                logs[src] = err
    objs = [os.path.join(OUT_DIR, os.path.basename(s)[:-3] + ".o") for s in srcs]
    if todo or not os.path.exists(LIB):
        cmd = [nvcc(), *ARCH, "-shared", "-o", LIB + ".tmp", *objs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n" + res.stderr)
        os.replace(LIB + ".tmp", LIB)
    if verbose_ptxas:
        for src, err in logs.items():
            print(f"== {os.path.basename(src)}\n{err}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
