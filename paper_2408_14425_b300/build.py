"""Build step of librcx.so: nvcc for sm_103a, in-tree (next to this file)."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "librcx.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(HERE, "csrc", "*.h")) + \
        glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + [os.path.join(ROOT, "include", "rcx.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    m = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= m for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles every CUDA source to an object in parallel (one nvcc per file), then links
    librcx.so; the library is replaced atomically."""
    if not force and up_to_date():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    extra = os.environ.get("RCX_NVCC_FLAGS", "").split()   # e.g. -DRCX_MIN_CTAS=6
    obj_dir = os.path.join(HERE, "_build", f"p{os.getpid()}")
    os.makedirs(obj_dir, exist_ok=True)
    common = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xptxas", "-v" if verbose else "-O3", "-I", os.path.join(ROOT, "include"), *extra]
    objs = [os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o") for src in sources()]

    def compile_one(pair):
        src, obj = pair
        subprocess.check_call([*common, "-c", src, "-o", obj])

    with ThreadPoolExecutor(max_workers=max(1, min(len(objs), os.cpu_count() or 1))) as ex:
        list(ex.map(compile_one, zip(sources(), objs)))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([NVCC, *ARCH, "--shared", *objs, "-o", tmp])
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    os.rmdir(obj_dir)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
