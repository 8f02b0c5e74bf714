"""Build libpat.so in-tree with nvcc for sm_103a (no cmake; sources compiled in parallel)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpat.so")
SOURCES = ["pat_api.cu", "pat_run.cu", "pat_zpass.cu", "pat_sample.cu", "pat_solver.cu", "pat_unet.cu",
           "pat_unet_tc.cu"] + [
    f"pat_plane_nx{n}.cu" for n in (8, 16, 32, 64, 128, 256)] + [
    f"pat_line_l{n}.cu" for n in (8, 16, 32, 64, 128, 256)]
HEADERS = ["pat_fft.cuh", "pat_internal.h", "pat_kargs.h", "pat_plane.cuh", "pat_line.cuh",
           os.path.join("..", "..", "include", "pat.h"), os.path.join("..", "..", "include", "pat_unet.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [__file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    tmpdir = os.path.join(HERE, "_build")
    os.makedirs(tmpdir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(tmpdir, src.replace(".cu", f".{os.getpid()}.o"))
        cmd = [cc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([cc, *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"])
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
