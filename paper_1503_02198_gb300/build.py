"""Build the CUDA library libssd.so in-tree (paper_1503_02198_gb300/_build/).

One -gencode (sm_103a), three translation units compiled in parallel (host
driver, FP64 engine, FP32 engine), then linked into a shared library that
exports the C ABI of include/ssd.h.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libssd.so")
# debug build: kernels check every index read from the mesh and mortar tables
# (-DSSD_DEBUG); a bad one raises a device flag that sd_sync reports
LIB_DEBUG = os.path.join(OUT, "libssd_debug.so")
SOURCES = ["ssd_api.cu", "ssd_f64.cu", "ssd_f32.cu", "ssd_f32s.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", *ARCH, *extra]


def build(force: bool = False, verbose: bool = False, extra=(), debug: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    lib_path = LIB_DEBUG if debug else LIB
    tag = "_debug" if debug else ""
    extra = (*extra, "-DSSD_DEBUG") if debug else tuple(extra)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "ssd.h")]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= newest:
        return lib_path
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT, os.path.splitext(src)[0] + tag + ".o")
        cmd = [cc, *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
        if verbose:
            sys.stderr.write(res.stdout + res.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib_path + f".tmp{os.getpid()}"
    cudalib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(cc))), "lib64")
    cmd = [cc, *ARCH, "-shared", *objs, "-o", tmp, "-lcudart", "-Xlinker", "-rpath", "-Xlinker", cudalib]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else (), debug="--debug" in sys.argv))
