"""Build the in-tree CUDA library libcq.so for sm_103a with nvcc.

Each translation unit under csrc/ is compiled in parallel, then linked into
paper_2506_10092_gb300/libcq.so.  No CMake; nvcc and g++ only.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcq.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
           "-Xcompiler", "-Wall", "-Xcudafe", "--diag_suppress=177"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


GEN = os.path.join(HERE, "gen")
GEN_LIB = os.path.join(HERE, "libcqgen.so")


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Build libcq.so (the query library) and libcqgen.so (the device-side
    input generator); returns the path of libcq.so."""
    os.makedirs(BUILD, exist_ok=True)
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(HERE, "..", "include", "cq.h")]
    gen_headers = [os.path.join(HERE, "..", "include", "cq_gen.h")]
    nvcc = _nvcc()
    jobs = []
    objs = []
    gen_objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            cmd = [nvcc] + ARCH + NVFLAGS + list(extra_flags) + ["-c", src, "-o", obj]
            jobs.append(cmd)
    for src in sorted(glob.glob(os.path.join(GEN, "*.cu"))):
        obj = os.path.join(BUILD, "gen_" + os.path.basename(src)[:-3] + ".o")
        gen_objs.append(obj)
        if force or _stale(obj, [src] + gen_headers):
            jobs.append([nvcc] + ARCH + NVFLAGS + list(extra_flags) + ["-c", src, "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + p.stdout + p.stderr)
        return p.stdout + p.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out)
    for lib, lib_objs in ((LIB, objs), (GEN_LIB, gen_objs)):
        if force or _stale(lib, lib_objs):
            tmp = lib + f".tmp{os.getpid()}"
            run([nvcc] + ARCH + ["-shared", "-o", tmp] + lib_objs + ["-lpthread"])
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
