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


# Device headers compiled again at run time for shape-specialised kernels
# (cq_jit.cu): (name as included, path).
JIT_HEADERS = [
    ("cq_fast.cuh", os.path.join(CSRC, "cq_fast.cuh")),
    ("cq_rowpath.cuh", os.path.join(CSRC, "cq_rowpath.cuh")),
    ("cq_phases.cuh", os.path.join(CSRC, "cq_phases.cuh")),
    ("cq_device.cuh", os.path.join(CSRC, "cq_device.cuh")),
    ("cq_desc.h", os.path.join(CSRC, "cq_desc.h")),
    ("../../include/cq.h", os.path.join(HERE, "..", "include", "cq.h")),
]
JIT_INC = os.path.join(BUILD, "cq_jit_headers.inc")


def _write_jit_headers() -> None:
    """Embed the device headers' text in a C++ include for cq_jit.cu."""
    parts = ["static const JitHeader kJitHeaders[] = {"]
    for name, path in JIT_HEADERS:
        text = open(path).read()
        if ")cqjit\"" in text:
            raise RuntimeError(f"{path}: contains the raw-string delimiter")
        parts.append(f'  {{"{name}", R"cqjit({text})cqjit"}},')
    parts.append("};")
    parts.append(f"static const int kNumJitHeaders = {len(JIT_HEADERS)};")
    out = "\n".join(parts) + "\n"
    if not os.path.exists(JIT_INC) or open(JIT_INC).read() != out:
        with open(JIT_INC + ".tmp", "w") as f:
            f.write(out)
        os.replace(JIT_INC + ".tmp", JIT_INC)


def _cuda_lib_dir(nvcc: str) -> str:
    import shutil
    path = nvcc if os.path.sep in nvcc else (shutil.which(nvcc) or "/usr/local/cuda/bin/nvcc")
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(path))), "lib64")


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Build libcq.so (the query library) and libcqgen.so (the device-side
    input generator); returns the path of libcq.so."""
    os.makedirs(BUILD, exist_ok=True)
    _write_jit_headers()
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(HERE, "..", "include", "cq.h"), JIT_INC]
    gen_headers = [os.path.join(HERE, "..", "include", "cq_gen.h")]
    nvcc = _nvcc()
    jobs = []
    objs = []
    gen_objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            cmd = [nvcc] + ARCH + NVFLAGS + list(extra_flags) + ["-I", BUILD, "-c", src, "-o", obj]
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
    cuda_lib = _cuda_lib_dir(nvcc)
    for lib, lib_objs, libs in ((LIB, objs, ["-L" + cuda_lib, "-lnvrtc", "-Xlinker", "-rpath=" + cuda_lib]),
                                (GEN_LIB, gen_objs, [])):
        if force or _stale(lib, lib_objs):
            tmp = lib + f".tmp{os.getpid()}"
            run([nvcc] + ARCH + ["-shared", "-o", tmp] + lib_objs + libs + ["-lpthread"])
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
