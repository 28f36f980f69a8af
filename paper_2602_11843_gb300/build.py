"""Build libneumann_gb300.so in-tree for sm_103a (GB300).

Each translation unit is compiled in parallel; host C++ is compiled with
-ffp-contract=off so the host-side coefficient refinement gives the same bits
on x86-64 and aarch64. The library links the CUDA runtime dynamically and
resolves the driver's tensor-map encoder at run time, so it loads on a machine
without a GPU driver.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_NAME = "libneumann_gb300.so"
LIB_PATH = os.path.join(HERE, LIB_NAME)
BUILD_DIR = os.path.join(ROOT, "_build")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["kernels_simt.cu", "kernels_tc.cu", "kernels_resident.cu", "noalloc.cu"]
CPP_SOURCES = ["plan.cpp", "approx_kernels.cpp"]


def _cmds():
    inc = ["-I", INCLUDE, "-I", CSRC, "-I", os.path.join(CUDA_HOME, "include")]
    out = []
    for src in CU_SOURCES:
        obj = os.path.join(BUILD_DIR, src + ".o")
        out.append((obj, [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                          "-Xcompiler", "-ffp-contract=off", *inc, "-c", os.path.join(CSRC, src), "-o", obj]))
    cxx = shutil.which("g++") or "c++"
    for src in CPP_SOURCES:
        obj = os.path.join(BUILD_DIR, src + ".o")
        out.append((obj, [cxx, "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", *inc, "-c",
                          os.path.join(CSRC, src), "-o", obj]))
    return out


def _stale(obj: str, src_deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in src_deps)


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile and link; returns the library path. Raises RuntimeError on failure."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "neumann.h"))
    jobs = []
    for obj, cmd in _cmds():
        src = cmd[cmd.index("-c") + 1]
        if force or _stale(obj, [src, *headers]):
            jobs.append((obj, cmd))

    def run(job):
        obj, cmd = job
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        return obj, r

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 2))) as ex:
        for obj, r in ex.map(run, jobs):
            if r.returncode != 0:
                raise RuntimeError(f"compile failed for {obj}:\n{r.stdout}\n{r.stderr}")
            if verbose and r.stderr.strip():
                print(r.stderr, file=sys.stderr)
    objs = [obj for obj, _ in _cmds()]
    if force or jobs or not os.path.exists(LIB_PATH) or _stale(LIB_PATH, objs):
        cxx = shutil.which("g++") or "c++"
        libdir = os.path.join(CUDA_HOME, "lib64")
        if not os.path.isdir(libdir):
            libdir = os.path.join(CUDA_HOME, "lib")
        cmd = [cxx, "-shared", "-o", LIB_PATH + ".tmp", *objs, "-L", libdir, "-lcudart",
               f"-Wl,-rpath,{libdir}", "-lpthread"]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(LIB_PATH + ".tmp", LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
