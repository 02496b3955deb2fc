"""In-tree build of libpmgfr.so for sm_103a (nvcc, no cmake).

Translation units compile in parallel; the CUDA runtime is linked statically
so that the library only needs the driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libpmgfr.so")
# objects are kept per host architecture (x86_64 builds must never be linked on aarch64)
BUILD_DIR = os.path.join(HERE, "_build", platform.machine())
ARCH_STAMP = os.path.join(OUT_DIR, ".arch")

CUDA_SOURCES = ["k_residual.cu", "k_volume_dw.cu", "k_blocks.cu", "k_misc.cu", "k_fused.cu", "k_viscous.cu", "k_loop.cu", "k_krylov.cu", "k_factor_cluster.cu",
                "k3_residual.cu", "k3_blocks.cu", "k3_misc.cu", "k3_viscous.cu", "k_tile.cu", "api.cu"]
CXX_SOURCES = ["host_tables.cpp", "host_tables3.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpmgfr")


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(BUILD_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "pmgfr.h"))
    jobs = []
    objs = []
    for src in CUDA_SOURCES + CXX_SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD_DIR, src.rsplit(".", 1)[0] + ".o")
        objs.append(obj)
        if force or _stale(obj, [path] + headers):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                   "-I", CSRC, "-c", path, "-o", obj]
            if src.endswith(".cpp"):
                cmd = [nvcc, "-x", "c++", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", CSRC,
                       "-c", path, "-o", obj]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    stamp = open(ARCH_STAMP).read().strip() if os.path.exists(ARCH_STAMP) else ""
    if force or jobs or not os.path.exists(LIB) or stamp != platform.machine():
        tmp = LIB + ".tmp"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
        with open(ARCH_STAMP, "w") as f:
            f.write(platform.machine())
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
