"""In-tree build of ``libblest.so`` for sm_103a (nvcc for the CUDA translation
units, g++ for the host-only one, compiled in parallel, linked with nvcc)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libblest.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

CU_SOURCES = ["api.cu", "bfs_kernel.cu", "bvss_build.cu", "msbfs_kernel.cu", "parents.cu", "server.cu", "static_scratch.cu", "stats.cu"]
CPP_SOURCES = ["host_graph.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "blest.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link the library if it is missing or older than a source."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", f"-I{INCLUDE}"]
    jobs = []
    for src in CU_SOURCES:
        obj = os.path.join(OUT_DIR, src + ".o")
        jobs.append([nvcc, *ARCH, *common, "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread",
                     "-Xptxas", "-v" if verbose else "-O3", "-c", os.path.join(CSRC, src), "-o", obj])
    for src in CPP_SOURCES:
        obj = os.path.join(OUT_DIR, src + ".o")
        jobs.append(["g++", *common, "-fPIC", "-pthread", "-Wall", "-c", os.path.join(CSRC, src), "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(run, jobs))
    failed = [(c, r) for c, r in results if r.returncode != 0]
    for c, r in results:
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(c) + "\n" + r.stdout + r.stderr)
    if failed:
        raise RuntimeError(f"building libblest failed in {len(failed)} translation unit(s); see stderr")
    objs = [os.path.join(OUT_DIR, s + ".o") for s in CU_SOURCES + CPP_SOURCES]
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-Xcompiler", "-pthread", *objs, "-o", tmp],
                       capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("linking libblest.so failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
