"""Build the in-tree CUDA library libidpdgsem.so for sm_103a.

Each polynomial degree N = 1..7 is its own translation unit (k_inst.cu with
IDP_NP = N + 1) so the kernels compile in parallel; the host runtime and the
C ABI are in idp_host.cu. The library is written next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libidpdgsem.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-diag-suppress", "177"]
NPS = list(range(2, 9))


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))] + \
        [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def _newest_source() -> float:
    return max(os.path.getmtime(p) for p in _sources())


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _compile(args):
    src, obj, defs = args
    cmd = [_nvcc(), *ARCH, *FLAGS, *defs, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{r.stderr[-4000:]}")
    return obj


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of libidpdgsem.so."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_source():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tasks = [(os.path.join(CSRC, "k_inst.cu"), os.path.join(BUILD, f"k_np{n}.o"), [f"-DIDP_NP={n}"]) for n in NPS]
    tasks.append((os.path.join(CSRC, "idp_host.cu"), os.path.join(BUILD, "idp_host.o"), []))
    tasks.append((os.path.join(CSRC, "k_probe.cu"), os.path.join(BUILD, "k_probe.o"), []))
    tasks.append((os.path.join(CSRC, "k_noalloc.cu"), os.path.join(BUILD, "k_noalloc.o"), []))
    tasks.append((os.path.join(CSRC, "k_remesh.cu"), os.path.join(BUILD, "k_remesh.o"), []))
    # 3D (N = 1..4): one translation unit per degree, and its host runtime
    tasks += [(os.path.join(CSRC, "k_inst3d.cu"), os.path.join(BUILD, f"k3d_np{n}.o"), [f"-DIDP3_NP={n}"])
              for n in (2, 3, 4, 5)]
    tasks.append((os.path.join(CSRC, "idp3d_host.cu"), os.path.join(BUILD, "idp3d_host.o"), []))
    jobs = jobs or min(len(tasks), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(_compile, tasks))
    cmd = [_nvcc(), *ARCH, "-shared", "-o", LIB + ".tmp", *objs, "-lcudart"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
