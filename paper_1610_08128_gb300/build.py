"""Builds the CUDA library librcm_gb300.so (sm_103a) in-tree with nvcc.

Each translation unit compiles in parallel to an object under _build/, then nvcc links the shared
library into _lib/. Only one -gencode target is built: compute_103a -> sm_103a (GB300).
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ_DIR = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "librcm_gb300.so")
SOURCES = [*(f"rcm_kern_grid{w}.cu" for w in (32, 64, 128, 256, 512, 1024)), "rcm_kern_grid512_async.cu",
           "rcm_kern_grid512_hybrid.cu",
           "rcm_kern_small.cu", "rcm_kern_components.cu",
           "rcm_batch.cu", "rcm_capi.cu", "rcm_prep.cu", "rcm_single.cu", "rcm_server.cu", "rcm_validate.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Kernel templates are instantiated once, in their own translation units, and launched from the
# host code of another: their host stubs need ordinary (not file-static) linkage.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-static-global-template-stub=false", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-Xcompiler", "-Wall"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps(src: str):
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".hpp", ".h"))]
    hdrs.append(os.path.join(os.path.dirname(HERE), "include", "rcm.h"))
    return [os.path.join(CSRC, src)] + hdrs


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(verbose: bool = False, ptxas_info: bool = False, force: bool = False) -> str:
    os.makedirs(OBJ_DIR, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    exe = nvcc()

    def compile_one(src):
        obj = os.path.join(OBJ_DIR, src.replace(".cu", ".o"))
        if not force and not _stale(obj, _deps(src)):
            return obj, ""
        cmd = [exe, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            if log:
                print(log)
    if force or _stale(LIB_PATH, objs):
        cmd = [exe, *ARCH, "-shared", "-o", LIB_PATH, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    return LIB_PATH


if __name__ == "__main__":
    import sys

    print(build(verbose=True, ptxas_info="-v" in sys.argv, force="-f" in sys.argv))
