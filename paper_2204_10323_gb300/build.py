"""Build the C-ABI shared library ``libflood_gb300.so`` in-tree.

CUDA sources are compiled by nvcc for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``), the host runtime by g++ against
PyTorch's c10 / c10_cuda (device memory and streams come from PyTorch), and
both are linked with the shared CUDA runtime.  Objects go to ``_build/`` next
to this file; every translation unit is compiled in parallel and only when its
sources changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import json
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libflood_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# translation units compiled without FMA contraction (bookkeeping kept in the
# plain definition's rounding order); the step kernels use explicit intrinsics
NO_FMAD = {"epoch.cu"}


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found")


def _torch_paths():
    import torch
    from torch.utils import cpp_extension as ce
    inc = [p for p in ce.include_paths() if os.path.isdir(p)]
    lib = os.path.join(os.path.dirname(torch.__file__), "lib")
    abi = int(bool(torch._C._GLIBCXX_USE_CXX11_ABI))
    return inc, lib, abi


def _deps():
    hdrs = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(p) for p in hdrs)


def _stale(obj: str, src: str, hdr_time: float) -> bool:
    return not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_time)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libflood_gb300.so."""
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    hdr_time = _deps()
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    tinc, tlib, abi = _torch_paths()
    jobs = []
    objs = []
    database = []                  # compile_commands.json: the command of every translation unit
    for src in cu:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [nvcc, "-c", src, "-o", obj, "-O3", "-std=c++17", "-lineinfo", *ARCH,
               "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE, "-Xptxas", "-v"]
        if os.path.basename(src) in NO_FMAD:
            cmd += ["-fmad=false"]
        database.append({"directory": BUILD, "file": src, "arguments": cmd})
        if force or _stale(obj, src, hdr_time):
            jobs.append(cmd)
    for src in cpp:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = ["g++", "-c", src, "-o", obj, "-O2", "-std=c++17", "-fPIC", f"-D_GLIBCXX_USE_CXX11_ABI={abi}",
               "-I", CSRC, "-I", INCLUDE, "-I", os.path.join(cuda, "include")]
        for p in tinc:
            cmd += ["-isystem", p]
        database.append({"directory": BUILD, "file": src, "arguments": cmd})
        if force or _stale(obj, src, hdr_time):
            jobs.append(cmd)
    with open(os.path.join(BUILD, "compile_commands.json"), "w") as f:
        json.dump(database, f, indent=1)
    logs = []
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            logs = list(ex.map(_run, jobs))
    if jobs or force or not os.path.exists(LIB):
        cudalib = os.path.join(cuda, "lib64")
        tmp = LIB + ".tmp"
        _run(["g++", "-shared", "-o", tmp, *objs, "-L", tlib, "-lc10", "-lc10_cuda", "-L", cudalib, "-lcudart",
              f"-Wl,-rpath,{tlib}", f"-Wl,-rpath,{cudalib}"])
        os.replace(tmp, LIB)
    if verbose:
        for l in logs:
            sys.stdout.write(l)
    with open(os.path.join(BUILD, "ptxas.log"), "a") as f:
        for l in logs:
            f.write(l)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
