"""Build the engine's shared library in-tree for sm_103a.

``python -m paper_1802_03084_gb300.build`` (or :func:`build`) compiles the CUDA
sources with nvcc (one -gencode, sm_103a) and the host C ABI with g++ using
``-ffp-contract=off`` (the FP64 plan tables are plain IEEE arithmetic in the
stated order), in parallel, and links ``lib/librealfast_gb300.so``.
Objects go to ``_build/``.  A rebuild happens only when a source or header is
newer than the library.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys
from typing import List

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIBNAME = "librealfast_gb300.so"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _sources():
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                 + glob.glob(os.path.join(INCLUDE, "*.h")))
    return cu, cpp, hdr


def _run(cmd: List[str], verbose: bool) -> str:
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(verbose: bool = False, force: bool = False, ptxas_verbose: bool = False) -> str:
    cu, cpp, hdr = _sources()
    out = lib_path()
    newest = max(os.path.getmtime(f) for f in cu + cpp + hdr + [__file__])
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    inc = ["-I" + INCLUDE, "-I" + CSRC, "-I" + os.path.join(home, "include")]
    jobs = []
    for src in cu:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
               "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off"] + inc + ["-c", src, "-o", obj]
        if ptxas_verbose:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, obj))
    for src in cpp:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-Wall"] + inc + \
              ["-c", src, "-o", obj]
        jobs.append((cmd, obj))
    logs = []
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        futs = [ex.submit(_run, cmd, verbose) for cmd, _ in jobs]
        for f in futs:
            logs.append(f.result())
    objs = [o for _, o in jobs]
    tmp = out + ".tmp"
    _run([nvcc, ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl",
                                                                           "-lpthread"], verbose)
    os.replace(tmp, out)
    if ptxas_verbose:
        print("\n".join(l for l in logs if l.strip()))
    return out


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(verbose=v, force="--force" in sys.argv, ptxas_verbose="--ptxas" in sys.argv))
