"""Builds libism.so (the CUDA library behind include/ism.h) in-tree.

Every translation unit under csrc/ is compiled by nvcc for sm_103a only, in
parallel, then linked into paper_2104_13347_gb300/libism.so with the static
CUDA runtime.  Rebuilds only what changed (by modification time).
--bounds-check builds libism_checked.so instead (ISM_BOUNDS_CHECK: kernels
record out-of-range indices, see ism_debug_bounds); select it at run time
with ISM_LIB=libism_checked.so.  --host-sanitize builds libism_san.so, whose
host code (argument checks, planning, the serving layer) carries
AddressSanitizer and UndefinedBehaviorSanitizer; a process that loads it
must preload the ASan runtime.
Usage: python -m paper_2104_13347_gb300.build  [--force] [--verbose] [--bounds-check]
       [--host-sanitize]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libism.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libism_checked.so")
BUILD_SAN = os.path.join(HERE, "_build_san")
LIB_SAN = os.path.join(HERE, "libism_san.so")
# (one flag per -Xcompiler: nvcc splits its argument at commas)
SAN = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined",
       "-Xcompiler", "-fno-omit-frame-pointer", "-Xcompiler", "-fno-sanitize-recover=undefined"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libism.so")


def _flags(verbose: bool, bounds_check: bool = False, host_sanitize: bool = False):
    f = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
         "-I", os.path.join(ROOT, "include"), "--expt-relaxed-constexpr"]
    if bounds_check:
        f += ["-DISM_BOUNDS_CHECK"]
    if host_sanitize:
        f += ["-g", *SAN]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    hs.append(os.path.join(ROOT, "include", "ism.h"))
    return max(os.path.getmtime(h) for h in hs if os.path.exists(h))


def build(force: bool = False, verbose: bool = False, bounds_check: bool = False,
          host_sanitize: bool = False) -> str:
    if bounds_check and host_sanitize:
        raise ValueError("choose one of bounds_check and host_sanitize")
    BUILD = (BUILD_CHECKED if bounds_check else BUILD_SAN if host_sanitize
             else globals()["BUILD"])
    LIB = LIB_CHECKED if bounds_check else LIB_SAN if host_sanitize else globals()["LIB"]
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hm = _headers_mtime()
    exe = nvcc()
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hm):
            jobs.append((s, o))

    def compile_one(so):
        s, o = so
        cmd = [exe, *_flags(verbose, bounds_check, host_sanitize), "-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(s)}:\n{r.stderr}")
        os.replace(o + ".tmp", o)
        return r.stderr

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for msg in ex.map(compile_one, jobs):
                if verbose and msg:
                    sys.stderr.write(msg)
    if force or jobs or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(o) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [exe, "-shared", *ARCH, *(SAN if host_sanitize else []), "-o", tmp, *objs,
               "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv,
                bounds_check="--bounds-check" in sys.argv,
                host_sanitize="--host-sanitize" in sys.argv))
