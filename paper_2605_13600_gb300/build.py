"""Build libscoup.so (sm_103a) in-tree with nvcc; no CMake.

Each .cu under csrc/ is compiled to an object in parallel and the objects are
linked into ``paper_2605_13600_gb300/libscoup.so``.  ``preprocess.cu`` is
compiled with ``--fmad=false`` so its binary32 projection is evaluated with
every operation rounded, in source order.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libscoup.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-Xptxas", "-warn-spills"]
PER_FILE = {"preprocess.cu": ["--fmad=false"]}


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libscoup.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(os.path.dirname(HERE), "include", "scoup.h")]


def _digest(cmd, deps) -> str:
    """SHA-256 of the compile command and the contents of every input."""
    h = hashlib.sha256("\0".join(cmd).encode())
    for d in deps:
        with open(d, "rb") as f:
            h.update(hashlib.sha256(f.read()).digest())
    return h.hexdigest()


def _stale(target: str, digest: str) -> bool:
    """A target is rebuilt unless it exists and its stamp holds the digest of
    its current inputs (file times alone miss a shipped, newer binary)."""
    stamp = target + ".sha256"
    if not (os.path.exists(target) and os.path.exists(stamp)):
        return True
    with open(stamp) as f:
        return f.read().strip() != digest


def _stamp(target: str, digest: str) -> None:
    with open(target + ".sha256", "w") as f:
        f.write(digest + "\n")


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    hdrs = _headers()
    objs = []
    jobs = []
    for src in srcs:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH, *COMMON, *PER_FILE.get(os.path.basename(src), []), "-c", src, "-o", obj]
        dig = _digest(cmd[1:], [src] + hdrs)
        if force or _stale(obj, dig):
            jobs.append((cmd, obj, dig))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            results = list(ex.map(lambda j: subprocess.run(j[0], capture_output=True, text=True), jobs))
        for (cmd, obj, dig), r in zip(jobs, results):
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
            _stamp(obj, dig)
    link = [*ARCH, "-shared"]
    lib_dig = _digest(link, objs)
    if force or jobs or _stale(LIB, lib_dig):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *link, "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link of libscoup.so failed")
        os.replace(tmp, LIB)
        _stamp(LIB, lib_dig)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
