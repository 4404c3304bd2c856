"""In-tree build of liblcq.so for sm_103a (GB300) with nvcc; no cmake.

Translation units compile in parallel into paper_2006_02545_gb300/_build/ and link into
paper_2006_02545_gb300/_build/liblcq.so.  Re-running only rebuilds when a source or
header is newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblcq.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["lcq_kernels.cu", "lcq_adjoint.cu", "lcq_nearlist.cu", "lcq_api.cpp",
           "lcq_tables.cpp", "lcq_noalloc.cu", "lcq_peaks.cu",
           "lcq_selftest.cu"]
DEGREES = range(1, 11)   # lcq_deg.cu is built once per patch degree (-DLCQ_DEG=d)


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblcq")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "lcq.h"))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
                     "-I" + INCLUDE, "-I" + CSRC]
    jobs = []
    units = [(src, []) for src in SOURCES] + [("lcq_deg.cu", [f"-DLCQ_DEG={d}"]) for d in DEGREES]
    for src, defs in units:
        stem = os.path.splitext(src)[0] + (defs[0].split("=")[1] if defs else "")
        obj = os.path.join(BUILD, stem + ".o")
        cmd = [nvcc] + common + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd[1:1] = ["--extended-lambda", "-Xptxas", "-v"] if verbose else ["--extended-lambda"]
        else:
            cmd[1:1] = ["-x", "cu"]
        jobs.append((src + " ".join(defs), obj, cmd))

    def run(job):
        src, obj, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r

    with ThreadPoolExecutor(max_workers=min(len(jobs), max(4, os.cpu_count() or 4))) as ex:
        results = list(ex.map(run, jobs))
    for src, r in results:
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr[-8000:]}")
    tmp = LIB + ".tmp"
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + [o for _, o, _ in jobs] + ["-lcudart"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
