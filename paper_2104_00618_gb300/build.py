"""Builds libvct.so in-tree with nvcc for sm_103a (GB300).

Translation units compile in parallel; the library is rebuilt only when a
source, header or flag changes (a hash stamp sits next to it).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libvct.so")

SOURCES = ["vct_api.cu", "mips.cu", "trace.cu", "trace_bwd.cu", "noalloc.cu", "voxelize.cu",
           "bricks.cu", "pipeline.cu", "gbuffer.cu"]
HEADERS = [os.path.join(CSRC, "vct_internal.cuh"), os.path.join(CSRC, "trace_common.cuh"),
           os.path.join(CSRC, "voxelize.cuh"), os.path.join(CSRC, "gbuffer.cuh"),
           os.path.join(INCLUDE, "vct.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvct")


def _stamp(extra_flags) -> str:
    h = hashlib.sha1()
    for f in [os.path.join(CSRC, s) for s in SOURCES] + HEADERS:
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS + list(extra_flags)).encode())
    return h.hexdigest()


def build(verbose: bool = False, extra_flags=(), force: bool = False) -> str:
    """Compile (if needed) and return the path of libvct.so."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = _stamp(extra_flags)
    stamp_file = LIB + ".stamp"
    if (not force and os.path.exists(LIB) and os.path.exists(stamp_file)
            and open(stamp_file).read().strip() == stamp):
        return LIB
    cc = nvcc()
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [cc, *NVCC_FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        logs = list(ex.map(compile_one, zip(SOURCES, objs)))
    if verbose:
        for log in logs:
            print(log)
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
