"""Builds libvct.so in-tree with nvcc for sm_103a (GB300).

Translation units compile in parallel; a library is rebuilt only when a
source, header or flag changes (a hash stamp sits next to it).  Two variants:
the release library `libvct.so` and `libvct_debug_bounds.so`, compiled with
-DVCT_DEBUG_BOUNDS (every computed index checked against its array before
the access; see include/vct.h).
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
# variant -> (extra nvcc flags, library file name)
VARIANTS = {"release": ((), "libvct.so"),
            "debug_bounds": (("-DVCT_DEBUG_BOUNDS",), "libvct_debug_bounds.so")}

SOURCES = ["vct_api.cu", "mips.cu", "trace.cu", "trace_bwd.cu", "noalloc.cu", "voxelize.cu",
           "bricks.cu", "pipeline.cu", "gbuffer.cu"]
HEADERS = [os.path.join(CSRC, "vct_internal.cuh"), os.path.join(CSRC, "trace_common.cuh"),
           os.path.join(CSRC, "voxelize.cuh"), os.path.join(CSRC, "gbuffer.cuh"),
           os.path.join(INCLUDE, "vct.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def library_file(variant: str = "release") -> str:
    return os.path.join(BUILD, VARIANTS[variant][1])


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


def build(verbose: bool = False, extra_flags=(), force: bool = False,
          variant: str = "release") -> str:
    """Compile (if needed) and return the path of the variant's library."""
    flags, _ = VARIANTS[variant]
    extra_flags = tuple(flags) + tuple(extra_flags)
    lib_path = library_file(variant)
    obj_dir = os.path.join(BUILD, variant)
    os.makedirs(obj_dir, exist_ok=True)
    stamp = _stamp(extra_flags)
    stamp_file = lib_path + ".stamp"
    if (not force and os.path.exists(lib_path) and os.path.exists(stamp_file)
            and open(stamp_file).read().strip() == stamp):
        return lib_path
    cc = nvcc()
    objs = [os.path.join(obj_dir, s.replace(".cu", ".o")) for s in SOURCES]

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
    tmp = lib_path + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return lib_path


def build_all(verbose: bool = False) -> list:
    """Every variant, compiled concurrently; returns the library paths."""
    with cf.ThreadPoolExecutor(max_workers=len(VARIANTS)) as ex:
        return list(ex.map(lambda v: build(verbose=verbose, variant=v), VARIANTS))


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
