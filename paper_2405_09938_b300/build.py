"""Build the in-tree CUDA library ``libharm.so`` for sm_103a with nvcc.

Run as ``python -m paper_2405_09938_b300.build`` or call :func:`build`. The
shared library is written next to this file, so it travels with the source tree.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libharm.so")
PEAKS_LIB = os.path.join(HERE, "libharm_peaks.so")  # arithmetic-pipe microbenchmarks (include/harm_peaks.h)
SOURCES = ["harm_scene.cu", "harm_dispatch.cu", "harm_batch.cu", "harm_noalloc.cu", "harm_host.cu", "echo_plain.cu",
           "echo_mixed.cu",
           "echo_mixed_cwm.cu", "echo_mixed_lut.cu", "echo_mixed_cwm_lut.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f != "peaks.cu"]
    files.append(os.path.join(INCLUDE, "harm.h"))
    return files


def up_to_date(lib=LIB, deps=None) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in (deps if deps is not None else _deps()))


def build_peaks(force: bool = False) -> str:
    """Build libharm_peaks.so (one translation unit, no dependence on libharm)."""
    deps = [os.path.join(CSRC, "peaks.cu"), os.path.join(INCLUDE, "harm_peaks.h")]
    if not force and up_to_date(PEAKS_LIB, deps):
        return PEAKS_LIB
    tmp = PEAKS_LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc_path(), "-shared", os.path.join(CSRC, "peaks.cu"), "-o", tmp] + ARCH + [
        "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed on peaks.cu")
    os.replace(tmp, PEAKS_LIB)
    return PEAKS_LIB


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    build_peaks(force)
    if not force and up_to_date():
        return LIB
    nvcc = nvcc_path()
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I" + INCLUDE, "-I" + CSRC] + list(extra)
    if verbose:
        flags += ["-Xptxas", "-v"]
    objs = [os.path.join(objdir, src.replace(".cu", ".o")) for src in SOURCES]

    def compile_one(src, obj):
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + flags
        return src, subprocess.run(cmd, capture_output=True, text=True)

    # the translation units are independent: compile them in parallel
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda a: compile_one(*a), zip(SOURCES, objs)))
    for src, r in results:
        if verbose or r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s" % src)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
