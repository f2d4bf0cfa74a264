"""Build the library in-tree: paper_2506_17650_gb300/liblpop.so for sm_103a.

Every translation unit is compiled by nvcc in parallel and linked into one
shared object with the CUDA runtime linked statically.  Usage::

    python -m paper_2506_17650_gb300.build [--verbose-ptxas]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblpop.so")
LIB_CHECKED = os.path.join(HERE, "liblpop_checked.so")

SOURCES = ["api.cu", "kernels_iter.cu", "kernels_check.cu", "kernels_setup.cu", "host_layout.cpp", "device_layout.cu",
           "noalloc.cu", "batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return path


def _compile(src: str, verbose_ptxas: bool, build_dir: str = BUILD, defines=()) -> str:
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3,-pthread", *defines,
           "-I", os.path.join(HERE, "..", "include"), "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cu"):
        cmd[1:1] = ["--expt-relaxed-constexpr"]
        if verbose_ptxas:
            cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    if verbose_ptxas and res.stderr:
        sys.stderr.write(res.stderr)
    return obj


def build(verbose_ptxas: bool = False, force: bool = False, checked: bool = False) -> str:
    """Compile and link; returns the path of the shared library.  checked=True
    builds the debug variant liblpop_checked.so instead (-DLPOP_CHECK_BOUNDS:
    every gather's index checked against the vector it reads, violations
    counted and skipped; read with lpop_bad_gathers)."""
    lib_path = LIB_CHECKED if checked else LIB
    build_dir = BUILD + "_checked" if checked else BUILD
    os.makedirs(build_dir, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "lpop.h")]
    if not force and os.path.exists(lib_path):
        lib_mtime = os.path.getmtime(lib_path)
        if all(os.path.getmtime(d) <= lib_mtime for d in deps):
            return lib_path
    defines = ("-DLPOP_CHECK_BOUNDS",) if checked else ()
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas, build_dir, defines), SOURCES))
    tmp = lib_path + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-Xcompiler", "-pthread", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"linking failed:\n{' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose_ptxas="--verbose-ptxas" in sys.argv, force=True))
