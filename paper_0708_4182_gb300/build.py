"""Build the CUDA library in-tree with nvcc for sm_103a (GB300).

``python -m paper_0708_4182_gb300.build`` or ``build()`` compiles
``csrc/lbm_ewod.cu`` (which includes the fused step kernel) into
``_build/liblbm_ewod.so``. The library links the shared CUDA runtime so that
it shares streams and the primary context with PyTorch.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "liblbm_ewod.so")
SOURCES = [os.path.join(CSRC, "lbm_ewod.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "lbm_step.cuh"), os.path.join(ROOT, "include", "lbm_ewod.h")]
UNET_LIB = os.path.join(BUILD, "libunet_bf16.so")
UNET_SOURCES = [os.path.join(CSRC, "unet_bf16.cu")]
UNET_DEPS = UNET_SOURCES + [os.path.join(ROOT, "include", "unet_bf16.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return cand


def command(out: str = LIB, verbose_ptxas: bool = False, sources=None) -> list[str]:
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-shared",
           "-cudart", "shared", "-I", os.path.join(ROOT, "include"), "-o", out, *(sources or SOURCES)]
    if verbose_ptxas:
        cmd.insert(1, "-Xptxas=-v")
    return cmd


def up_to_date(lib=LIB, deps=DEPS) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in deps)


def _start(lib, sources, verbose_ptxas):
    tmp = lib + f".{os.getpid()}.tmp"
    proc = subprocess.Popen(command(tmp, verbose_ptxas, sources), stdout=subprocess.PIPE,
                            stderr=subprocess.PIPE, text=True)
    return proc, tmp, lib


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Build both libraries (the lattice Boltzmann step and the U-Net
    kernels), compiling them in parallel; returns the step library's path."""
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    if force or not up_to_date(LIB, DEPS):
        jobs.append(_start(LIB, SOURCES, verbose_ptxas))
    if force or not up_to_date(UNET_LIB, UNET_DEPS):
        jobs.append(_start(UNET_LIB, UNET_SOURCES, verbose_ptxas))
    errors = []
    for proc, tmp, lib in jobs:
        out, err = proc.communicate()
        if proc.returncode != 0:
            errors.append(out + err)
            continue
        if verbose_ptxas:
            sys.stderr.write(err)
        os.replace(tmp, lib)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
