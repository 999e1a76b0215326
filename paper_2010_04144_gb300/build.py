"""Build the sm_103a extension libhemegb.so in-tree (nvcc + g++, no cmake).

The shared library exports the C ABI declared in include/hemegb.h.  The CUDA
runtime is linked statically, so the library needs only the NVIDIA driver.
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libhemegb.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, object name, extra flags): hg_sc_part.cu once per (storage, scheme, launch parity)
# combination of the stream-collide kernels, so the heavy instantiations compile in parallel
_PARTS = [(s, c, p) for s in (0, 1, 2) for c, p in ((0, 2), (1, 0), (1, 1), (1, 2))]
UNITS = ([("hg_sc_part.cu", f"hg_sc_{s}{c}{p}", [f"-DHG_PART_S={s}", f"-DHG_PART_SCHEME={c}",
                                                   f"-DHG_PART_PAR={p}"]) for s, c, p in _PARTS]
         + [("hg_kernels.cu", "hg_kernels", []), ("hg_host.cpp", "hg_host", []), ("hg_noalloc.cu", "hg_noalloc", [])])
SOURCES = sorted({u[0] for u in UNITS})
HEADERS = ["hg_internal.h", "hg_device.cuh", os.path.join("..", "..", "include", "hemegb.h")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(p) > t for p in deps)


def _compile_cmd(src: str, obj: str, verbose_ptxas: bool, extra=()) -> list:
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", *extra, "-c", src, "-o", obj]
        if verbose_ptxas:
            cmd.insert(1, "-Xptxas=-v")
        return cmd
    return ["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", f"-I{CUDA_HOME}/include",
            "-c", src, "-o", obj]


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    objs, procs = [], []
    for f, name, extra in UNITS:
        obj = os.path.join(BUILD, name + ".o")
        objs.append(obj)
        procs.append((name, subprocess.Popen(_compile_cmd(os.path.join(CSRC, f), obj, verbose_ptxas, extra),
                                             stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                             text=True)))
    errs = []
    for f, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errs.append(f"{f}:\n{out}")
        elif verbose_ptxas and out:
            print(out)
    if errs:
        raise RuntimeError("hemegb build failed:\n" + "\n".join(errs))
    tmp = LIB + ".tmp"
    link = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static", "-Xcompiler", "-pthread"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("hemegb link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
