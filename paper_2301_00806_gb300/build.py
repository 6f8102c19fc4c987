"""Build libwpm.so in-tree with nvcc for sm_103a (GB300).

The search kernels are compiled once per size class (wpm_class.cu with -DWPM_CLASS_ID=k),
in parallel with the other translation units, then linked into one shared library with the
CUDA runtime linked statically. Objects are rebuilt only when a source or header is newer.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libwpm.so")
N_CLASSES = 9
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _flags(extra=()):
    return ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                   "-I", CSRC] + list(extra)


def _units(checked: bool):
    """(source, object, extra flags) of every translation unit."""
    extra = ["-DWPM_CHECKED=1"] if checked else []
    tag = "_chk" if checked else ""
    units = [
        (os.path.join(CSRC, "wpm_kernels.cu"), os.path.join(BUILD, f"wpm_kernels{tag}.o"), extra),
        (os.path.join(CSRC, "wpm_runtime.cpp"), os.path.join(BUILD, f"wpm_runtime{tag}.o"), extra),
        (os.path.join(CSRC, "wpm_noalloc.cu"), os.path.join(BUILD, f"wpm_noalloc{tag}.o"), extra),
        (os.path.join(CSRC, "wpm_engine.cpp"), os.path.join(BUILD, f"wpm_engine{tag}.o"), extra),
        (os.path.join(CSRC, "wpm_sweep.cu"), os.path.join(BUILD, f"wpm_sweep{tag}.o"), extra),
        (os.path.join(CSRC, "wpm_post.cu"), os.path.join(BUILD, f"wpm_post{tag}.o"), extra),
        (os.path.join(CSRC, "wpm_iso.cpp"), os.path.join(BUILD, f"wpm_iso{tag}.o"), extra),
        (os.path.join(CSRC, "wpm_sphere.cpp"), os.path.join(BUILD, f"wpm_sphere{tag}.o"), extra),
        (os.path.join(CSRC, "wpm_link.cpp"), os.path.join(BUILD, f"wpm_link{tag}.o"), extra),
        (os.path.join(CSRC, "wpm_peak.cu"), os.path.join(BUILD, f"wpm_peak{tag}.o"), extra),
    ]
    for k in range(N_CLASSES):
        units.append((os.path.join(CSRC, "wpm_class.cu"), os.path.join(BUILD, f"wpm_class{k}{tag}.o"),
                      extra + [f"-DWPM_CLASS_ID={k}"]))
    return units


def _newest_input(src: str) -> float:
    deps = [src, os.path.join(INCLUDE, "wpm.h")] + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(CSRC, "*.cuh"))
    return max(os.path.getmtime(p) for p in deps)


def build(force: bool = False, checked: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libwpm.so (libwpm_chk.so when checked)."""
    os.makedirs(BUILD, exist_ok=True)
    lib = LIB if not checked else os.path.join(BUILD, "libwpm_chk.so")
    nvcc = _nvcc()
    units = _units(checked)
    todo = [u for u in units
            if force or not os.path.exists(u[1]) or os.path.getmtime(u[1]) < _newest_input(u[0])]

    def compile_one(u):
        src, obj, extra = u
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [nvcc] + _flags(extra) + ["-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)} {extra}:\n{r.stderr}")
        if verbose and r.stderr.strip():
            sys.stderr.write(r.stderr)
        os.replace(tmp, obj)
        return obj

    if todo:
        with ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            list(ex.map(compile_one, todo))
    objs = [u[1] for u in units]
    if force or todo or not os.path.exists(lib) or \
            os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, checked="--checked" in sys.argv, verbose=True))
