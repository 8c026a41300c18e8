"""Build step for libcn_b300.so (the C-ABI library declared in include/cn.h).

nvcc compiles csrc/cn_api.cu for sm_103a only (B300); the shared CUDA runtime is
linked so the library and PyTorch use one runtime instance in a process.
"""
from __future__ import annotations

import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libcn_b300.so")
# the CN_DEBUG build: every global-memory access of the kernels bounds-checked
# against the buffers the enqueuing call registered (include/cn.h)
DEBUG_LIB = os.path.join(PKG, "libcn_b300_debug.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

SOURCES = [os.path.join(CSRC, "cn_api.cu"), os.path.join(CSRC, "cn_noalloc.cu"), os.path.join(CSRC, "cn_probe.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [
    os.path.join(ROOT, "include", "cn.h")]

FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17", "-shared",
         "-Xcompiler", "-fPIC", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in DEPS if os.path.exists(p))


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile the library (debug: the CN_DEBUG build) in-tree if it is missing
    or older than its sources."""
    lib = DEBUG_LIB if debug else LIB
    if not force and not needs_build(lib):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, *FLAGS, *(["-DCN_DEBUG"] if debug else []), "-o", tmp, *SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> None:
    """Both libraries, the default and the CN_DEBUG build, compiled in parallel."""
    import threading
    errs = []

    def one(dbg):
        try:
            build(force=force, debug=dbg)
        except Exception as e:  # re-raised below
            errs.append(e)
    ts = [threading.Thread(target=one, args=(d,)) for d in (False, True)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errs:
        raise errs[0]


if __name__ == "__main__":
    build(force=True, verbose=True)
    build(force=True, debug=True)
