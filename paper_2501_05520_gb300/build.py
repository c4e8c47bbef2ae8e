"""Compile the CUDA library libptca.so for sm_103a (in-tree, no cmake).

Each translation unit is compiled in parallel with nvcc and the objects are linked
into paper_2501_05520_gb300/lib/libptca.so.  Rebuilds only when a source or header is
newer than the library.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libptca.so")
# The debug build: the same sources compiled with PT_DEBUG (device-side bounds checks
# that report a failing index through a status bit instead of making the access).
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(LIBDIR, "libptca_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                     "-I", CSRC, "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
            + glob.glob(os.path.join(PKG, "tools", "*.cpp")))


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    if not debug and not os.path.exists(os.path.join(LIBDIR, "serve_load")):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          debug: bool = False) -> str:
    """Build libptca.so (debug: libptca_debug.so, compiled with PT_DEBUG); returns its
    path.  Raises RuntimeError on compile errors."""
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(debug):
        return lib
    bdir = BUILD_DEBUG if debug else BUILD
    os.makedirs(bdir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = _nvcc()
    flags = NVCC_FLAGS + (["-DPT_DEBUG"] if debug else []) + (extra_flags or [])

    def compile_one(src: str) -> str:
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise subprocess.CalledProcessError(res.returncode, cmd, res.stdout, res.stderr)
        if verbose and (res.stdout or res.stderr):
            print(res.stdout + res.stderr)
        return obj

    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        try:
            objs = list(ex.map(compile_one, srcs))
        except subprocess.CalledProcessError as e:
            raise RuntimeError(f"nvcc failed:\n{' '.join(e.cmd)}\n{e.stdout}\n{e.stderr}") from None
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, lib)
    if not debug:
        build_tools()
    return lib


TOOLS = os.path.join(PKG, "tools")
SERVE_LOAD = os.path.join(LIBDIR, "serve_load")


def build_tools() -> str:
    """The native open-loop load generator of the request server (lib/serve_load),
    linked against libptca.so."""
    cxx = os.environ.get("CXX", "g++")
    tmp = SERVE_LOAD + f".tmp{os.getpid()}"
    subprocess.check_call([cxx, "-std=c++17", "-O2", "-pthread", "-I", INCLUDE,
                           os.path.join(TOOLS, "serve_load.cpp"), "-L", LIBDIR, "-lptca",
                           "-Wl,-rpath,$ORIGIN", "-o", tmp])
    os.replace(tmp, SERVE_LOAD)
    return SERVE_LOAD


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
