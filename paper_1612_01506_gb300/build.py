"""Build the in-tree native libraries of the package.

``build()`` compiles the CUDA library (``csrc/*.cu``, ``csrc/*.cpp``) for
sm_103a with nvcc into ``_build/<machine>/libsm.so`` and the input generator
(``synth/synth.c``) with gcc. Translation units compile in parallel; a unit
is rebuilt only when a source or header is newer than its object file.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build", platform.machine())
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(OUT, "libsm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra: list[str], out: str = OUT) -> str:
    obj = os.path.join(out, os.path.basename(src) + ".o")
    if _stale(obj, [src] + _headers()):
        cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, "-I", CSRC, *extra, "-c", src, "-o", obj + ".tmp"]
        subprocess.check_call(cmd)
        os.replace(obj + ".tmp", obj)
    return obj


def build_lib(verbose_ptxas: bool = False, out: str = OUT, defines: tuple[str, ...] = ()) -> str:
    """Compile and link libsm.so into `out` (extra -D `defines` for tuning builds)."""
    os.makedirs(out, exist_ok=True)
    lib = os.path.join(out, "libsm.so")
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    extra = (["-Xptxas", "-v"] if verbose_ptxas else []) + [f"-D{d}" for d in defines]
    with cf.ThreadPoolExecutor(max_workers=max(1, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, out), srcs))
    if _stale(lib, objs):
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", lib + ".tmp", *objs])
        os.replace(lib + ".tmp", lib)
    return lib


def build() -> str:
    from . import synth
    synth.build()
    return build_lib()


if __name__ == "__main__":
    print(build())
