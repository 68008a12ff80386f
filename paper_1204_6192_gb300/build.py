"""Build libhsg.so (the CUDA library behind include/hsg.h) for sm_103a with nvcc.

Each translation unit compiles in parallel; the objects link into one shared
library next to this file.  No torch, cmake or setuptools involved.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhsg.so")
# the same library with device bounds checks compiled in (-DHSG_CHECK)
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libhsg_check.so")
SOURCES = ["hsg_api.cu", "hsg_sweep.cu", "hsg_aux.cu", "hsg_persist.cu", "hsg_noalloc.cu",
           "hsg_overlap.cu", "hsg_multihit.cu", "hsg_fused.cu", "hsg_wave.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps() -> list:
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hdrs + [os.path.join(ROOT, "include", "hsg.h")]


def source_hash() -> str:
    """Hash of every source file of the library (to tell whether a stored profile is current)."""
    import hashlib
    h = hashlib.sha256()
    for f in sorted(SOURCES) + sorted(os.path.basename(d) for d in _deps()):
        p = os.path.join(CSRC, f) if os.path.exists(os.path.join(CSRC, f)) else os.path.join(ROOT, "include", f)
        with open(p, "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in [src] + _deps())


def build(verbose: bool = False, force: bool = False, extra_flags=None, check: bool = False) -> str:
    """Build libhsg.so (check=True: libhsg_check.so, with the device bounds
    checks of HSG_CHECK compiled in) and return its path."""
    build_dir, lib = (BUILD_CHECK, LIB_CHECK) if check else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(ROOT, "include")] + list(extra_flags or [])
    if check:
        flags.append("-DHSG_CHECK")
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        if force or verbose or _stale(o, s):
            p = subprocess.run([cc, "-c", s, "-o", o] + flags, capture_output=True, text=True)
            if p.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{p.stderr}")
            return o, p.stderr
        return o, ""

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    objs = [r[0] for r in results]
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    if force or not os.path.exists(lib) or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        tmp = lib + ".tmp"
        p = subprocess.run([cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"],
                           capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("link failed:\n" + p.stderr)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
