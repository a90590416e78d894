"""Build libarrow_gb300.so in-tree for sm_103a (nvcc + g++, no cmake).

Translation units are compiled in parallel into ``paper_2402_19364_gb300/_build``
and linked into ``paper_2402_19364_gb300/libarrow_gb300.so``.  A unit is rebuilt
when its source or any header under ``csrc/`` or ``include/`` is newer than
its object.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = PKG / "libarrow_gb300.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++20", "-Xcompiler", "-fPIC", "-I", str(ROOT / "include")]
CXX_FLAGS = ["-O3", "-std=c++20", "-fPIC", "-Wall", "-I", str(ROOT / "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and Path(c).exists():
            return c
    raise RuntimeError("nvcc not found: the arrow library needs the CUDA toolkit to build")


def _headers_mtime() -> float:
    hs = list(CSRC.glob("*.h")) + list(CSRC.glob("*.cuh")) + list((ROOT / "include").glob("*.h"))
    return max((h.stat().st_mtime for h in hs), default=0.0)


def _units():
    nvcc = _nvcc()
    cxx = os.environ.get("CXX", "g++")
    units = []
    for src in sorted(CSRC.glob("*.cu")):
        obj = BUILD / (src.stem + ".cu.o")
        units.append((src, obj, [nvcc, *ARCH, *NVCC_FLAGS, "-c", str(src), "-o", str(obj)]))
    for src in sorted(CSRC.glob("*.cpp")):
        obj = BUILD / (src.stem + ".cpp.o")
        units.append((src, obj, [cxx, *CXX_FLAGS, "-c", str(src), "-o", str(obj)]))
    return units


def build(force: bool = False, verbose: bool = False) -> Path:
    BUILD.mkdir(exist_ok=True)
    hdr = _headers_mtime()
    procs = []
    objs = []
    for src, obj, cmd in _units():
        objs.append(obj)
        if not force and obj.exists() and obj.stat().st_mtime >= max(src.stat().st_mtime, hdr):
            continue
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("arrow library build failed:\n" + msg)
    newest = max(o.stat().st_mtime for o in objs)
    if force or procs or not LIB.exists() or LIB.stat().st_mtime < newest:
        cmd = [_nvcc(), *ARCH, "-shared", "-o", str(LIB), *map(str, objs), "-lpthread"]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("arrow library link failed:\n" + r.stdout.decode(errors="replace"))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
