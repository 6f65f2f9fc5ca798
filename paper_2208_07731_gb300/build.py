"""Build the CUDA library libisdf.so in-tree for sm_103a (nvcc, no cmake).

Each .cu file is compiled to an object in parallel, then linked into one
shared library next to this file. The library exports only the C ABI
declared in include/isdf.h.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libisdf.so")
OBJDIR = os.path.join(ROOT, "_build", "obj")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps_mtime() -> float:
    files = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "isdf.h")]
    return max(os.path.getmtime(f) for f in files)


STAMP = LIB + ".stamp"


def _toolchain(nvcc: str) -> str:
    """What the library was built with: nvcc's version line, the host machine and the flags. A library
    built elsewhere (another toolchain or CPU architecture) is rebuilt, not reused."""
    try:
        ver = subprocess.run([nvcc, "--version"], capture_output=True, text=True).stdout.strip().splitlines()[-1]
    except Exception:
        ver = "unknown"
    return "|".join([ver, os.uname().machine, " ".join(ARCH + FLAGS)])


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libisdf.so unless an up-to-date one built by this toolchain on this machine type exists.
    Reports on stderr which of the two happened."""
    nvcc = _nvcc()
    tool = _toolchain(nvcc)
    stamp = open(STAMP).read() if os.path.exists(STAMP) else ""
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime() and stamp == tool):
        print(f"libisdf: reusing {LIB} (sources unchanged, same toolchain)", file=sys.stderr)
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
        cmd = [nvcc] + ARCH + FLAGS + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(tool)
    print(f"libisdf: compiled {len(objs)} sources into {LIB}", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
