"""Build the CUDA library libbid.so in-tree for sm_103a.

Each translation unit compiles in parallel (nvcc for .cu, g++ for .cpp) into
``_build/``; the shared object is linked next to this file.  Host code uses
no target-specific flags so that it builds on x86-64 and aarch64 alike.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbid.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _cmd(src: str, obj: str, cuda: str):
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if src.endswith(".cu"):
        return [os.path.join(cuda, "bin", "nvcc"), "-std=c++17", "-O3", ARCH, "-lineinfo",
                "-Xcompiler", "-fPIC,-fopenmp", "-Xptxas", "-O3", *inc, "-c",
                os.path.join(CSRC, src), "-o", obj]
    return ["g++", "-std=c++17", "-O3", "-fPIC", "-fopenmp", "-Wall", "-Wno-unused-function",
            "-I", os.path.join(cuda, "include"), *inc, "-c", os.path.join(CSRC, src), "-o", obj]


def _stamp() -> str:
    h = hashlib.sha256()
    for f in _sources() + ["internal.h", "dense.h"]:
        p = os.path.join(CSRC, f)
        if os.path.exists(p):
            h.update(f.encode())
            h.update(open(p, "rb").read())
    h.update(open(os.path.join(ROOT, "include", "bid.h"), "rb").read())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    cuda = _cuda_home()
    os.makedirs(OUT, exist_ok=True)
    stamp_file = os.path.join(OUT, "stamp")
    stamp = _stamp()
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file) \
            and open(stamp_file).read() == stamp:
        return LIB
    objs, cmds = [], []
    for s in _sources():
        obj = os.path.join(OUT, s.rsplit(".", 1)[0] + (".cu.o" if s.endswith(".cu") else ".o"))
        objs.append(obj)
        cmds.append(_cmd(s, obj, cuda))

    def run(c):
        r = subprocess.run(c, capture_output=True, text=True)
        return c, r

    with cf.ThreadPoolExecutor(max_workers=min(8, len(cmds))) as ex:
        for c, r in ex.map(run, cmds):
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(c) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("compilation failed: " + c[-3])
    link = [os.path.join(cuda, "bin", "nvcc"), "-shared", ARCH, "-Xcompiler", "-fopenmp",
            "-o", LIB + ".tmp", *objs, "-lgomp"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
