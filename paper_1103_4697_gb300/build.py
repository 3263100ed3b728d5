"""Builds libgbres.so in-tree for sm_103a (GB300).

Each translation unit under csrc/ is compiled by nvcc in parallel, then linked
into paper_1103_4697_gb300/_build/libgbres.so.  A unit is recompiled when its
source, any csrc header, include/gbres.h or the flags changed.
"""

from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgbres.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-Xptxas", "-O3",
                "-I" + os.path.join(ROOT, "include"), "-DNDEBUG"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgbres")


def _digest(src: str) -> str:
    h = hashlib.sha256()
    h.update(" ".join(FLAGS).encode())
    deps = [src, os.path.join(ROOT, "include", "gbres.h")]
    deps += sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh")))
    for d in deps:
        with open(d, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def build(verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    units = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    objs = []

    def compile_one(u: str) -> str:
        src = os.path.join(CSRC, u)
        obj = os.path.join(OUT, u[:-3] + "." + _digest(src) + ".o")
        if not os.path.exists(obj):
            cmd = [nvcc] + FLAGS + ["-c", src, "-o", obj + ".tmp"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {u}:\n{r.stdout}\n{r.stderr}")
            if verbose and r.stderr.strip():
                print(r.stderr)
            os.replace(obj + ".tmp", obj)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(units))) as ex:
        objs = list(ex.map(compile_one, units))
    stamp = hashlib.sha256("".join(objs).encode()).hexdigest()[:16]
    stamp_file = os.path.join(OUT, "libgbres.stamp")
    if os.path.exists(LIB) and os.path.exists(stamp_file) and open(stamp_file).read() == stamp:
        return LIB
    cmd = [nvcc] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    for f in os.listdir(OUT):      # drop objects of older source versions
        p = os.path.join(OUT, f)
        if f.endswith(".o") and p not in objs:
            os.remove(p)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
