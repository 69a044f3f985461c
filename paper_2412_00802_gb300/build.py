"""Build the sm_103a shared library ``libhedl.so`` in-tree with nvcc.

Every translation unit is compiled in parallel for the one target GB300
architecture (``-gencode arch=compute_103a,code=sm_103a``) and linked with the
static CUDA runtime into ``paper_2412_00802_gb300/libhedl.so``.  The library
exposes only the C ABI declared in ``include/hedl.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libhedl.so")
SOURCES = ["api.cu", "exec.cu", "plain.cu", "kb.cu", "noalloc.cu", "tune.cu", "mlp.cu", "umma.cu", "plan.cpp",
           "devplan.cu", "search.cpp"]
HEADERS = ["hedl_internal.h", "device_common.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include")]


# the files that define the batched interpreter (its kernels and the plans it runs)
INTERPRETER = ["exec.cu", "device_common.cuh", "hedl_internal.h", "plan.cpp"]


def _code_only(text: str) -> str:
    """C/C++ source without comments and with whitespace runs collapsed (string literals kept)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"':                                   # string literal, escapes included
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def interpreter_digest() -> str:
    """Digest of the interpreter's code (comments and layout ignored) and build flags:
    recorded ncu counters stay valid while it is unchanged."""
    h = hashlib.sha256()
    for f in INTERPRETER:
        with open(os.path.join(CSRC, f), encoding="utf-8") as fh:
            h.update(f.encode() + _code_only(fh.read()).encode())
    # flags without paths: the checkout's location must not change the digest
    h.update(" ".join(a for a in ARCH + FLAGS if not os.path.isabs(a)).encode())
    return h.hexdigest()


def _digest() -> str:
    h = hashlib.sha256()
    for f in SOURCES + HEADERS:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    with open(os.path.join(ROOT, "include", "hedl.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, src + ".o")
        cmd = [NVCC, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
