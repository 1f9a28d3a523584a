"""Build libpdas.so in-tree: every csrc/*.cu compiled by nvcc for sm_103a
(GB300), in parallel, then linked into paper_1502_03543_gb300/_lib/libpdas.so.

Run ``python -m paper_1502_03543_gb300.build`` (or call ``build()``).  The
CUDA runtime is linked statically; the driver entry point for tensor maps is
fetched at run time, so the library needs no libcuda at link time.
"""
from __future__ import annotations

import concurrent.futures
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
OBJ_DIR = os.path.join(OUT_DIR, "obj")
LIB_PATH = os.path.join(OUT_DIR, "libpdas.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + INCLUDE, "-I" + CSRC] + ARCH


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers_digest() -> str:
    h = hashlib.sha1()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".cuh", ".h")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode() + fh.read())
    h.update(" ".join(NVCC_FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile and link libpdas.so; returns its path.  Raises on failure."""
    os.makedirs(OBJ_DIR, exist_ok=True)
    nvcc = _nvcc()
    digest = _headers_digest()
    stamp = os.path.join(OBJ_DIR, "headers.sha1")
    stale_headers = force or not os.path.exists(stamp) or open(stamp).read() != digest
    srcs = _sources()
    flags = NVCC_FLAGS + list(extra_flags)

    def obj_of(src):
        return os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + ".o")

    def compile_one(src):
        obj = obj_of(src)
        if not stale_headers and os.path.exists(obj) and os.path.getmtime(obj) >= os.path.getmtime(src):
            return obj, ""
        cmd = [nvcc, "-c", src, "-o", obj] + flags
        proc = subprocess.run(cmd, capture_output=True, text=True)
        if proc.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), proc.stderr))
        return obj, proc.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for obj, err in results:
            if err.strip():
                sys.stderr.write(err)
    objs = [o for o, _ in results]
    tmp = LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), proc.stderr))
    os.replace(tmp, LIB_PATH)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
