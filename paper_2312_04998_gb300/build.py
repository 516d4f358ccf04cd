"""Builds libstoich.so (all CUDA kernels and the C ABI) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked with the
static CUDA runtime; a content hash of the sources and flags skips rebuilds.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libstoich.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-I", os.path.join(ROOT, "include"),
         "-I", CSRC]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libstoich.so")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _digest(srcs, extra):
    h = hashlib.sha256()
    for p in srcs + sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")) + \
            [os.path.join(ROOT, "include", "stoich.h")]:
        h.update(p.encode())
        with open(p, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS + extra).encode())
    return h.hexdigest()


PHASE_LIB = os.path.join(PKG, "libstoich_phases.so")


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, phase_clocks: bool = False) -> str:
    """Compile and link; returns the path of the shared library.  With
    phase_clocks the refresh kernel's per-phase cycle counters are compiled
    in (-DSM_PHASE_CLOCKS) and the result is libstoich_phases.so, built in
    its own folder; the regular library is not touched."""
    nvcc = _nvcc()
    srcs = sources()
    extra = ["-Xptxas", "-v"] if ptxas_v else []
    if phase_clocks:
        extra = extra + ["-DSM_PHASE_CLOCKS"]
    lib_out = PHASE_LIB if phase_clocks else LIB
    build_dir = BUILD + ("_phases" if phase_clocks else "")
    digest = _digest(srcs, extra)
    stamp = os.path.join(build_dir, "stamp")
    if not force and os.path.exists(lib_out) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return lib_out
    os.makedirs(build_dir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        cmd = [nvcc] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc] + FLAGS + ["-x", "c++", "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{res.stderr}")
        return obj, res.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose or ptxas_v:
        for obj, err in results:
            if err.strip():
                print(f"== {os.path.basename(obj)}\n{err}")
    tmp = lib_out + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lpthread"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, lib_out)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return lib_out


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="--ptxas-v" in sys.argv))
