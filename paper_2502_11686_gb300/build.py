"""Builds libks.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into one shared library next to
this file.  Nothing is installed into site-packages.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libks.so")
BUILD_DIR = os.path.join(HERE, "_build")
GENCODE = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", GENCODE, "-Xcompiler", "-fPIC",
              "-Xcompiler", "-O2", "-I", INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


SMALL_UNIT = "ks_small_n.cu"   # compiled once per state dimension N = 1..SMALL_NMAX
SMALL_NMAX = 8
MED_UNIT = "ks_med_n.cu"       # compiled once per N in MED_NS
MED_NS = (12, 16, 24, 32, 48, 64)


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def units():
    """(source, object name, extra flags) of every translation unit."""
    out = []
    for src in sources():
        base = os.path.basename(src)[:-3]
        if os.path.basename(src) == SMALL_UNIT:
            for n in range(1, SMALL_NMAX + 1):
                out.append((src, f"{base}{n}.o", [f"-DKS_SMALL_N={n}"]))
        elif os.path.basename(src) == MED_UNIT:
            for n in MED_NS:
                out.append((src, f"{base}{n}.o", [f"-DKS_MED_N={n}"]))
        else:
            out.append((src, base + ".o", []))
    return out


def _headers_digest() -> str:
    h = hashlib.sha256()
    files = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")))
    files.append(os.path.join(INCLUDE, "ks.h"))
    for f in files:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _digest() -> str:
    h = hashlib.sha256()
    files = sources() + sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")))
    files.append(os.path.join(INCLUDE, "ks.h"))
    for f in files:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile and link libks.so; skipped when the sources are unchanged since the last build."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    stamp = os.path.join(BUILD_DIR, "stamp")
    dig = _digest() + ":" + " ".join(extra_flags)
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    cc = nvcc()
    objs = []

    hdr = _headers_digest()

    def compile_one(unit):
        src, oname, defs = unit
        obj = os.path.join(BUILD_DIR, oname)
        cmd = [cc, *NVCC_FLAGS, *defs, *extra_flags, "-c", src, "-o", obj]
        h = hashlib.sha256(hdr.encode() + " ".join(cmd).encode())
        with open(src, "rb") as fh:
            h.update(fh.read())
        ustamp = obj + ".stamp"
        if not force and os.path.exists(obj) and os.path.exists(ustamp) and open(ustamp).read() == h.hexdigest():
            return obj   # this unit and every header unchanged
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        with open(ustamp, "w") as fh:
            fh.write(h.hexdigest())
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, units()))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, "-shared", GENCODE, "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
