"""Compile libhh.so in-tree: the C++ host builder and the sm_103a kernels.

    python -m paper_2604_09147_gb300.build            # build if sources changed
    python -m paper_2604_09147_gb300.build --force

Translation units are compiled in parallel: host C++ with g++ (no FMA
contraction outside the dense linear algebra, so the tree and the partition
are decided by the same floating-point operations on x86-64 and aarch64),
device code with nvcc for sm_103a only.
The CUDA runtime is linked statically, so the library depends only on the
driver.
"""
from __future__ import annotations

import argparse
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libhh.so")
BUILD_DIR = os.path.join(HERE, "_build")

HOST_SRCS = ["builder.cpp", "linalg.cpp", "hhio.cpp", "shard.cpp"]
CUDA_SRCS = ["kernels.cu", "stream.cu", "tc.cu", "mr.cu", "dense_tc.cu", "capi.cu", "construct.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found (set NVCC or install the CUDA toolkit)")


def _digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)) + ["../../include/hh.h"]:
        p = os.path.normpath(os.path.join(CSRC, name))
        if os.path.isfile(p):
            h.update(name.encode())
            with open(p, "rb") as f:
                h.update(f.read())
    h.update(" ".join(ARCH).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libhh.so if missing or stale; returns its path."""
    stamp = os.path.join(BUILD_DIR, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", CSRC, "-I", os.path.join(ROOT, "include")]
    host_flags = ["-O3", "-std=c++17", "-fPIC", "-ffp-contract=off", "-pthread", "-Wall"]
    jobs = []
    objs = []
    for s in HOST_SRCS:
        o = os.path.join(BUILD_DIR, s + ".o")
        flags = list(host_flags)
        if s == "linalg.cpp":   # dense kernels of the compression: contraction allowed
            flags[flags.index("-ffp-contract=off")] = "-ffp-contract=fast"
        jobs.append(["g++", *flags, *inc, "-c", os.path.join(CSRC, s), "-o", o])
        objs.append(o)
    for s in CUDA_SRCS:
        o = os.path.join(BUILD_DIR, s + ".o")
        jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "--expt-relaxed-constexpr", *inc, "-c", os.path.join(CSRC, s), "-o", o])
        objs.append(o)
    procs = []
    for j in jobs:
        if verbose:
            print(" ".join(j), flush=True)
        procs.append((j, subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for j, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(" ".join(j) + "\n" + out.decode(errors="replace"))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if errors:
        raise RuntimeError("compilation failed:\n" + "\n".join(errors))
    tmp = LIB + ".tmp"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-pthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    a = ap.parse_args(argv)
    print(build(force=a.force, verbose=a.verbose))
    return 0


if __name__ == "__main__":
    sys.exit(main())
