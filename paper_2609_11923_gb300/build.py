"""Builds libcfr.so in-tree for sm_103a (nvcc + g++, translation units in parallel)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libcfr.so")
BUILD = os.path.join(HERE, "_build")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# --fmad=false: no contraction of a*b+c, so FP64 kernels round exactly like
# the plain definition (bitwise parity in the FP64 mode).
NVFLAGS = ARCH + ["-O3", "-lineinfo", "--fmad=false", "-std=c++17", "-Xcompiler", "-fPIC"]
CU_UNITS = ["cfr_api", "k_bwd32", "k_bwd64", "k_pers32", "k_pers64", "k_br", "k_batch32", "k_batch64", "k_batchbr", "mlp"]
# FP32-only units may contract a*b+c into one FMA (deterministic, and the
# FP32 mode is held to the exploitability tolerance, not to bitwise parity).
FMA_UNITS = {"k_bwd32", "k_pers32", "k_batch32"}
CPP_UNITS = ["compile"]


def _sources():
    out = []
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            out.append(os.path.join(CSRC, f))
    out.append(os.path.join(HERE, "..", "include", "cfr.h"))
    out.append(os.path.join(HERE, "..", "include", "mlp.h"))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(verbose: bool = False, force: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    objs = []
    for u in CU_UNITS:
        obj = os.path.join(BUILD, u + ".o")
        flags = [("--fmad=true" if (f == "--fmad=false" and u in FMA_UNITS) else f) for f in NVFLAGS]
        cmd = [NVCC] + flags + ["-c", os.path.join(CSRC, u + ".cu"), "-o", obj]
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for u in CPP_UNITS:
        obj = os.path.join(BUILD, u + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-c", os.path.join(CSRC, u + ".cpp"), "-o", obj]
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stdout.write(" ".join(cmd) + "\n" + out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(cmd[-3] if "-c" in cmd else cmd)
    if failed:
        raise RuntimeError("libcfr build failed: %s" % failed)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-lpthread", "-ldl"]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv)
