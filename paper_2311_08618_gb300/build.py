"""Builds libh2eig.so in-tree for sm_103a (nvcc + g++, translation units in
parallel, no cmake).  Usage: python -m paper_2311_08618_gb300.build"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libh2eig.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _sources():
    cu = ["h2_build.cu", "h2_factor.cu", "h2_noalloc.cu", "h2_matvec.cu"]
    cpp = ["h2_plan.cpp", "h2_api.cpp"]
    return [os.path.join(CSRC, f) for f in cu], [os.path.join(CSRC, f) for f in cpp]


def _stale(srcs):
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(os.path.dirname(HERE), "include", "h2eig.h")]
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def build(force: bool = False, verbose: bool = False) -> str:
    cu, cpp = _sources()
    if not force and not _stale(cu + cpp):
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I" + os.path.join(os.path.dirname(HERE), "include")]
    cmds = []
    objs = []
    for s in cu:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(o)
        cmds.append([nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", *inc,
                     "-Xcompiler", "-fPIC,-ffp-contract=off", "-c", s, "-o", o])
    for s in cpp:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(o)
        cmds.append([nvcc, "-x", "cu", *ARCH, "-O3", "-std=c++17", *inc,
                     "-Xcompiler", "-fPIC,-ffp-contract=off", "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        list(ex.map(run, cmds))
    tmp = OUT + ".tmp"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
