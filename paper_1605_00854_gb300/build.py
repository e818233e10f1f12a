"""Build the native library ``libpbn.so`` in-tree.

The CUDA translation unit is compiled by nvcc for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``) and the host C++ by g++; both are
compiled in parallel and linked with nvcc into ``paper_1605_00854_gb300/_build``.
Run ``python -m paper_1605_00854_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libpbn.so")
GENCODE = "arch=compute_103a,code=sm_103a"

CU_SOURCES = ["pbn_sim.cu", "pbn_batch.cu", "pbn_batch1024.cu"]
CPP_SOURCES = ["pbn_host.cpp", "pbn_jit.cpp"]
HEADERS = ["pbn_internal.h", "pbn_image.h", "pbn_device.cuh", "pbn_interp.cuh", "pbn_team.cuh", "pbn_batch.cuh",
           "pbn_batch_interp.cuh"]
# the interpreter's batch work-item function as relocatable device code, linked at run
# time into the batch modules of pbn_batch_compile
ITEM_SOURCE = "pbn_batch_item.cu"
ITEM_CUBIN = os.path.join(OUT, "pbn_batch_item.cubin")
CUDA_INC = "/usr/local/cuda/include"


def _embed_device_header():
    """Write the device headers as C++ raw strings for the plan and batch compilers."""
    for name, inc in (("pbn_device.cuh", "pbn_device_cuh.inc"), ("pbn_batch.cuh", "pbn_batch_cuh.inc")):
        src = os.path.join(CSRC, name)
        dst = os.path.join(OUT, inc)
        text = open(src).read()
        body = 'R"PBNSRC(' + text + ')PBNSRC"\n'
        if not os.path.exists(dst) or open(dst).read() != body:
            with open(dst, "w") as f:
                f.write(body)


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpbn.so")
    return cand


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    proc = subprocess.run(cmd, capture_output=True, text=True)
    if proc.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + proc.stdout + proc.stderr)
    return proc.stdout + proc.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libpbn.so if any source changed; return its path."""
    os.makedirs(OUT, exist_ok=True)
    _embed_device_header()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", OUT]
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "pbn.h")]
    nvcc = _nvcc()
    jobs = []
    objs = []
    for src in CU_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src + ".o")
        objs.append(o)
        if force or _newer(o, [s] + hdrs):
            jobs.append([nvcc, "-gencode", GENCODE, "-O3", "-lineinfo", "-std=c++17",
                         "-Xcompiler", "-fPIC", "-Xptxas", "-v", *inc, "-c", s, "-o", o])
    item = os.path.join(CSRC, ITEM_SOURCE)
    if force or _newer(ITEM_CUBIN, [item] + hdrs):
        jobs.append([nvcc, "-arch=sm_103a", "-rdc=true", "-cubin", "-O3", "-lineinfo", "-std=c++17",
                     "-maxrregcount=128", *inc, item, "-o", ITEM_CUBIN])
    for src in CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src + ".o")
        objs.append(o)
        if force or _newer(o, [s] + hdrs + [os.path.join(OUT, "pbn_device_cuh.inc"),
                                            os.path.join(OUT, "pbn_batch_cuh.inc")]):
            jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", *inc, "-I", CUDA_INC, "-c", s, "-o", o])
    logs = []
    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            logs = list(ex.map(_run, jobs))
    if force or jobs or _newer(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        _run([nvcc, "-shared", "-gencode", GENCODE, "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"])
        os.replace(tmp, LIB)
    if verbose:
        for l in logs:
            sys.stdout.write(l)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
