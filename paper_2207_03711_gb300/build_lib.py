"""Build the in-tree CUDA library libmpsvqe.so for sm_103a (GB300).

Five translation units compiled in parallel (host.cpp with g++; kernels.cu, api.cu,
tc_gemm.cu and env_tc.cu with nvcc), linked with nvcc into paper_2207_03711_gb300/libmpsvqe.so.
The CUDA runtime is linked statically, so the library only needs the driver.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libmpsvqe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the MPS-VQE library needs the CUDA toolkit to build")


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def build(force=False, verbose=False):
    srcs = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(ROOT, "include", "mpsvqe.h"), __file__])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", CSRC, "-I", os.path.join(ROOT, "include")]
    jobs = [
        # no FMA contraction: the host arithmetic rounds the same on x86-64 and aarch64
        ["g++", "-O2", "-fPIC", "-std=c++17", "-Wall", "-pthread", "-ffp-contract=off", *inc, "-c",
         os.path.join(CSRC, "host.cpp"),
         "-o", os.path.join(OBJ, "host.o")],
    ]
    for name in ("kernels", "api", "tc_gemm", "env_tc"):
        jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *inc,
                     "-c", os.path.join(CSRC, name + ".cu"), "-o", os.path.join(OBJ, name + ".o")])
    with ThreadPoolExecutor(len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    tmp = LIB + ".tmp"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, os.path.join(OBJ, "host.o"), os.path.join(OBJ, "kernels.o"),
          os.path.join(OBJ, "api.o"), os.path.join(OBJ, "tc_gemm.o"),
          os.path.join(OBJ, "env_tc.o"), "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
