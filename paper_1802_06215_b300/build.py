"""Builds the CUDA library libdsp.so in-tree for sm_103a (B300).

Device code is compiled with --fmad=false and IEEE division/sqrt so that every
FP32 operation of the car model is one correctly rounded operation; host code
with -ffp-contract=off for the same reason.
"""
import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libdsp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-lineinfo", "-O3", "--fmad=false", "-prec-div=true", "-prec-sqrt=true", "-std=c++17",
                  "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "-I", os.path.join(ROOT, "include")]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.hpp")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))


def _compile(src):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    hdr_t = max(os.path.getmtime(h) for h in _headers())
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_t):
        return obj
    subprocess.check_call(["nvcc"] + NVFLAGS + ["-c", src, "-o", obj + ".tmp"])
    os.replace(obj + ".tmp", obj)
    return obj


def build(force=False, jobs=8):
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in glob.glob(os.path.join(BUILD, "*.o")):
            os.remove(f)
    srcs = _sources()
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(_compile, srcs))
    if os.path.exists(LIB) and all(os.path.getmtime(o) <= os.path.getmtime(LIB) for o in objs):
        return LIB
    subprocess.check_call(["nvcc"] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs +
                          ["-lcudart", "-lpthread"])
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
