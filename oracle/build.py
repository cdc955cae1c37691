"""Builds the CPU oracle (test infrastructure) into oracle/liboracle.so.

Plain g++ with IEEE semantics: no fast-math, no FMA contraction, so each FP32
operation of the driving model is one correctly rounded operation.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = ["capi.cpp"]
OUT = os.path.join(HERE, "liboracle.so")


def build(force=False):
    srcs = [os.path.join(HERE, s) for s in SRC if os.path.exists(os.path.join(HERE, s))]
    deps = srcs + [os.path.join(HERE, f) for f in os.listdir(HERE) if f.endswith(".hpp")]
    if not force and os.path.exists(OUT):
        t = os.path.getmtime(OUT)
        if all(os.path.getmtime(d) <= t for d in deps):
            return OUT
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-mno-fma", "-Wall", "-o", OUT + ".tmp"] + srcs
    subprocess.check_call(cmd)
    os.replace(OUT + ".tmp", OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True))
