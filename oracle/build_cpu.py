"""Builds oracle/libcpu_mt.so (the multithreaded CPU baseline, cpu_mt.cpp) with g++ and
OpenMP.  Test and measurement infrastructure: the library never links it."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_mt.cpp")
LIB = os.path.join(HERE, "libcpu_mt.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cxx = os.environ.get("CXX") or shutil.which("g++") or "g++"
    tmp = LIB + ".tmp"
    r = subprocess.run([cxx, "-O3", "-fopenmp", "-shared", "-fPIC", "-std=c++17", SRC, "-o", tmp],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"g++ failed on {SRC}:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    return LIB
