"""Builds the host-thread emulation of libiblbm.so (TEST INFRASTRUCTURE).

The library's own sources (kernels, C ABI, server) are compiled with g++ and
-DIBLBM_EMULATE against cuda_emu.h / emu_runtime.cpp, giving
tests/emu/libiblbm_emu.so with the same exported symbols.  The CPU test suite
loads it to run the kernel logic without a GPU; the product never does."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_2609_02298_b300", "csrc")
LIB = os.path.join(HERE, "libiblbm_emu.so")
SOURCES = [os.path.join(CSRC, f) for f in ("kernels.cu", "api.cu", "server.cu", "noalloc.cu")] + \
          [os.path.join(HERE, "emu_runtime.cpp")]


def build(force=False):
    deps = SOURCES + [os.path.join(HERE, "cuda_emu.h"), __file__, os.path.join(ROOT, "include", "iblbm.h")] + \
        [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(d) <= os.path.getmtime(LIB) for d in deps):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    # -Bsymbolic: the library's CUDA runtime calls bind to the emulation in this
    # library even when the real libcudart is already loaded in the process.
    cmd = ["g++", "-std=c++20", "-O2", "-g", "-fPIC", "-shared", "-Wl,-Bsymbolic", "-DIBLBM_EMULATE",
           "-Wno-attributes",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", HERE, "-I", "/usr/local/cuda/include",
           "-x", "c++"] + SOURCES[:-1] + ["-x", "none", SOURCES[-1], "-o", tmp, "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
