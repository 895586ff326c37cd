"""Build step for the FP64 CPU oracle (test infrastructure only).

Compiles ``haar_oracle.c`` with the system C compiler into
``oracle/_build/libhaar_oracle.so``, and the benchmark's FP32 CPU baseline
``cpu_baseline.c`` into ``oracle/_build/libhaar_cpu_baseline.so``.  Plain
ISO C11, no SIMD intrinsics and no architecture flags, so both build the
same way on x86_64 and aarch64 and give identical results on both.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "haar_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libhaar_oracle.so")
# the FP32 CPU baseline of the benchmark (cpu_baseline.c; not the oracle)
CPU_LOOP_SRC = os.path.join(HERE, "cpu_baseline.c")
CPU_LOOP_LIB = os.path.join(OUT_DIR, "libhaar_cpu_baseline.so")


def _compile(src: str, lib: str, opt: str, force: bool) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(src)):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [os.environ.get("CC", "gcc"), opt, "-std=c11", "-fPIC", "-shared",
           "-fno-fast-math", "-ffp-contract=off", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile the oracle (and the CPU baseline beside it) if a library is
    missing or older than its source; returns the oracle's path."""
    _compile(CPU_LOOP_SRC, CPU_LOOP_LIB, "-O3", force)
    return _compile(SRC, LIB, "-O2", force)


def build_baseline(force: bool = False) -> str:
    """Compile the FP32 CPU baseline only; returns its path."""
    return _compile(CPU_LOOP_SRC, CPU_LOOP_LIB, "-O3", force)


if __name__ == "__main__":
    print(build(force=True))
    print(build_baseline())
