"""Compile the FP64 oracle (test infrastructure) into oracle/_build/liborc.so.

The oracle is plain C++ with OpenMP and no FMA contraction, so its arithmetic is the IEEE double
arithmetic written in the source.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "yee_oracle.cpp")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liborc.so")


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file into a shared library at `out` (the flags of the oracle)."""
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", src, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Build the oracle shared library if it is missing or older than its source; return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    return compile_source(SRC, LIB)


if __name__ == "__main__":
    print(build(force=True))
