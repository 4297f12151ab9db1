"""Compile the CPU oracle's C library (test infrastructure; see ``oracle/__init__.py``)."""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "liboracle.so")


def build_oracle(verbose: bool = False) -> str:
    """gcc -O2 -fopenmp -shared; portable flags only (the same source builds on x86 and Arm)."""
    src = os.path.join(_HERE, "gabp_oracle.c")
    out = library_path()
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, src, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(verbose=True))
