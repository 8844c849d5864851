"""Build the C oracle into oracle/liboracle.so (gcc, FP64, no FP contraction).

Test infrastructure: the oracle is compiled so that the checker exists; it is
never linked into the product library.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vlbm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-Wall"]


def build(src: str = SRC, out: str = LIB, extra: list[str] | None = None, force: bool = False) -> str:
    """Compile `src` to the shared library `out`; returns the output path."""
    if (not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src)
            and os.path.getmtime(out) >= os.path.getmtime(os.path.join(HERE, "vlbm_oracle.h"))):
        return out
    cmd = ["gcc", *CFLAGS, "-I", HERE, *(extra or []), src, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
