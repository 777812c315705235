"""Build step for the C oracle (test infrastructure only).

Compiles ``fd_oracle.c`` into ``oracle/_build/liboracle_fd.so`` with plain
gcc, ``-O2 -ffp-contract=off`` (no fused multiply-adds), with OpenMP when the
compiler has it.  Host code only; no CPU-specific flags, so the same source
builds on x86_64 and aarch64.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fd_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle_fd.so")


def _compile(extra):
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
           "-Wall", *extra, "-o", LIB + ".tmp", SRC, "-lm"]
    return subprocess.run(cmd, capture_output=True, text=True)


def build(force=False):
    """Compile the oracle library if it is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    res = _compile(["-fopenmp"])
    if res.returncode != 0:  # no OpenMP runtime: single-threaded build
        res = _compile([])
    if res.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + res.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
