"""Compile the FP64 CPU oracle into ``oracle/liboracle.so``.

Test infrastructure only: the oracle is the checker of the CUDA path, and only
the test suite, the smoke check and the benchmark's CPU-baseline leg load it.
Plain gcc, FP64, ``-ffp-contract=off`` so that no fused multiply-add changes
the rounding of the written-out definitions; OpenMP over independent nodes
when the compiler supports it (it does not reorder arithmetic within a node).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["cmmrt_oracle.c", "h37_oracle.c", "hlat_oracle.c"]
LIB = os.path.join(HERE, "liboracle.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in SOURCES
               if os.path.exists(os.path.join(HERE, s)))


def build(force: bool = False) -> str:
    """Build the oracle library if missing or older than its sources; return its path."""
    if not force and not _stale():
        return LIB
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = base + ["-fopenmp"] + srcs + ["-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP runtime: build single-threaded
        cmd = base + srcs + ["-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
