"""Build the CPU oracle (oracle/lco.c) into oracle/_build/liblco.so.

Test infrastructure only.  The oracle is compiled with
``-O2 -ffp-contract=off`` so that GCC never fuses a multiply and an add into
one rounding (it would on aarch64 otherwise): every binary64 operation the
source writes is then exactly one IEEE round-to-nearest-even operation.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liblco.so")
SOURCES = [os.path.join(HERE, "lco.c")]
HEADERS = [os.path.join(HERE, "lco.h")]

CFLAGS = [
    "-std=gnu99",
    "-O2",
    "-ffp-contract=off",
    "-fno-fast-math",
    "-fPIC",
    "-shared",
    "-Wall",
    "-Wextra",
]


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(s) > t for s in SOURCES + HEADERS + [__file__])


def build_oracle(force: bool = False) -> str:
    """Compile the oracle if needed and return the path of the shared object."""
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc"] + CFLAGS + ["-o", tmp] + SOURCES + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
