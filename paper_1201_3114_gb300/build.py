"""Build liblorenzcipher.so (the C ABI of include/lc.h) in-tree for sm_103a.

Translation units are compiled in parallel with nvcc and linked into
paper_1201_3114_gb300/_build/liblorenzcipher.so.  Device code is compiled
with --fmad=false so that no multiply-add is ever contracted: the kernels
must round every binary64 operation exactly once, as written.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_NAME = "liblorenzcipher.so"
LIB_PATH = os.path.join(BUILD_DIR, LIB_NAME)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3",
    "-lineinfo",
    "--fmad=false",
    "-std=c++17",
    "-Xcompiler", "-fPIC",
    "-Xcompiler", "-ffp-contract=off",
    "-Xcompiler", "-Wall",
    "-I", os.path.join(ROOT, "include"),
]
SOURCES = ["cipher.cu", "api.cu", "keysched.cpp", "probe.cu", "noalloc.cu", "softfp_eval.cu",
           "stats.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return "nvcc"


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(ROOT, "include", "lc.h"))
    out.append(os.path.abspath(__file__))
    return out


CHECKED_DIR = os.path.join(BUILD_DIR, "checked")
CHECKED_LIB_PATH = os.path.join(BUILD_DIR, "liblorenzcipher_checked.so")


def _stale(lib) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    """Compile (if anything changed) and return the path of the library.
    checked=True builds the checked variant (-DLC_CHECKED: kernels validate
    every part-table entry before use) into its own file."""
    lib = CHECKED_LIB_PATH if checked else LIB_PATH
    obj_dir = CHECKED_DIR if checked else BUILD_DIR
    if checked:
        extra_flags = list(extra_flags) + ["-DLC_CHECKED"]
    if not force and not _stale(lib):
        return lib
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(obj_dir, src + ".o")
        cmd = [cc] + NVCC_FLAGS + list(extra_flags) + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd += ["-x", "c++"]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
