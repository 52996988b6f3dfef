"""Build the CUDA library in-tree: paper_2206_01683_b300/libfishlbm.so (sm_103a)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libfishlbm.so")
DEBUG_LIB = os.path.join(HERE, "libfishlbm_debug.so")   # index checks on (-DFG_DEBUG_BOUNDS)
SOURCES = [os.path.join(CSRC, "fishlbm.cu"), os.path.join(CSRC, "noalloc.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".cu"))] + [
    os.path.join(ROOT, "include", "fishlbm.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
         "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr"]


def build(force=False, verbose=False, extra=(), debug=False):
    out = DEBUG_LIB if debug else LIB
    if not force and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(p) <= t for p in DEPS):
            return out
    cmd = [NVCC] + FLAGS + (["-DFG_DEBUG_BOUNDS"] if debug else []) + list(extra) + ["-o", out + ".tmp"] + SOURCES
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if a != "--debug"]
    print(build(force=True, verbose=True, extra=args, debug="--debug" in sys.argv[1:]))
