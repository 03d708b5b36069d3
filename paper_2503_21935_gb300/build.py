"""Build the mgx CUDA library in-tree for sm_103a.

1. The process compiler writes csrc/generated/programs.inc (op tables and colour
   matrices of the built-in processes).
2. nvcc compiles csrc/mgx.cu into libmgx.so next to this file.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libmgx.so")
GENERATED = os.path.join(HERE, "csrc", "generated", "programs.inc")
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("mgx.cu", "peaks.cu", "phase_space.cu", "mlp.cu", "unweight.cu")]
HEADERS = [os.path.join(HERE, "csrc", f) for f in ("mgx_kernel.cuh", "mgx_ops.cuh", "real.cuh", "umma.cuh", "colour_tc.cuh", "philox.cuh")] + \
          [os.path.join(ROOT, "include", "mgx.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_2503_21935_gb300.gen import emit
    gen_dir = os.path.join(HERE, "gen")
    gen_srcs = [os.path.join(gen_dir, f) for f in os.listdir(gen_dir) if f.endswith(".py")]
    if force or _stale(GENERATED, gen_srcs):
        emit.emit(GENERATED)
    deps = SOURCES + HEADERS + [GENERATED]
    if not force and not _stale(LIB, deps):
        return LIB
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "--threads", "4",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(HERE, "csrc"),
           "-o", LIB + ".tmp", *SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
