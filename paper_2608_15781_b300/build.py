"""Build the CUDA library in-tree: ``python -m paper_2608_15781_b300.build``.

Compiles ``csrc/api.cu`` (which includes the kernels) for sm_103a with nvcc
into ``paper_2608_15781_b300/libcglbm.so``.  The C ABI is declared in
``include/cglbm.h`` at the repository root.
"""
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libcglbm.so")
SOURCES = [os.path.join(PKG, "csrc", "api.cu")]
DEPENDS = SOURCES + [os.path.join(PKG, "csrc", f) for f in ("kernels.cuh", "lattice.cuh", "compact.cuh", "adjoint.cuh", "layout.cuh")] + [
    os.path.join(ROOT, "include", "cglbm.h")]

NVCC_FLAGS = [
    "-O3", "-std=c++17", "-lineinfo",
    "-gencode", "arch=compute_103a,code=sm_103a",
    "--expt-relaxed-constexpr",
    "-Xcompiler", "-fPIC,-O2",
    "-shared",
]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in DEPENDS)


def build(force=False, verbose=False, ptxas_info=False):
    if not force and up_to_date():
        return LIB
    cmd = [nvcc()] + NVCC_FLAGS + ["-I", os.path.join(ROOT, "include"), "-I", os.path.join(PKG, "csrc")]
    if ptxas_info:
        cmd += ["-Xptxas", "-v"]
    cmd += ["-o", LIB] + SOURCES
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    if verbose or ptxas_info:
        sys.stdout.write(res.stdout + res.stderr)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True, ptxas_info="-v" in sys.argv)
