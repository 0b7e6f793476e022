"""Build libpic.so (the sm_103a CUDA kernels and the C-ABI) in-tree.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_1912_04064_gb300/libpic.so`` with the static CUDA runtime.  nvcc
cross-compiles for sm_103a without a GPU.
"""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libpic.so")
BUILD = os.path.join(HERE, "_build")
UNITS = ["api", "particle_step", "fields", "particles", "noalloc", "runtime", "pic3d", "poisson"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-I" + os.path.join(ROOT, "include")]


def _sources():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "pic.h"))
    return deps


def _compile(unit):
    src = os.path.join(CSRC, unit + ".cu")
    obj = os.path.join(BUILD, unit + ".o")
    subprocess.run(["nvcc"] + ARCH + FLAGS + ["-c", src, "-o", obj], check=True)
    return obj


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(p) for p in _sources())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(_compile, UNITS))
    tmp = LIB + ".tmp%d" % os.getpid()
    # cuFFT (shared, from the CUDA toolkit) serves the initial Poisson solve
    subprocess.run(["nvcc"] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs +
                   ["-lcufft"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
