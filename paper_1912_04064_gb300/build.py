"""Build libpic.so (the sm_103a CUDA kernels and the C-ABI) in-tree.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_1912_04064_gb300/libpic.so`` with the static CUDA runtime.  nvcc
cross-compiles for sm_103a without a GPU.

``build(checked=True)`` (or ``python -m paper_1912_04064_gb300.build
--checked``) builds ``libpic_checked.so`` instead: the same library with
-DPIC_CHECKED, whose kernels test every guarded shared-tile, bucket and
global index and record an out-of-range one in the context's device error
word (reported as PIC_ECUDA) instead of making the access.  The binding
loads it when the environment has PIC_CHECKED=1.
"""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libpic.so")
LIB_CHECKED = os.path.join(HERE, "libpic_checked.so")
BUILD = os.path.join(HERE, "_build")
UNITS = ["api", "particle_step", "fields", "particles", "noalloc", "runtime", "pic3d", "poisson"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-I" + os.path.join(ROOT, "include")]


def _sources():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "pic.h"))
    return deps


def _compile(unit, checked=False):
    src = os.path.join(CSRC, unit + ".cu")
    obj = os.path.join(BUILD + ("_checked" if checked else ""), unit + ".o")
    extra = ["-DPIC_CHECKED"] if checked else []
    subprocess.run(["nvcc"] + ARCH + FLAGS + extra + ["-c", src, "-o", obj], check=True)
    return obj


def build(force: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    newest = max(os.path.getmtime(p) for p in _sources())
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    os.makedirs(BUILD + ("_checked" if checked else ""), exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(lambda u: _compile(u, checked), UNITS))
    tmp = lib + ".tmp%d" % os.getpid()
    # cuFFT (shared, from the CUDA toolkit) serves the initial Poisson solve
    subprocess.run(["nvcc"] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs +
                   ["-lcufft"], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys

    print(build(force=True, checked="--checked" in sys.argv))
