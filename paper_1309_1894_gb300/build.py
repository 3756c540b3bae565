"""Build ``libwxpy.so`` in-tree with nvcc for sm_103a (GB300).

Every translation unit under ``csrc/`` is compiled in parallel into
``csrc/_build/*.o`` and linked into ``libwxpy.so`` next to this file.  Nothing
is installed anywhere else.  ``--fmad=false`` keeps any multiply-add the
compiler might see from being fused; the kernels also use the explicitly
rounded ``__dmul_rn`` / ``__dadd_rn`` intrinsics, which are never fused.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(CSRC, "_build")
LIBRARY = os.path.join(HERE, "libwxpy.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = [*ARCH, "-O3", "-lineinfo", "--fmad=false", "-std=c++17",
              "-Xcompiler", "-fPIC,-Wall", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwxpy.so")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def headers() -> list[str]:
    return (sorted(glob.glob(os.path.join(CSRC, "*.cuh")))
            + sorted(glob.glob(os.path.join(CSRC, "*.h")))
            + sorted(glob.glob(os.path.join(INCLUDE, "*.h"))))


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str) -> str:
    obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
    if _stale(obj, [src, *headers(), __file__]):
        cmd = [nvcc(), *NVCC_FLAGS, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}{r.stdout}")
    return obj


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile and link libwxpy.so (incremental unless ``force``); returns its path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    srcs = sources()
    if force:
        for o in glob.glob(os.path.join(BUILD_DIR, "*.o")):
            os.remove(o)
    jobs = jobs or min(len(srcs), max(2, os.cpu_count() or 2))
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(_compile, srcs))
    if force or _stale(LIBRARY, objs):
        tmp = LIBRARY + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of libwxpy.so failed:\n{r.stderr}{r.stdout}")
        os.replace(tmp, LIBRARY)
    if verbose:
        print(f"built {LIBRARY}")
    return LIBRARY


# ---- the host family (libwxpy_cpu.so): plain gcc, no CUDA ------------------

CPU_DIR = os.path.join(HERE, "cpu")
CPU_BUILD_DIR = os.path.join(CPU_DIR, "_build")
CPU_LIBRARY = os.path.join(HERE, "libwxpy_cpu.so")
# Every flavour keeps the product and the sum separately rounded.
CPU_COMMON = ["-fPIC", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-Wall",
              "-I", INCLUDE, "-I", CPU_DIR]


def cpu_flavours() -> list[list[str]]:
    """Flags of flavours 0, 1, 2.  Flavour 2 adds the CPU target of the machine
    the library is built on (Grace's Neoverse V2 on the GPU machine, with SVE
    disabled: the box's kernel does not expose it, so SVE code would trap);
    elsewhere it adds loop unrolling, and never -march=native."""
    import platform
    f2 = (["-O3", "-mcpu=neoverse-v2+nosve"] if platform.machine() == "aarch64"
          else ["-O3", "-funroll-loops"])
    return [["-O2", "-fno-tree-vectorize"], ["-O3"], f2]


def gcc() -> str:
    for cand in (shutil.which("gcc"), "/usr/bin/gcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("gcc not found")


def _cpu_compile(args: tuple[str, list[str], str]) -> str:
    src, flags, obj = args
    deps = [src, os.path.join(CPU_DIR, "cpu_internal.h"), os.path.join(INCLUDE, "wxpy_cpu.h"),
            os.path.join(INCLUDE, "wxpy.h"), __file__]
    if _stale(obj, deps):
        r = subprocess.run([gcc(), *CPU_COMMON, *flags, "-c", src, "-o", obj],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"gcc failed on {os.path.basename(obj)}:\n{r.stderr}{r.stdout}")
    return obj


def build_cpu(force: bool = False, verbose: bool = False) -> str:
    """Compile the kernel file once per flavour plus the library, link
    libwxpy_cpu.so next to this file; returns its path."""
    os.makedirs(CPU_BUILD_DIR, exist_ok=True)
    if force:
        for o in glob.glob(os.path.join(CPU_BUILD_DIR, "*.o")):
            os.remove(o)
    flavours = cpu_flavours()
    names = ",".join('"' + " ".join(f) + '"' for f in flavours)
    jobs = [(os.path.join(CPU_DIR, "kernels.c"), [*f, f"-DFLAVOUR_TABLE=wxc_table_f{i}"],
             os.path.join(CPU_BUILD_DIR, f"kernels_f{i}.o")) for i, f in enumerate(flavours)]
    jobs.append((os.path.join(CPU_DIR, "wxpy_cpu.c"), ["-O2", f"-DWXC_FLAVOUR_FLAGS={names}"],
                 os.path.join(CPU_BUILD_DIR, "wxpy_cpu.o")))
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(_cpu_compile, jobs))
    if force or _stale(CPU_LIBRARY, objs):
        tmp = CPU_LIBRARY + f".tmp{os.getpid()}"
        r = subprocess.run([gcc(), "-shared", "-o", tmp, *objs, "-lpthread"],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of libwxpy_cpu.so failed:\n{r.stderr}{r.stdout}")
        os.replace(tmp, CPU_LIBRARY)
    if verbose:
        print(f"built {CPU_LIBRARY}")
    return CPU_LIBRARY


if __name__ == "__main__":
    build(verbose=True)
    build_cpu(verbose=True)
