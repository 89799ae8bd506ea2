"""Builds libgbmc.so (the C-ABI library of include/mc.h) for sm_103a, in tree.

Every .cu file under csrc/ is one translation unit; they compile in parallel
with nvcc and link into a shared library next to this file.  The build is
skipped when the library is newer than every source and header.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(ROOT, "_build", "obj")
LIB = os.path.join(PKG, "libgbmc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cuda, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(ROOT, "include", "mc.h"), os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


# Host-code sanitizer variant (AddressSanitizer + UndefinedBehaviorSanitizer
# on the host side of every translation unit: argument checks, plan set-up,
# marshalling); the device code is unchanged.  Built apart from the release
# library and loaded through GBMC_LIBRARY by the sanitizer tests.
SANITIZE_FLAGS = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined",
                  "-Xcompiler", "-fno-omit-frame-pointer", "-Xcompiler", "-fno-sanitize-recover=undefined"]
SANITIZE_LIB = os.path.join(ROOT, "_build", "asan", "libgbmc.so")
# Debug variant: the device code's bounds checks (GBMC_DEBUG, mc_debug_status).
DEBUG_FLAGS = ["-DGBMC_DEBUG=1"]
DEBUG_LIB = os.path.join(ROOT, "_build", "debug", "libgbmc.so")


def build(force: bool = False, verbose: bool = False, jobs: int | None = None, sanitize: bool = False,
          debug: bool = False) -> str:
    variant = "asan" if sanitize else ("debug" if debug else None)
    lib = {None: LIB, "asan": SANITIZE_LIB, "debug": DEBUG_LIB}[variant]
    obj_dir = os.path.join(ROOT, "_build", variant, "obj") if variant else OBJ
    if not force and (up_to_date() if not variant else
                      os.path.exists(lib) and all(os.path.getmtime(f) <= os.path.getmtime(lib) for f in _inputs())):
        return lib
    os.makedirs(obj_dir, exist_ok=True)
    nvcc = _nvcc()
    srcs = sources()
    extra = SANITIZE_FLAGS if sanitize else (DEBUG_FLAGS if debug else [])

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.splitext(os.path.basename(src))[0] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs or os.cpu_count() or 4) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", *extra, "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
