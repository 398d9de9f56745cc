"""In-tree build of libgbpme.so for sm_103a (GB300) with nvcc.

Each CUDA translation unit under ``csrc/`` is compiled in parallel to an object file under
``_build/`` and linked into ``lib/libgbpme.so`` against cuFFT (the only library call on the
path: the two 3D transforms) with the CUDA runtime linked statically. Up-to-date outputs are
reused unless ``force`` is set. The pair-term unit is compiled without implicit multiply-add
contraction (its multiply-adds are written out), so that its fused and list-driven kernels
round identically.
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
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIBNAME = "libgbpme.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# per-unit flags: no implicit contraction where two kernels must round the same expressions
# identically
UNIT_FLAGS = {"pair.cu": ["-fmad=false"]}


def find_nvcc() -> str:
    for cand in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return os.path.join(cand, "bin", "nvcc")
    p = shutil.which("nvcc")
    if p:
        return p
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


BOUNDS_LIBNAME = "libgbpme_bounds.so"


def lib_path(bounds: bool = False) -> str:
    return os.path.join(LIBDIR, BOUNDS_LIBNAME if bounds else LIBNAME)


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, bounds: bool = False) -> str:
    """Compile and link the library; returns the path of the shared object. bounds: the
    index-checking variant (-DGBPME_BOUNDS, libgbpme_bounds.so, objects in _build/bounds)."""
    nvcc = find_nvcc()
    cuda_home = os.path.dirname(os.path.dirname(nvcc))
    bdir = os.path.join(BUILD, "bounds") if bounds else BUILD
    os.makedirs(bdir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    out = lib_path(bounds)
    headers = [d for d in _deps() if not d.endswith(".cu")]
    if not force and not _stale(out, _deps()):
        return out
    cflags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if ptxas_info:
        cflags += ["-Xptxas", "-v"]
    if bounds:
        cflags += ["-DGBPME_BOUNDS"]

    def compile_one(src: str):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        if force or _stale(obj, [src] + headers):
            cmd = [nvcc, "-c", src, "-o", obj] + cflags + UNIT_FLAGS.get(os.path.basename(src), [])
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
            if verbose or ptxas_info:
                print(r.stdout + r.stderr)
        return obj

    srcs = _sources()
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = out + ".tmp"
    cmd = ([nvcc, "-shared", "-o", tmp] + objs + ARCH +
           ["-lcufft", "-cudart", "static", "-Xlinker", f"-rpath,{os.path.join(cuda_home, 'lib64')}"])
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                bounds="--bounds" in sys.argv))
