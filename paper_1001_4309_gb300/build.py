"""Build the sm_103a CUDA libraries in-tree.

* ``libshifted_fresnel.so`` -- the product library: each ``csrc/*.cu``
  translation unit is compiled in parallel with nvcc for
  ``arch=compute_103a,code=sm_103a`` and linked with the static CUDA runtime.
* ``libsf_plain.so`` -- the paper's per-view procedure with cuFFT
  (``csrc_plain/``), a timed comparison only; the product library does not
  use it.

Both land in ``paper_1001_4309_gb300/_build/``.
"""

from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB_NAME = "libshifted_fresnel.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + INCLUDE, "-I" + CSRC]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def library_path():
    return os.path.join(BUILD, LIB_NAME)


PLAIN_SRC = os.path.join(PKG, "csrc_plain", "sf_plain.cu")
PLAIN_LIB = "libsf_plain.so"


def plain_library_path():
    return os.path.join(BUILD, PLAIN_LIB)


def build_plain(force=False):
    """Compile the cuFFT comparison library if needed; returns its path."""
    lib = plain_library_path()
    deps = [PLAIN_SRC, os.path.join(INCLUDE, "shifted_fresnel.h")]
    if not force and os.path.exists(lib) and all(os.path.getmtime(d) <= os.path.getmtime(lib) for d in deps):
        return lib
    os.makedirs(BUILD, exist_ok=True)
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-shared", PLAIN_SRC, "-o", tmp, "-lcufft", "-L" + cuda_lib,
           "-Xlinker", "-rpath=" + cuda_lib]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {PLAIN_SRC}:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))) + \
        [os.path.join(INCLUDE, "shifted_fresnel.h")]


def up_to_date():
    lib = library_path()
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force=False, verbose=False, extra_flags=()):
    """Compile and link the library if needed; returns its path."""
    if not force and up_to_date():
        return library_path()
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = _sources()
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = library_path() + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, library_path())
    return library_path()


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra_flags=("-Xptxas", "-v") if "-v" in sys.argv else ()))
    print(build_plain(force="--force" in sys.argv))
