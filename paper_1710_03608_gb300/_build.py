"""Compile libctd.so (the CTD CUDA library) in-tree for sm_103a with nvcc.

Translation units compile in parallel; the shared library is linked only
when a source or header is newer than it."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libctd.so")
TORCH_SHIM = os.path.join(HERE, "libctd_torch.so")
TORCH_SHIM_SRC = os.path.join(CSRC, "ctd_torch_alloc.cpp")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
SOURCES = ["ctd_stream.cu", "ctd_sample.cu", "ctd_spmm.cu", "ctd_dense.cu", "ctd_filter.cu", "ctd_api.cu",
           "ctd_dynamic.cu", "ctd_noalloc.cu", "ctd_batch.cu",
           "ctd_serve.cu", "ctd_cfill.cu", "ctd_detect.cu", "ctd_matricize.cu",
           "ctd_nway.cu", "ctd_real.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
            "-I" + INCLUDE, "-I" + CSRC, *extra]


def _deps_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh"))]
    paths += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    paths.append(__file__)
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Build libctd.so if needed; return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    objs = []

    def one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [cc, ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def build_torch_shim(force: bool = False) -> str:
    """Build libctd_torch.so (PyTorch's caching allocator as the library's
    allocator hook) against the installed torch's headers; return its path."""
    if (not force and os.path.exists(TORCH_SHIM)
            and os.path.getmtime(TORCH_SHIM) >= max(os.path.getmtime(TORCH_SHIM_SRC),
                                                    os.path.getmtime(__file__))):
        return TORCH_SHIM
    import torch
    from torch.utils import cpp_extension
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "include")
    incs = [*cpp_extension.include_paths(), cuda_inc]
    libdir = os.path.join(os.path.dirname(torch.__file__), "lib")
    abi = int(torch._C._GLIBCXX_USE_CXX11_ABI)
    tmp = TORCH_SHIM + ".tmp"
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-fvisibility=hidden",
           f"-D_GLIBCXX_USE_CXX11_ABI={abi}", *[f"-I{p}" for p in incs], TORCH_SHIM_SRC,
           "-o", tmp, f"-L{libdir}", "-lc10_cuda", "-lc10", f"-Wl,-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"torch allocator shim failed to build:\n{r.stderr}")
    os.replace(tmp, TORCH_SHIM)
    return TORCH_SHIM


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
