"""Build ``libbcgb300.so`` in-tree with nvcc for sm_103a.

Eight translation units compiled in parallel, then linked with the static
CUDA runtime into ``paper_2605_14780_gb300/_lib/libbcgb300.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
SOURCES = ["plan.cpp", "prune.cpp", "quadrature.cpp", "kernels.cu", "geometry.cu", "sync.cu",
           "fused.cu", "pack.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-I", os.path.join(ROOT, "include")]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def _compile(src, obj, extra):
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


SANITIZE = ["-O1", "-g", "-Xcompiler",
            "-fsanitize=address,-fsanitize=undefined,-fno-omit-frame-pointer"]
HOST_SOURCES = ("plan.cpp", "prune.cpp", "quadrature.cpp")


def build_library(force=False, extra_flags=(), sanitize=False):
    """Compile and link the library; returns its path.

    ``sanitize`` builds a separate copy (``_lib/sanitize/``) whose host
    translation units (plan builder, pruning, quadrature rows) carry the
    address and undefined-behaviour sanitizers, for host-only checks with
    the sanitizer runtimes preloaded; its kernels are the regular ones."""
    out_dir = os.path.join(OUT_DIR, "sanitize") if sanitize else OUT_DIR
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libbcgb300.so")
    srcs = [os.path.join(CSRC, s) for s in SOURCES] + [
        os.path.join(CSRC, "bc_internal.h"), os.path.join(CSRC, "prune.h"),
        os.path.join(CSRC, "quadrature.h"),
        os.path.join(ROOT, "include", "bc.h")]
    if not force and os.path.exists(lib):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(lib) >= newest and not extra_flags:
            return lib
    objs = [os.path.join(out_dir, s.replace(".", "_") + ".o") for s in SOURCES]

    def flags(src):
        return list(extra_flags) + (SANITIZE if sanitize and src in HOST_SOURCES else [])
    with ThreadPoolExecutor(len(SOURCES)) as ex:
        list(ex.map(lambda a: _compile(a[0], a[1], flags(a[0])), zip(SOURCES, objs)))
    cmd = [nvcc(), *ARCH, "-shared", "-o", lib + ".tmp", *objs,
           "-cudart", "static"]
    if sanitize:
        cmd += ["-Xcompiler", "-fsanitize=address,-fsanitize=undefined"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(lib + ".tmp", lib)
    for o in objs:
        os.remove(o)
    return lib


if __name__ == "__main__":
    print(build_library(force=True))
