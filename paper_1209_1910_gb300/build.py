"""Build libtinv.so in-tree with nvcc for sm_103a (its translation units compiled in parallel).

    python -m paper_1209_1910_gb300.build [--force] [--verbose]
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libtinv.so")
OBJDIR = os.path.join(HERE, "_build")
SOURCES = ["tinv_kernels.cu", "tinv_api.cu", "tinv_noalloc.cu", "tinv_bisect.cu",
           "tinv_server.cu", "tinv_eig.cu", "tinv_bdsvd.cu", "tinv_tune.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "tinv.h"))
    return files


def build(force: bool = False, verbose: bool = False, debug: bool = False,
          profile: bool = False, sanitize: bool = False) -> str:
    """Compile libtinv.so, or a diagnostic variant with its own library file and objects:
    profile=True gives libtinv_prof.so (per-CTA phase cycle counts of the cluster kernel),
    debug=True libtinv_debug.so (device bounds checks, TINV_DEBUG), sanitize=True
    libtinv_asan.so (host code under AddressSanitizer and UBSan; load it with the ASan runtime
    preloaded).  Variants combine, e.g. libtinv_debug_asan.so."""
    suffix = ("_prof" if profile else "") + ("_debug" if debug else "") + ("_asan" if sanitize else "")
    lib = LIB.replace("libtinv.so", "libtinv%s.so" % suffix)
    objdir = OBJDIR + suffix
    if not force and os.path.exists(lib):
        if os.path.getmtime(lib) >= max(os.path.getmtime(f) for f in _deps()):
            return lib
    os.makedirs(objdir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "--expt-relaxed-constexpr", "-I", INCLUDE]
    # one flag per option: -Xcompiler splits its argument at commas
    san = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined",
           "-Xcompiler", "-fno-omit-frame-pointer"]
    if verbose:
        flags += ["-Xptxas", "-v"]
    if debug:
        flags += ["-DTINV_DEBUG=1"]
    if profile:
        flags += ["-DTINV_PHASE_PROFILE=1"]
    if sanitize:
        flags += san

    def compile_one(src):
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"] + (san if sanitize else [])
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
