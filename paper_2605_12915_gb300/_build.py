"""Build libaf.so (the C-ABI library) in-tree with nvcc for sm_103a."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libaf.so")
SOURCES = ["af_api.cu", "af_noalloc.cu", "af_fc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _deps():
    deps = [os.path.join(ROOT, "include", "af.h"), os.path.abspath(__file__)]
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh", ".h")):
            deps.append(os.path.join(CSRC, f))
    return deps


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force=False, verbose=False, extra_flags=(), out=None):
    """Compile the CUDA sources into paper_2605_12915_gb300/libaf.so (or `out`,
    e.g. a debug variant built with extra_flags).  Rebuilds when a source is
    newer than the library."""
    lib = out or LIB
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= t for d in _deps()):
            return lib
    # -fmad=false: no implicit multiply-add contraction.  Every value that two
    # CTAs compute redundantly (tile-boundary points and edge fluxes) must round
    # identically in every unrolled copy of the code, or conservation breaks;
    # the hot loops use explicit fma() where fusion is wanted.
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC",
             *extra_flags]
    # one object per translation unit, compiled in parallel, then one link
    objs, procs = [], []
    for src in SOURCES:
        tag = os.path.splitext(os.path.basename(lib))[0]
        obj = os.path.join(CSRC, "_build", tag, src.replace(".cu", ".o"))
        os.makedirs(os.path.dirname(obj), exist_ok=True)
        cmd = [nvcc(), *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append(subprocess.Popen(cmd, cwd=CSRC))
        objs.append(obj)
    failed = [p.args for p in procs if p.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, failed[0])
    cmd = [nvcc(), *ARCH, "-shared", "-o", lib + ".tmp", *objs]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd, cwd=CSRC)
    os.replace(lib + ".tmp", lib)
    return lib
