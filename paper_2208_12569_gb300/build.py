"""Build libfqsl.so (the CUDA library behind include/fqsl.h) in-tree with nvcc
for sm_103a. Translation units compile in parallel into _build/, then link."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libfqsl.so")
# the roofline probes (include/fqsl_probes.h): a separate small library that
# the benchmark loads; not part of the product ABI
PROBES_SRC = os.path.join(PKG, "probes", "roofline_probes.cu")
PROBES_LIB = os.path.join(PKG, "libfqsl_probes.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]
# Translation units whose FP64 arithmetic must round like a plain evaluation
# of the method (no fused multiply-add contraction): the FP64 tracers, the curl
# grid and the Q assembly. The FP32 tracers keep contraction.
NO_FMAD = {"trace_f64.cu", "trace_rect_f64.cu", "trace_rk38_f64.cu", "trace_rect_rk38_f64.cu", "field.cu", "assemble.cu"}


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the fqsl CUDA library cannot be built")
    return exe


def _deps():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  [os.path.join(INCLUDE, "fqsl.h"), os.path.abspath(__file__)])


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_probes(force: bool = False) -> str:
    """Compile the roofline probes into libfqsl_probes.so. Returns its path."""
    deps = [PROBES_SRC, os.path.join(INCLUDE, "fqsl_probes.h"), os.path.abspath(__file__)]
    if not force and not _stale(PROBES_LIB, deps):
        return PROBES_LIB
    tmp = PROBES_LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-shared", PROBES_SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (PROBES_SRC, r.stdout, r.stderr))
    os.replace(tmp, PROBES_LIB)
    return PROBES_LIB


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile every csrc/*.cu for sm_103a and link libfqsl.so (and the roofline
    probes' libfqsl_probes.so). Returns the path of libfqsl.so."""
    build_probes(force)
    deps = _deps()
    if not force and not _stale(LIB, deps):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    exe = nvcc()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        fmad = ["--fmad=false"] if os.path.basename(src) in NO_FMAD else []
        cmd = [exe, *ARCH, *NVCC_FLAGS, *fmad, *extra_flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True))
