"""Build the CUDA library libmixfft.so in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into one
shared object next to this file.  No torch headers are involved: the library
is a plain C ABI (include/mixfft.h) over the CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmixfft.so")
# debug build: every shared- and global-memory index of the generic and
# fixed-size transform kernels and the tangent pass checked (MF_DEBUG, see
# common.cuh)
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libmixfft_debug.so")
# trace build: device timestamps between the phases of a load history's
# graph (MF_TRACE, read back with mf_trace_read)
BUILD_TRACE = os.path.join(HERE, "_build_trace")
LIB_TRACE = os.path.join(HERE, "libmixfft_trace.so")
SOURCES = ["transform.cu", "transform2_f32.cu", "transform2_f64.cu", "pointwise.cu", "cg.cu", "history.cu",
           "mixfft.cu", "noalloc.cu", "cufft_path.cu", "adjoint.cu", "transform2_dw.cu",
           "constitutive_dw.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-Xptxas", "-v"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def _compile(src, verbose, debug=False, trace=False):
    obj = os.path.join(BUILD_DEBUG if debug else (BUILD_TRACE if trace else BUILD), src.replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, *FLAGS, *(["-DMF_DEBUG"] if debug else []), *(["-DMF_TRACE"] if trace else []), "-c",
           os.path.join(CSRC, src), "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stderr}")
    if verbose:
        sys.stderr.write(res.stderr)
    return obj


def build(verbose: bool = False, force: bool = False, debug: bool = False, trace: bool = False) -> str:
    """Compile libmixfft.so (or, with debug, libmixfft_debug.so: the same
    library with the bounds checks of MF_DEBUG; with trace,
    libmixfft_trace.so: with the phase timestamps of MF_TRACE) unless it is
    newer than every source; returns its path."""
    out = LIB_DEBUG if debug else (LIB_TRACE if trace else LIB)
    os.makedirs(BUILD_DEBUG if debug else (BUILD_TRACE if trace else BUILD), exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(os.path.dirname(HERE), "include", "mixfft.h")]
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(d) for d in deps)):
        return out
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, debug, trace), SOURCES))
    tmp = out + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lcufft"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force=True, debug="--debug" in sys.argv))
