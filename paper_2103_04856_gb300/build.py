"""Build the CUDA library libpfc.so in-tree for sm_103a (GB300).

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into one shared library with the CUDA runtime linked statically, so the
library does not depend on which libcudart the Python process has loaded.

    python -m paper_2103_04856_gb300.build [--debug]

--debug builds libpfc_debug.so beside the library instead: its kernels fill
their shared-memory staging with NaN before use, so that a read of a cell no
load wrote shows up in the parity tests (run them with
PFC_LIBRARY=<path of libpfc_debug.so>).
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libpfc.so")
DEBUG_LIB = os.path.join(HERE, "libpfc_debug.so")
SOURCES = ["pfc_fused.cu", "pfc_fused_sym.cu", "pfc_fused_slab.cu", "pfc_fused_uni.cu", "pfc_plain.cu", "pfc_api.cu", "pfc_noalloc.cu", "pfc_hflow.cu", "pfc_diag.cu", "pfc_surface.cu", "pfc_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _flags(debug: bool):
    # -ftz=true: FP32 denormals flush to zero (values below 1e-38 carry no
    # weight in the energy), so reciprocal square roots need no range fix-ups
    f = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
         "--expt-relaxed-constexpr", "-ftz=true"] + ARCH
    if debug:
        f += ["-DPFC_DEBUG=1"]
    return f


def build(debug: bool = False, verbose: bool = False, out: str | None = None) -> str:
    out = out or (DEBUG_LIB if debug else LIB)
    tmpdir = os.path.join(HERE, "_build_debug" if debug else "_build")
    os.makedirs(tmpdir, exist_ok=True)
    cc = nvcc()
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    objs = [os.path.join(tmpdir, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    extra = ["-Xptxas", "-v"] if verbose else []

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [cc, "-c", src, "-o", obj] + _flags(debug) + extra
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if verbose:
        for lg in logs:
            sys.stderr.write(lg)
    tmp = out + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--debug", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true", help="print ptxas register/spill usage")
    a = ap.parse_args()
    print(build(debug=a.debug, verbose=a.verbose))
