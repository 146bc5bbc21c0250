"""Build the CUDA library in-tree: paper_2403_11651_gb300/_build/libcoolchic.so.

Every translation unit is compiled for sm_103a only (``-gencode arch=compute_103a,
code=sm_103a``), in parallel, then linked with nvcc into one shared library exposing the
C ABI of include/coolchic.h.  Rebuilds only when a source or header is newer than the
library.  ``python -m paper_2403_11651_gb300.build [--force]``.

``--trace`` builds a second library, _build/libcoolchic_trace.so, from all sources as one
translation unit with CC_TRACE defined: every kernel's first block then records its start
time (``%globaltimer``) and name hash in a device buffer read by ``cc_trace_dump``
(see trace.py).  The default library is not affected.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libcoolchic.so")
TRACE_LIB = os.path.join(BUILD, "libcoolchic_trace.so")
SOURCES = ["cc_arm.cu", "cc_syn.cu", "cc_iter.cu", "cc_capi.cu", "cc_noalloc.cu", "cc_codec.cu", "cc_warm.cu"]
HEADERS = [os.path.join(CSRC, "cc_internal.cuh"), os.path.join(CSRC, "cc_laplace.cuh"),
           os.path.join(CSRC, "cc_tc.cuh"), os.path.join(CSRC, "cc_tc16.cuh"),
           os.path.join(ROOT, "include", "coolchic.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-Xcompiler", "-ffp-contract=off"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return path


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    if not force and not _stale(LIB, srcs + HEADERS + [__file__]):
        return LIB
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src).replace(".cu", ".o"))
        if force or _stale(obj, [src] + HEADERS + [__file__]):
            cmd = [cc, *ARCH, *FLAGS, "-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            if verbose:
                sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def build_trace(force: bool = False) -> str:
    """The traced library: one translation unit (the trace buffer is a single device
    symbol) compiled with CC_TRACE."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    if not force and not _stale(TRACE_LIB, srcs + HEADERS + [__file__]):
        return TRACE_LIB
    unit = os.path.join(BUILD, "trace_unit.cu")
    with open(unit, "w") as f:
        f.write("".join(f'#include "{s}"\n' for s in srcs))
    tmp = TRACE_LIB + ".tmp"
    cmd = [nvcc(), *ARCH, *FLAGS, "-DCC_TRACE", "-shared", unit, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on the traced unit:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, TRACE_LIB)
    return TRACE_LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--trace", action="store_true", help="build the traced library instead")
    ap.add_argument("-v", "--verbose", action="store_true")
    a = ap.parse_args()
    print(build_trace(force=a.force) if a.trace else build(force=a.force, verbose=a.verbose))
