"""Builds libqc_eloc.so in-tree with nvcc for sm_103a (GB300) only.

Each .cu under csrc/ compiles to an object in _build/ (in parallel), then one shared
library is linked next to this file.  ``-Xptxas -v`` output is kept in
_build/ptxas_<unit>.log for register / spill / shared-memory checks.

``build(checked=True)`` makes libqc_eloc_checked.so from the same sources with QC_CHECKED
defined: every table, integral and work-list index in the kernels is then bounds-checked
(an index out of range sets QC_FLAG_BOUNDS and the call returns QC_ERR_BOUNDS).  It is a
testing build; the product library has no such checks.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libqc_eloc.so")
LIB_CHECKED = os.path.join(HERE, "libqc_eloc_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = ["qc_api.cu", "qc_batch.cu", "qc_server.cu", "qc_kernels.cu", "qc_kernels_diag.cu", "qc_batch_kernels.cu", "qc_static.cu", "qc_grad.cu", "qc_dedup.cu", "qc_full.cu", "qc_probe.cu", "qc_join.cu"]


def _nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqc_eloc")
    return exe


def _sources():
    srcs = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".cu", ".h", ".cuh"))]
    srcs.append(os.path.join(ROOT, "include", "qc_eloc.h"))
    return srcs


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(lib):
        return lib
    nvcc = _nvcc()
    out = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(out, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-Xptxas", "-v"]
    if checked:
        common += ["-DQC_CHECKED"]
    procs = []
    objs = []
    for u in UNITS:
        obj = os.path.join(out, u.replace(".cu", ".o"))
        log = os.path.join(out, f"ptxas_{u.replace('.cu', '')}.log")
        objs.append(obj)
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, u), "-o", obj]
        f = open(log, "w")
        procs.append((u, subprocess.Popen(cmd, stdout=f, stderr=subprocess.STDOUT), f, log))
    failed = []
    for u, p, f, log in procs:
        rc = p.wait()
        f.close()
        text = open(log).read()
        if rc != 0:
            failed.append((u, text))
        elif verbose:
            sys.stdout.write(text)
        if "warning" in text and rc == 0:
            sys.stderr.write(f"[libqc_eloc] compiler warnings in {u}:\n" +
                             "\n".join(l for l in text.splitlines() if "warning" in l) + "\n")
    if failed:
        msg = "\n".join(f"--- {u} ---\n{t}" for u, t in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
