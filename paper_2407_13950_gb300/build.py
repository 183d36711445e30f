"""Build libmsqoc.so in-tree (paper_2407_13950_gb300/_build/) with nvcc for sm_103a.

The sweep kernels are templated on (levels L, subsystems q); ``csrc/inst_sweep.cu`` is compiled
once per supported shape so the objects build in parallel.  No cmake, no torch extension
machinery: plain ``nvcc -c`` per unit and one ``nvcc -shared`` link.
"""
from __future__ import annotations

import concurrent.futures
import hashlib
import os
import shutil
import subprocess
import sys
from typing import List, Optional

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmsqoc.so")

ARCH = "-gencode=arch=compute_103a,code=sm_103a"
SHAPES = [(2, q) for q in range(1, 7)] + [(3, q) for q in range(1, 6)]
# host code without floating-point contraction: the compensated FP32 arithmetic of msqoc_split.cuh
# also runs on the host (self-tests), where a fused multiply-add would break its error terms
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-Xcompiler", "-ffp-contract=off",
          "-diag-suppress", "1444", ARCH]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found (set NVCC or put the CUDA toolkit on PATH)")
    return cand


def _sources_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for fn in sorted(os.listdir(d)):
            if fn.endswith((".cu", ".cuh", ".h")):
                with open(os.path.join(d, fn), "rb") as f:
                    h.update(fn.encode())
                    h.update(f.read())
    h.update(" ".join(CFLAGS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()[:16]


def _units() -> List[tuple]:
    units = [("msqoc_api", os.path.join(CSRC, "msqoc_api.cu"), []),
             ("dispatch", os.path.join(CSRC, "dispatch.cu"), []),
             ("batch", os.path.join(CSRC, "msqoc_batch.cu"), []),
             ("peak", os.path.join(CSRC, "msqoc_peak.cu"), []),
             ("lbfgs", os.path.join(CSRC, "msqoc_lbfgs.cu"), []),
             ("selftest", os.path.join(CSRC, "msqoc_selftest.cu"), [])]
    for L, q in SHAPES:
        units.append((f"sweep_L{L}_Q{q}", os.path.join(CSRC, "inst_sweep.cu"), [f"-DMSQOC_L={L}", f"-DMSQOC_Q={q}"]))
    return units


def build(force: bool = False, jobs: Optional[int] = None, verbose: bool = False) -> str:
    """Compile (if sources changed) and return the path of libmsqoc.so."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp.txt")
    digest = _sources_digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read().strip() == digest:
        return LIB
    nvcc = _nvcc()
    units = _units()
    objdir = os.path.join(BUILD, "obj")
    os.makedirs(objdir, exist_ok=True)

    def compile_unit(u):
        name, src, defs = u
        obj = os.path.join(objdir, name + ".o")
        cmd = [nvcc, *CFLAGS, "-I", INCLUDE, *defs, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr.strip():
            sys.stderr.write(r.stderr)
        return obj

    jobs = jobs or max(1, min(len(units), os.cpu_count() or 4))
    with concurrent.futures.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(compile_unit, units))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
