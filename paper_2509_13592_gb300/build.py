"""Build the C-ABI library ``libbccb.so`` for sm_103a with nvcc (in-tree).

Usage: ``python -m paper_2509_13592_gb300.build`` (or ``build()``).  Each
translation unit compiles in its own nvcc process, in parallel; the objects go to
``paper_2509_13592_gb300/_build`` and the shared library next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbccb.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]

L2_VALUES = (16, 32, 64, 128, 256)


def _units():
    units = [("api", "api.cu", []), ("setup_fp64", "setup_fp64.cu", []),
             ("fused_dispatch", "fused_dispatch.cu", []), ("noalloc", "noalloc.cu", []),
             ("multipass", "multipass.cu", []), ("peaks", "peaks.cu", []),
             ("dense", "dense.cu", []), ("fma_rate", "fma_rate.cu", [])]
    for l2 in L2_VALUES:
        units.append((f"fused_L2_{l2}", "fused_inst.cu", [f"-DBCCB_L2={l2}"]))
    return units


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libbccb.so")
    return cand


def _compile(nvcc, name, src, extra, verbose):
    obj = os.path.join(BUILD, name + ".o")
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {name}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(jobs: int | None = None, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    units = _units()
    jobs = jobs or int(os.environ.get("BCCB_BUILD_JOBS", "0")) or min(len(units), os.cpu_count() or 4)
    objs, logs = [], []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = [ex.submit(_compile, nvcc, n, s, e, verbose) for (n, s, e) in units]
        for f in futs:
            o, log = f.result()
            objs.append(o)
            logs.append(log)
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        sys.stderr.write("\n".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
