"""Build the solver library ``libfdlbm.so`` in-tree for GB300 (sm_103a).

Plain nvcc: each translation unit of ``csrc/`` compiles in parallel to an object file,
then one link step produces a shared library with the C ABI of ``include/fdlbm.h``
(static CUDA runtime, no torch types). Usage: ``python -m paper_1804_07588_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfdlbm.so")
SOURCES = ["fdlbm_kernels.cu", "fdlbm_local_tau.cu", "fdlbm_ledger_detail.cu", "fdlbm_store_bf16.cu",
           "fdlbm_store_fp16.cu", "fdlbm3d_kernels.cu", "fdlbm3d_ledger_detail.cu", "fdlbm3d_store_bf16.cu",
           "fdlbm3d_store_fp16.cu", "fdlbm_api.cu", "net_kernels.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfdlbm.so")


def _inputs_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "fdlbm.h"))
    files.append(os.path.join(HERE, "..", "include", "fdlbm_net.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _inputs_mtime():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nv = nvcc()
    # -fmad=false: no implicit contraction of a * b + c; the kernels write their fused
    # multiply-adds explicitly (fmaf), so every instantiation of the same arithmetic (plain
    # or exact-accounts step, single or batched lattice) rounds identically.
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                    "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]
    # extra nvcc flags, e.g. -DFDLBM_THREADS_PER_SM=1024 to change the register budget
    flags += os.environ.get("FDLBM_NVCC_FLAGS", "").split()
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [nv, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
