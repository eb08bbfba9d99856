"""Build of the CUDA library (sm_103a) with nvcc, in-tree.

Each translation unit compiles in parallel; the FP64 unit is compiled with
--fmad=false so its arithmetic is rounded operation by operation.  Host code
is compiled with -ffp-contract=off for the same reason (the run constants).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
          "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-Xcompiler", "-fno-fast-math"]
# (source, extra flags, object name): the instantiation units compile once
# per lattice (and 16-bit type), so the jobs run in parallel.
UNITS = [("lbm_api.cu", [], "lbm_api.o"),
         ("lbm_noalloc.cu", [], "lbm_noalloc.o"),
         ("lbm_batch_api.cu", [], "lbm_batch_api.o")]
for _lat in range(3):
    UNITS.append(("lbm_inst_f64.cu", ["--fmad=false", f"-DLBM_LAT={_lat}"], f"lbm_inst_f64_{_lat}.o"))
    UNITS.append(("lbm_inst_f32.cu", [f"-DLBM_LAT={_lat}"], f"lbm_inst_f32_{_lat}.o"))
    for _bf in range(2):
        UNITS.append(("lbm_inst_f16.cu", [f"-DLBM_LAT={_lat}", f"-DLBM_BF16={_bf}"],
                      f"lbm_inst_{'bf16' if _bf else 'f16'}_{_lat}.o"))


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources_mtime() -> float:
    m = 0.0
    for root in (CSRC, os.path.join(HERE, "..", "include")):
        for f in os.listdir(root):
            m = max(m, os.path.getmtime(os.path.join(root, f)))
    return m


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    cc = nvcc()

    def compile_unit(item):
        src, extra, oname = item
        obj = os.path.join(BUILD, oname)
        cmd = [cc, *ARCH, *COMMON, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=min(len(UNITS), max(2, os.cpu_count() or 2))) as ex:
        results = list(ex.map(compile_unit, UNITS))
    if verbose or ptxas_info:
        for obj, err in results:
            if err:
                print(f"== {os.path.basename(obj)}\n{err}", file=sys.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
