"""Build librca (the CUDA library behind include/rca.h) in-tree for sm_103a.

``python -m paper_2511_21647_gb300.build`` compiles every translation unit
under csrc/ with nvcc in parallel and links paper_2511_21647_gb300/_build/librca.so.
``build(checked=True)`` links the checked variant _build/librca_checked.so
(-DRCA_CHECKED: shared-memory ring slots, staged rows and queue indexes are
bounds-checked and a violation sets RCA_ERR_BOUNDS in the status word); the
binding loads it when RCA_LIBRARY=checked.
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
LIB = os.path.join(BUILD, "librca.so")
LIB_CHECKED = os.path.join(BUILD, "librca_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# translation units and their extra flags (the FP64 table and tracking
# kernels keep every rounding as written: no fused multiply-add contraction)
UNITS = {
    "api.cu": [],
    "tables.cu": ["-fmad=false"],
    "beamform.cu": [],
    "batch_c32.cu": [],
    "batch_c16f.cu": [],
    "batch_c16bf.cu": [],
    "localize.cu": [],
    "cnn.cu": [],
    "track.cu": ["-fmad=false", "-Xcompiler", "-ffp-contract=off"],
    "motion.cu": [],
    "svd.cu": [],
    "separate.cu": [],
    "peak.cu": [],
}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return [u for u in UNITS if os.path.exists(os.path.join(CSRC, u))]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "rca.h"))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(lib):
        return lib
    objdir = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(objdir, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                     "-I", os.path.join(ROOT, "include"), *(["-DRCA_CHECKED"] if checked else []), *extra]

    def compile_one(unit):
        src = os.path.join(CSRC, unit)
        obj = os.path.join(objdir, unit.replace(".cu", ".o"))
        cmd = [cc, "-c", src, "-o", obj, *common, *UNITS[unit]]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {unit}:\n{r.stderr}")
        return obj, r.stderr

    units = _sources()
    with cf.ThreadPoolExecutor(max_workers=len(units)) as ex:
        results = list(ex.map(compile_one, units))
    if verbose:
        for _, err in results:
            sys.stderr.write(err)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", *ARCH, "-o", tmp, *[o for o, _ in results], "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> list:
    """the release and the checked library, compiled concurrently"""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build, force, False, (), c) for c in (False, True)]
        return [f.result() for f in futs]


if __name__ == "__main__":
    if "--checked" in sys.argv:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked=True))
    else:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
