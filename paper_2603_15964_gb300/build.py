"""Build ``liblmep.so`` (the C ABI of include/lmep.h) for sm_103a, in-tree.

Each CUDA translation unit is compiled by its own nvcc process in parallel,
then the objects are linked into one shared library next to this file.  The
CUDA runtime is linked statically, so the library needs only the driver.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "liblmep.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["lmep_set_fb_f64.cu", "lmep_set_fb_f32.cu", "lmep_expm_f64_hi.cu", "lmep_expm_f32_hi.cu",
           "lmep_frozen_set.cu", "lmep_expm_f64.cu", "lmep_expm_f32.cu", "lmep_adjoint.cu", "lmep_api.cu",
           "lmep_expm.cu", "lmep_apply.cu", "lmep_apply_f64.cu", "lmep_apply_stream.cu", "lmep_apply_rk4.cu", "lmep_apply_rk4_f64.cu", "lmep_apply_pw.cu", "lmep_apply_pw_f64.cu", "lmep_peak.cu", "lmep_noalloc.cu",
           "lmep_spectral.cu", "lmep_wide.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-fvisibility=hidden"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found; the LMEP CUDA library cannot be built")


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra or [])
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = OUT + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    if verbose:
        print(f"built {OUT}")
    return OUT


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
