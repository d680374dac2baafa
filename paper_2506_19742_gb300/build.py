"""Builds libnhcbct.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel; the shared library lands next to this
file. Run ``python -m paper_2506_19742_gb300.build`` or call ``build()``.
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
LIB = os.path.join(HERE, "libnhcbct.so")
SOURCES = ["nh_train_f32.cu", "nh_train_bf16.cu", "nh_train_f16.cu", "nh_field_f32.cu", "nh_field_bf16.cu",
           "nh_field_f16.cu", "nh_api.cu", "nh_field.cu", "nh_adam.cu", "nh_project.cu", "nh_probe.cu",
           "nh_ssim.cu", "nh_mask.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _flags(debug: bool):
    f = ARCH + ["-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
                "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]
    f += ["-O0", "-G"] if debug else ["-O3"]
    return f


def _compile(src: str, debug: bool, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(debug)
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(HERE, "..", "include", "nhcbct.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, debug: bool = False, verbose: bool = False) -> str:
    """Compiles the CUDA sources (if changed) and links libnhcbct.so; returns its path.
    Processes that build at the same time (one per GPU under torchrun) take turns on
    a file lock, so only the first one compiles."""
    if not force and not _stale():
        return LIB
    import fcntl
    os.makedirs(BUILD, exist_ok=True)
    with open(os.path.join(BUILD, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            if not force and not _stale():
                return LIB
            return _build_locked(debug, verbose)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(debug: bool, verbose: bool) -> str:
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, debug, verbose), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [_nvcc(), "-shared", "-o", tmp] + objs + ARCH + [
        "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, debug="--debug" in sys.argv, verbose="-v" in sys.argv))
