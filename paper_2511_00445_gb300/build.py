"""Build libtwofluid.so in-tree with nvcc for sm_103a (GB300).

Each .cu translation unit is compiled in parallel, then linked into one
shared library next to this file.  The CUDA runtime is linked statically, so
the library only needs the NVIDIA driver at run time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libtwofluid.so"
LIB_PATH = os.path.join(HERE, LIB_NAME)
# The bounds-check build (-DTF_BOUNDS_CHECK): the hot kernels check their
# shared-memory and global indices and report TF_ERR_BOUNDS instead of
# accessing out of range (tests/test_gpu_bounds_check.py).
BC_LIB_PATH = os.path.join(HERE, "libtwofluid_bc.so")
BC_BUILD_DIR = os.path.join(HERE, "_build_bc")

SOURCES = ["tf_api.cu", "tf_step.cu", "tf_observe.cu", "tf_fused.cu", "tf_ensemble.cu", "nn_surrogate.cu",
           "tf_noalloc.cu"]
HEADERS = ["tf_internal.h", "tf_device.cuh", "tf_ptx.cuh", "tf_pair.cuh", "tf_fused.cuh", "tf_strip.cuh",
           "tf_check.cuh", "nn_tc.cuh"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC] + ARCH


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA 13 toolkit required)")


def _newest_input_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "twofluid.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _is_native(path: str) -> bool:
    """True when the ELF file at path matches this machine's architecture."""
    import platform
    try:
        with open(path, "rb") as fh:
            head = fh.read(20)
    except OSError:
        return False
    if head[:4] != b"\x7fELF":
        return False
    machine = int.from_bytes(head[18:20], "little")
    want = {"x86_64": 62, "aarch64": 183, "arm64": 183}.get(platform.machine(), -1)
    return machine == want


def _fresh(path: str) -> bool:
    return os.path.exists(path) and _is_native(path) and os.path.getmtime(path) >= _newest_input_mtime()


def up_to_date() -> bool:
    return _fresh(LIB_PATH) and _fresh(BC_LIB_PATH)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile and link the library and its bounds-check build (all
    translation units of both in one parallel pass); returns the library's path."""
    if not force and up_to_date():
        return LIB_PATH
    nvcc = nvcc_path()
    os.makedirs(BUILD_DIR, exist_ok=True)
    os.makedirs(BC_BUILD_DIR, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(job) -> str:
        src, out_dir, defs = job
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *NVCC_FLAGS, *defs, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src} {' '.join(defs)}:\n{res.stderr}")
        if verbose or ptxas_info:
            sys.stderr.write(res.stderr)
        return obj

    jobs = [(f, BUILD_DIR, []) for f in SOURCES] + [(f, BC_BUILD_DIR, ["-DTF_BOUNDS_CHECK"]) for f in SOURCES]
    with ThreadPoolExecutor(max_workers=min(len(jobs), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(compile_one, jobs))
    for path, group in ((LIB_PATH, objs[:len(SOURCES)]), (BC_LIB_PATH, objs[len(SOURCES):])):
        tmp = path + ".tmp"
        res = subprocess.run([nvcc, "-shared", *ARCH, "-o", tmp, *group], capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stderr}")
        os.replace(tmp, path)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
