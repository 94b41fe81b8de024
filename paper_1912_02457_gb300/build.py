"""Build libswe (the CUDA C-ABI library) in-tree for sm_103a with nvcc.

``python -m paper_1912_02457_gb300.build`` or ``build()`` compiles every
translation unit under csrc/ in parallel and links
paper_1912_02457_gb300/_build/libswe.so (static CUDA runtime, so the library
only needs the driver at run time).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libswe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
              "-I", os.path.join(ROOT, "include"), "-I", CSRC]
# per-file flags: the FP32 fast path uses the approximate reciprocal and
# square root (about 1 ulp) and flushes denormal results to zero (FP32
# values below 1.2e-38, far below any depth, level or momentum the scheme
# resolves; 4% on the coastal 1024 step); the reference kernels stay IEEE
FILE_FLAGS = {"swe_stage_fast.cu": ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]}


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _paths(variant):
    """Output folder and library of a build variant ("" is the product)."""
    out = os.path.join(OUT_DIR, variant) if variant else OUT_DIR
    return out, os.path.join(out, "libswe.so")


def _stale(extra_flags, variant=""):
    out_dir, lib = _paths(variant)
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    deps += glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)]
    stamp = os.path.join(out_dir, "flags.txt")
    want = " ".join(extra_flags)
    if not os.path.exists(stamp) or open(stamp).read() != want:
        return True
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=(), variant: str = "") -> str:
    out_dir, lib = _paths(variant)
    os.makedirs(out_dir, exist_ok=True)
    extra_flags = list(extra_flags)
    if not force and not _stale(extra_flags, variant):
        return lib
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *FILE_FLAGS.get(os.path.basename(src), []),
               *extra_flags, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(os.path.join(out_dir, "flags.txt"), "w") as fh:
        fh.write(" ".join(extra_flags))
    return lib


def build_debug(force: bool = False) -> str:
    """The bounds-checked variant (_build/debug/libswe.so): every global
    access of the FP32 stage kernels checks its offset against the extent of
    its buffer; a violation is skipped and reported as SWE_ERR_BOUNDS with
    the source line in swe_info.error_cell. A test tool, slower than the
    product."""
    return build(force=force, extra_flags=["-DSWE_DEBUG_BOUNDS"], variant="debug")


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
