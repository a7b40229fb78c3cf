"""Build libowqs.so in-tree for sm_103a (GB300).

Host C++ goes through g++, the kernels through nvcc with
-gencode arch=compute_103a,code=sm_103a; the objects are linked into one
shared library with the CUDA runtime linked statically, so the library has
no dependency beyond the CUDA driver (libcuda).  Objects go to _build/ next to this file.

build(bounds_check=True) makes the debug library libowqs_checked.so
(objects in _build_checked/): the kernels compiled with OWQS_BOUNDS_CHECK,
which checks every global access of the pass kernels against the extent of
its buffer and reports a failed check as an error of the run.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libowqs.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libowqs_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# owqs_group_seq.cu is compiled once per slice of the sequence table
# (kGroupSeqSlices in csrc/owqs_group_c64.cuh)
SEQ_SOURCE = "owqs_group_seq.cu"
SEQ_SLICES = 8


def cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found; set CUDA_HOME")


def sources():
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    return cpp, cu


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build step failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(verbose: bool = False, ptxas_info: bool = False, bounds_check: bool = False) -> str:
    cuda = cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    bdir, lib = (BUILD_CHECKED, LIB_CHECKED) if bounds_check else (BUILD, LIB)
    os.makedirs(bdir, exist_ok=True)
    cpp, cu = sources()
    inc = ["-I", INCLUDE, "-I", CSRC, "-I", os.path.join(cuda, "include")]
    defs = ["-DOWQS_BOUNDS_CHECK"] if bounds_check else []
    jobs = []
    for f in cpp:
        obj = os.path.join(bdir, f[:-4] + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function", *defs, *inc, "-c",
                     os.path.join(CSRC, f), "-o", obj])
    cu_objs = []
    for f in cu:
        extra = ["-Xptxas", "-v"] if ptxas_info else []
        # the sequence-specialised group kernels compile in SEQ_SLICES parallel parts
        variants = [(f"_{k}", [f"-DOWQS_SEQ_SLICE={k}"]) for k in range(SEQ_SLICES)] if f == SEQ_SOURCE else [("", [])]
        for suffix, vdefs in variants:
            obj = os.path.join(bdir, f[:-3] + suffix + ".o")
            cu_objs.append(obj)
            jobs.append([nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                         "--expt-relaxed-constexpr", *defs, *vdefs, *extra, *inc, "-c", os.path.join(CSRC, f),
                         "-o", obj])
    logs = []
    with cf.ThreadPoolExecutor(max_workers=min(max(4, os.cpu_count() or 4), len(jobs))) as ex:
        for out in ex.map(_run, jobs):
            logs.append(out)
    objs = [os.path.join(bdir, f[:-4] + ".o") for f in cpp] + cu_objs
    tmp = lib + ".tmp"
    logs.append(_run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]))
    os.replace(tmp, lib)
    text = "\n".join(x for x in logs if x.strip())
    if verbose and text:
        print(text)
    return text


def ensure_built(bounds_check: bool = False) -> str:
    """Build if the library is missing or older than a source file."""
    srcs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cpp", ".cu", ".h", ".cuh", ".inc"))]
    srcs.append(os.path.join(INCLUDE, "owqs.h"))
    lib = LIB_CHECKED if bounds_check else LIB
    if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(s) for s in srcs):
        build(bounds_check=bounds_check)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
