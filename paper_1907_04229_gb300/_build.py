"""Compile the CUDA sources of this package for sm_103a (in-tree build): libcptr.so, and the
bounds-checking variant libcptr_check.so (-DCPTR_CHECK: every index a hot-path kernel reads from a
table is checked against its array; a failure is recorded, the access skipped, and the call
returns CPTR_ECHECK)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcptr.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-Xptxas", "-O3"]


VARIANTS = {"": (LIB, BUILD, []), "check": (os.path.join(HERE, "libcptr_check.so"), os.path.join(BUILD, "check"),
                                            ["-DCPTR_CHECK"])}


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = glob.glob(os.path.join(CSRC, "*")) + [os.path.join(HERE, "..", "include", "cptr.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, variant: str = "") -> str:
    lib, bdir, defs = VARIANTS[variant]
    if not force and not _stale(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    objs = [os.path.join(bdir, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def compile_one(pair):
        s, o = pair
        # the model assembly rounds every product and sum on its own (no fused multiply-add)
        extra = ["-fmad=false"] if os.path.basename(s) == "model.cu" else []
        cmd = [NVCC, *ARCH, *FLAGS, *defs, *extra, "-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(s)}:\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if verbose:
        for l in logs:
            if l.strip():
                print(l)
    tmp = lib + ".tmp"
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lpthread"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib
