"""Build liber.so, the C-ABI CUDA library, in-tree for sm_103a (nvcc, no cmake).

Each translation unit is compiled in parallel; the shared object lands next to this
file.  Host code is plain C++17 so the same sources build on x86-64 and aarch64.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = ["er_grid.cu", "er_pcg.cu", "er_fp32.cu", "er_noalloc.cu", "er_batch.cu", "er_unet_kernels.cu",
       "er_surrogate.cu", "er_pairs.cu", "er_stack.cu", "er_mg.cu"]
LIB = os.path.join(HERE, "liber.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _compile(src: str, obj: str, extra: list[str]) -> str:
    cmd = [nvcc(), "-c", os.path.join(HERE, "csrc", src), "-o", obj, *ARCH, "-lineinfo", "-O3",
           "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
           "--expt-relaxed-constexpr", *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(verbose_ptxas: bool = False, force: bool = False) -> str:
    srcs = [os.path.join(HERE, "csrc", s) for s in SRC]
    hdrs = [os.path.join(HERE, "csrc", h) for h in ("er_internal.h", "er_common.cuh", "er_unet.h")] + [
        os.path.join(ROOT, "include", "er.h")]
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in srcs + hdrs + [__file__])
        if os.path.getmtime(LIB) >= newest and not verbose_ptxas:
            return LIB
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    objs = [os.path.join(bdir, s.replace(".cu", ".o")) for s in SRC]
    with cf.ThreadPoolExecutor(len(SRC)) as ex:
        logs = list(ex.map(lambda a: _compile(*a, extra), zip(SRC, objs)))
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lcudart", "-lpthread"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose_ptxas:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose_ptxas="-v" in sys.argv, force=True))
