"""Build the CUDA library in-tree: paper_2408_06880_gb300/_lib/libsparse_lbm.so.

One nvcc per translation unit, compiled in parallel, for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``), then linked with a static CUDA
runtime.  Rebuilds only what changed (sources, headers or flags)."""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libsparse_lbm.so")

SOURCES = ["api.cu", "lists.cu", "aa_dispatch.cu", "aa_q19_f32.cu", "aa_q19_f16.cu", "aa_q19_bf16.cu",
           "aa_q27_f32.cu", "aa_q27_f16.cu", "aa_q27_bf16.cu", "macro.cu", "dense.cu", "pool.cu", "pull.cu",
           "convert.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: every multiply and add is rounded separately, in program order,
# so all kernel instantiations (launch shapes, batched or not) produce the same
# bits for the same cell.  The kernels are memory-bound; the unfused FP work
# does not show.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _digest(extra: list[str]) -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "sparse_lbm.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + FLAGS + extra).encode())
    return h.hexdigest()


def build(verbose: bool = False, ptxas_v: bool = False, jobs: int | None = None) -> str:
    """Compile and link if anything changed; return the library path."""
    extra = ["-Xptxas", "-v"] if ptxas_v else []
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest(extra)
    if os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig and not ptxas_v:
        return LIB
    nvcc = _nvcc()

    def compile_one(src: str):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_v:
        for obj, log in results:
            if log.strip():
                print(f"== {os.path.basename(obj)}\n{log}", file=sys.stderr)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_v="-v" in sys.argv))
