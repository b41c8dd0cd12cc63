"""Build libhf.so (the CUDA library behind include/hf.h) in-tree.

Regenerates the per-class recurrence header, compiles every translation
unit under csrc/ for sm_103a in parallel with nvcc and links them with
cuBLAS and cuSOLVER.  Objects go to ``_build/`` next to this file; the
library to ``libhf.so`` in this package directory.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# heaviest first, so the long compiles start early
SOURCES = ["rys_thread.cu", "eri_d6.cu", "eri_d5.cu", "eri_d4.cu", "eri_d3.cu", "eri_d2.cu", "eri_d1.cu", "eri_sp.cu",
           "rys.cu", "grad.cu", "api.cu", "basis.cu", "onee.cu", "scf.cu", "batch.cu", "serve.cu", "noalloc.cu", "multi.cu",
           "mp2.cu"]
KERNEL_HEADERS = ["eri.cuh", "eri_classes.cuh", "hf_device.h", "rys.cuh", "df64.cuh"]
HEADERS = KERNEL_HEADERS + ["hf_internal.h", "scf_internal.h", "multi.h", "../../include/hf.h"]
LMAX = 2


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, *extra]


def _stamp(src, flags):
    h = hashlib.sha256()
    h.update(" ".join(flags).encode())
    deps = KERNEL_HEADERS if os.path.basename(src).startswith("eri_") else HEADERS
    for f in [src] + [os.path.join(CSRC, x) for x in deps]:
        if os.path.exists(f):
            with open(f, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


def _compile(src, flags, verbose, out_dir=OUT):
    path = os.path.join(CSRC, src)
    obj = os.path.join(out_dir, src.replace(".cu", ".o"))
    stamp_file = obj + ".stamp"
    st = _stamp(path, flags)
    if os.path.exists(obj) and os.path.exists(stamp_file) and open(stamp_file).read() == st:
        return obj, False
    cmd = [_nvcc(), *flags, "-c", path, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    with open(stamp_file, "w") as fh:
        fh.write(st)
    return obj, True


def build(verbose: bool = False, jobs: int | None = None, extra_flags=(), out_dir: str = OUT,
          lib: str = LIB) -> str:
    os.makedirs(out_dir, exist_ok=True)
    subprocess.run([sys.executable, os.path.join(CSRC, "gen_eri.py"),
                    os.path.join(CSRC, "eri_classes.cuh"), str(LMAX)], check=True)
    flags = _flags(extra_flags)
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    jobs = jobs or min(len(srcs), max(2, os.cpu_count() or 2))
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, flags, verbose, out_dir), srcs))
    objs = [o for o, _ in results]
    rebuilt = any(r for _, r in results) or not os.path.exists(lib)
    if rebuilt:
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcublas", "-lcusolver"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


def build_bounds_checked(verbose: bool = False) -> str:
    """The same library with -DHF_BOUNDS_CHECK (every index of the J/K
    kernels checked before use) as libhf_bcheck.so, objects in _build_bcheck/.
    Load it with HF_LIB=<path> for small test cases."""
    return build(verbose, extra_flags=("-DHF_BOUNDS_CHECK",), out_dir=os.path.join(HERE, "_build_bcheck"),
                 lib=os.path.join(HERE, "libhf_bcheck.so"))


if __name__ == "__main__":
    print(build(verbose=True))
