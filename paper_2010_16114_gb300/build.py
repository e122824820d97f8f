"""Build libcoxgb.so (the C-ABI library: the Cox solver and the NMF) in-tree for sm_103a with nvcc."""
from __future__ import annotations

import hashlib
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libcoxgb.so")
SOURCES = ["api.cu", "setup.cu", "scans.cu", "gemm_tc.cu", "gemm_f4.cu", "gemv.cu", "path.cu", "active.cu", "nmf.cu"]
HEADERS = ["internal.h", "ptx.cuh", "nmf_gemm.cuh", "gemm_kernel.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing",
          f"-I{os.path.join(ROOT, 'include')}"]


def _digest(extra: list[str]) -> str:
    h = hashlib.sha256()
    for f in SOURCES + HEADERS:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    for hdr in ("coxgb.h", "nmfgb.h"):
        with open(os.path.join(ROOT, "include", hdr), "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + CFLAGS + extra).encode())
    return h.hexdigest()


def build(force: bool = False, extra_flags: list[str] | None = None, verbose: bool = False) -> str:
    """Compile every translation unit in parallel and link libcoxgb.so.

    Skips the work when the library is newer than a stamp of the sources."""
    extra = list(extra_flags or [])
    stamp = LIB + ".stamp"
    dig = _digest(extra)
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == dig:
                return LIB
    bdir = os.path.join(CSRC, "_build")
    os.makedirs(bdir, exist_ok=True)

    def compile_one(src: str) -> str:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = ["nvcc", *ARCH, *CFLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = ["nvcc", *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
