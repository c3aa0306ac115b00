"""Build libftgemm.so for sm_103a with nvcc (one object per translation unit,
compiled in parallel, then linked).  The library lands in
``paper_2305_01024_gb300/_build/libftgemm.so`` (git-ignored)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libftgemm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xcompiler", "-Wall"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(HERE, "..", "include", "*.h")))


def _digest(path: str, extra: list[str]) -> str:
    h = hashlib.sha256()
    for p in [path] + extra:
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()[:16]


def build(verbose: bool = False, jobs: int | None = None, ptxas_info: bool = False) -> str:
    """Compile every csrc/*.cu and link libftgemm.so; skip objects whose
    sources and headers are unchanged."""
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = _sources()
    heads = _headers()
    cc = nvcc()
    jobs = jobs or max(1, min(len(srcs), os.cpu_count() or 4))

    def compile_one(src):
        base = os.path.splitext(os.path.basename(src))[0]
        dig = _digest(src, heads)
        obj = os.path.join(OUT_DIR, f"{base}.{dig}.o")
        if os.path.exists(obj) and not ptxas_info:
            return obj, ""
        cmd = [cc] + ARCH + NVCC_FLAGS + ["-c", src, "-o", obj + ".tmp"]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(compile_one, srcs))
    objs = [o for o, _ in results]
    if verbose or ptxas_info:
        for _, log in results:
            if log:
                sys.stdout.write(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    # drop stale objects of earlier source versions
    keep = set(objs)
    for o in glob.glob(os.path.join(OUT_DIR, "*.o")):
        if o not in keep:
            os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
