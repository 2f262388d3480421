"""In-tree build of libtc.so (nvcc, sm_103a only).

Each .cu file compiles to an object in parallel, then nvcc links the shared
library against the shared CUDA runtime (so device pointers and streams are
those of any other runtime user in the process, e.g. PyTorch).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libtc.so")

SOURCES = ["api.cu", "count.cu", "levels.cu", "rank.cu", "rows.cu", "isect.cu", "scan.cu", "csr.cu", "batch.cu", "serve.cu", "alg3.cu", "list.cu",
           "noalloc.cu", "graphs.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "tc.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    tmpdir = tempfile.mkdtemp(dir=LIBDIR, prefix="obj_")
    try:
        def compile_one(src):
            obj = os.path.join(tmpdir, src.replace(".cu", ".o"))
            cmd = [nvcc()] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
            if verbose and r.stderr.strip():
                print(r.stderr)
            return obj

        with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
            objs = list(ex.map(compile_one, SOURCES))
        home = os.path.dirname(os.path.dirname(nvcc()))
        libdir = os.path.join(home, "lib64")
        fd, tmp_lib = tempfile.mkstemp(suffix=".so", dir=LIBDIR)
        os.close(fd)
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp_lib] + objs + \
              ["-Xlinker", "-rpath," + libdir, "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
        os.replace(tmp_lib, LIB)
    finally:
        shutil.rmtree(tmpdir, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
