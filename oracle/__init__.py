"""CPU oracle for exact triangle counting (D. A. Bader, "Fast Triangle Counting").

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and never calls it; the
CUDA library never calls it either.

Everything runs in ``oracle.c`` (plain serial C, built with gcc into
``_lib/liboracle.so``); this module only marshals numpy arrays.  See the
header of ``oracle.c`` for which passage of the paper each function follows
and for the readings taken where the paper is silent.

Pins (tests/test_oracle_pins.py) tie it to things other than itself: brute
force over all triples, trace(A^3)/6, closed forms (K_n, wheels, friendship
graphs, bipartite graphs, cycles, grids with diagonals), BFS-distance
characterisation of the levels, relabelling invariance and disjoint-union
additivity, and agreement of the four formulations (definition, Algorithm 3,
Algorithm 4 in both vertex orders).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")

UNVISITED = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile oracle.c (serial, -O2) into ``_lib/liboracle.so``."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_LIBDIR, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_LIBDIR)
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp],
                   check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_build_csr.argtypes = [ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p, _u64p, _u32p]
            lib.oracle_build_csr.restype = ctypes.c_int64
            lib.oracle_count_definition.argtypes = [ctypes.c_uint32, _u64p, _u32p]
            lib.oracle_count_definition.restype = ctypes.c_uint64
            lib.oracle_vertex_counts.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u64p]
            lib.oracle_vertex_counts.restype = ctypes.c_uint64
            lib.oracle_alg4.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int, _u32p, _u64p]
            lib.oracle_alg4.restype = ctypes.c_int
            lib.oracle_list_definition.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u32p, ctypes.c_uint64]
            lib.oracle_list_definition.restype = ctypes.c_uint64
            lib.oracle_alg3.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_int]
            lib.oracle_alg3.restype = ctypes.c_uint64
            _lib = lib
    return _lib


def _csr_args(row_ptr, col):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    col = np.ascontiguousarray(col, dtype=np.uint32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.uint32)
    return len(row_ptr) - 1, row_ptr, col


def build_csr(n: int, src, dst):
    """Tuples -> (row_ptr uint64[n+1], col uint32[2m]): symmetric, loop-free, de-duplicated, rows ascending."""
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    t = len(src)
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    col = np.zeros(max(2 * t, 1), dtype=np.uint32)
    s = src if t else np.zeros(1, np.uint32)
    d = dst if t else np.zeros(1, np.uint32)
    k = _load().oracle_build_csr(n, t, s, d, row_ptr, col)
    if k < 0:
        raise ValueError("tuple names a vertex id >= n")
    return row_ptr, col[:k].copy()


def count_definition(row_ptr, col) -> int:
    """T from the definition (pairwise adjacent triples, each counted once)."""
    n, rp, c = _csr_args(row_ptr, col)
    return int(_load().oracle_count_definition(n, rp, c))


def vertex_counts(row_ptr, col):
    """(T, t[v]) with t[v] the number of triangles containing v."""
    n, rp, c = _csr_args(row_ptr, col)
    tv = np.zeros(max(n, 1), dtype=np.uint64)
    T = int(_load().oracle_vertex_counts(n, rp, c, tv))
    return T, tv[:n]


def list_definition(row_ptr, col):
    """Every triangle once: uint32 array (T, 3) of id triples a < b < c, rows in lexicographic order."""
    n, rp, c = _csr_args(row_ptr, col)
    lib = _load()
    T = int(lib.oracle_list_definition(n, rp, c, np.zeros(3, np.uint32), 0))
    out = np.zeros(3 * max(T, 1), dtype=np.uint32)
    lib.oracle_list_definition(n, rp, c, out, T)
    return out[:3 * T].reshape(T, 3)


def alg4(row_ptr, col, degree_order: bool = True) -> dict:
    """Algorithm 4 (BaderD when degree_order, else Bader): T, its two parts, |E0|, levels, L[]."""
    n, rp, c = _csr_args(row_ptr, col)
    L = np.zeros(max(n, 1), dtype=np.uint32)
    out = np.zeros(5, dtype=np.uint64)
    if _load().oracle_alg4(n, rp, c, int(degree_order), L, out) != 0:
        raise MemoryError("oracle_alg4: allocation failed")
    return {"T": int(out[0]), "T_same": int(out[1]), "T_cross": int(out[2]),
            "E0": int(out[3]), "levels": int(out[4]), "L": L[:n]}


def alg3(row_ptr, col, degree_order: bool = True) -> int:
    """Algorithm 3 (cover-edge rule) total."""
    n, rp, c = _csr_args(row_ptr, col)
    return int(_load().oracle_alg3(n, rp, c, int(degree_order)))
