"""Seeded synthetic graph inputs, shared by the CPU oracle and the CUDA library.

Every function returns raw edge tuples ``(n, src, dst)`` as numpy ``uint32``
arrays.  Nothing here builds a CSR or counts anything: symmetrising, dropping
self-loops, removing duplicates and sorting rows is left to the consumer, so
the oracle and the CUDA path each do it with their own code.

The large families (R-MAT, Erdos-Renyi, Chung-Lu, grid with diagonals) are in
``graphgen.c`` (counter-based SplitMix64 draws, OpenMP loops whose output does
not depend on the thread count).  The small closed-form families used to pin
the oracle (complete, wheel, bipartite, cycle, Petersen, friendship, ...) are
plain numpy below.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

U32 = np.uint32
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile graphgen.c into ``_lib/libgraphgen.so`` (OpenMP when gcc has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_LIBDIR, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_LIBDIR)
    os.close(fd)
    base = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:3] + ["-fopenmp"] + base[3:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.gg_permutation.argtypes = [ctypes.c_uint32, ctypes.c_uint64, _u32p]
            lib.gg_permutation.restype = None
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, _u32p, _u32p]
            lib.gg_rmat.restype = None
            lib.gg_er.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, _u32p, _u32p]
            lib.gg_er.restype = ctypes.c_uint64
            lib.gg_chung_lu.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.c_int, _u32p, _u32p, _f64p]
            lib.gg_chung_lu.restype = None
            lib.gg_grid.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64,
                                    _u32p, _u32p, ctypes.POINTER(ctypes.c_uint64)]
            lib.gg_grid.restype = ctypes.c_uint64
            lib.gg_draws.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, _u64p]
            lib.gg_draws.restype = None
            _lib = lib
    return _lib


# ----------------------------------------------------------------------------- large families

def draws(seed: int, stream: int, first: int, count: int) -> np.ndarray:
    """Raw counter-based SplitMix64 draws (for testing the generator itself)."""
    out = np.empty(count, dtype=np.uint64)
    _load().gg_draws(seed, stream, first, count, out)
    return out


def permutation(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=U32)
    _load().gg_permutation(n, seed, out)
    return out


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True):
    """R-MAT with ``edge_factor * 2**scale`` tuples (Graph500-style parameters by default)."""
    n = 1 << scale
    t = edge_factor * n
    src = np.empty(t, dtype=U32)
    dst = np.empty(t, dtype=U32)
    q = lambda x: min(int(x * 4294967296.0), 0xFFFFFFFF)
    _load().gg_rmat(scale, t, q(a), q(a + b), q(a + b + c), seed, int(permute), src, dst)
    return n, src, dst


def er(n: int, m: int, seed: int):
    """Erdos-Renyi G(n, m): exactly m distinct loop-free undirected pairs."""
    m = min(m, n * (n - 1) // 2)
    src = np.empty(m, dtype=U32)
    dst = np.empty(m, dtype=U32)
    k = _load().gg_er(n, m, seed, src, dst)
    return n, src[:k], dst[:k]


def chung_lu(n: int, gamma: float = 2.1, mean_deg: float = 32.0, n_tuples: int | None = None,
             seed: int = 3, permute: bool = True):
    """Chung-Lu power-law tuples; ``n_tuples`` defaults to mean_deg * n / 2."""
    if n_tuples is None:
        n_tuples = int(mean_deg * n / 2)
    src = np.empty(n_tuples, dtype=U32)
    dst = np.empty(n_tuples, dtype=U32)
    stats = np.zeros(2, dtype=np.float64)
    _load().gg_chung_lu(n, gamma, mean_deg, n_tuples, seed, int(permute), src, dst, stats)
    return n, src, dst


def grid(rows: int, cols: int, p: float = 0.3, seed: int = 4):
    """Grid with random diagonals; returns ``(n, src, dst, n_diagonals)``.

    With at most one diagonal per cell every triangle lies inside one cell and
    each diagonal closes exactly two, so the triangle count is 2 * n_diagonals.
    """
    cap = rows * (cols - 1) + (rows - 1) * cols + (rows - 1) * (cols - 1)
    src = np.empty(max(cap, 1), dtype=U32)
    dst = np.empty(max(cap, 1), dtype=U32)
    nd = ctypes.c_uint64(0)
    k = _load().gg_grid(rows, cols, p, seed, src, dst, ctypes.byref(nd))
    return rows * cols, src[:k], dst[:k], int(nd.value)


# ----------------------------------------------------------------------------- small closed-form families

def _pairs(n, pairs):
    if len(pairs) == 0:
        return n, np.zeros(0, U32), np.zeros(0, U32)
    arr = np.asarray(pairs, dtype=np.int64)
    return n, arr[:, 0].astype(U32), arr[:, 1].astype(U32)


def complete(n: int):
    """K_n: C(n, 3) triangles."""
    iu = np.triu_indices(n, 1)
    return n, iu[0].astype(U32), iu[1].astype(U32)


def wheel(rim: int):
    """Hub 0 joined to a cycle 1..rim.  rim >= 4 gives rim triangles; rim = 3 is K_4 (4)."""
    pairs = [(0, i) for i in range(1, rim + 1)]
    pairs += [(i, i % rim + 1) for i in range(1, rim + 1)]
    return _pairs(rim + 1, pairs)


def complete_bipartite(a: int, b: int):
    """K_{a,b}: bipartite, 0 triangles."""
    pairs = [(i, a + j) for i in range(a) for j in range(b)]
    return _pairs(a + b, pairs)


def cycle(n: int):
    """C_n: 0 triangles for n >= 4, 1 for n = 3."""
    return _pairs(n, [(i, (i + 1) % n) for i in range(n)])


def path(n: int):
    return _pairs(n, [(i, i + 1) for i in range(n - 1)])


def star(leaves: int):
    return _pairs(leaves + 1, [(0, i) for i in range(1, leaves + 1)])


def petersen():
    """Petersen graph: outer 5-cycle, inner pentagram, five spokes; girth 5, 0 triangles."""
    pairs = [(i, (i + 1) % 5) for i in range(5)]
    pairs += [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    pairs += [(i, 5 + i) for i in range(5)]
    return _pairs(10, pairs)


def friendship(k: int):
    """Friendship (windmill) graph F_k: k triangles sharing vertex 0."""
    pairs = []
    for i in range(k):
        a, b = 1 + 2 * i, 2 + 2 * i
        pairs += [(0, a), (0, b), (a, b)]
    return _pairs(2 * k + 1, pairs)


def grid_plain(rows: int, cols: int):
    """Grid without diagonals: bipartite, 0 triangles."""
    return grid(rows, cols, p=0.0, seed=0)[:3]


def random_tree(n: int, seed: int):
    """Random recursive tree: vertex i > 0 attaches to a uniform earlier vertex (0 triangles)."""
    if n <= 1:
        return n, np.zeros(0, U32), np.zeros(0, U32)
    r = draws(seed, 0x54524545, 0, n)
    parent = [int((int(r[i]) >> 32) * i >> 32) for i in range(1, n)]
    return _pairs(n, [(p, i) for p, i in zip(parent, range(1, n))])


def gnp(n: int, p: float, seed: int):
    """Small G(n, p) via one draw per unordered pair (for property tests)."""
    iu = np.triu_indices(n, 1)
    r = draws(seed, 0x474E5000, 0, len(iu[0]))
    keep = (r >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0) < p
    return n, iu[0][keep].astype(U32), iu[1][keep].astype(U32)


def disjoint_union(graphs):
    """Vertex-disjoint union of tuple graphs (ids shifted); triangle counts add."""
    n0 = 0
    srcs, dsts = [], []
    for n, s, d in graphs:
        srcs.append(s.astype(np.int64) + n0)
        dsts.append(d.astype(np.int64) + n0)
        n0 += n
    if not srcs:
        return 0, np.zeros(0, U32), np.zeros(0, U32)
    return n0, np.concatenate(srcs).astype(U32), np.concatenate(dsts).astype(U32)


def relabel(graph, perm):
    """Apply vertex permutation ``perm`` (old id -> new id); triangle count unchanged."""
    n, s, d = graph
    perm = np.asarray(perm, dtype=U32)
    return n, perm[s], perm[d]


def with_noise(graph, seed: int, dup_frac: float = 0.2, loop_frac: float = 0.05, flip: bool = True):
    """Add duplicate tuples, self-loops and reversed copies (they must not change the graph)."""
    n, s, d = graph
    t = len(s)
    if t == 0 or n == 0:
        return graph
    r = draws(seed, 0x4E4F4953, 0, 3 * t + 3)
    nd = int(dup_frac * t)
    nl = int(loop_frac * n) + 1
    idx = ((r[:nd] >> np.uint64(32)) * np.uint64(t) >> np.uint64(32)).astype(np.int64)
    loops = ((r[t:t + nl] >> np.uint64(32)) * np.uint64(n) >> np.uint64(32)).astype(U32)
    ds, dd = s[idx], d[idx]
    if flip:
        ds, dd = dd, ds
    return n, np.concatenate([s, ds, loops]).astype(U32), np.concatenate([d, dd, loops]).astype(U32)


# ----------------------------------------------------------------------------- named workloads

@dataclass(frozen=True)
class Spec:
    """One synthetic graph: family plus parameters; ``make()`` returns its tuples."""
    kind: str          # "rmat" | "er" | "chung_lu" | "grid"
    n: int
    param: float       # rmat: edge factor; er: mean degree; chung_lu: mean degree; grid: p
    seed: int

    def make(self):
        if self.kind == "rmat":
            return rmat(int(round(math.log2(self.n))), int(self.param), seed=self.seed)
        if self.kind == "er":
            return er(self.n, int(self.param * self.n / 2), self.seed)
        if self.kind == "chung_lu":
            return chung_lu(self.n, 2.1, self.param, seed=self.seed)
        if self.kind == "grid":
            side = int(round(math.sqrt(self.n)))
            return grid(side, side, self.param, self.seed)[:3]
        raise ValueError(self.kind)


def batch_specs(count: int, seed: int = 5, n_lo: int = 64, n_hi: int = 65536):
    """The mixed batch: n log-uniform in [n_lo, n_hi]; R-MAT (scale floor(log2 n),
    edge factor uniform in [8, 32]) or Erdos-Renyi (mean degree uniform in [4, 64])
    by a fair coin; per-graph seeds derived from ``seed``."""
    r = draws(seed, 0x42415443, 0, 4 * count)
    unit = lambda x: float(int(x) >> 11) * (1.0 / 9007199254740992.0)
    specs = []
    for i in range(count):
        u = unit(r[4 * i])
        n = int(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo))))
        n = max(n_lo, min(n_hi, n))
        coin = unit(r[4 * i + 1]) < 0.5
        gseed = int(r[4 * i + 3] >> np.uint64(1)) | 1
        if coin:
            scale = int(math.floor(math.log2(n)))
            ef = 8 + int(unit(r[4 * i + 2]) * 25)
            specs.append(Spec("rmat", 1 << scale, ef, gseed))
        else:
            d = 4.0 + unit(r[4 * i + 2]) * 60.0
            specs.append(Spec("er", n, d, gseed))
    return specs
