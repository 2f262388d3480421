"""Pins of the CPU oracle to things other than itself (no GPU).

Every check compares the oracle with an independent source of truth:
brute force over all vertex triples, trace(A^3)/6 from an integer dense
matrix product, closed forms of graph families, BFS distances from a library
routine (scipy.sparse.csgraph), hand-worked fixtures in tests/golden/, and
invariants (relabelling, disjoint unions).  A dropped term, a flipped
comparison or a wrong index in any oracle function fails at least one test
here.
"""
import itertools
import math
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

scipy_sparse = pytest.importorskip("scipy.sparse")
from scipy.sparse import csgraph  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr_of(graph):
    n, s, d = graph[:3]
    return oracle.build_csr(n, s, d)


def dense(rp, col):
    n = len(rp) - 1
    A = np.zeros((n, n), dtype=np.int64)
    for v in range(n):
        A[v, col[rp[v]:rp[v + 1]]] = 1
    return A


def brute_triangles(A):
    """All triples i < j < k with the three adjacencies (vectorised over k)."""
    n = A.shape[0]
    t = 0
    for i in range(n):
        for j in range(i + 1, n):
            if A[i, j]:
                t += int(np.sum(A[i, j + 1:] & A[j, j + 1:]))
    return t


def brute_triangle_list(A):
    n = A.shape[0]
    out = []
    for i, j, k in itertools.combinations(range(n), 3):
        if A[i, j] and A[j, k] and A[i, k]:
            out.append((i, j, k))
    return out


def all_counts(rp, col):
    r4d = oracle.alg4(rp, col, True)
    r4 = oracle.alg4(rp, col, False)
    return {
        "definition": oracle.count_definition(rp, col),
        "alg4_degree": r4d["T"],
        "alg4_id": r4["T"],
        "alg3_degree": oracle.alg3(rp, col, True),
        "alg3_id": oracle.alg3(rp, col, False),
        "vertex_sum": int(oracle.vertex_counts(rp, col)[1].sum()) // 3,
    }


# --------------------------------------------------------------------- CSR construction

def test_build_csr_matches_set_construction():
    n, s, d = gg.with_noise(gg.gnp(40, 0.2, 11), seed=3)
    rp, col = oracle.build_csr(n, s, d)
    pairs = {(int(a), int(b)) for a, b in zip(s, d) if a != b}
    pairs |= {(b, a) for a, b in pairs}
    for v in range(n):
        assert list(col[rp[v]:rp[v + 1]]) == sorted(b for a, b in pairs if a == v)
    assert rp[-1] == len(pairs)


def test_build_csr_noise_invariant_and_rejects_bad_ids():
    g = gg.rmat(8, 8, seed=9)
    rp0, c0 = csr_of(g)
    rp1, c1 = csr_of(gg.with_noise(g, seed=5))
    assert np.array_equal(rp0, rp1) and np.array_equal(c0, c1)
    with pytest.raises(ValueError):
        oracle.build_csr(4, np.array([0, 1], np.uint32), np.array([1, 4], np.uint32))


def test_build_csr_empty_and_isolated():
    rp, col = oracle.build_csr(5, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    assert list(rp) == [0] * 6 and len(col) == 0
    r = oracle.alg4(rp, col)
    assert r["T"] == 0 and r["E0"] == 0 and list(r["L"]) == [0] * 5 and r["levels"] == 1
    rp, col = oracle.build_csr(0, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    assert oracle.alg4(rp, col)["T"] == 0 and oracle.count_definition(rp, col) == 0


# --------------------------------------------------------------------- brute force / trace

@pytest.mark.parametrize("seed,n,p", [(1, 12, 0.5), (2, 30, 0.3), (3, 60, 0.15), (4, 90, 0.4), (5, 7, 1.0)])
def test_every_formulation_matches_brute_force(seed, n, p):
    rp, col = csr_of(gg.gnp(n, p, seed))
    A = dense(rp, col)
    bf = brute_triangles(A)
    for name, t in all_counts(rp, col).items():
        assert t == bf, name


def test_vertex_counts_match_brute_force():
    rp, col = csr_of(gg.gnp(25, 0.35, 8))
    A = dense(rp, col)
    tv = np.zeros(25, dtype=np.int64)
    for (i, j, k) in brute_triangle_list(A):
        tv[[i, j, k]] += 1
    T, got = oracle.vertex_counts(rp, col)
    assert T == len(brute_triangle_list(A))
    assert np.array_equal(got.astype(np.int64), tv)


@pytest.mark.parametrize("seed,n,p", [(8, 25, 0.35), (9, 40, 0.2), (10, 12, 1.0), (11, 6, 0.0)])
def test_triangle_list_matches_brute_force(seed, n, p):
    """The listing is exactly the set of adjacent triples, each once, in lexicographic order."""
    rp, col = csr_of(gg.gnp(n, p, seed))
    A = dense(rp, col)
    got = oracle.list_definition(rp, col)
    assert got.shape == (len(brute_triangle_list(A)), 3)
    assert [tuple(int(x) for x in r) for r in got] == brute_triangle_list(A)


@pytest.mark.parametrize("n", [0, 3, 7, 12])
def test_triangle_list_complete_graph(n):
    rp, col = csr_of(gg.complete(n))
    got = oracle.list_definition(rp, col)
    assert [tuple(int(x) for x in r) for r in got] == list(itertools.combinations(range(n), 3))


def test_triangle_list_agrees_with_the_counts_on_rmat():
    rp, col = csr_of(gg.rmat(10, 16, seed=1))
    got = oracle.list_definition(rp, col)
    T, tv = oracle.vertex_counts(rp, col)
    assert len(got) == T == oracle.count_definition(rp, col)
    assert np.array_equal(np.bincount(got.ravel(), minlength=len(rp) - 1).astype(np.uint64), tv)
    assert np.all((got[:, 0] < got[:, 1]) & (got[:, 1] < got[:, 2]))


@pytest.mark.parametrize("graph", ["rmat10", "rmat9_ef32", "er2048"])
def test_trace_a_cubed(graph):
    if graph == "rmat10":
        g = gg.rmat(10, 16, seed=1)
    elif graph == "rmat9_ef32":
        g = gg.rmat(9, 32, seed=7)
    else:
        g = gg.er(2048, 30000, seed=2)
    rp, col = csr_of(g)
    A = dense(rp, col).astype(np.float64)
    # float64 products are exact here: entries of A^3 stay far below 2^53
    tr = int(round(np.trace(A @ A @ A)))
    assert tr % 6 == 0
    for name, t in all_counts(rp, col).items():
        assert t == tr // 6, name


# --------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 9, 17, 40])
def test_complete_graph(n):
    rp, col = csr_of(gg.complete(n))
    for name, t in all_counts(rp, col).items():
        assert t == math.comb(n, 3), name


@pytest.mark.parametrize("rim", [3, 4, 5, 10, 101])
def test_wheel(rim):
    rp, col = csr_of(gg.wheel(rim))
    want = 4 if rim == 3 else rim
    for name, t in all_counts(rp, col).items():
        assert t == want, name


@pytest.mark.parametrize("k", [1, 2, 7, 50])
def test_friendship(k):
    rp, col = csr_of(gg.friendship(k))
    for name, t in all_counts(rp, col).items():
        assert t == k, name


@pytest.mark.parametrize("graph", [
    gg.complete_bipartite(7, 9), gg.cycle(4), gg.cycle(11), gg.path(30), gg.star(40),
    gg.petersen(), gg.grid_plain(13, 17), gg.random_tree(200, 4)])
def test_triangle_free(graph):
    rp, col = csr_of(graph)
    for name, t in all_counts(rp, col).items():
        assert t == 0, name


def test_cycle3():
    rp, col = csr_of(gg.cycle(3))
    assert set(all_counts(rp, col).values()) == {1}


@pytest.mark.parametrize("rows,cols,p,seed", [(9, 11, 0.3, 4), (64, 48, 0.3, 1), (40, 40, 1.0, 2), (30, 2, 0.5, 3)])
def test_grid_with_diagonals(rows, cols, p, seed):
    n, s, d, ndiag = gg.grid(rows, cols, p, seed)
    rp, col = oracle.build_csr(n, s, d)
    for name, t in all_counts(rp, col).items():
        assert t == 2 * ndiag, name


# --------------------------------------------------------------------- BFS levels (Algorithm 4, BFS loop)

def _check_levels(rp, col, L, degree_order):
    """L must be the hop distance from each component's root, where the root is
    the component's first vertex in the working order."""
    n = len(rp) - 1
    deg = np.diff(rp).astype(np.int64)
    M = scipy_sparse.csr_matrix((np.ones(len(col)), col.astype(np.int64), rp.astype(np.int64)), shape=(n, n))
    ncomp, comp = csgraph.connected_components(M, directed=False)
    for c in range(ncomp):
        members = np.flatnonzero(comp == c)
        if degree_order:
            root = min(members, key=lambda v: (-deg[v], v))
        else:
            root = members.min()
        dist = csgraph.shortest_path(M, unweighted=True, indices=[root])[0]
        assert np.array_equal(L[members], dist[members].astype(np.uint32))


@pytest.mark.parametrize("degree_order", [True, False])
@pytest.mark.parametrize("graph", ["rmat10", "disjoint", "grid", "er"])
def test_levels_are_bfs_distances_from_canonical_roots(graph, degree_order):
    if graph == "rmat10":
        g = gg.rmat(10, 16, seed=1)
    elif graph == "disjoint":
        g = gg.disjoint_union([gg.rmat(7, 4, seed=3), gg.cycle(9), gg.star(5), gg.complete(1), gg.wheel(6),
                               gg.path(12)])
    elif graph == "grid":
        g = gg.grid(20, 30, 0.3, 4)[:3]
    else:
        g = gg.er(3000, 4000, 6)
    rp, col = csr_of(g)
    r = oracle.alg4(rp, col, degree_order)
    _check_levels(rp, col, r["L"], degree_order)
    # E0 recounted from the levels, and the number of levels
    src = np.repeat(np.arange(len(rp) - 1), np.diff(rp).astype(np.int64))
    assert r["E0"] * 2 == int(np.sum(r["L"][src] == r["L"][col]))
    assert r["levels"] == (int(r["L"].max()) + 1 if len(r["L"]) else 0)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_same_and_cross_split_matches_triangle_classification(seed):
    """T_same = triangles with all three vertices on one level; T_cross = the
    rest, each of which has exactly one horizontal edge (BFS levels differ by at
    most one along an edge)."""
    rp, col = csr_of(gg.disjoint_union([gg.gnp(45, 0.2, seed), gg.gnp(20, 0.5, seed + 10)]))
    A = dense(rp, col)
    for degree_order in (True, False):
        r = oracle.alg4(rp, col, degree_order)
        L = r["L"].astype(np.int64)
        same = cross = 0
        for (i, j, k) in brute_triangle_list(A):
            lv = [L[i], L[j], L[k]]
            assert max(lv) - min(lv) <= 1
            if lv[0] == lv[1] == lv[2]:
                same += 1
            else:
                horiz = (lv[0] == lv[1]) + (lv[1] == lv[2]) + (lv[0] == lv[2])
                assert horiz == 1
                cross += 1
        assert (r["T_same"], r["T_cross"]) == (same, cross)


# --------------------------------------------------------------------- invariants

def test_relabelling_invariance():
    g = gg.rmat(11, 16, seed=2)
    rp, col = csr_of(g)
    base = all_counts(rp, col)
    perm = gg.permutation(g[0], 77)
    rp2, col2 = csr_of(gg.relabel(g, perm))
    assert all_counts(rp2, col2) == base
    r1, r2 = oracle.alg4(rp, col, True), oracle.alg4(rp2, col2, True)
    # degree classes move with the vertices; the level histogram is invariant
    # unless a degree tie decides a root, so compare T parts only
    assert r1["T"] == r2["T"]


def test_disjoint_union_adds():
    parts = [gg.rmat(8, 16, seed=s) for s in (1, 2, 3)] + [gg.complete(12), gg.wheel(9)]
    tot = 0
    for p in parts:
        rp, col = csr_of(p)
        tot += oracle.count_definition(rp, col)
    rp, col = csr_of(gg.disjoint_union(parts))
    for name, t in all_counts(rp, col).items():
        assert t == tot, name


# --------------------------------------------------------------------- hand-worked fixtures

def _read_fixture(path):
    spec = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        spec[key] = vals
    n = int(spec["n"][0])
    pairs = [tuple(int(x) for x in e.split("-")) for e in spec["edges"]]
    return n, pairs, spec


@pytest.mark.parametrize("name", sorted(f for f in os.listdir(GOLDEN) if f.startswith("worked_")))
def test_hand_worked_fixture(name):
    n, pairs, spec = _read_fixture(os.path.join(GOLDEN, name))
    s = np.array([a for a, b in pairs], np.uint32)
    d = np.array([b for a, b in pairs], np.uint32)
    rp, col = oracle.build_csr(n, s, d)
    r = oracle.alg4(rp, col, spec["order"][0] == "degree")
    assert list(r["L"]) == [int(x) for x in spec["L"]]
    for key in ("E0", "levels", "T", "T_same", "T_cross"):
        assert r[key] == int(spec[key][0]), key
    assert oracle.count_definition(rp, col) == int(spec["T"][0])


# --------------------------------------------------------------------- generator sanity

def test_generators_are_deterministic_and_in_range():
    a = gg.rmat(12, 16, seed=1)
    b = gg.rmat(12, 16, seed=1)
    c = gg.rmat(12, 16, seed=2)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert not np.array_equal(a[1], c[1])
    assert a[1].max() < 4096 and a[2].max() < 4096
    n, s, d = gg.er(5000, 20000, 3)
    assert len(s) == 20000 and np.all(s < d)
    assert len(np.unique(s.astype(np.uint64) * 5000 + d)) == 20000
    p = gg.permutation(1000, 5)
    assert np.array_equal(np.sort(p), np.arange(1000))


def test_generator_draws_are_splitmix64():
    # Counter-based SplitMix64: draw i of a stream is the SplitMix64 mixing
    # function applied to key + (i + 1) * golden gamma.
    golden = 0x9E3779B97F4A7C15

    def mix(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        return z ^ (z >> 31)

    key = mix((1 * golden) ^ 0x524D4154 & 0xFFFFFFFFFFFFFFFF)
    want = [mix((key + (i + 1) * golden) & 0xFFFFFFFFFFFFFFFF) for i in range(4)]
    assert [int(x) for x in gg.draws(1, 0x524D4154, 0, 4)] == want
