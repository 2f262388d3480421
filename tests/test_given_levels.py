"""Counting with levels supplied by the caller (tc_count_with_levels).

The count is exact for any labelling in which the ends of every edge differ
by at most one level; the expected values come from the oracle alone: T is
the plain definition on the whole graph, t_same the plain definition on the
subgraph of horizontal edges (both ends on one level), |E0| the number of
horizontal edges.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
scipy_sparse = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import paper_2309_09064_gb300 as tc
    return tc


@pytest.fixture(scope="module")
def ctx(tc):
    c = tc.tc_create(0)
    yield c
    tc.tc_destroy(c)


GRAPHS = {
    "rmat10": gg.rmat(10, 16, seed=1),
    "er4096": gg.er(4096, 60000, seed=2),
    "grid33x47": gg.grid(33, 47, 0.3, 4)[:3],
    "union": gg.disjoint_union([gg.rmat(7, 8, seed=3), gg.cycle(9), gg.complete(6), gg.wheel(6),
                                (3, np.zeros(0, np.uint32), np.zeros(0, np.uint32))]),
    "chung_lu4096": gg.chung_lu(4096, 2.1, 32.0, seed=3),
}


def expected(rp, col, L):
    """T, t_same, |E0| for levels L from the oracle's plain definition."""
    n = len(rp) - 1
    src = np.repeat(np.arange(n, dtype=np.uint32), np.diff(rp).astype(np.int64))
    horiz = L[src] == L[col]
    T = oracle.count_definition(rp, col)
    hrp, hcol = oracle.build_csr(n, src[horiz], col[horiz])
    return T, oracle.count_definition(hrp, hcol), int(horiz.sum()) // 2


def bfs_levels_from(rp, col, roots):
    """Hop distances from the given roots (one per component); unreached vertices get 0."""
    n = len(rp) - 1
    A = scipy_sparse.csr_matrix((np.ones(len(col)), col.astype(np.int64), rp.astype(np.int64)), shape=(n, n))
    dist = csgraph.shortest_path(A, unweighted=True, directed=False, indices=roots)
    dist = np.atleast_2d(dist).min(axis=0)
    dist[~np.isfinite(dist)] = 0
    return dist.astype(np.uint32)


def run(tc, ctx, graph, L):
    n, s, d = graph
    g = tc.tc_build_csr(ctx, n, s, d)
    try:
        Ld = torch.from_numpy(L.astype(np.uint32).view(np.int32)).cuda()
        return tc.tc_count_with_levels(ctx, g, Ld)
    finally:
        tc.tc_graph_free(g)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_other_bfs_roots(tc, ctx, name):
    n, s, d = GRAPHS[name]
    rp, col = oracle.build_csr(n, s, d)
    labels = csgraph.connected_components(
        scipy_sparse.csr_matrix((np.ones(len(col)), col.astype(np.int64), rp.astype(np.int64)), shape=(n, n)),
        directed=False)[1]
    rng = np.random.default_rng(7)
    roots = [int(rng.choice(np.flatnonzero(labels == c))) for c in np.unique(labels)]
    L = bfs_levels_from(rp, col, roots)
    T, st = run(tc, ctx, GRAPHS[name], L)
    eT, esame, eE0 = expected(rp, col, L)
    assert T == eT == st["triangles"]
    assert (st["t_same"], st["t_cross"]) == (esame, eT - esame)
    assert st["horizontal_edges"] == eE0
    assert st["levels"] == (int(L.max()) + 1 if n else 0)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_all_on_one_level(tc, ctx, name):
    """Every edge horizontal: all triangles are counted inside G0."""
    n, s, d = GRAPHS[name]
    rp, col = oracle.build_csr(n, s, d)
    T, st = run(tc, ctx, GRAPHS[name], np.zeros(n, np.uint32))
    assert T == oracle.count_definition(rp, col)
    assert (st["t_same"], st["t_cross"]) == (T, 0)
    assert st["horizontal_edges"] == len(col) // 2


@pytest.mark.parametrize("name", ["rmat10", "grid33x47"])
def test_own_levels_round_trip(tc, ctx, name):
    """The levels tc_count_levels returns give the same count and split."""
    n, s, d = GRAPHS[name]
    g = tc.tc_build_csr(ctx, n, s, d)
    try:
        L = torch.zeros(n, dtype=torch.int32, device="cuda")
        T0, st0 = tc.tc_count_levels(ctx, g, L)
        T1, st1 = tc.tc_count_with_levels(ctx, g, L)
    finally:
        tc.tc_graph_free(g)
    assert T0 == T1
    for k in ("t_same", "t_cross", "horizontal_edges", "levels"):
        assert st0[k] == st1[k]


def test_levels_two_apart_are_rejected(tc, ctx):
    n, s, d = GRAPHS["rmat10"]
    rp, col = oracle.build_csr(n, s, d)
    L = bfs_levels_from(rp, col, [0])
    x = int(np.argmax(np.diff(rp)))  # a vertex with neighbours, now two levels above all of them
    L[x] = L.max() + 2
    with pytest.raises(tc.TcError):
        run(tc, ctx, GRAPHS["rmat10"], L)
    # the context stays usable
    T, _ = run(tc, ctx, GRAPHS["rmat10"], np.zeros(n, np.uint32))
    assert T == oracle.count_definition(rp, col)
