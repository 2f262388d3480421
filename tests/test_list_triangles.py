"""Triangle listing (tc_list_triangles) against the oracle's listing from the
definition: the same set of vertex triples, each exactly once, through every
intersection class (tiny, warp, block, hub), both table kinds and both
working orders; the capacity contract (too small: TC_ERR_CAPACITY with T)
and the degenerate graphs."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import paper_2309_09064_gb300 as tc
    return tc


GRAPHS = {
    "K40": gg.complete(40),
    "wheel101": gg.wheel(101),
    "rmat10": gg.rmat(10, 16, seed=1),
    "rmat12_ef32": gg.rmat(12, 32, seed=3),
    "er4096": gg.er(4096, 60000, seed=2),
    "grid33x47": gg.grid(33, 47, 0.3, 4)[:3],
    "union": gg.disjoint_union([gg.rmat(7, 8, seed=3), gg.cycle(9), gg.complete(6), gg.wheel(6),
                                (3, np.zeros(0, np.uint32), np.zeros(0, np.uint32))]),
    "chung_lu4096": gg.chung_lu(4096, 2.1, 32.0, seed=3),
}
TUNINGS = {
    "default": {},
    "warp_block_hub": {"warp_cap": 4, "block_cap": 32, "task_work": 100, "tiny_cap": 0},
    "all_hub": {"warp_cap": 1, "block_cap": 1, "task_work": 1, "tiny_cap": 0},
    "tiny64": {"tiny_cap": 64},
    "buckets": {"table_kind": 1, "warp_cap": 8, "block_cap": 64, "tiny_cap": 0},
    "split_block": {"warp_cap": 1, "block_cap": 13107, "task_work": 256, "tiny_cap": 0, "block_bits_log2": 10},
    "flat_all": {"flat_cap": 4096, "tiny_cap": 0},
}
SENTINEL = 0x7EADBEEF


def canonical(triples):
    """Rows sorted within, then the rows in lexicographic order."""
    t = np.sort(np.asarray(triples, dtype=np.uint32).reshape(-1, 3), axis=1)
    return t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))]


def list_on_gpu(tc, c, graph, capacity=None):
    n, s, d = graph
    g = tc.tc_build_csr(c, n, s, d)
    try:
        if capacity is None:
            T0, _ = tc.tc_count(c, g)
            capacity = T0 + 5  # room to spare: rows past T are scratch
        out = torch.full((3 * max(capacity, 1),), SENTINEL, dtype=torch.int32, device="cuda")
        T, st = tc.tc_list_triangles(c, g, out if capacity else None, capacity)
    finally:
        tc.tc_graph_free(g)
    return T, st, out.cpu().numpy().view(np.uint32)


def check_listing(T, got, rp, col):
    want = oracle.list_definition(rp, col)
    assert T == len(want) == oracle.count_definition(rp, col)
    assert np.array_equal(canonical(got[:3 * T]), want)


@pytest.mark.parametrize("tuning", sorted(TUNINGS))
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_listing(tc, name, tuning):
    n, s, d = GRAPHS[name]
    rp, col = oracle.build_csr(n, s, d)
    c = tc.tc_create(0)
    try:
        if TUNINGS[tuning]:
            tc.tc_set_tuning(c, **TUNINGS[tuning])
        T, st, got = list_on_gpu(tc, c, GRAPHS[name])
    finally:
        tc.tc_destroy(c)
    check_listing(T, got, rp, col)
    assert st["triangles"] == T == st["t_same"] + st["t_cross"]


@pytest.mark.parametrize("name", ["rmat10", "union", "chung_lu4096"])
def test_listing_id_order(tc, name):
    n, s, d = GRAPHS[name]
    rp, col = oracle.build_csr(n, s, d)
    c = tc.tc_create(0, order=tc.TC_ORDER_ID)
    try:
        T, st, got = list_on_gpu(tc, c, GRAPHS[name])
    finally:
        tc.tc_destroy(c)
    check_listing(T, got, rp, col)


def test_listing_rows_follow_the_method(tc):
    """Every row {u, v, w}: u -> v is an edge on one level (Algorithm 4 intersects across horizontal edges
    only) and w is adjacent to both."""
    n, s, d = GRAPHS["rmat12_ef32"]
    rp, col = oracle.build_csr(n, s, d)
    c = tc.tc_create(0)
    try:
        g = tc.tc_build_csr(c, n, s, d)
        L = torch.zeros(n, dtype=torch.int32, device="cuda")
        T, _ = tc.tc_count_levels(c, g, L)
        out = torch.zeros(3 * T, dtype=torch.int32, device="cuda")
        T2, _ = tc.tc_list_triangles(c, g, out, T)
        tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(c)
    assert T2 == T
    rows = out.cpu().numpy().view(np.uint32).reshape(-1, 3).astype(np.int64)
    lv = L.cpu().numpy()
    assert np.all(lv[rows[:, 0]] == lv[rows[:, 1]])
    adj = set(zip(np.repeat(np.arange(n), np.diff(rp).astype(np.int64)).tolist(), col.tolist()))
    for u, v, w in rows[:: max(1, len(rows) // 5000)]:
        assert (u, v) in adj and (u, w) in adj and (v, w) in adj


def test_capacity_too_small(tc):
    n, s, d = GRAPHS["rmat10"]
    rp, col = oracle.build_csr(n, s, d)
    T_want = oracle.count_definition(rp, col)
    c = tc.tc_create(0)
    try:
        g = tc.tc_build_csr(c, n, s, d)
        out = torch.full((3 * (T_want - 1),), SENTINEL, dtype=torch.int32, device="cuda")
        with pytest.raises(tc.TcError) as e:
            tc.tc_list_triangles(c, g, out, T_want - 1)
        assert e.value.status == tc.TC_ERR_CAPACITY and e.value.triangles == T_want
        with pytest.raises(tc.TcError) as e:
            tc.tc_list_triangles(c, g, None, 0)
        assert e.value.triangles == T_want
        # exactly T fits; the context stays usable, and a plain count after it agrees
        out = torch.zeros(3 * T_want, dtype=torch.int32, device="cuda")
        T, _ = tc.tc_list_triangles(c, g, out, T_want)
        assert T == T_want
        assert np.array_equal(canonical(out.cpu().numpy().view(np.uint32)), oracle.list_definition(rp, col))
        assert tc.tc_count(c, g)[0] == T_want
        tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(c)


@pytest.mark.parametrize("graph", [
    (0, np.zeros(0, np.uint32), np.zeros(0, np.uint32)),
    (5, np.zeros(0, np.uint32), np.zeros(0, np.uint32)),
    gg.cycle(1000),
    gg.complete_bipartite(20, 30),
])
def test_no_triangles(tc, graph):
    c = tc.tc_create(0)
    try:
        n, s, d = graph
        g = tc.tc_build_csr(c, n, s, d)
        T, st = tc.tc_list_triangles(c, g, None, 0)
        tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(c)
    assert T == 0 and st["triangles"] == 0


def test_listing_larger_rmat(tc):
    """R-MAT scale 15 (about 0.5 M edges, several million triangles): every task class at default
    tuning, element by element."""
    n, s, d = gg.rmat(15, 16, seed=11)
    rp, col = oracle.build_csr(n, s, d)
    c = tc.tc_create(0)
    try:
        T, st, got = list_on_gpu(tc, c, (n, s, d))
    finally:
        tc.tc_destroy(c)
    check_listing(T, got, rp, col)
