"""Triangles through every vertex (tc_count_vertices) against the oracle's
per-vertex counts, through every intersection class (tiny, warp, block,
hub) and both working orders; the counts sum to 3T."""
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
}


def vertex_count(tc, c, graph):
    n, s, d = graph
    g = tc.tc_build_csr(c, n, s, d)
    try:
        out = torch.full((max(n, 1),), -1, dtype=torch.int64, device="cuda")
        T, st = tc.tc_count_vertices(c, g, out)
    finally:
        tc.tc_graph_free(g)
    return T, st, out.cpu().numpy()[:n].astype(np.uint64)


@pytest.mark.parametrize("tuning", sorted(TUNINGS))
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_vertex_counts(tc, name, tuning):
    n, s, d = GRAPHS[name]
    rp, col = oracle.build_csr(n, s, d)
    T_oracle, want = oracle.vertex_counts(rp, col)
    c = tc.tc_create(0)
    try:
        if TUNINGS[tuning]:
            tc.tc_set_tuning(c, **TUNINGS[tuning])
        T, st, got = vertex_count(tc, c, GRAPHS[name])
    finally:
        tc.tc_destroy(c)
    assert T == T_oracle == oracle.count_definition(rp, col)
    assert np.array_equal(got, want.astype(np.uint64))
    assert int(got.sum()) == 3 * T


@pytest.mark.parametrize("name", ["rmat10", "union"])
def test_vertex_counts_id_order(tc, name):
    n, s, d = GRAPHS[name]
    rp, col = oracle.build_csr(n, s, d)
    c = tc.tc_create(0, order=tc.TC_ORDER_ID)
    try:
        T, st, got = vertex_count(tc, c, GRAPHS[name])
    finally:
        tc.tc_destroy(c)
    assert np.array_equal(got, oracle.vertex_counts(rp, col)[1].astype(np.uint64))


def test_plain_count_unchanged_after_vertex_mode(tc):
    """A vertex-mode count leaves no state behind: tc_count after it agrees."""
    n, s, d = GRAPHS["rmat12_ef32"]
    rp, col = oracle.build_csr(n, s, d)
    c = tc.tc_create(0)
    try:
        vertex_count(tc, c, GRAPHS["rmat12_ef32"])
        g = tc.tc_build_csr(c, n, s, d)
        T, st = tc.tc_count(c, g)
        tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(c)
    assert T == oracle.count_definition(rp, col)
