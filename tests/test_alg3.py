"""Algorithm 3 as a comparison kernel (tc_count_alg3) against the oracle:
T equal to the oracle's Algorithm 3 and to the definition, and the same
t_same / t_cross / |E0| split as the oracle's Algorithm 4 (both count every
triangle from the same horizontal edges), in both working orders."""
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
    "rmat14": gg.rmat(14, 16, seed=5),
    "er4096": gg.er(4096, 60000, seed=2),
    "grid33x47": gg.grid(33, 47, 0.3, 4)[:3],
    "union": gg.disjoint_union([gg.rmat(7, 8, seed=3), gg.cycle(9), gg.complete(6), gg.wheel(6),
                                (3, np.zeros(0, np.uint32), np.zeros(0, np.uint32))]),
    "chung_lu4096": gg.chung_lu(4096, 2.1, 32.0, seed=3),
    "empty": (0, np.zeros(0, np.uint32), np.zeros(0, np.uint32)),
    "isolated5": (5, np.zeros(0, np.uint32), np.zeros(0, np.uint32)),
    "bipartite": gg.complete_bipartite(20, 30),
}


@pytest.mark.parametrize("degree_order", [True, False])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_alg3_matches_oracle(tc, name, degree_order):
    n, s, d = GRAPHS[name]
    rp, col = oracle.build_csr(n, s, d)
    c = tc.tc_create(0, order=tc.TC_ORDER_DEGREE if degree_order else tc.TC_ORDER_ID)
    try:
        g = tc.tc_build_csr(c, n, s, d)
        T, st = tc.tc_count_alg3(c, g)
        T4, st4 = tc.tc_count(c, g)
        tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(c)
    want = oracle.alg4(rp, col, degree_order)
    assert T == oracle.alg3(rp, col, degree_order) == oracle.count_definition(rp, col) == T4
    assert (st["t_same"], st["t_cross"]) == (want["T_same"], want["T_cross"])
    assert st["horizontal_edges"] == want["E0"] == st4["horizontal_edges"]
    # Algorithm 3 reads both full rows of every horizontal edge: at least as much as Algorithm 4 probes
    assert st["probes"] >= st4["probes"]
