"""tc_count_noalloc: the count for callers that cannot allocate device memory.

It must give the same results as the allocating entry point (tc_count), call
after call, although every call reuses the same fixed scratch array.  This
file is collected last so that a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import paper_2309_09064_gb300 as tc
    return tc


def _device_csr(tc, ctx, graph):
    n, s, d = graph[:3]
    g = tc.tc_build_csr(ctx, n, s, d)
    rp, col = tc.tc_graph_copy_out(ctx, g)
    T, st = tc.tc_count(ctx, g)
    tc.tc_graph_free(g)
    trp = torch.from_numpy(rp.view(np.int64)).cuda()
    tcol = torch.from_numpy(col.view(np.int32) if len(col) else np.zeros(1, np.int32)).cuda()
    return n, len(col), trp, tcol, (T, st["t_same"], st["t_cross"])


@pytest.mark.parametrize("order_name", ["degree", "id"])
def test_noalloc_matches_tc_count_two_calls_in_a_row(tc, order_name):
    order = tc.TC_ORDER_DEGREE if order_name == "degree" else tc.TC_ORDER_ID
    ctx = tc.tc_create(0, order=order)
    try:
        graphs = [gg.rmat(12, 16, seed=3), gg.disjoint_union([gg.rmat(9, 8, seed=4), gg.wheel(40), gg.complete(30),
                                                             gg.path(7), gg.star(9)]),
                  gg.er(20000, 150000, seed=5)]
        for graph in graphs:
            n, slots, trp, tcol, want = _device_csr(tc, ctx, graph)
            for _ in range(2):  # the shared array keeps the previous call's contents
                out = torch.full((4,), -1, dtype=torch.int64, device="cuda")
                tc.tc_count_noalloc(trp, tcol, n, slots, out, order=order)
                torch.cuda.synchronize()
                got = [int(x) for x in out.cpu().numpy().view(np.uint64)]
                assert got[3] == 0
                assert tuple(got[:3]) == want
    finally:
        tc.tc_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_array(tc):
    rp = torch.zeros(70000, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(tc.TcError) as e:
        tc.tc_count_noalloc(rp, col, 69999, 0, out)
    assert e.value.status == tc.TC_ERR_INVALID
    with pytest.raises(tc.TcError):
        tc.tc_count_noalloc(rp[:11], col, 10, (1 << 20) + 2, out)
