"""tc_count_noalloc: the count for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc when they need a count (code inside
another allocator's callback, a memory pool that already owns the whole
device).  The entry point keeps all its scratch in one fixed device array of
the library.  It must give the oracle's exact results (T and its split into
triangles inside G0 and cross-level triangles), call after call, although
every call reuses that array; and after the first call on the device, a call
must not change the device's free memory.  This file is collected last so
that a run that stops at the first failure has already run every other test;
it also passes on its own in a fresh process.
"""
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


def _oracle(graph, degree_order):
    rp, col = oracle.build_csr(*graph[:3])
    r = oracle.alg4(rp, col, degree_order)
    return rp, col, (r["T"], r["T_same"], r["T_cross"])


def _device(rp, col):
    trp = torch.from_numpy(rp.astype(np.uint64).view(np.int64)).cuda()
    tcol = torch.from_numpy(col.view(np.int32) if len(col) else np.zeros(1, np.int32)).cuda()
    return trp, tcol


def _run(tc, trp, tcol, n, slots, order, stream=None):
    out = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    if stream is None:
        tc.tc_count_noalloc(trp, tcol, n, slots, out, order=order)
        torch.cuda.synchronize()
    else:
        tc.tc_count_noalloc(trp, tcol, n, slots, out, order=order, stream=stream)
        stream.synchronize()
    return [int(x) for x in out.cpu().numpy().view(np.uint64)]


def _many_components():
    parts = []
    for i in range(2400):
        k = i % 6
        parts.append(gg.complete(3) if k == 0 else gg.complete(4) if k == 1 else gg.path(5) if k == 2
                     else gg.star(4) if k == 3 else gg.wheel(5) if k == 4 else gg.cycle(6))
    return gg.disjoint_union(parts)


def _matching(n):
    src = np.arange(0, n, 2, dtype=np.uint32)
    return n, src, src + 1


GRAPHS = {
    "rmat12": lambda: gg.rmat(12, 16, seed=3),
    "mixed_union": lambda: gg.disjoint_union([gg.rmat(9, 8, seed=4), gg.wheel(40), gg.complete(30),
                                              gg.path(7), gg.star(9)]),
    "er20000": lambda: gg.er(20000, 150000, seed=5),
    "many_components": _many_components,
    "matching65536": lambda: _matching(65536),
    "limit_rmat16": lambda: gg.rmat(16, 8, seed=7),
}


@pytest.mark.parametrize("order_name", ["degree", "id"])
@pytest.mark.parametrize("name", list(GRAPHS))
def test_noalloc_matches_the_oracle_two_calls_in_a_row(tc, name, order_name):
    order = tc.TC_ORDER_DEGREE if order_name == "degree" else tc.TC_ORDER_ID
    graph = GRAPHS[name]()
    rp, col, want = _oracle(graph, order_name == "degree")
    n = len(rp) - 1
    if name == "limit_rmat16":
        assert n == 65536 and len(col) > 900_000  # at the limits: n = 65536, close to 2^20 slots
    trp, tcol = _device(rp, col)
    for _ in range(2):  # the shared array keeps the previous call's contents
        got = _run(tc, trp, tcol, n, len(col), order)
        assert got[3] == 0
        assert tuple(got[:3]) == want


def test_noalloc_equals_tc_count(tc):
    ctx = tc.tc_create(0)
    try:
        n, s, d = gg.rmat(11, 16, seed=9)
        g = tc.tc_build_csr(ctx, n, s, d)
        T, st = tc.tc_count(ctx, g)
        rp, col = tc.tc_graph_copy_out(ctx, g)
        tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(ctx)
    trp, tcol = _device(rp, col)
    assert _run(tc, trp, tcol, n, len(col), tc.TC_ORDER_DEGREE)[:3] == [T, st["t_same"], st["t_cross"]]


def test_noalloc_on_a_caller_stream(tc):
    rp, col, want = _oracle(gg.rmat(10, 16, seed=1), True)
    trp, tcol = _device(rp, col)
    s = torch.cuda.Stream()
    for _ in range(2):
        got = _run(tc, trp, tcol, len(rp) - 1, len(col), tc.TC_ORDER_DEGREE, stream=s)
        assert got == [*want, 0]


def test_noalloc_allocates_nothing_after_the_first_call(tc):
    rp, col, want = _oracle(gg.rmat(13, 16, seed=11), True)
    trp, tcol = _device(rp, col)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    n = len(rp) - 1
    tc.tc_count_noalloc(trp, tcol, n, len(col), out)  # first call on the device: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        tc.tc_count_noalloc(trp, tcol, n, len(col), out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert [int(x) for x in out.cpu().numpy().view(np.uint64)] == [*want, 0]


def test_noalloc_reports_a_row_ptr_beyond_its_array_on_the_device(tc):
    # the host sees slots = 0; the kernel reads row_ptr[n] > 2^20, writes [0, 0, 0, 1] and touches nothing else
    n = 10
    rp = np.zeros(n + 1, dtype=np.uint64)
    rp[n] = (1 << 20) + 5
    trp = torch.from_numpy(rp.view(np.int64)).cuda()
    tcol = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _run(tc, trp, tcol, n, 0, tc.TC_ORDER_DEGREE) == [0, 0, 0, 1]


def test_noalloc_rejects_sizes_beyond_its_array(tc):
    rp = torch.zeros(70000, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(tc.TcError) as e:
        tc.tc_count_noalloc(rp, col, 69999, 0, out)
    assert e.value.status == tc.TC_ERR_INVALID
    with pytest.raises(tc.TcError):
        tc.tc_count_noalloc(rp[:11], col, 10, (1 << 20) + 2, out)


def test_noalloc_empty_graph(tc):
    trp = torch.zeros(1, dtype=torch.int64, device="cuda")
    tcol = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _run(tc, trp, tcol, 0, 0, tc.TC_ORDER_DEGREE) == [0, 0, 0, 0]
