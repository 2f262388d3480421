"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Counts, the G0 / cross split, |E0|, the number of levels and the level of
every vertex must be bit-exact (integer work).  The CSR built by
tc_build_csr must equal the oracle's CSR bit for bit.
"""
import json
import math
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "configs.json")


@pytest.fixture(scope="module")
def tc():
    import paper_2309_09064_gb300 as tc
    return tc


@pytest.fixture(scope="module")
def ctx(tc):
    c = tc.tc_create(0)
    yield c
    tc.tc_destroy(c)


@pytest.fixture(scope="module")
def ctx_id(tc):
    c = tc.tc_create(0, order=tc.TC_ORDER_ID)
    yield c
    tc.tc_destroy(c)


def small_graphs():
    out = {
        "empty0": (0, np.zeros(0, np.uint32), np.zeros(0, np.uint32)),
        "isolated5": (5, np.zeros(0, np.uint32), np.zeros(0, np.uint32)),
        "one_edge": gg.path(2),
        "K1": gg.complete(1), "K3": gg.complete(3), "K4": gg.complete(4), "K40": gg.complete(40),
        "wheel3": gg.wheel(3), "wheel4": gg.wheel(4), "wheel101": gg.wheel(101),
        "friendship50": gg.friendship(50), "bip7x9": gg.complete_bipartite(7, 9),
        "cycle3": gg.cycle(3), "cycle11": gg.cycle(11), "petersen": gg.petersen(),
        "star40": gg.star(40), "tree300": gg.random_tree(300, 4),
        "grid33x47": gg.grid(33, 47, 0.3, 4)[:3], "gridfull20": gg.grid(20, 20, 1.0, 2)[:3],
        "gnp90": gg.gnp(90, 0.3, 4), "gnp200": gg.gnp(200, 0.05, 5),
        "rmat6": gg.rmat(6, 16, seed=1), "rmat10": gg.rmat(10, 16, seed=1), "rmat12_ef32": gg.rmat(12, 32, seed=3),
        "er4096": gg.er(4096, 60000, seed=2), "chung_lu4096": gg.chung_lu(4096, 2.1, 32.0, seed=3),
        "union": gg.disjoint_union([gg.rmat(7, 8, seed=3), gg.cycle(9), gg.star(5), gg.complete(1), gg.wheel(6),
                                    gg.path(12), gg.complete(7), (3, np.zeros(0, np.uint32), np.zeros(0, np.uint32))]),
        "noisy_rmat9": gg.with_noise(gg.rmat(9, 16, seed=8), seed=1),
    }
    return out


SMALL = small_graphs()


def gpu_count(tc, ctx, graph):
    n, s, d = graph[:3]
    g = tc.tc_build_csr(ctx, n, s, d)
    L = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    T, st = tc.tc_count_levels(ctx, g, L)
    rp, col = tc.tc_graph_copy_out(ctx, g)
    tc.tc_graph_free(g)
    return T, st, L.cpu().numpy().view(np.uint32)[:n], rp, col


def assert_parity(T, st, L, rp, col, graph, degree_order=True):
    n, s, d = graph[:3]
    orp, ocol = oracle.build_csr(n, s, d)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol), "CSR differs"
    ref = oracle.alg4(orp, ocol, degree_order)
    assert T == ref["T"]
    assert st["triangles"] == T
    assert (st["t_same"], st["t_cross"]) == (ref["T_same"], ref["T_cross"])
    assert st["horizontal_edges"] == ref["E0"]
    assert st["levels"] == ref["levels"]
    assert np.array_equal(L, ref["L"])
    assert st["n"] == n and st["m"] == len(ocol) // 2


@pytest.mark.parametrize("name", sorted(SMALL))
def test_small_graph_parity_degree_order(tc, ctx, name):
    g = SMALL[name]
    assert_parity(*gpu_count(tc, ctx, g), g, degree_order=True)


@pytest.mark.parametrize("name", ["rmat10", "union", "grid33x47", "gnp90", "wheel101", "er4096"])
def test_small_graph_parity_id_order(tc, ctx_id, name):
    g = SMALL[name]
    assert_parity(*gpu_count(tc, ctx_id, g), g, degree_order=False)


@pytest.mark.parametrize("caps", [(1, 1, 1), (4, 32, 1), (8, 64, 100), (32, 32, 64)])
@pytest.mark.parametrize("name", ["rmat10", "rmat12_ef32", "union", "K40", "chung_lu4096"])
def test_every_intersection_class(tc, name, caps):
    """Tiny class caps send rows of small graphs through the warp, block and
    global-table (hub) kernels, with maximal task splitting."""
    c = tc.tc_create(0)
    try:
        tc.tc_set_tuning(c, warp_cap=caps[0], block_cap=caps[1], task_work=caps[2], tiny_cap=0)
        g = SMALL[name]
        assert_parity(*gpu_count(tc, c, g), g)
    finally:
        tc.tc_destroy(c)


@pytest.mark.parametrize("bits", [0, 10, 11, 12, 14, 18, 20])
@pytest.mark.parametrize("name", ["rmat10", "rmat12_ef32", "union", "K40", "chung_lu4096", "er4096", "rmat15",
                                  "two_hubs"])
@pytest.mark.parametrize("order_name", ["degree", "id"])
def test_block_class_split_set(tc, name, bits, order_name):
    """Block-class sets split at rank 2^bits (a shared bitmap below, the cuckoo
    table above; the rows stage puts the low ranks of every level-spanning part
    first): with 2^bits below, inside and above the rank range of the graph,
    probe pieces take the bitmap, the table, or both id by id; every row whose
    set holds two or more ranks goes to the block class.  Under the id order
    the ranks are the ids."""
    c = tc.tc_create(0, order=tc.TC_ORDER_DEGREE if order_name == "degree" else tc.TC_ORDER_ID)
    try:
        tc.tc_set_tuning(c, warp_cap=1, block_cap=13107, task_work=256, tiny_cap=0, block_bits_log2=bits)
        g = {"rmat15": lambda: gg.rmat(15, 16, seed=2), "two_hubs": two_hub_graph}.get(name, lambda: SMALL[name])()
        T, st, L, rp, col = gpu_count(tc, c, g)
        if name != "two_hubs":  # its hub rows stay in the hub class
            assert st["class_probes"][2] == 0 and st["class_probes"][1] > st["class_probes"][0]
        assert_parity(T, st, L, rp, col, g, degree_order=order_name == "degree")
    finally:
        tc.tc_destroy(c)


@pytest.mark.parametrize("bits", [10, 11, 12])
@pytest.mark.parametrize("name", ["rmat12_ef32", "chung_lu4096", "union", "rmat10"])
def test_hub_class_split_set(tc, name, bits):
    """Every row with a set of two or more ranks goes to the hub class, split at
    rank 2^bits: low pieces in the shared bitmap, high pieces behind the
    prefilter of the high ranks, and rows ranked at or above 2^bits (whose A
    tails may hold high ranks) probing both, id by id."""
    c = tc.tc_create(0)
    try:
        tc.tc_set_tuning(c, warp_cap=1, block_cap=1, task_work=64, hub_task_work=64, tiny_cap=0,
                         block_bits_log2=bits)
        g = SMALL[name]
        T, st, L, rp, col = gpu_count(tc, c, g)
        assert st["class_probes"][2] > st["class_probes"][0] + st["class_probes"][1]
        assert_parity(T, st, L, rp, col, g)
    finally:
        tc.tc_destroy(c)


@pytest.mark.parametrize("hub_group", [1, 2, 3, 32])
@pytest.mark.parametrize("name", ["rmat12_ef32", "chung_lu4096", "union"])
def test_hub_groups_on_two_streams(tc, name, hub_group):
    """Plain counts run consecutive hub groups on the context's stream and a
    side stream, each with its own bitmaps and task counter; with one to
    three rows per group every group boundary is crossed many times, and the
    per-vertex counts (one stream) must agree with the same tuning."""
    c = tc.tc_create(0)
    try:
        tc.tc_set_tuning(c, warp_cap=1, block_cap=1, task_work=64, hub_task_work=64, tiny_cap=0,
                         hub_group=hub_group)
        g = SMALL[name]
        T, st, L, rp, col = gpu_count(tc, c, g)
        assert st["class_rows"][2] > 0
        assert_parity(T, st, L, rp, col, g)
        gr = tc.tc_build_csr(c, *g[:3])
        out = torch.zeros(g[0], dtype=torch.int64, device="cuda")
        Tv, _ = tc.tc_count_vertices(c, gr, out)
        tc.tc_graph_free(gr)
        assert Tv == T and int(out.sum()) == 3 * T
        # a new stream for the context: the side stream is made again beside it
        st2 = torch.cuda.Stream()
        tc.tc_set_stream(c, st2)
        T2 = gpu_count(tc, c, g)[0]
        tc.tc_set_stream(c, None)
        assert T2 == T
    finally:
        tc.tc_destroy(c)


@pytest.mark.parametrize("tiny", [1, 8, 64])
@pytest.mark.parametrize("name", ["rmat10", "grid33x47", "union", "wheel101", "er4096"])
def test_tiny_merge_class(tc, name, tiny):
    """Rows up to `tiny` go to the thread-per-row merge kernel, the rest to the tables."""
    c = tc.tc_create(0)
    try:
        tc.tc_set_tuning(c, tiny_cap=tiny)
        g = SMALL[name]
        assert_parity(*gpu_count(tc, c, g), g)
    finally:
        tc.tc_destroy(c)


def two_hub_graph(leaves=20000, extra=3000, seed=5):
    """Hubs A (vertex 0) and B (vertex 1) joined to each other and to `leaves`
    leaves; A also has a private pendant so it is the root.  B sits on level 1
    with all leaves, and its hashed row exceeds the shared-memory cap, so it
    takes the global-table kernel with the default tuning."""
    pairs = [(0, 1), (0, leaves + 2)]
    pairs += [(0, 2 + i) for i in range(leaves)] + [(1, 2 + i) for i in range(leaves)]
    r = gg.draws(seed, 0x48554221, 0, 2 * extra)
    for i in range(extra):
        a = 2 + int(r[2 * i] % np.uint64(leaves))
        b = 2 + int(r[2 * i + 1] % np.uint64(leaves))
        pairs.append((a, b))
    arr = np.array(pairs, dtype=np.uint32)
    return leaves + 3, arr[:, 0].copy(), arr[:, 1].copy()


def test_hub_kernel_default_tuning(tc, ctx):
    g = two_hub_graph()
    assert_parity(*gpu_count(tc, ctx, g), g)


@pytest.mark.parametrize("scale", [14, 16])
def test_rmat_medium(tc, ctx, scale):
    g = gg.rmat(scale, 16, seed=scale)
    assert_parity(*gpu_count(tc, ctx, g), g)


def test_device_tuples_and_borrowed_csr(tc, ctx):
    n, s, d = gg.rmat(11, 16, seed=4)
    g = tc.tc_build_csr(ctx, n, torch.from_numpy(s.view(np.int32)).cuda(), torch.from_numpy(d.view(np.int32)).cuda())
    T, _ = tc.tc_count(ctx, g)
    rp, col = oracle.build_csr(n, s, d)
    assert T == oracle.count_definition(rp, col)
    trp = torch.from_numpy(rp.view(np.int64)).cuda()
    tcol = torch.from_numpy(col.view(np.int32)).cuda()
    gb = tc.tc_graph_from_csr(ctx, trp, tcol, flags=tc.TC_BORROW | tc.TC_VALIDATE)
    T2, _ = tc.tc_count(ctx, gb)
    gh = tc.tc_graph_from_csr(ctx, rp, col, flags=tc.TC_COPY | tc.TC_VALIDATE)
    T3, _ = tc.tc_count(ctx, gh)
    assert T == T2 == T3
    for x in (g, gb, gh):
        tc.tc_graph_free(x)


def test_validation_rejects_malformed_csr(tc, ctx):
    rp, col = oracle.build_csr(*gg.wheel(6))
    cases = []
    bad = col.copy(); bad[0], bad[1] = bad[1], bad[0]; cases.append((rp, bad))            # unsorted row
    bad = col.copy(); bad[1] = bad[0]; cases.append((rp, bad))                             # repeat
    bad = col.copy(); bad[0] = 0; cases.append((rp, bad))                                  # self-loop at row 0
    bad = col.copy(); bad[-1] = 99; cases.append((rp, bad))                                # id >= n
    rp2, col2 = oracle.build_csr(*gg.path(3))
    asym = np.array([0, 1, 2, 3], np.uint64), np.array([1, 0, 0], np.uint32)             # 2 -> 0 without 0 -> 2
    cases.append(asym)
    bad_rp = rp.copy(); bad_rp[3] = bad_rp[-1] + 50; cases.append((bad_rp, col))            # row past the end
    for r, c in cases:
        with pytest.raises(tc.TcError) as e:
            tc.tc_graph_from_csr(ctx, r, c, flags=tc.TC_COPY | tc.TC_VALIDATE)
        assert e.value.status == tc.TC_ERR_INVALID
    g = tc.tc_graph_from_csr(ctx, rp2, col2, flags=tc.TC_VALIDATE)
    assert tc.tc_validate(ctx, g)
    tc.tc_graph_free(g)


def test_build_csr_rejects_bad_ids(tc, ctx):
    with pytest.raises(tc.TcError) as e:
        tc.tc_build_csr(ctx, 4, np.array([0, 1], np.uint32), np.array([1, 4], np.uint32))
    assert e.value.status == tc.TC_ERR_INVALID


def test_torch_stream(tc):
    s = torch.cuda.Stream()
    c = tc.tc_create(0, stream=s)
    try:
        n, src, dst = gg.rmat(10, 16, seed=1)
        g = tc.tc_build_csr(c, n, src, dst)
        T, _ = tc.tc_count(c, g)
        rp, col = oracle.build_csr(n, src, dst)
        assert T == oracle.count_definition(rp, col)
        tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(c)


def test_repeated_counts_are_identical(tc, ctx):
    n, s, d = gg.rmat(13, 16, seed=2)
    g = tc.tc_build_csr(ctx, n, s, d)
    runs = [tc.tc_count(ctx, g) for _ in range(5)]
    tc.tc_graph_free(g)
    assert len({T for T, _ in runs}) == 1
    # stats.launches counts the kernels of one call: the same for every repeat
    launches = {st["launches"] for _, st in runs}
    assert len(launches) == 1 and 0 < launches.pop() < 1000


# ------------------------------------------------------------------------- batched and served forms

def batch_graphs(count, seed, n_hi=4096):
    return [spec.make() for spec in gg.batch_specs(count, seed=seed, n_hi=n_hi)]


@pytest.mark.parametrize("small_slots", [0, 1 << 10, 1 << 22])
@pytest.mark.parametrize("order_name", ["degree", "id"])
def test_batch_equals_loop_and_oracle(tc, small_slots, order_name):
    """Graphs up to small_slots CSR slots take the one-launch kernel (a block per
    graph), the others the union pipeline (0: all of them), in one batch."""
    order = tc.TC_ORDER_DEGREE if order_name == "degree" else tc.TC_ORDER_ID
    c = tc.tc_create(0, order=order)
    try:
        tc.tc_set_tuning(c, batch_small_slots=small_slots)
        graphs = batch_graphs(96, seed=5) + [SMALL[k] for k in ("empty0", "isolated5", "K40", "union", "wheel101",
                                                                  "grid33x47", "tree300", "friendship50")]
        gs = [tc.tc_build_csr(c, *g[:3]) for g in graphs]
        batched = tc.tc_count_batch(c, gs)
        again = tc.tc_count_batch(c, gs[::-1])
        looped = [tc.tc_count(c, g)[0] for g in gs]
        ref = [oracle.count_definition(*oracle.build_csr(*g[:3])) for g in graphs]
        for g in gs:
            tc.tc_graph_free(g)
        assert list(batched) == looped == ref
        assert list(again) == ref[::-1]
    finally:
        tc.tc_destroy(c)


def test_served_results_alone_and_in_the_mix(tc):
    c = tc.tc_create(0)
    try:
        graphs = batch_graphs(200, seed=6)
        gs = [tc.tc_build_csr(c, *g[:3]) for g in graphs]
        alone = [tc.tc_count(c, g)[0] for g in gs]
        tickets = [tc.tc_submit(c, g) for g in gs]
        got = {}
        import time
        deadline = time.time() + 120
        while len(got) < len(tickets) and time.time() < deadline:
            for i, t in enumerate(tickets):
                if i not in got:
                    r = tc.tc_poll(c, t)
                    if r is not None:
                        got[i] = r
        assert len(got) == len(tickets)
        assert [got[i] for i in range(len(gs))] == alone
        # one more request on its own after the mix, with its latency
        t = tc.tc_submit(c, gs[3])
        while (r := tc.tc_poll_ex(c, t)) is None:
            pass
        assert r[0] == alone[3] and r[1] > 0
        with pytest.raises(tc.TcError):
            tc.tc_poll(c, t)  # a ticket is released once its result has been read
        for g in gs:
            tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(c)


# ------------------------------------------------------------------------- full-size workloads (stored oracle values)

def _golden():
    if not os.path.exists(GOLDEN):
        pytest.skip("tests/golden/configs.json not generated")
    return json.load(open(GOLDEN))


FULL = {
    "rmat20": lambda: gg.rmat(20, 16, seed=1),
    "er20": lambda: gg.er(1 << 20, 1 << 24, seed=2),
    "rmat24": lambda: gg.rmat(24, 16, seed=1),
    "chung_lu23": lambda: gg.chung_lu(1 << 23, 2.1, 32.0, seed=3),
    "grid4096": lambda: gg.grid(4096, 4096, 0.3, seed=4),
}


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_against_stored_oracle(tc, ctx, name):
    import hashlib
    gold = _golden()
    if name not in gold:
        pytest.skip(f"{name} not in configs.json")
    ref = gold[name]
    g = FULL[name]()
    n, s, d = g[:3]
    dev_s = torch.from_numpy(s.view(np.int32)).cuda()
    dev_d = torch.from_numpy(d.view(np.int32)).cuda()
    gr = tc.tc_build_csr(ctx, n, dev_s, dev_d)
    del dev_s, dev_d
    L = torch.empty(n, dtype=torch.int32, device="cuda")
    T, st = tc.tc_count_levels(ctx, gr, L)
    rp, col = tc.tc_graph_copy_out(ctx, gr)
    tc.tc_graph_free(gr)
    h = hashlib.sha256()
    h.update(rp.astype("<u8").tobytes())
    h.update(col.astype("<u4").tobytes())
    assert h.hexdigest() == ref["csr_sha256"]
    assert (T, st["t_same"], st["t_cross"], st["horizontal_edges"], st["levels"]) == \
        (ref["T"], ref["T_same"], ref["T_cross"], ref["E0"], ref["levels"])
    Lh = L.cpu().numpy().view(np.uint32)
    assert hashlib.sha256(Lh.astype("<u4").tobytes()).hexdigest() == ref["levels_sha256"]
    if "grid_diagonals" in ref:
        assert T == 2 * ref["grid_diagonals"]


def test_autotuner_keeps_counts_and_sets_a_valid_tuning(tc, tmp_path):
    from paper_2309_09064_gb300 import autotune
    c = tc.tc_create(0)
    try:
        graphs = [tc.tc_build_csr(c, *gg.rmat(13, 16, seed=3)), tc.tc_build_csr(c, *SMALL["union"])]
        want = [tc.tc_count(c, g)[0] for g in graphs]
        cache = str(tmp_path / "tune.json")
        best, table = autotune.autotune(c, graphs, reps=1, cache_path=cache)
        assert table and tc.tc_get_tuning(c) == best
        assert list(tc.tc_count_batch(c, graphs)) == want
        again, table2 = autotune.autotune(c, graphs, cache_path=cache)  # served from the cache
        assert again == best and table2 == []
        for g in graphs:
            tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(c)


@pytest.mark.parametrize("nshards", [1, 2, 3, 8])
def test_shards_sum_to_the_count(tc, ctx, nshards):
    for graph in (gg.rmat(14, 16, seed=2), two_hub_graph(), SMALL["union"]):
        g = tc.tc_build_csr(ctx, *graph[:3])
        T, _ = tc.tc_count(ctx, g)
        parts = [tc.tc_count_shard(ctx, g, k, nshards)[0] for k in range(nshards)]
        tc.tc_graph_free(g)
        assert sum(parts) == T


@pytest.mark.parametrize("bits", [0, 19])
@pytest.mark.parametrize("nshards", [2, 3, 5, 8])
def test_shards_agree_on_rows_of_degree_above_8192(tc, nshards, bits):
    """Every shard recomputes the rows, and its tasks are slices of F(u): the
    block-filled rows (degree above 8192) must come out in the same order on
    every run, or shards would cut a row's slices from different orders."""
    c = tc.tc_create(0)
    try:
        tc.tc_set_tuning(c, warp_cap=64, block_cap=1024, task_work=4096, hub_task_work=4096, max_v=64,
                         block_bits_log2=bits)
        n, s, d = gg.rmat(17, 16, seed=3)
        g = tc.tc_build_csr(c, n, s, d)
        assert tc.tc_graph_info(g)[1] > 0
        T, st = tc.tc_count(c, g)
        assert st["class_rows"][2 if bits == 0 else 1] > nshards  # hub (or split block) rows, many tasks
        for _ in range(3):
            parts = [tc.tc_count_shard(c, g, k, nshards)[0] for k in range(nshards)]
            assert sum(parts) == T
        tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(c)


def test_bounded_device_wait_times_out_and_context_survives(tc):
    c = tc.tc_create(0)
    try:
        assert tc.tc_selftest_barrier(c, 200) == tc.TC_ERR_TIMEOUT
        g = tc.tc_build_csr(c, *SMALL["rmat10"])
        T, _ = tc.tc_count(c, g)  # the context still works
        rp, col = oracle.build_csr(*SMALL["rmat10"])
        assert T == oracle.count_definition(rp, col)
        tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(c)


def test_injected_allocation_failure_is_reported_and_recovered(tc, monkeypatch):
    monkeypatch.setenv("TC_FAIL_ALLOC_AT", "1")
    c = tc.tc_create(0)  # the variable is read here
    monkeypatch.delenv("TC_FAIL_ALLOC_AT")
    try:
        n, s, d = SMALL["rmat10"]
        rp, col = oracle.build_csr(n, s, d)
        with pytest.raises(tc.TcError) as e:
            tc.tc_graph_from_csr(c, rp, col)  # its first allocation fails
        assert e.value.status == tc.TC_ERR_OOM
        g = tc.tc_graph_from_csr(c, rp, col)  # the next one succeeds
        assert tc.tc_count(c, g)[0] == oracle.count_definition(rp, col)
        tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(c)


def test_queue_full_reports_busy(tc):
    c = tc.tc_create(0, max_queue=4)
    try:
        g = tc.tc_build_csr(c, *gg.rmat(12, 16, seed=9))
        want = tc.tc_count(c, g)[0]
        tickets, busy = [], 0
        for _ in range(2000):
            try:
                tickets.append(tc.tc_submit(c, g))
            except tc.TcError as e:
                assert e.status == tc.TC_ERR_BUSY
                busy += 1
        assert busy > 0
        for t in tickets:
            while (r := tc.tc_poll(c, t)) is None:
                pass
            assert r == want
        tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(c)
