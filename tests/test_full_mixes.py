"""The batched and served forms at their full sizes, against the oracle.

Exact counts are the method's output (Sec. III: an integer, the number of
triangles), so every graph of the 8,192-graph batch and every request of the
served stream must equal the oracle's Algorithm 4 count, stored per graph in
tests/golden/batches.json by tests/golden/make_golden.py (which calls only
the generators and the oracle).
"""
import json
import os
import random
import time

import numpy as np
import pytest

import graphgen as gg


BATCHES = os.path.join(os.path.dirname(__file__), "golden", "batches.json")


def _gold(name):
    if not os.path.exists(BATCHES):
        pytest.skip("tests/golden/batches.json not generated")
    data = json.load(open(BATCHES))
    if name not in data:
        pytest.skip(f"{name} not in batches.json")
    return data[name]


@pytest.fixture(scope="module")
def tc():
    pytest.importorskip("torch")
    import paper_2309_09064_gb300 as tc
    return tc


def _build_all(tc, ctx, makers):
    graphs = []
    for make in makers:
        n, s, d = make()[:3]
        graphs.append(tc.tc_build_csr(ctx, n, s, d))
    return graphs


@pytest.mark.gpu
def test_batch_of_8192_graphs_equals_the_oracle_graph_by_graph(tc):
    gold = _gold("batch8192")
    specs = gg.batch_specs(8192, seed=5)
    assert len(specs) == gold["count"] == 8192
    ctx = tc.tc_create(0)
    try:
        graphs = _build_all(tc, ctx, [sp.make for sp in specs])
        assert [tc.tc_graph_info(g)[1] // 2 for g in graphs] == gold["m"]
        counts = [int(x) for x in tc.tc_count_batch(ctx, graphs)]
        assert counts == gold["T"]
        # a second batch over the same graphs (arena reused) gives the same counts
        assert [int(x) for x in tc.tc_count_batch(ctx, graphs)] == gold["T"]
        for g in graphs:
            tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(ctx)


@pytest.mark.gpu
def test_served_pool_equals_the_oracle_request_by_request(tc):
    gold = _gold("serve_pool")
    specs = gg.batch_specs(1024, seed=6)
    makers = [sp.make for sp in specs] + [lambda s=s: gg.rmat(20, 16, seed=s) for s in (100, 101)]
    assert len(makers) == gold["count"]
    ctx = tc.tc_create(0)
    try:
        graphs = _build_all(tc, ctx, makers)
        assert [tc.tc_graph_info(g)[1] // 2 for g in graphs] == gold["m"]
        rng = random.Random(6)
        # every graph once, then a random stream with 1% large requests, in arrival order
        reqs = list(range(len(graphs)))
        rng.shuffle(reqs)
        for _ in range(3000):
            reqs.append(len(specs) + rng.randrange(2) if rng.random() < 0.01 else rng.randrange(len(specs)))
        pending, got = {}, {}
        deadline = time.time() + 600
        i = 0
        while (i < len(reqs) or pending) and time.time() < deadline:
            for _ in range(64):  # submissions arrive while earlier ones are on the device
                if i < len(reqs):
                    pending[tc.tc_submit(ctx, graphs[reqs[i]])] = i
                    i += 1
            for t, k in list(pending.items()):
                r = tc.tc_poll(ctx, t)
                if r is not None:
                    got[k] = r
                    del pending[t]
        assert len(got) == len(reqs)
        wrong = [(k, reqs[k], got[k], gold["T"][reqs[k]]) for k in range(len(reqs)) if got[k] != gold["T"][reqs[k]]]
        assert wrong == []
        for g in graphs:
            tc.tc_graph_free(g)
    finally:
        tc.tc_destroy(ctx)


def test_stored_batch_counts_are_self_consistent():
    """The stored lists match their digests (a truncated or edited file fails here, on any machine)."""
    import hashlib
    for name in ("batch8192", "serve_pool"):
        gold = _gold(name)
        h = hashlib.sha256(np.array(gold["T"], dtype="<u8").tobytes()).hexdigest()
        assert h == gold["T_sha256"] and sum(gold["T"]) == gold["T_total"] and len(gold["T"]) == gold["count"]
