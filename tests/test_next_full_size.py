"""Per-vertex counts and the triangle listing at R-MAT scale 20, against the oracle.

At this size the per-vertex counts pass the block-private shared counters of
the 1,024 highest ranks and the listing fills many output chunks from the
global cursor and compacts them, paths the small parity graphs do not reach.
The expected values are SHA-256 digests written by tests/golden/make_golden.py
from the oracle's per-vertex counts (uint64, little-endian) and its triangle
list as sorted keys a << 40 | b << 20 | c with a < b < c (uint64).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "configs.json")


@pytest.fixture(scope="module")
def rmat20():
    if not os.path.exists(GOLDEN):
        pytest.skip("tests/golden/configs.json not generated")
    ref = json.load(open(GOLDEN)).get("rmat20", {})
    if "list_keys_sha256" not in ref:
        pytest.skip("R-MAT 20 listing digest not stored")
    import paper_2309_09064_gb300 as tc
    ctx = tc.tc_create(0)
    n, s, d = gg.rmat(20, 16, seed=1)
    g = tc.tc_build_csr(ctx, n, s, d)
    yield tc, ctx, g, n, ref
    tc.tc_graph_free(g)
    tc.tc_destroy(ctx)


def test_vertex_counts_rmat20_equal_the_oracle(rmat20):
    tc, ctx, g, n, ref = rmat20
    out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    T, _ = tc.tc_count_vertices(ctx, g, out)
    tv = out.cpu().numpy().view(np.uint64)
    assert int(tv.sum()) == ref["vertex_counts_sum"] == 3 * T == 3 * ref["T"]
    assert hashlib.sha256(tv.astype("<u8").tobytes()).hexdigest() == ref["vertex_counts_sha256"]


def test_triangle_list_rmat20_equals_the_oracle(rmat20):
    tc, ctx, g, n, ref = rmat20
    cap = ref["T"]
    triples = torch.empty(3 * cap, dtype=torch.int32, device="cuda")
    T, _ = tc.tc_list_triangles(ctx, g, triples, cap)
    assert T == ref["T"]
    t = triples.view(cap, 3).to(torch.int64)
    del triples
    t, _ = torch.sort(t, dim=1)
    keys = (t[:, 0] << 40) | (t[:, 1] << 20) | t[:, 2]
    del t
    keys, _ = torch.sort(keys)
    assert bool((keys[1:] > keys[:-1]).all())  # every triangle once
    h = hashlib.sha256(keys.cpu().numpy().astype("<u8").tobytes()).hexdigest()
    assert h == ref["list_keys_sha256"]
