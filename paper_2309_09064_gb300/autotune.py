"""Autotuner for the launch-shape knobs of the intersection stage.

The knobs (``tc_tuning`` in ``include/tc.h``) decide how hashed rows are
classed (warp / block / hub caps), how big the shared tables, slices and hub
prefilters are (hence how many blocks fit on an SM), and how much probe work a
task carries.  ``autotune`` times every candidate on sample graphs through the
C ABI (``tc_count`` for one graph, ``tc_count_batch`` for several), requires
every candidate to return the same exact counts, keeps the fastest on the
context and returns it.  Results can be cached in a JSON file keyed by a
coarse signature of the workload (log2 of n, m and the largest degree), so a
service can tune once per graph family.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import (TcError, tc_count, tc_count_batch, tc_get_tuning, tc_graph_info, tc_set_tuning)

# Candidate overrides of the default tuning.  Pairs of (block_cap, max_v) and
# (hub_filter_log2, max_v) trade table / prefilter size against blocks per SM.
CANDIDATES = [
    {},
    {"block_cap": 8192, "max_v": 1024},
    {"block_cap": 8192, "max_v": 1024, "hub_filter_log2": 19},
    {"hub_filter_log2": 19, "max_v": 1024},
    {"block_cap": 8192, "max_v": 1024, "hub_filter_log2": 19, "hub_group": 8},
    {"block_cap": 8192, "max_v": 1024, "hub_filter_log2": 19, "hub_group": 4},
    {"warp_cap": 512},
    {"warp_cap": 2048, "warps_per_block": 4},
    {"task_work": 1048576, "hub_task_work": 262144, "hub_group": 8},
    {"task_work": 65536, "hub_task_work": 131072},
    {"task_work": 524288, "hub_task_work": 1048576},
    {"block_threads": 512, "hub_threads": 512, "block_cap": 8192, "max_v": 1024, "hub_filter_log2": 19},
    {"table_kind": 1, "block_cap": 16384},
    {"block_cap": 13107},
    {"flat_cap": 0},
    {"flat_cap": 256},
    {"block_bits_log2": 0},
    {"block_bits_log2": 18},
    {"block_bits_log2": 20},
    {"hub_task_work": 1048576},
    {"task_work": 2097152, "warp_task_work": 16384},
    {"max_v": 1024},
    {"batch_small_slots": 16384},
    {"batch_small_slots": 65536},
    {"batch_small_slots": 262144},
]


def signature(ctx, graphs) -> str:
    """Coarse workload key: rounded log2 of vertices, edges and graph count."""
    n = sum(tc_graph_info(g)[0] for g in graphs)
    m = sum(tc_graph_info(g)[1] for g in graphs) // 2
    lg = lambda x: int(round(math.log2(max(x, 1))))
    return f"n2^{lg(n)}-m2^{lg(m)}-g{lg(len(graphs))}"


def _run(ctx, graphs):
    if len(graphs) == 1:
        return [tc_count(ctx, graphs[0])[0]]
    return [int(x) for x in tc_count_batch(ctx, graphs)]


def autotune(ctx, graphs, candidates=None, reps: int = 2, cache_path: str | None = None, verbose: bool = False):
    """Pick the fastest valid candidate for `graphs`; returns (best knobs, table of results)."""
    graphs = list(graphs)
    cache_path = cache_path or os.environ.get("TC_AUTOTUNE_CACHE")
    key = signature(ctx, graphs)
    if cache_path and os.path.exists(cache_path):
        cached = json.load(open(cache_path)).get(key)
        if cached:
            tc_set_tuning(ctx, **cached)
            return cached, []
    base = tc_get_tuning(ctx)
    want = _run(ctx, graphs)
    results = []
    best, best_ms = None, float("inf")
    for cand in candidates or CANDIDATES:
        knobs = dict(base)
        knobs.update(cand)
        try:
            tc_set_tuning(ctx, **knobs)
        except TcError:
            continue
        got = _run(ctx, graphs)  # warm-up, and the exactness check
        if got != want:
            raise RuntimeError(f"tuning {cand} changed the counts")
        t0 = time.perf_counter()
        for _ in range(reps):
            _run(ctx, graphs)
        ms = (time.perf_counter() - t0) / reps * 1e3
        results.append({"knobs": cand, "ms": ms})
        if verbose:
            print(f"  {ms:9.2f} ms  {cand}")
        if ms < best_ms:
            best, best_ms = knobs, ms
    tc_set_tuning(ctx, **best)
    if cache_path:
        data = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
        data[key] = best
        with open(cache_path, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
    return best, results
