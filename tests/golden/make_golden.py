"""Write tests/golden/configs.json: oracle results for the full-size workloads.

Calls only the generators and the CPU oracle (never the CUDA library).  For
each workload it stores n, the CSR size, a SHA-256 of the oracle's CSR
(row_ptr as little-endian uint64, then col as uint32), and the Algorithm 4
results under the degree order: T, T_same, T_cross, |E0|, number of levels,
the level histogram and a SHA-256 of the level array (uint32).

It also writes tests/golden/batches.json: the oracle's T and m of every
graph of the batched mix (8,192 graphs) and of the served pool (1,024
graphs of the same mix plus two R-MAT scale-20 graphs), and, into the
rmat20 record, SHA-256 digests of the per-vertex counts (uint64) and of the
triangle list as sorted keys a << 40 | b << 20 | c (a < b < c, uint64).

Run: python tests/golden/make_golden.py [name ...]   (R-MAT scale 24 takes tens of minutes)
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs.json")
OUT_BATCHES = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batches.json")

WORKLOADS = {
    "rmat10": lambda: gg.rmat(10, 16, seed=1),
    "rmat20": lambda: gg.rmat(20, 16, seed=1),
    "er20": lambda: gg.er(1 << 20, 1 << 24, seed=2),
    "rmat24": lambda: gg.rmat(24, 16, seed=1),
    "chung_lu23": lambda: gg.chung_lu(1 << 23, 2.1, 32.0, seed=3),
    "grid4096": lambda: gg.grid(4096, 4096, 0.3, seed=4),
}


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def host():
    """Where the oracle times were taken: machine, CPU model, cores (the oracle is serial: one thread)."""
    import platform
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.split(":")[0].strip().lower() in ("model name", "cpu part") and not model:
                model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    return {"machine": platform.machine(), "cpu_model": model, "cpus": os.cpu_count(), "threads_used": 1}


def run(name):
    t0 = time.time()
    g = WORKLOADS[name]()
    n, s, d = g[:3]
    rp, col = oracle.build_csr(n, s, d)
    t1 = time.time()
    r = oracle.alg4(rp, col, True)
    t2 = time.time()
    L = r["L"]
    rec = {
        "n": int(n), "tuples": int(len(s)), "slots": int(rp[-1]), "m": int(rp[-1]) // 2,
        "csr_sha256": sha(rp.astype("<u8"), col.astype("<u4")),
        "T": r["T"], "T_same": r["T_same"], "T_cross": r["T_cross"], "E0": r["E0"], "levels": r["levels"],
        "level_hist": [int(x) for x in np.bincount(L.astype(np.int64))],
        "levels_sha256": sha(L.astype("<u4")),
        "oracle_seconds": {"build_csr": round(t1 - t0, 2), "alg4": round(t2 - t1, 2)},
        "oracle_host": host(),
    }
    if len(g) == 4:
        rec["grid_diagonals"] = int(g[3])
    if name in ("rmat10", "rmat20", "er20"):
        rec["T_definition"] = oracle.count_definition(rp, col)
        assert rec["T_definition"] == rec["T"]
    return rec


def _batch_one(desc):
    """Oracle T and m of one graph of a mix; desc is a batch Spec or ("rmat", scale, ef, seed)."""
    g = desc.make() if isinstance(desc, gg.Spec) else gg.rmat(desc[1], desc[2], seed=desc[3])
    rp, col = oracle.build_csr(*g[:3])
    return oracle.alg4(rp, col, True)["T"], int(rp[-1]) // 2


BATCHES = {
    "batch8192": ("gg.batch_specs(8192, seed=5)", lambda: list(gg.batch_specs(8192, seed=5))),
    "serve_pool": ("gg.batch_specs(1024, seed=6) + [gg.rmat(20, 16, seed=100), gg.rmat(20, 16, seed=101)]",
                   lambda: list(gg.batch_specs(1024, seed=6)) + [("rmat", 20, 16, 100), ("rmat", 20, 16, 101)]),
}


def run_batch(name, procs):
    import multiprocessing as mp
    what, make = BATCHES[name]
    descs = make()
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_batch_one, descs, chunksize=8)
    T = [int(t) for t, _ in res]
    return {"graphs": what, "count": len(descs), "T": T, "m": [int(m) for _, m in res],
            "T_sha256": sha(np.array(T, dtype="<u8")), "T_total": sum(T),
            "oracle_seconds": round(time.time() - t0, 2), "oracle_procs": procs}


def list_keys(rp, col):
    """The oracle's triangle list as sorted uint64 keys a << 40 | b << 20 | c (a < b < c < 2^20)."""
    t = oracle.list_definition(rp, col).astype(np.uint64)
    return (t[:, 0] << np.uint64(40)) | (t[:, 1] << np.uint64(20)) | t[:, 2]


def run_next_rmat20():
    rp, col = oracle.build_csr(*gg.rmat(20, 16, seed=1))
    T, tv = oracle.vertex_counts(rp, col)
    keys = list_keys(rp, col)
    assert len(keys) == T and np.all(keys[1:] > keys[:-1])
    return {"vertex_counts_sha256": sha(tv.astype("<u8")), "vertex_counts_sum": int(tv.sum()),
            "list_keys_sha256": sha(keys.astype("<u8"))}


def main(names):
    procs = max(1, min(8, os.cpu_count() or 1))
    batch_names = [x for x in names if x in BATCHES]
    if batch_names:
        bdata = json.load(open(OUT_BATCHES)) if os.path.exists(OUT_BATCHES) else {}
        for name in batch_names:
            bdata[name] = run_batch(name, procs)
            print(name, bdata[name]["count"], bdata[name]["T_total"], bdata[name]["oracle_seconds"], flush=True)
            with open(OUT_BATCHES, "w") as f:
                json.dump(bdata, f, sort_keys=True, separators=(",", ":"))
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    if "next_rmat20" in names:
        data.setdefault("rmat20", {}).update(run_next_rmat20())
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
    for name in [x for x in names if x in WORKLOADS]:
        data[name] = run(name)
        print(name, {k: v for k, v in data[name].items() if k not in ("level_hist",)}, flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS) + list(BATCHES) + ["next_rmat20"])
