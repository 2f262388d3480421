"""Write tests/golden/configs.json: oracle results for the full-size workloads.

Calls only the generators and the CPU oracle (never the CUDA library).  For
each workload it stores n, the CSR size, a SHA-256 of the oracle's CSR
(row_ptr as little-endian uint64, then col as uint32), and the Algorithm 4
results under the degree order: T, T_same, T_cross, |E0|, number of levels,
the level histogram and a SHA-256 of the level array (uint32).

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
    }
    if len(g) == 4:
        rec["grid_diagonals"] = int(g[3])
    if name in ("rmat10", "rmat20", "er20"):
        rec["T_definition"] = oracle.count_definition(rp, col)
        assert rec["T_definition"] == rec["T"]
    return rec


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        data[name] = run(name)
        print(name, {k: v for k, v in data[name].items() if k not in ("level_hist",)}, flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
