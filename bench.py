"""Benchmark: exact triangle counting on one GB300 (edges counted per second).

Default workload: R-MAT scale 24 (16,777,216 vertices, edge factor 16,
A/B/C/D = 0.57/0.19/0.19/0.05, seed 1, symmetrised, de-duplicated, no
self-loops), one exact count per step through the C ABI (tc_count) on the
device-resident CSR.  The CSR is larger than L2, so steps need no flush.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload rmat24|rmat20|er20|chung_lu23|grid4096|rmat10]

One JSON line on rank 0.  `value` = undirected edges counted per second over
the whole job (N replicas of the count, one per GPU: weak scaling), measured
with CUDA events on the library's stream, max over ranks.  `e2e` is the same
metric through the public API from pinned host buffers (CSR upload, count,
8-byte result back).  `roofline` is the dominant kernel of the count (by
device time), algorithmic bytes / its event-timed duration against the
measured HBM copy bandwidth.  `cpu_baseline` times the CPU oracle (serial C,
Algorithm 4) on a bounded sample of the same generator.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

WORKLOADS = {
    "rmat24": dict(kind="rmat", scale=24, edge_factor=16, seed=1),
    "rmat22": dict(kind="rmat", scale=22, edge_factor=16, seed=1),
    "rmat20": dict(kind="rmat", scale=20, edge_factor=16, seed=1),
    "rmat10": dict(kind="rmat", scale=10, edge_factor=16, seed=1),
    "er20": dict(kind="er", n=1 << 20, m=1 << 24, seed=2),
    "chung_lu23": dict(kind="chung_lu", n=1 << 23, gamma=2.1, mean_deg=32.0, seed=3),
    "grid4096": dict(kind="grid", rows=4096, cols=4096, p=0.3, seed=4),
}
CPU_SAMPLE = dict(kind="rmat", scale=18, edge_factor=16, seed=1)
L2_BYTES = 129 * 1024 * 1024


def make_tuples(w):
    if w["kind"] == "rmat":
        return gg.rmat(w["scale"], w["edge_factor"], seed=w["seed"])
    if w["kind"] == "er":
        return gg.er(w["n"], w["m"], w["seed"])
    if w["kind"] == "chung_lu":
        return gg.chung_lu(w["n"], w["gamma"], w["mean_deg"], seed=w["seed"])
    if w["kind"] == "grid":
        return gg.grid(w["rows"], w["cols"], w["p"], w["seed"])[:3]
    raise ValueError(w)


def config_of(name, w, n, m, extra=None):
    c = {"workload": name, "n": int(n), "m": int(m), **{k: v for k, v in w.items() if k != "kind"},
         "family": w["kind"], "order": "degree (BaderD)",
         "l2": "no flush: col array alone exceeds L2" if 4 * 2 * m > L2_BYTES else "inputs smaller than L2"}
    if w["kind"] == "rmat":
        c["abcd"] = [0.57, 0.19, 0.19, 0.05]
    if extra:
        c.update(extra)
    return c


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline_run(repeats=5):
    """The CPU oracle (serial C, Algorithm 4 under the degree order) on R-MAT
    scale 18 of the same generator: edges/s = m / mean oracle time."""
    import oracle
    n, s, d = make_tuples(CPU_SAMPLE)
    rp, col = oracle.build_csr(n, s, d)
    m = len(col) // 2
    times = []
    T = None
    for _ in range(repeats):
        t0 = time.perf_counter()
        T = oracle.alg4(rp, col, True)["T"]
        times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    return {"value": m / mean, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"R-MAT scale 18 (n=262144, m={m}, seed 1, same generator and A-D), "
                      f"oracle Algorithm 4 (serial C, 1 thread), mean of {repeats} runs, "
                      f"{mean:.2f} s each, T={T}"}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    n, s, d = make_tuples(CPU_SAMPLE)
    rp, col = oracle.build_csr(n, s, d)
    m = len(col) // 2
    for _ in range(args.warmup):
        oracle.alg4(rp, col, True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.alg4(rp, col, True)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    value = m / dt
    w = WORKLOADS[args.workload]
    line = {"metric": "edges/sec counted (exact)", "value": value, "unit": "edges/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "impl": "reference",
            "config": config_of(args.workload, w, 0, 0, {"reference_sample": "R-MAT scale 18, seed 1"}),
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: oracle Algorithm 4 (serial C) on R-MAT scale 18 "
                                       f"(m={m}) of the same generator"},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat24", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    world, rank, local = dist_setup()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2309_09064_gb300 as tc

    w = WORKLOADS[args.workload]
    n, s, d = make_tuples(w)
    stream = torch.cuda.current_stream()
    ctx = tc.tc_create(local, stream=stream)
    ts = torch.from_numpy(s.view(np.int32)).cuda()
    td = torch.from_numpy(d.view(np.int32)).cuda()
    g = tc.tc_build_csr(ctx, n, ts, td)
    del ts, td
    torch.cuda.synchronize()
    n_, slots, _, _ = tc.tc_graph_info(g)
    m = slots // 2

    T0 = None
    for _ in range(max(args.warmup, 0)):
        T0, _ = tc.tc_count(ctx, g)

    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record(stream)
    for _ in range(args.steps):
        T, st = tc.tc_count(ctx, g)
        stats.append(st)
        assert T0 is None or T == T0, "count changed between steps"
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clock_info = clocks.stop()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * m / (ms / 1e3)

    # dominant kernel of the count by device time, from the library's own events
    def mean(key, i=None):
        xs = [st[key][i] if i is not None else st[key] for st in stats]
        return sum(xs) / len(xs)

    kernels = {
        "k_isect_warp": (mean("ms_class", 0), mean("class_bytes", 0)),
        "k_isect_block<shared>": (mean("ms_class", 1), mean("class_bytes", 1)),
        "k_isect_block<global>": (mean("ms_class", 2), mean("class_bytes", 2)),
    }
    dom = max(kernels, key=lambda k: kernels[k][0])
    dom_ms, dom_bytes = kernels[dom]
    peak, peak_kind = measured_peaks()
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else 0.0
    whole_gbs = mean("alg_bytes") / (ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
                "bytes_per_launch": dom_bytes, "ms_per_launch": dom_ms,
                "whole_count": {"alg_bytes": mean("alg_bytes"), "achieved": whole_gbs, "frac": whole_gbs / peak}}

    # end to end through the public API from pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        rp_h, col_h = tc.tc_graph_copy_out(ctx, g)
        rp_p = torch.from_numpy(rp_h.view(np.int64)).pin_memory()
        col_p = torch.from_numpy(col_h.view(np.int32)).pin_memory()
        out = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            g2 = tc.tc_graph_from_csr(ctx, rp_p, col_p, flags=tc.TC_COPY)
            T2, _ = tc.tc_count(ctx, g2)
            tc.tc_graph_free(g2)
            out.append(T2)
        dt = (time.perf_counter() - t0) / args.e2e_steps
        assert all(x == T0 for x in out)
        e2e = {"value": world * m / dt, "unit": "edges/s",
               "h2d_bytes_per_step": int(rp_p.numel() * 8 + col_p.numel() * 4), "d2h_bytes_per_step": 8 + 208,
               "ms_per_step": dt * 1e3}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_run()

    last = stats[-1]
    line = {
        "metric": "edges/sec counted (exact)", "value": value, "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": config_of(args.workload, w, n_, m, {"parallelism": f"replicas x{world}"}),
        "triangles": T0, "t_same": last["t_same"], "t_cross": last["t_cross"],
        "horizontal_edges": last["horizontal_edges"], "levels": last["levels"],
        "stage_ms": {"levels": mean("ms_levels"), "rows": mean("ms_mark"), "intersect": mean("ms_isect"),
                     "isect_warp": mean("ms_class", 0), "isect_block": mean("ms_class", 1),
                     "isect_hub": mean("ms_class", 2)},
        "roofline": roofline, "gpu_launches": int(sum(st["launches"] for st in stats)),
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clock_info,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    tc.tc_graph_free(g)
    tc.tc_destroy(ctx)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
