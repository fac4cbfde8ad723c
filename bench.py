"""Benchmark of the MAP hot path on GB300: GTEPS + fraction of the HBM roofline.

One step = one full MAP run (every outer iteration: dense round, frontier rounds to the
fix-point, self-map test, elimination) over the 2^26-vertex layered no-cycle graph
(4,000 layers, geometric out-degree with mean 4, 92 % forward edges, back edges over 50
layers, 1 % accepting, accepting vertices on no cycle), inputs resident in HBM.

    metric  MAP edge relaxations/s, GTEPS = (m x outer iterations) / device time
            (every fix-point examines every edge at least once)
    e2e     the same metric through the C ABI from pinned host buffers: map_create
            (host-to-device copy, validation, transpose) + map_run + map output
            device-to-host + map_destroy, every step
    roofline  the dense-round kernel: algorithmic bytes per launch / its CUDA-event time
    cpu_baseline  the CPU oracle on the first outer iterations of the same graph

Under torchrun (N > 1) every rank solves its own replica of the graph on its own GPU
(MAP on one graph does not shard; independent graphs do): scaling "weak".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="layered-2^26v-4000L", n=1 << 26, layers=4000, seed=3, D=16, window=50,
                acc_p=0.01, fwd_p=0.92, mean_degree=4)
METRIC = "MAP edge relaxations/s (GTEPS)"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling (SM clock, throttle reasons) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [line for line in out.splitlines() if line.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The oracle as it stands, on the host cores, each step a bounded sample of the workload."""
    ws, rank, _ = dist_init()
    if rank != 0:
        return 0
    import mapgen
    import oracle

    oracle.build()
    g = mapgen.layered_64m()
    sample_outer = args.cpu_outer
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; warm-up steps are not repeated on the CPU
    t0 = time.perf_counter()
    edges = 0
    for _ in range(args.steps):
        r = oracle.run_graph(g, max_outer=sample_outer)
        edges += g.m * r.outer
    dt = time.perf_counter() - t0
    v = edges / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": dict(WORKLOAD, l2="inputs larger than L2 (1.34 GB CSR)"),
            "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": f"first {sample_outer} outer iterations of the same graph per step"},
            "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(g, outer):
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    r = oracle.run_graph(g, max_outer=outer)
    dt = time.perf_counter() - t0
    return {"value": g.m * r.outer / dt / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"first {r.outer} outer iterations of the same graph ({dt:.1f} s, single thread, "
                      f"including the oracle's own set-up)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--sched", type=int, default=0, help="0 = synchronous rounds (canonical), 1 = asynchronous")
    ap.add_argument("--cpu-outer", type=int, default=3, help="outer iterations in the CPU-oracle sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--n", type=int, default=None, help="override vertex count (smaller runs, not the bench line)")
    args = ap.parse_args()

    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import mapgen
    import paper_0912_2555_gb300 as pkg
    from paper_0912_2555_gb300 import build as gpu_build

    ws, rank, local = dist_init()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        gpu_build.build()
    if ws > 1:
        dist.barrier()
    lib = pkg.load()

    n = args.n or WORKLOAD["n"]
    layers = WORKLOAD["layers"] if args.n is None else max(8, round(n / 16777))
    g = mapgen.layered_graph(n, layers, WORKLOAD["seed"], D=WORKLOAD["D"], window=WORKLOAD["window"],
                             acc_p=WORKLOAD["acc_p"], fwd_p=WORKLOAD["fwd_p"])
    stream = torch.cuda.current_stream()
    rp = torch.from_numpy(g.rowptr.view(np.int32)).cuda()
    ci = torch.from_numpy(g.colidx.view(np.int32)).cuda()
    ab = torch.from_numpy(pkg.pack_bits(g.acc).view(np.int32)).cuda()
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    h = pkg.map_create(g.n, rp, ci, ab, stream)

    def step(flags=0):
        return pkg.map_run(h, sched=args.sched, flags=flags, map_out=out)

    for _ in range(max(args.warmup, 3)):
        r0 = step()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    results = []
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            results.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    edges = sum(r.edges_total for r in results)
    value = edges * ws / (ms / 1e3) / 1e9

    # roofline of the dominant kernel (the dense round): algorithmic bytes per launch over its
    # CUDA-event time.  Events cannot sit inside the graph's loop bodies, so this pass runs
    # the same kernels stepped from the host, with events around every dense launch.
    prof = [step(pkg.MAP_FLAG_PROFILE) for _ in range(2)]
    dense_launches = sum(r.dense_launches for r in prof)
    dense_ms = sum(r.dense_ms for r in prof)
    words = (g.n + 31) // 32
    dense_bytes = 4 * (g.n + 1) + 4 * g.m + 4 * g.n  # rowptr + colidx (flags in bit 31) + map writes
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = dense_bytes * dense_launches / (dense_ms / 1e3) / 1e9 if dense_ms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "kernel": "k_dense (round 1 of each outer iteration)", "bytes_per_launch": dense_bytes,
                "launch_ms": dense_ms / max(dense_launches, 1),
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s",
                "share_of_step": (dense_ms / len(prof)) / (ms / args.steps) if ms else None,
                "timing": "CUDA events around each dense launch in 2 extra host-stepped runs"}
    phases = {"dense_ms_per_run": dense_ms / len(prof), "rounds_ms_per_run": sum(r.round_ms for r in prof) / len(prof),
              "check_ms_per_run": sum(r.check_ms for r in prof) / len(prof),
              "frontier_rows_per_run": prof[0].frontier_rows, "stepped_run_ms": prof[0].device_ms}

    # end to end through the C ABI from pinned host buffers
    hp = [torch.from_numpy(x.view(np.int32)).pin_memory() for x in (g.rowptr, g.colidx, pkg.pack_bits(g.acc))]
    hout = torch.empty(g.n, dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_edges = 0
    for _ in range(args.e2e_steps):
        h2 = pkg.map_create(g.n, hp[0], hp[1], hp[2], stream)
        try:
            r2 = pkg.map_run(h2, sched=args.sched, map_out=hout)
        finally:
            pkg.map_destroy(h2)
        e2e_edges += r2.edges_total
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = None if args.e2e_steps == 0 else {"value": e2e_edges / e2e_s / 1e9 * ws, "unit": "GTEPS",
           "h2d_bytes_per_step": 4 * (g.n + 1) + 4 * g.m + 4 * words, "d2h_bytes_per_step": 4 * g.n,
           "includes": "map_create (H2D, validation, transpose) + map_run + map D2H + map_destroy"}

    line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(WORKLOAD, n=g.n, m=g.m, layers=layers, sched="sync" if args.sched == 0 else "async",
                           outer_iters=r0.outer, rounds_per_run=sum(r0.rounds),
                           relaxations_per_run=r0.relaxations, verdict=r0.verdict,
                           l2="inputs larger than L2 (CSR 1.34 GB vs 129 MB L2); no flush",
                           parallelism="replicas" if ws > 1 else "single GPU"),
            "roofline": roofline, "phases": phases, "e2e": e2e, "gpu_launches": sum(r.launches for r in results),
            "clocks": clk.summary()}
    pkg.map_destroy(h)
    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(g, args.cpu_outer)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
