"""Benchmark of the MAP hot path on GB300: GTEPS + fraction of the HBM roofline.

One step = one full MAP run (every outer iteration: dense round, frontier rounds to the
fix-point, self-map test, elimination) over the 2^26-vertex layered no-cycle graph
(4,000 layers, geometric out-degree with mean 4, 92 % forward edges, back edges over 50
layers, 1 % accepting, accepting vertices on no cycle), inputs resident in HBM.

    metric  MAP edge relaxations/s, GTEPS = (m x outer iterations) / device time of K runs queued
            back to back in one call (map_opts.repeat)
            (every fix-point examines every edge at least once), timed on the asynchronous
            in-place schedule (same maps, verdict and outer count as the synchronous one, which
            is timed after it and reported as `other_schedule` with its canonical counts)
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
import faulthandler
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


# DRAM traffic of one k_dense launch, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of a sparse-write launch (outer iteration 4, 4 loads in flight per lane)
# on the layered graph of 2^24 vertices (1,000 layers, m = 67,111,361), whose algorithmic bytes
# are 339,748,616: 342.05 MB read + 8.77 MB written = 350.8 MB, 1.03 x the algorithmic bytes.
# Valid only for the kernel source it was taken on (a hash of the dense-round section of the
# kernel file, which holds k_dense and its helpers).
DENSE_TRAFFIC = {"dense_section_sha256_16": "adcfe7b01e8bba66", "bytes": 350_819_328,
                 "algorithmic_bytes": 339_748_616, "case": "layered 2^24 vertices, m = 67,111,361, outer iteration 4"}


def _dense_traffic(dense_bytes):
    import hashlib

    path = os.path.join(ROOT, "paper_0912_2555_gb300", "csrc", "map_kernels.cuh")
    try:
        text = open(path, "rb").read()
    except OSError:
        return None, "kernel source not found"
    # the kernel's source: the dense-round section of the file (k_dense and its helpers)
    a = text.find(b"// ------------------------------------------------------------ dense round --")
    b = text.find(b"// ------------------------------------------------------------ push rounds --")
    sha = hashlib.sha256(text[a:b] if 0 <= a < b else text).hexdigest()[:16]
    if sha != DENSE_TRAFFIC["dense_section_sha256_16"]:
        return None, "kernel changed since the ncu capture"
    scale = dense_bytes / DENSE_TRAFFIC["algorithmic_bytes"]
    return DENSE_TRAFFIC["bytes"] * scale, (f"ncu capture on {DENSE_TRAFFIC['case']}, scaled by the ratio of "
                                             f"algorithmic bytes ({scale:.3f})")


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling (SM clock, throttle reasons) every period_ms.  The sampler starts before the
    warm-up (it needs a moment to start); mark_start() / mark_end() bracket the timed region, and
    summary() keeps the samples stamped inside it (the nearest one if the region is shorter than
    the sampling interval)."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: int = 200):
        self.index = index
        self.period_ms = period_ms  # (nvidia-smi's queries take driver locks: sample no faster than needed)
        self.proc = None
        self.t_start = self.t_end = None

    def mark_start(self):
        import datetime

        self.t_start = datetime.datetime.now()

    def mark_end(self):
        import datetime

        self.t_end = datetime.datetime.now()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.period_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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

    def stamps(self):
        """The time stamp of every sample taken (nvidia-smi's own, host clock)."""
        import datetime

        out = []
        for line in getattr(self, "lines", []):
            try:
                out.append(datetime.datetime.strptime(line.split(",")[0].strip(), "%Y/%m/%d %H:%M:%S.%f"))
            except ValueError:
                continue
        return out

    def summary(self):
        import datetime

        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []  # (time, sm MHz, max MHz, reasons)
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                t = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                t = None  # an unexpected time format: no filtering by time
            try:
                rows.append((t, float(f[1]), float(f[2]), {nm for nm, val in zip(names, f[5:9])
                                                          if val.lower().startswith("active")}))
            except ValueError:
                continue
        window = "timed region"
        sel = rows
        if any(r[0] is None for r in rows):
            window = "whole sampling (no time stamps)"
        elif self.t_start is not None and self.t_end is not None and rows:
            sel = [r for r in rows if self.t_start <= r[0] <= self.t_end]
            if not sel:  # a region shorter than the interval: the sample nearest to it
                mid = self.t_start + (self.t_end - self.t_start) / 2
                sel = [min(rows, key=lambda r: abs((r[0] - mid).total_seconds()))]
                window = "nearest sample"
        reasons = set().union(*[r[3] for r in sel]) if sel else set()
        return {"sm_mhz": statistics.median([r[1] for r in sel]) if sel else None,
                "sm_max_mhz": sel[-1][2] if sel else None, "reasons": sorted(reasons), "samples": len(sel),
                "window": window}


def queries_per_window(stamps, windows, lead_ms=50):
    """For each (start, end) window: the clock samples stamped inside it or up to lead_ms before
    its start (a query holds driver locks while it runs, so one that began just before a window
    can still stall a CUDA call inside it)."""
    import datetime

    lead = datetime.timedelta(milliseconds=lead_ms)
    return [sum(1 for t in stamps if a - lead <= t <= b) for a, b in windows]


def replica_value(ms, edges, device="cuda"):
    """Whole-job GTEPS of independent replicas (one per rank): the edges all ranks processed
    over the slowest rank's time.  Returns (GTEPS, slowest ms, total edges)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        import torch

        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e = torch.tensor([float(edges)], dtype=torch.float64, device=device)
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
        ms, edges = float(t.item()), float(e.item())
    return edges / (ms / 1e3) / 1e9, ms, edges


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(g, layers=None):
    """The workload both arms time: the graph recipe and its size (nothing measured)."""
    return dict(WORKLOAD, n=g.n, m=g.m, layers=layers or WORKLOAD["layers"],
                l2="inputs larger than L2 (CSR 1.34 GB vs 129 MB L2); no flush")


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
            "data": "synthetic",
            "config": workload_config(g),
            "run": {"impl": "CPU oracle (synchronous rounds)", "placement": "host, 1 thread"},
            "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
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
    return {"value": g.m * r.outer / dt / 1e9, "unit": "GTEPS", "cores": 1, "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"first {r.outer} outer iterations of the same graph ({dt:.1f} s, single thread, "
                      f"including the oracle's own set-up)"}


def doubling_bytes(n, rounds):
    """Algorithmic bytes of the pointer-doubling fix-point of one run (one entry per row at most):
    per outer iteration an initial pass (rowptr 4(n+1), the entries 4n at most, the dense round's
    values 4n read, the 8-byte (value, pointer) pairs 8n written: 20n) and, for each of its
    rounds after the dense one, a pass that reads the pairs (8n), gathers one pair per vertex (8n)
    and writes the next pairs (8n): 24n.  An outer iteration whose dense round gave no vertex a
    value (one round) makes no pass at all.  rounds: the run's rounds per outer iteration."""
    return sum(20 * n + 24 * n * (k - 1) for k in rounds if k > 1)


def configs_leg(pkg, np, torch, stream, peak, steps=10):
    """The two other single-graph workloads, resident in HBM, both schedules: the 16,384-vertex
    random graph (both variants; latency-bound, reported in microseconds per run) and the
    8 x 7 lock-step process product (2 x 7^8 vertices; GTEPS, and the run against the HBM roofline:
    one minimal pass over the matrix per outer iteration -- rowptr 4(n + 1), colidx 4m and one
    4-byte gather per edge -- over the run time)."""
    import mapgen

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(g):
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
        h = pkg.map_create(g.n, dev(g.rowptr), dev(g.colidx), dev(pkg.pack_bits(g.acc)), stream)
        out = {}
        try:
            for sched, name in ((1, "async"), (0, "sync")):
                # this graph's run choices for this schedule, by measurement (the start included)
                out[f"autotune_{name}"] = pkg.map_autotune(h, sched)
                for _ in range(3):
                    r = pkg.map_run(h, sched=sched)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(steps):
                    r = pkg.map_run(h, sched=sched)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / steps
                alg = (4 * (g.n + 1) + 8 * g.m) * r.outer
                out[name] = {"us_per_run": ms * 1e3, "gteps": g.m * r.outer / (ms / 1e3) / 1e9,
                             "verdict": r.verdict, "witness": r.witness, "outer": r.outer,
                             "rounds": sum(r.rounds), "relaxations": r.relaxations,
                             "phases_ms": {"dense": r.dense_ms, "rounds": r.round_ms, "check": r.check_ms},
                             "roofline": {"bytes_per_run": alg, "achieved_gbs": alg / (ms / 1e3) / 1e9,
                                          "peak_gbs": peak, "frac": alg / (ms / 1e3) / 1e9 / peak}}
                # a graph whose rows hold one entry at most, asynchronous with the dense start: the
                # fix-point is pointer doubling (k_func); its own roofline from a host-stepped run
                # with CUDA events around each launch
                if sched == 1 and g.m and int(np.diff(g.rowptr).max()) <= 1:
                    rp = pkg.map_run(h, sched=sched, flags=pkg.MAP_FLAG_PROFILE)
                    if rp.dense_ms > 0 and rp.round_ms > 0:
                        b = doubling_bytes(g.n, rp.rounds)
                        out[name]["doubling_roofline"] = {
                            "kernel": "k_func", "passes": [k - 1 for k in rp.rounds], "bytes_per_run": b,
                            "ms_per_run": rp.round_ms, "achieved_gbs": b / (rp.round_ms / 1e3) / 1e9,
                            "peak_gbs": peak, "frac": b / (rp.round_ms / 1e3) / 1e9 / peak,
                            "timing": "CUDA events around the fix-point launch of a host-stepped run"}
        finally:
            pkg.map_destroy(h)
        return out

    res = {}
    for variant in ("cycle", "nocycle"):
        g = mapgen.random_16k(variant)
        res[f"random-16k-{variant}"] = dict(n=g.n, m=g.m, **timed(g))
    g = mapgen.product_8x7()
    res["product-8x7"] = dict(n=g.n, m=g.m, **timed(g))
    return res


def batched_leg(pkg, np, torch, stream, count=256, steps=2):
    """256 graphs (sizes log-uniform in [1e3, 2e6], 40 % with a planted accepting cycle, layered
    recipe) in one batched run, against the same 256 graphs run one after another with map_run,
    under both schedules: the asynchronous one (the headline's) and the synchronous one, whose
    canonical round and relaxation counts are compared too.  For each schedule map_autotune picks
    the batch's run choices (start included) first; the one-by-one runs use the same start.
    Inputs resident in HBM in both legs; device time by CUDA events; jobs/s = graphs / time."""
    import mapgen

    sizes, planted, seeds = mapgen.batch_plan(count=count, lo=1000, hi=2_000_000, frac_cycle=0.4, seed=4)
    gs = [mapgen.batch_graph(int(sz), bool(p), int(sd)) for sz, p, sd in zip(sizes, planted, seeds)]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    items = [(g.n, dev(g.rowptr), dev(g.colidx), dev(pkg.pack_bits(g.acc))) for g in gs]
    hb = pkg.map_batch_create(items, stream)
    singles = [pkg.map_create(it[0], it[1], it[2], it[3], stream) for it in items]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": f"{count} layered graphs, n log-uniform in [1e3, 2e6], 40 % planted cycles, seed 4",
           "vertices": int(sum(g.n for g in gs)), "edges": int(sum(g.m for g in gs))}
    try:
        for sched, name in ((1, "async"), (0, "sync")):
            t_tune = time.perf_counter()
            tune = pkg.map_autotune(hb, sched)  # this batch's run choices, by measurement
            t_tune = time.perf_counter() - t_tune
            res = pkg.map_batch_run(hb, count, sched=sched)  # warm-up (builds the graph)
            sflags = pkg.MAP_FLAG_FRONTIER_START if tune["frontier_start"] else pkg.MAP_FLAG_DENSE_START
            for h in singles:
                pkg.map_run(h, sched=sched, flags=sflags)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(steps):
                res = pkg.map_batch_run(hb, count, sched=sched)
            e1.record(stream)
            torch.cuda.synchronize()
            batch_ms = e0.elapsed_time(e1) / steps
            e0.record(stream)
            seq = None
            for _ in range(steps):
                seq = [pkg.map_run(h, sched=sched, flags=sflags) for h in singles]
            e1.record(stream)
            torch.cuda.synchronize()
            seq_ms = e0.elapsed_time(e1) / steps
            key = lambda r: (r.verdict, r.witness, r.outer) + ((tuple(r.rounds), r.relaxations) if sched == 0 else ())
            same = all(key(a) == key(b) for a, b in zip(res, seq))
            edges = sum(r.edges_total for r in res)
            out[name] = {"cycles_found": int(sum(r.verdict for r in res)), "batch_ms": batch_ms, "sequential_ms": seq_ms,
                         "jobs_per_s_batched": count / (batch_ms / 1e3),
                         "jobs_per_s_sequential": count / (seq_ms / 1e3), "speedup": seq_ms / batch_ms,
                         "gteps_batched": edges / (batch_ms / 1e3) / 1e9,
                         "start": "frontier" if tune["frontier_start"] else "dense",
                         "results_identical": bool(same),
                         "compared": "verdict, witness, outer" + (", rounds, relaxations" if sched == 0 else ""),
                         "autotune": dict(tune, seconds=t_tune)}
    finally:
        pkg.map_destroy(hb)
        for h in singles:
            pkg.map_destroy(h)
    # the headline schedule's figures at the top level
    out.update({k: out["async"][k] for k in ("batch_ms", "sequential_ms", "jobs_per_s_batched", "jobs_per_s_sequential",
                                           "speedup", "gteps_batched", "results_identical")})
    out["sched"] = "async"
    return out


def serving_leg(pkg, np, rates=(50, 100, 200, 500, 1000, 2000), jobs=2000, max_arrival_s=12.0, slots=8):
    """Poisson arrivals of verification jobs (sizes lognormal, median 1e5, sigma 1.5, within
    [1e3, 1e7]; half process products with 4-9 processes of 5-7 states, half layered graphs),
    served with continuous admission and batching by `slots` workers (the jobs queued behind the
    one a worker takes share its run), against the same schedule served one job at a time in
    arrival order (one worker, no batching), and, at the rates where jobs queue up, against
    `slots` workers running one job each (no batching).  All serve every job on the asynchronous schedule
    (same verdict, witness, outer count and map as the synchronous one).  Latency = submission to
    result, end to end (copy to the device, set-up, run, map back), split per job into the wait
    for a worker, map_create and the run with the map's copy back.  `jobs` arrivals per rate, but
    no more than `max_arrival_s` seconds of arrivals (so the bench stays within minutes: 600 and
    1,200 jobs at 50 and 100 per second).  The graphs are generated before the clock starts."""
    import threading
    from concurrent.futures import ThreadPoolExecutor

    import mapgen

    arr = mapgen.arrivals(jobs, 1.0, seed=5)  # times at rate 1/s; scaled per rate below
    with ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:  # the generator releases the GIL
        graphs = list(ex.map(lambda i: mapgen.arrival_graph(arr, i), range(jobs)))
    bits = [pkg.pack_bits(g.acc) for g in graphs]

    def serve(rate, nslots, max_batch=0):
        t_arr = arr["t"] / rate
        k = int(min(jobs, max(1, np.searchsorted(t_arr, max_arrival_s))))
        sub, done = [0.0] * k, [None] * k
        ids, res = [None] * k, [None] * k
        with pkg.Server(slots=nslots, max_batch=max_batch) as sv:
            t0 = time.perf_counter()

            def submitter():
                for i in range(k):
                    wait = t0 + t_arr[i] - time.perf_counter()
                    if wait > 0:
                        time.sleep(wait)
                    g = graphs[i]
                    sub[i] = time.perf_counter()
                    ids[i] = sv.submit(g.n, g.rowptr, g.colidx, bits[i], sched=pkg.MAP_SCHED_ASYNC)

            th = threading.Thread(target=submitter)
            th.start()
            left = set(range(k))
            while left:
                for i in list(left):
                    if ids[i] is None:
                        continue
                    got = sv.poll(ids[i], want_map=False)
                    if got is not None:
                        done[i] = time.perf_counter()
                        res[i] = got[0]
                        left.discard(i)
                time.sleep(0.0002)
            th.join()
        lat = np.array([d - s0 for d, s0 in zip(done, sub)]) * 1e3
        span = max(done) - t0

        def pct(x):
            x = np.asarray(x)
            return {"p50": float(np.percentile(x, 50)), "p99": float(np.percentile(x, 99))}

        return {"jobs": k, "jobs_per_s": k / span, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "jobs_per_run_mean": float(np.mean([r.batch_jobs for r in res])),
                "jobs_per_run_max": int(max(r.batch_jobs for r in res)),
                "phases_ms": {"wait_for_worker": pct([r.queue_ms for r in res]),
                              "map_create": pct([r.setup_ms for r in res]),
                              "run_and_map_back": pct([r.run_ms for r in res])}}

    out = {"workload": f"up to {jobs} jobs per rate ({max_arrival_s:.0f} s of arrivals at most), lognormal sizes "
                       "(median 1e5, sigma 1.5, [1e3, 1e7]), half process products, half layered graphs, seed 5, "
                       "asynchronous schedule",
           "vertices": int(sum(g.n for g in graphs)), "slots": slots, "rates": {}}
    for rate in rates:
        r = {"continuous": serve(rate, slots), "fifo_one_at_a_time": serve(rate, 1, max_batch=1)}
        if rate >= 500:
            r["continuous_no_batching"] = serve(rate, slots, max_batch=1)
        out["rates"][str(rate)] = r
    return out


def main():
    faulthandler.enable()  # a fatal signal prints every thread's Python stack
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--sched", type=int, default=1,
                    help="timed schedule: 1 = asynchronous in-place sweeps (default), 0 = synchronous rounds; "
                         "the other schedule is timed after it and reported beside it")
    ap.add_argument("--cpu-outer", type=int, default=3, help="outer iterations in the CPU-oracle sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--n", type=int, default=None, help="override vertex count (smaller runs, not the bench line)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched leg (256 graphs)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg (Poisson arrivals)")
    ap.add_argument("--no-tune", action="store_true", help="skip map_autotune on the bench graph (library defaults)")
    ap.add_argument("--start", default="dense", choices=["dense", "frontier"],
                    help="round 1 of every outer iteration: the dense round over the whole matrix (default, the "
                         "headline) or MAP_FLAG_FRONTIER_START on every step (profiling that path; no dense roofline)")
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
    # the handle's run choices by measurement on this graph (pull threshold, block-local passes,
    # one-block rounds, launch shapes, dense-round loads in flight); the start stays the one asked
    # for (the headline streams the whole matrix in every outer iteration)
    t_tune = time.perf_counter()
    tune = pkg.map_autotune(h, args.sched) if not args.no_tune else None
    t_tune = time.perf_counter() - t_tune

    start_flags = pkg.MAP_FLAG_FRONTIER_START if args.start == "frontier" else pkg.MAP_FLAG_DENSE_START

    def step(flags=0, repeat=0):
        return pkg.map_run(h, sched=args.sched, flags=flags | start_flags, map_out=out, repeat=repeat)

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    results = []
    with Clocks(local) as clk:
        # warm-up: at least W steps, and at least 0.4 s so that the clock sampler is running
        t_w = time.perf_counter()
        for _ in range(max(args.warmup, 3)):
            r0 = step()
        while time.perf_counter() - t_w < 0.4:
            step()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk.mark_start()
        e0.record(stream)
        # the K steps queued back to back in one call (map_opts.repeat): no host step between runs
        rk = step(repeat=args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
        results = [rk] * args.steps  # (every run of the K gives the same result; rk is the last)
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    value, ms, _ = replica_value(ms, sum(r.edges_total for r in results), device="cuda")

    # the other schedule on the same graph and steps, reported beside the headline (both give the
    # same maps, verdict and outer count; only the synchronous one has the canonical round counts)
    other = 1 - args.sched
    for _ in range(3):
        pkg.map_run(h, sched=other, flags=start_flags, map_out=out)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    ores = [pkg.map_run(h, sched=other, flags=start_flags, map_out=out, repeat=args.steps)] * args.steps
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ovalue, oms, _ = replica_value(e0.elapsed_time(e1), sum(r.edges_total for r in ores), device="cuda")
    other_line = {"sched": "sync" if other == 0 else "async", "value": ovalue, "unit": "GTEPS",
                  "ms_per_step": oms / args.steps, "rounds_per_run": sum(ores[0].rounds),
                  "relaxations_per_run": ores[0].relaxations,
                  "work_ratio": ores[0].relaxations / (g.m * ores[0].outer) if ores[0].outer else None,
                  "canonical_counts": bool(ores[0].inner_canonical),
                  "same_result": (ores[0].verdict, ores[0].witness, ores[0].outer) == (r0.verdict, r0.witness,
                                                                                       r0.outer)}

    # round 1 pushed from the accepting vertices (MAP_FLAG_FRONTIER_START) instead of the dense
    # round: the same maps, verdict and outer count from far fewer edges when the accepting set is
    # small.  Reported beside the headline as time and pushes per run: it does not examine every
    # edge in every outer iteration, so m x outer / time would not be an edge rate.
    fs = pkg.MAP_FLAG_FRONTIER_START

    def fstep(repeat=0):
        return pkg.map_run(h, sched=args.sched, flags=fs, map_out=out, repeat=repeat)

    for _ in range(3):
        fstep()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    fres = [fstep(repeat=args.steps)] * args.steps
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    fms = e0.elapsed_time(e1) / args.steps
    frontier_line = {"flag": "MAP_FLAG_FRONTIER_START", "sched": "sync" if args.sched == 0 else "async",
                     "ms_per_run": fms, "headline_ms_per_run": ms / args.steps,
                     "relaxations_per_run": fres[0].relaxations,
                     "relaxations_are": "pushes made" if args.sched == 1 else "canonical count of the synchronous schedule",
                     "sweeps_per_run": sum(fres[0].rounds),
                     "same_result": (fres[0].verdict, fres[0].witness, fres[0].outer) == (r0.verdict, r0.witness,
                                                                                          r0.outer)}

    # roofline of the dominant kernel (the dense round): algorithmic bytes per launch over its
    # CUDA-event time.  Events cannot sit inside the graph's loop bodies, so this pass runs
    # the same kernels stepped from the host, with events around every dense launch.
    prof = [step(pkg.MAP_FLAG_PROFILE) for _ in range(2)]
    dense_launches = sum(r.dense_launches for r in prof)
    dense_ms = sum(r.dense_ms for r in prof)
    # algorithmic bytes of one run's dense launches: every launch streams rowptr + colidx (flags in
    # bit 31) and writes the stale bitmap (n / 8); the first also writes every map value (4n), the
    # later ones read the bitmap (n / 8) and write only the rows that get or lose a value (not
    # counted: a lower bound, about 1 % of the rows on this graph)
    outer = prof[0].outer
    words = (g.n + 31) // 32
    stream_bytes = 4 * (g.n + 1) + 4 * g.m + g.n // 8
    run_dense_bytes = outer * stream_bytes + 4 * g.n + (outer - 1) * (g.n // 8)
    dense_bytes = run_dense_bytes / outer  # average per launch
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = dense_bytes * dense_launches / (dense_ms / 1e3) / 1e9 if dense_ms > 0 else None
    traffic, traffic_note = _dense_traffic(dense_bytes)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic, "traffic_note": traffic_note,
                "kernel": "k_dense (round 1 of each outer iteration)", "bytes_per_launch": dense_bytes,
                "launch_ms": dense_ms / max(dense_launches, 1),
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s",
                "share_of_step": (dense_ms / len(prof)) / (ms / args.steps) if ms else None,
                "timing": "CUDA events around each dense launch in 2 extra host-stepped runs"}
    # the whole run against the same peak: the dense launches' bytes (push rounds and checks add
    # scattered traffic that is not counted) over the timed run
    run_ms = ms / args.steps
    run_roofline = {"bytes_per_run": run_dense_bytes, "ms_per_run": run_ms,
                    "achieved": run_dense_bytes / (run_ms / 1e3) / 1e9 if run_ms else None, "peak": peak,
                    "unit": "GB/s", "frac": run_dense_bytes / (run_ms / 1e3) / 1e9 / peak if run_ms else None,
                    "counted": "dense-round bytes only"}
    # the timed runs' own phases: the kernels stamp %globaltimer at the end of every dense round,
    # fix-point loop and elimination (each phase runs from the end of the one before it)
    k = len(results)
    phases = {"dense_ms_per_run": sum(r.dense_ms for r in results) / k,
              "rounds_ms_per_run": sum(r.round_ms for r in results) / k,
              "check_ms_per_run": sum(r.check_ms for r in results) / k,
              "frontier_rows_per_run": results[0].frontier_rows,
              "source": "device %globaltimer stamps inside the timed graph runs",
              "stepped_events": {"dense_ms_per_run": dense_ms / len(prof),
                                 "rounds_ms_per_run": sum(r.round_ms for r in prof) / len(prof),
                                 "check_ms_per_run": sum(r.check_ms for r in prof) / len(prof),
                                 "run_ms": prof[0].device_ms,
                                 "source": "CUDA events around each launch of 2 host-stepped runs"}}

    # end to end through the C ABI from pinned host buffers, with the bench graph's handle gone
    # (one graph's work space in the device memory pool, as for a caller running one job at a time)
    pkg.map_destroy(h)
    hp = [torch.from_numpy(x.view(np.int32)).pin_memory() for x in (g.rowptr, g.colidx, pkg.pack_bits(g.acc))]
    hout = torch.empty(g.n, dtype=torch.int32).pin_memory()

    e2e_split = []  # host time of each call of each step (ms): create, run, destroy

    def e2e_step():
        t0 = time.perf_counter()
        h2 = pkg.map_create(g.n, hp[0], hp[1], hp[2], stream)
        t1 = time.perf_counter()
        try:
            r = pkg.map_run(h2, sched=args.sched, flags=start_flags, map_out=hout)
        finally:
            t2 = time.perf_counter()
            pkg.map_destroy(h2)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            e2e_split.append({"map_create": (t1 - t0) * 1e3, "map_run": (t2 - t1) * 1e3, "map_destroy": (t3 - t2) * 1e3,
                              "run_device_ms": None})
        e2e_split[-1]["run_device_ms"] = r.device_ms
        return r

    # each step timed on its own (host clock, device synchronised on both sides); the value is
    # taken at the median step, so that one step stalled on the host does not decide it, and
    # every step's time is reported with it
    import datetime

    e2e_ms, e2e_edges, e2e_win = [], 0, []
    with Clocks(local, period_ms=500) as e2e_clk:
        for _ in range(2 if args.e2e_steps else 0):
            e2e_step()  # warm-up: the device memory pool and the pinned control slots reach their size
        e2e_clk.mark_start()
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            w0 = datetime.datetime.now()
            t0 = time.perf_counter()
            e2e_edges = e2e_step().edges_total
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            e2e_win.append((w0, datetime.datetime.now()))
        e2e_clk.mark_end()
    e2e = None
    if args.e2e_steps:
        # clock queries that began in a step or up to 50 ms before it: a query holds driver locks
        # while it runs, and a CUDA call that meets one waits
        queries = queries_per_window(e2e_clk.stamps(), e2e_win, lead_ms=50)
        med = float(np.median(e2e_ms))
        e2e = {"value": e2e_edges / (med / 1e3) / 1e9 * ws, "unit": "GTEPS",
               "h2d_bytes_per_step": 4 * (g.n + 1) + 4 * g.m + 4 * words, "d2h_bytes_per_step": 4 * g.n,
               "ms_per_step_median": med, "ms_per_step": e2e_ms, "value_from": "median step",
               "calls_ms": e2e_split[-args.e2e_steps:],
               "clock_queries_per_step": queries,
               "clocks": e2e_clk.summary(),
               "includes": "map_create (H2D, validation, transpose) + map_run + map D2H + map_destroy"}

    line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(g, layers),
            "run": {"sched": "sync" if args.sched == 0 else "async", "start": args.start, "outer_iters": r0.outer,
                    "rounds_per_run": sum(r0.rounds), "relaxations_per_run": r0.relaxations,
                    # relaxations executed / (m x outer iterations): the edges the run examined per edge
                    # the metric counts (asynchronous: every push counted as one)
                    "work_ratio": r0.relaxations / (g.m * r0.outer) if r0.outer else None, "verdict": r0.verdict,
                    "placement": "replicas, one per GPU" if ws > 1 else "single GPU"},
            "roofline": roofline, "run_roofline": run_roofline, "phases": phases, "e2e": e2e,
            "other_schedule": other_line, "frontier_start": frontier_line,
            "autotune": dict(tune, seconds=t_tune) if tune else None,
            "gpu_launches": sum(r.launches for r in results),
            "clocks": clk.summary()}
    if not args.no_batch and args.n is None and ws == 1:
        line["configs"] = configs_leg(pkg, np, torch, stream, peak)
        line["batched"] = batched_leg(pkg, np, torch, stream)
    if not args.no_serve and args.n is None and ws == 1:
        line["serving"] = serving_leg(pkg, np)
    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(g, args.cpu_outer)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
