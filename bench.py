"""Benchmark: CSR edges/s of the threshold random hyperbolic graph generator.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

One step is the whole generator on one graph -- radius solve, sampling, band
structure, degree count, row offsets, neighbour write, row sort -- for the
workload n = 1e8, alpha = 0.55 (gamma = 2.1), kbar = 16, seed 3 with the FP32
filter + FP64 recheck, outputs resident in device memory.  ``value`` is
directed CSR entries (2m) per second over the timed steps.  The plain FP64
path on the same graph, the end-to-end rate through the host-buffer entry
point, the roofline of the dominant kernel, the clocks seen during the timed
region and the CPU oracle's rate on the host cores are reported beside it.

N > 1 (torchrun, one rank per GPU): every rank generates its own graph
(seed 3 + rank) -- independent problems, no data-path collective, weak
scaling.  --impl reference times the CPU oracle (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1501_03545_gb300 import workloads as W  # noqa: E402

METRIC = "CSR edges/sec at n=1e8 (FP32-filter vs plain FP64, same GB300), batched graphs/sec, p50/p99"
UNIT = "edges/s"
WORKLOAD = W.LARGE
# CPU-oracle sample: the same alpha, kbar and seed at a size the host cores
# finish in ~10-30 s (the band algorithm's per-entry cost grows only
# logarithmically with n).
ORACLE_SAMPLE_N = 2_000_000

# DRAM bytes per point of the dominant kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture at n = 4e6, divided by n), keyed by
# the hash of the code it was taken with (comments and whitespace ignored): a
# changed kernel reports null.
NCU_TRAFFIC = {"14e7a3ed74252b58": (313.544448e6 + 367.326976e6) / 4e6}


# Warp instructions of one launch of the dominant kernel at the timed workload
# (smsp__inst_executed.sum of one ncu capture at n = 1e8, a one-pass metric),
# keyed like the traffic record.
NCU_INSTRUCTIONS = {"14e7a3ed74252b58": 13121738271}

# issue slots per second at the maximum SM clock: 152 SMs x 4 schedulers x 2.07 GHz
ISSUE_PEAK = 152 * 4 * 2.07e9


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def code_digest(texts):
    """Hash of C/CUDA sources with comments and whitespace taken out."""
    h = hashlib.sha256()
    for src in texts:
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def source_hash():
    """Digest of the dominant kernel's sources: only a change of the code,
    not of its comments, voids the traffic record."""
    return code_digest(open(os.path.join(ROOT, "paper_1501_03545_gb300", "csrc", f)).read()
                       for f in ("hrg_query.cu", "hrg_common.cuh", "hrg_internal.h"))


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 10:
                    continue
                rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        load = [r for r in rows if (num(r[4]) or 0) >= 50] or rows
        sm = [num(r[1]) for r in load if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in load for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(load)}


def oracle_rate(n=ORACLE_SAMPLE_N):
    """The CPU oracle as it stands (sample + band structure + count + fill),
    timed on this host's cores: directed entries per second."""
    import oracle as O

    w = WORKLOAD
    t0 = time.perf_counter()
    R = O.solve_radius(n, w.alpha, w.kbar)
    r, phi = O.sample(n, w.alpha, R, w.seed)
    b = O.Bands(r, phi, R)
    off, col = b.csr()
    b.close()
    dt = time.perf_counter() - t0
    return {"value": float(off[-1]) / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": "oracle band algorithm, whole pipeline (sample, bands, count, fill) on the same alpha=%g, "
                      "kbar=%g, seed=%d at n=%d: %d entries in %.2f s" % (w.alpha, w.kbar, w.seed, n,
                                                                          int(off[-1]), dt),
            "seconds": dt}


def quadtree_rate(H, ctx, stream, n=500_000):
    """The paper's own generator (Algorithm 1 with the polar quadtree, from
    the oracle package) on the host cores, and the device on the same
    parameters: the 1e6-vertex workload's alpha, kbar and seed at n, where the
    quadtree's Poincare-disk coordinates still resolve (R = 25.1)."""
    import oracle as O
    import torch

    w = W.scaled(W.MEDIUM, n)
    t0 = time.perf_counter()
    R = O.solve_radius(w.n, w.alpha, w.kbar)
    r, phi = O.sample(w.n, w.alpha, R, w.seed)
    off, col, secs = O.quadtree_csr(r, phi, R, w.alpha, 64)
    dt = time.perf_counter() - t0
    ent = int(off[-1])
    del r, phi, off, col
    g = H.generate(ctx, w.n, w.alpha, w.kbar, w.seed, stream=stream)
    gent = g["stats"]["n_entries"]
    del g
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(3):
        g = H.generate(ctx, w.n, w.alpha, w.kbar, w.seed, stream=stream)
        del g
    b.record(stream)
    torch.cuda.synchronize()
    gms = a.elapsed_time(b) / 3
    return {"workload": w.name, "unit": UNIT, "leaf_capacity": 64, "cores": O.num_threads(),
            "cpu_value": ent / dt, "cpu_seconds": dt, "cpu_seconds_build_count_fill": list(secs),
            "cpu_entries": ent, "gpu_value": gent / (gms / 1e3), "gpu_ms": gms, "gpu_entries": gent}


def replica_seed(w, rank):
    """Seed of rank's graph: every rank generates an independent graph of the
    same workload (no data-path collective; the path does not shard)."""
    return w.seed + rank


def reduce_over_ranks(ms, entries, dist, device):
    """Whole-job timing: the slowest rank's timed milliseconds and the entries
    all ranks produced.  dist is None on one process."""
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    e = torch.tensor([float(entries)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


def run_serving(H, device, seconds, slots, rate=W.SERVE_RATE):
    """Replays the serving workload's Poisson arrivals (``rate`` requests/s)
    for `seconds` against an hrg_server; latency = done - submit (server
    clock)."""
    import queue

    reqs = [q for q in W.serving_requests(int(rate * seconds * 1.5) + 16, rate=rate) if q[0] <= seconds]
    srv = H.Server(device, slots=slots)
    try:
        # warm-up: grow every worker's resident workspace to the largest request size
        big = max(reqs, key=lambda q: q[1])
        warm = [srv.submit(big[1], big[2], big[3], big[4]) for _ in range(2 * slots)]
        for t in warm:
            srv.wait(t, timeout_s=300.0)
            srv.release(t)
        base = srv.counters()
        todo = queue.Queue()
        done = []
        lock = threading.Lock()

        def collect():
            while True:
                t = todo.get()
                if t is None:
                    return
                res = srv.wait(t, timeout_s=300.0)
                with lock:
                    done.append((res.status, res.submit_s, res.done_s, res.n_entries, res.batch_size))
                srv.release(t)

        cs = [threading.Thread(target=collect) for _ in range(8)]
        for c in cs:
            c.start()
        t0 = time.perf_counter()
        for (at, n, a, k, sd) in reqs:
            d = t0 + at - time.perf_counter()
            if d > 0:
                time.sleep(d)
            todo.put(srv.submit(n, a, k, sd))
        for _ in cs:
            todo.put(None)
        for c in cs:
            c.join()
        c1 = srv.counters()
    finally:
        srv.close()
    lat = sorted(1e3 * (d - s) for (_, s, d, _, _) in done)
    span = max(d for (_, _, d, _, _) in done) - min(s for (_, s, _, _, _) in done)
    ents = sum(e for (_, _, _, e, _) in done)
    q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))]
    return {"requests": len(done), "failed": sum(1 for x in done if x[0] != 0), "offered_rate_req_s": rate,
            "arrival_seconds": seconds, "span_s": span, "p50_ms": q(0.50), "p99_ms": q(0.99),
            "mean_ms": statistics.mean(lat), "throughput_entries_s": ents / span,
            "throughput_req_s": len(done) / span, "entries": ents,
            "mean_batch": (c1["batched_requests"] - base["batched_requests"]) / max(1, c1["batches"] - base["batches"]),
            "max_running": c1["max_running"], "slots": slots,
            "recipe": "Poisson arrivals at %g req/s, n log-uniform [1e3, 3e7], alpha U[0.55, 1.5], kbar U[4, 32], "
                      "seed 10000 + index, numpy draw seed %d" % (rate, W.SERVE_DRAW_SEED)}


def run_properties(H, ctx, stream, graphs):
    """Sec. 4.1 properties on the device (hrg_graph_props: degree tail
    exponent, triads, triangles, clustering) of freshly generated graphs, and
    Sec. 4.2's random long-range edges (hrg_add_random_edges, 0.5 % of m),
    each timed as the host wall time of the call (after one warm-up call up
    to n = 1e7; the calls return with their results), and the diameter
    bounds of Sec. 4.1 by double sweeps (hrg_diameter_bounds).  graphs:
    (workload, seed, d_min, properties and diameter of the graph with the
    long-range edges too)."""
    import torch

    def timed(f, warm):
        if warm:
            f()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = f()
        return r, (time.perf_counter() - t0) * 1e3

    out = {}
    for w, seed, d_min, lr_props in graphs:
        g = H.generate(ctx, w.n, w.alpha, w.kbar, seed, stream=stream)
        warm = w.n <= 10_000_000
        p, ms = timed(lambda: H.graph_props(ctx, g["row_off"], g["col_idx"], d_min=d_min, stream=stream), warm)
        p["ms"] = ms
        p["gamma_expected"] = 2 * w.alpha + 1
        (lo, hi, _, size), dms = timed(lambda: H.diameter_bounds(ctx, g["row_off"], g["col_idx"], stream=stream),
                                       False)
        p["diameter"] = {"lower": lo, "upper": hi, "component": size, "ms": dms}
        count = -(-p["entries"] // 400)  # ceil(0.005 m), m = entries / 2
        lr, lms = timed(lambda: H.add_random_edges(ctx, g["row_off"], g["col_idx"], count, 99, stream=stream), True)
        del g
        p["long_range"] = {"pairs": count, "added": lr["added"], "ms": lms}
        if lr_props:
            q = H.graph_props(ctx, lr["row_off"], lr["col_idx"], d_min=d_min, stream=stream)
            p["long_range"].update({k: q[k] for k in ("gamma", "triangles", "clustering", "avg_local_clustering")})
            lo, hi, _, size = H.diameter_bounds(ctx, lr["row_off"], lr["col_idx"], stream=stream)
            p["long_range"]["diameter"] = {"lower": lo, "upper": hi, "component": size}
        del lr
        out[w.name] = p
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    steps = []
    for _ in range(args.warmup):
        oracle_rate(args.oracle_n)
    for _ in range(args.steps):
        steps.append(oracle_rate(args.oracle_n))
    secs = sum(s["seconds"] for s in steps)
    entries = sum(s["value"] * s["seconds"] for s in steps)
    val = entries / secs
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD.name, "n": args.oracle_n, "alpha": WORKLOAD.alpha,
                       "kbar": WORKLOAD.kbar, "seed": WORKLOAD.seed, "path": "cpu oracle band algorithm"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": steps[-1]["cores"], "kind": "oracle",
                             "sample": steps[-1]["sample"]},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--update-steps", type=int, default=3, help="timed updates per move count (vertex movement)")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-slots", type=int, default=2)
    ap.add_argument("--oracle-n", type=int, default=ORACLE_SAMPLE_N)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-props", action="store_true", help="skip the graph properties (Sec. 4.1)")
    ap.add_argument("--n", type=int, default=0, help="profiling only: same alpha/kbar/seed at another n")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1501_03545_gb300 import _lib as H

    H.load()
    w = WORKLOAD if args.n <= 0 else W.scaled(WORKLOAD, args.n)
    seed = replica_seed(w, rank)
    ctx = H.Context(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    def step(fp64=False):
        return H.generate(ctx, w.n, w.alpha, w.kbar, seed, fp64_only=fp64, stream=stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    g = None
    for _ in range(max(3, args.warmup)):
        g = step()
        del g
    barrier()
    stats = []
    entries = 0
    with ClockSampler(local) as clk:
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            g = step()
            entries += g["stats"]["n_entries"]
            stats.append(g["stats"])
            del g
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    ms_max, total = reduce_over_ranks(ms, entries, dist, dev)
    value = total / (ms_max / 1e3)
    last = stats[-1]
    n_entries = last["n_entries"]

    # stage times (device, CUDA events on the job stream) averaged over the timed steps
    stage = {k: statistics.mean(s["stage_ms"][k] for s in stats) for k in stats[0]["stage_ms"]}

    # end to end through the host-buffer entry point (D2H of all outputs)
    e2e = None
    if args.e2e_steps > 0:
        n = w.n
        rh = torch.empty(n, dtype=torch.float64, pin_memory=True)
        ph = torch.empty(n, dtype=torch.float64, pin_memory=True)
        oh = torch.empty(n + 1, dtype=torch.int64, pin_memory=True)
        ch = torch.empty(int(n_entries * 1.01) + 1024, dtype=torch.int32, pin_memory=True)
        H.generate_host(ctx, n, w.alpha, w.kbar, seed, rh, ph, oh, ch)
        torch.cuda.synchronize()
        # each step is one call (generation + read-back into pinned host
        # memory, which the host's other tenants share: the spread between
        # steps is reported, the median is the value)
        per, d2h, chunks = [], [], 0
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            ne, hst = H.generate_host(ctx, n, w.alpha, w.kbar, seed, rh, ph, oh, ch)
            per.append(time.perf_counter() - t0)
            d2h.append(hst["d2h_ms"])
            chunks = hst["write_chunks"]
        es = statistics.median(per)
        srt = sorted(per)
        nbytes = int(16 * n + 8 * (n + 1) + 4 * ne)
        # the copies run from the sampler's end to the last range's read-back:
        # d2h_ms is that span on the copy stream, its rate the link's (when
        # the copies, not the generation, set the pace)
        e2e = {"value": ne / es, "unit": UNIT, "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": nbytes, "ms_per_step": 1e3 * es,
               "ms_min": 1e3 * srt[0], "ms_p90": 1e3 * srt[min(len(srt) - 1, int(0.9 * len(srt)))],
               "ms_steps": [round(1e3 * x, 1) for x in per], "statistic": "median over steps",
               "write_chunks": chunks, "d2h_ms_steps": [round(x, 1) for x in d2h],
               "d2h_span_gbs_median": round(nbytes / (statistics.median(d2h) * 1e6), 1) if d2h else None}
        del rh, ph, oh, ch

    # plain FP64 path on the same graph
    fp64 = None
    if args.fp64_steps > 0:
        g = step(fp64=True)
        del g
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.fp64_steps):
            g = step(fp64=True)
            del g
        b.record(stream)
        torch.cuda.synchronize()
        fms = a.elapsed_time(b) / args.fp64_steps
        fp64 = {"value": n_entries / (fms / 1e3), "unit": UNIT, "ms_per_step": fms}

    # vertex movement on the timed graph: k vertices moved (hrg_update_begin),
    # the update's device time against a full generation of the graph
    dynamic = None
    if args.update_steps > 0:
        import numpy as np

        g = step()
        R = g["stats"]["R"]
        r, phi, off, col = g["r"], g["phi"], g["row_off"], g["col_idx"]
        del g
        sel = torch.randint(0, w.n, (1 << 21,), generator=torch.Generator().manual_seed(5), device="cpu")
        sel = torch.unique(sel)
        dynamic = {"recipe": "moves of workloads.moves without radial jumps (75 % small steps, 10 % through phi = 0, "
                             "15 % to the rim) of distinct vertices; device time of begin + finish (CUDA events)",
                   "regenerate_ms": ms_max / args.steps}
        for k in (1000, 100_000):
            times, ents = [], 0
            for rep in range(args.update_steps + 1):
                rs, ps = r[sel.to(dev)].cpu().numpy(), phi[sel.to(dev)].cpu().numpy()
                # no jumps to uniform radii: at n = 1e8 each such vertex would see ~5e6 others
                ids, rn, pn = W.moves(rs, ps, R, k, 1000 * k + rep, jumps=0.0)
                ids = sel.numpy()[ids].astype(np.int32)
                ti, tr, tp = torch.tensor(ids), torch.tensor(rn), torch.tensor(pn)
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                u = H.update_points(ctx, r, phi, off, col, R, ti, tr, tp, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                if rep > 0:
                    times.append(a.elapsed_time(b))
                ents = u["stats"]["n_entries"]
                off, col = u["row_off"], u["col_idx"]
                del u
            t = statistics.median(times)
            dynamic["k%d" % k] = {"ms": t, "entries": ents, "vs_regenerate": t / dynamic["regenerate_ms"]}
        del r, phi, off, col

    # the batched workload: 4096 small graphs per call, with the band width and
    # hub threshold of each size class picked by the tuner (untimed), and with
    # the defaults
    batched = None
    if args.batch_steps > 0:
        from paper_1501_03545_gb300 import autotune

        items = W.batch_items()
        table = autotune.tune(ctx, items, stream=stream)
        tuned = H.BatchItems(autotune.apply(items, table))
        untuned = H.BatchItems(items)

        def time_batch(its):
            g = H.generate_batch(ctx, its, stream=stream)
            del g
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ent = 0
            for _ in range(args.batch_steps):
                g = H.generate_batch(ctx, its, stream=stream)
                ent = g["stats"]["n_entries"]
                nl = g["stats"]["launches"]
                del g
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / args.batch_steps, ent, nl

        bms, bent, bl = time_batch(tuned)
        dms, _, _ = time_batch(untuned)
        batched = {"graphs_per_s": len(items) / (bms / 1e3), "entries_per_s": bent / (bms / 1e3),
                   "ms_per_batch": bms, "graphs": len(items), "sum_n": sum(it[0] for it in items),
                   "entries_per_batch": bent, "launches_per_batch": bl,
                   "untuned_ms_per_batch": dms,
                   "tuned": {str(k): {"band_width": v[0], "hub_candidates": v[1]} for k, v in table.items()},
                   "recipe": "n log-uniform [1e3, 1e5], alpha U[0.55, 1.5], kbar from {4, 8, 16, 32}, seeds "
                             "1000..%d, parameters drawn with numpy seed %d" % (999 + len(items),
                                                                                 W.BATCH_DRAW_SEED)}

    # serving: Poisson arrivals of mixed requests, continuous batching
    serving = None
    serving_x3 = None
    if args.serve_seconds > 0 and rank == 0:
        serving = run_serving(H, local, args.serve_seconds, args.serve_slots)
        # the same mix at three times the rate (near the device's capacity):
        # requests wait for each other, so batches form
        serving_x3 = run_serving(H, local, min(3.0, args.serve_seconds), args.serve_slots, rate=3 * W.SERVE_RATE)

    # graph properties of Sec. 4.1 and the random long-range edges of Sec. 4.2
    # on the device: the 1e6-vertex workload (the size of the paper's property
    # study) and the timed graph
    props = None
    if not args.no_props and rank == 0:
        gamma3 = W.Workload("rhg_n2e5_a1.0_k10", 200_000, 1.0, 10.0, 4)  # gamma = 3, average degree 10
        props = run_properties(H, ctx, stream, [(W.MEDIUM, W.MEDIUM.seed, 30, True), (gamma3, gamma3.seed, 30, True),
                                                (w, seed, 48, False)])

    # roofline of the dominant kernel: the rim count pass (k_rim_sector), one
    # launch per graph, timed by the library's CUDA events around exactly that
    # launch on the job stream
    peak, peak_kind = peaks()
    n = w.n
    stage["count"] = stage["count_hub"] + stage["count_rim"]
    stage["write"] = stage["write_hub"] + stage["write_rim"]
    # algorithmic bytes per launch: the band structure read once (fixed-point
    # angle 8 B + FP32 {P, M, S, id} 16 B per point) and the degree written (4 B)
    algo = 28 * n
    achieved = algo / (stage["count_rim"] / 1e3) / 1e9
    traffic = NCU_TRAFFIC.get(source_hash())
    roof = {"bound": "hbm", "kernel": "k_rim_sector (rim count pass)", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind, "algorithmic_bytes": algo,
            "ms_per_launch": stage["count_rim"],
            "traffic": None if traffic is None else traffic * n,
            "query_csr_roofline": {
                "bytes": 4 * n_entries + 8 * (n + 1) + 2 * 16 * n,
                "ms": stage["count"] + stage["offsets"] + stage["write"] + stage["rowsort"]}}
    qc = roof["query_csr_roofline"]
    qc["frac"] = qc["bytes"] / (qc["ms"] / 1e3) / 1e9 / peak
    # its instruction-issue rate against the issue roof (the pass is far from
    # the HBM roof: a few per cent of DRAM throughput)
    inst = NCU_INSTRUCTIONS.get(source_hash()) if w.n == WORKLOAD.n else None
    roof["issue_roof"] = None if inst is None else {
        "warp_instructions": inst, "achieved": inst / (stage["count_rim"] / 1e3), "peak": ISSUE_PEAK,
        "unit": "warp instructions/s", "frac": inst / (stage["count_rim"] / 1e3) / ISSUE_PEAK,
        "peak_kind": "152 SMs x 4 schedulers x 2.07 GHz (maximum SM clock)"}

    cpu = quadtree = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_rate(args.oracle_n)
        cpu.pop("seconds", None)
        quadtree = quadtree_rate(H, ctx, stream)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64recheck", "data": "synthetic",
                "config": {"workload": w.name, "n": w.n, "alpha": w.alpha, "kbar": w.kbar, "seed": w.seed,
                           "path": "fp32 filter + fp64 recheck", "entries_per_step": n_entries,
                           "undirected_edges_per_s": value / 2,
                           "l2": "no flush: every step writes and reads >8 GB, far above the 126 MB L2"},
                "e2e": e2e, "roofline": roof, "clocks": clocks, "cpu_baseline": cpu,
                "gpu_launches": last.get("launches", 0) * args.steps, "ties": last["ties"],
                "fp64_plain": fp64, "batched": batched, "serving": serving, "serving_x3": serving_x3,
                "dynamic": dynamic, "stage_ms": stage,
                "paper_quadtree": quadtree,
                "job": {k: last[k] for k in ("R", "candidates", "rechecks", "ties", "bands", "hub_bands", "buckets",
                                             "hub_queries", "mid_rows", "big_rows", "mu", "rows_no_room",
                                             "hub_rows_retraversed", "heavy_retries")},
                "properties": props,
                # last, so that the end of the line carries the other workloads' figures
                "summary": {"ms_per_step": round(ms_max / args.steps, 2), "ties": last["ties"],
                            "fp64_plain_ms": fp64 and round(fp64["ms_per_step"], 2),
                            "fp32_vs_fp64": fp64 and round(fp64["ms_per_step"] / (ms_max / args.steps), 2),
                            "e2e_ms_median": e2e and round(e2e["ms_per_step"], 1),
                            "batched_graphs_per_s": batched and round(batched["graphs_per_s"]),
                            "batched_ms": batched and round(batched["ms_per_batch"], 2),
                            "serving_p50_ms": serving and round(serving["p50_ms"], 2),
                            "serving_p99_ms": serving and round(serving["p99_ms"], 2),
                            "serving_mean_batch": serving and round(serving["mean_batch"], 2),
                            "serving_x3_p50_ms": serving_x3 and round(serving_x3["p50_ms"], 2),
                            "serving_x3_p99_ms": serving_x3 and round(serving_x3["p99_ms"], 2),
                            "serving_x3_mean_batch": serving_x3 and round(serving_x3["mean_batch"], 2),
                            "update_k1000_ms": dynamic and round(dynamic["k1000"]["ms"], 2),
                            "update_k100000_ms": dynamic and round(dynamic["k100000"]["ms"], 2),
                            "rim_count_frac_of_hbm": round(roof["frac"], 4)}}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
