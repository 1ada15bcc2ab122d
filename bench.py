#!/usr/bin/env python
"""ProbeWalk bench: batched queries/s on one GB300 (and N GPUs by query sharding).

One step = one batch of the workload's queries through the whole hot path
(budget, pilot, walks, U-statistic, median-of-means), all walks of all
queries in one persistent launch.  `value` is timed with CUDA events on the
launch stream with inputs resident in HBM (pw_query_batch_device); `e2e` is
the same batch through the host-array entry point (pw_query_batch), pinned
staging, host-to-device and device-to-host copies included.  L2 is flushed
(256 MiB write) between timed steps, outside the timed events.

--impl reference times the CPU oracle (the plain serial walker) on the machine's
host cores on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/s at eps=0.1 (batched server vs 1-per-launch), walk-steps/s, p99 latency"

WORKLOADS = {
    "ba-1e5": dict(graph="ba-1e5", desc="Barabasi-Albert n=100000 m=5 (seed 1), int32 CSR", queries=1000, L=200,
                   eps=0.1, pair_seed=101, seed_seed=1001),
    "tiny-er200": dict(graph="tiny-er200", desc="Erdos-Renyi G(200, 8/199) + cycle (seed 0)", queries=64, L=32,
                       eps=0.2, pair_seed=100, seed_seed=200),
    "rmat-20": dict(graph="rmat-20", desc="R-MAT 2^20 ef16 (.57,.19,.19,.05) symmetrised, LCC (seed 2)",
                    queries=1000, L=500, eps=("uniform", 0.05, 0.2), pair_seed=102, seed_seed=1002),
    "rmat-24": dict(graph="rmat-24", desc="R-MAT 2^24 ef16 (.57,.19,.19,.05) symmetrised, LCC (seed 4), native generator",
                    queries=1000, L=1000, eps=("uniform", 0.05, 0.2), pair_seed=104, seed_seed=1004),
    "grid-2000": dict(graph="grid-2000", desc="2000x2000 grid, 5% edges deleted, LCC (seed 3), bipartite",
                      queries=1000, L=2000, eps=("choice", 0.05, 0.1, 0.2), pair_seed=103, seed_seed=1003),
}


def workload_eps(wl: dict, count: int, rank: int = 0) -> np.ndarray:
    from pw_inputs import eps_choice, eps_uniform

    e = wl["eps"]
    if isinstance(e, float):
        return np.full(count, e)
    if e[0] == "uniform":
        return eps_uniform(count, e[1], e[2], wl["pair_seed"] + 7919 * rank)
    return eps_choice(count, list(e[1:]), wl["pair_seed"] + 7919 * rank)

SECTOR_BYTES = 32  # one 16-byte neighbour record per transition lives in one 32-byte sector
L2_BYTES = 129 << 20
WALK_KERNEL_NAME = {1: "walk_kernel (per-visit probe evaluation)", 2: "walk_table_kernel (per-probe table)",
                    3: "walk_table_kernel and walk_kernel (walk kernel chosen per query)"}
# DRAM and L2 traffic of a walk kernel from one ncu capture on a small case of
# the same workload (null when no capture of the current kernel exists, or
# when the batch ran both walk kernels).  BA, table kernel, one launch of 8
# queries (5.2096e9 transitions): dram read+write 16.04 MB + 2.6 KB, the record
# array read once into L2 whatever the transitions, so the DRAM bytes are not
# scaled; lts__t_sectors 5.653e9, 1.085 sectors per transition, scaled.
WALK_TRAFFIC = {
    ("ba-1e5", 2): {"dram_per_launch": 16.041472e6 + 2560.0, "l2_per_transition": 5652706685 * 32 / 5.2096e9,
                    "note": "ncu capture of one 8-query launch: DRAM reads are the 16 MB record array, loaded once "
                            "into L2 (not scaled); L2 sectors scaled by transitions"},
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p.get("hbm_gbs", 6800.0), "measured"
    except OSError:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return parse_clock_lines(self.lines)


def parse_clock_lines(lines) -> dict:
    """Median SM clock, maximum SM clock and the throttle reasons seen Active in
    nvidia-smi CSV lines of ClockSampler.FIELDS (lines that do not parse are skipped)."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, x: float, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_inputs(wl: dict, rank: int):
    from pw_inputs import query_seeds, uniform_pairs, workload_graph

    host = workload_graph(wl["graph"])
    s, t = uniform_pairs(host.n, wl["queries"], wl["pair_seed"] + 7919 * rank)
    seeds = query_seeds(wl["queries"], wl["seed_seed"] + 7919 * rank)
    return host, s, t, seeds


def cpu_oracle_sample(host, s, t, seeds, wl, n_queries: int, probes_per_query: int, offset: int = 0):
    """The oracle, as it stands, on a bounded sample of the workload: for each
    of `n_queries` queries (one host thread each) its budget (pilot included)
    and its first `probes_per_query` probes.  Returns queries/s = (sum over the
    sampled queries of the fraction of their transitions done) / wall time."""
    import concurrent.futures as cf

    import oracle

    oracle.build()
    idx = [(offset + i) % s.size for i in range(n_queries)]

    eps_all = workload_eps(wl, s.size)

    def one(i):
        b = oracle.budget(host, int(s[i]), int(t[i]), float(eps_all[i]), wl["L"], int(seeds[i]))
        P = min(probes_per_query, b["K"])
        oracle.probe_q(host, int(s[i]), int(t[i]), wl["L"], int(seeds[i]), b["R"], np.arange(P))
        pilot = 2 * 64 * 32 * wl["L"]
        done = pilot + 2 * P * b["R"] * wl["L"]
        total = pilot + 2 * b["K"] * b["R"] * wl["L"]
        return done / total, done

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=n_queries) as ex:
        res = list(ex.map(one, idx))
    dt = time.perf_counter() - t0
    frac = sum(r[0] for r in res)
    steps = sum(r[1] for r in res)
    return frac / dt, dt, n_queries, steps / dt


def run_reference(args, wl, world, rank):
    """CPU oracle arm: each step is a bounded sample (budget plus the first
    probes of one query per host core), scaled to queries/s."""
    if rank != 0:
        return
    host, s, t, seeds = workload_inputs(wl, 0)
    threads = args.cpu_threads or os.cpu_count()
    vals, times = [], []
    for i in range(args.warmup + args.steps):
        qps, dt, nq, sps = cpu_oracle_sample(host, s, t, seeds, wl, threads, args.cpu_probes, offset=i * threads)
        if i >= args.warmup:
            vals.append(qps)
            times.append(dt)
    value = sum(vals) / len(vals)
    sample = (f"per step: budget (pilot included) and the first {args.cpu_probes} probes of each of {threads} queries, "
              f"one host thread per query; queries/s = completed fraction of the sampled queries / wall time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}; {wl['queries']} uniform pairs; L={wl['L']}; "
                                   f"eps={wl['eps']}; delta=0.01; PILOT budget c_B=0.5", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_server(pw, g, s, t, eps, L, seeds, params, want):
    """pw_server_*: a burst of the whole batch (capacity; every estimate must
    equal the batch entry point's), then Poisson arrivals at 0.5x and 0.9x of
    that capacity.  Latency = submit to completion, measured by the server."""
    from pw_inputs import poisson_arrivals

    nq = s.size
    srv = pw.pw_server_create(g.handle, params, 4 << 30)
    out = {}
    try:
        k = min(nq, 32)
        out["tune"] = pw.pw_server_tune(srv, s[:k], t[:k], eps[:k], L[:k], seeds[:k])
        out["tune"]["sample"] = f"first {k} queries, burst timed after a warm-up burst, per policy"
        t0 = time.perf_counter()
        tickets = [pw.pw_server_submit(srv, int(s[i]), int(t[i]), float(eps[i]), int(L[i]), int(seeds[i]))
                   for i in range(nq)]
        pw.pw_server_drain(srv, 600000)
        burst_s = time.perf_counter() - t0
        tk, b, st, lat = pw.pw_server_collect(srv, 4 * nq)
        order = {int(x): i for i, x in enumerate(tickets)}
        got = np.empty(nq)
        got[[order[int(x)] for x in tk]] = b
        assert np.all(st == 0) and np.array_equal(got, want), "server estimates differ from the batch entry point"
        cap_qps = nq / burst_s
        out["burst"] = {"queries": nq, "queries_per_s": cap_qps, "p50_ms": float(np.percentile(lat, 50)),
                        "p99_ms": float(np.percentile(lat, 99))}
        loads = []
        n_load = min(nq, 400)
        for frac in (0.5, 0.9):
            rate = frac * cap_qps
            arr = poisson_arrivals(n_load, rate, 4242 + int(100 * frac))
            t0 = time.perf_counter()
            for i in range(n_load):
                d = arr[i] - (time.perf_counter() - t0)
                if d > 0:
                    time.sleep(d)
                pw.pw_server_submit(srv, int(s[i]), int(t[i]), float(eps[i]), int(L[i]), int(seeds[i]))
            pw.pw_server_drain(srv, 600000)
            wall = time.perf_counter() - t0
            _, _, st, lat = pw.pw_server_collect(srv, 4 * nq)
            assert np.all(st == 0)
            loads.append({"offered_frac_of_capacity": frac, "offered_qps": rate, "achieved_qps": n_load / wall,
                          "queries": n_load, "p50_ms": float(np.percentile(lat, 50)),
                          "p99_ms": float(np.percentile(lat, 99))})
        out["poisson"] = loads
    finally:
        pw.pw_server_destroy(srv)
    return out


def run_serving(args, wl, world, rank, local):
    """Serving on the workload's graph: a burst of --burst queries measures the
    server's capacity, then Poisson streams of --queries queries arrive at
    --loads x that capacity; latency is submit to completion (p50, p99,
    p99.9), throughput is completions / wall time, clocks are sampled while the
    streams run.  Query pairs, eps and seeds follow the workload's recipe."""
    import torch

    from paper_2512_05460_gb300 import build as pwbuild
    from pw_inputs import poisson_arrivals, query_seeds, uniform_pairs, workload_graph

    pwbuild.build()
    from paper_2512_05460_gb300 import probewalk as pw

    torch.cuda.set_device(local)
    n = args.queries or 1000
    host = workload_graph(wl["graph"])
    s, t = uniform_pairs(host.n, n, wl["pair_seed"] + 7919 * rank)
    seeds = query_seeds(n, wl["seed_seed"] + 7919 * rank)
    eps = workload_eps(wl, n, rank)
    L = wl["L"]
    g = pw.Graph(host.row_ptr, host.col_idx, device=local)
    out = {}
    if not args.no_autotune:
        k = min(n, args.tune_sample)
        out["graph_tune"] = pw.pw_autotune(g.handle, s[:k], t[:k], eps[:k], np.full(k, L, np.int32), seeds[:k])
    srv = pw.pw_server_create(g.handle, None, 8 << 30)
    try:
        k = min(n, 32)
        out["tune"] = pw.pw_server_tune(srv, s[:k], t[:k], eps[:k], np.full(k, L, np.int32), seeds[:k])
        nb = min(n, args.burst)
        t0 = time.perf_counter()
        for i in range(nb):
            pw.pw_server_submit(srv, int(s[i]), int(t[i]), float(eps[i]), L, int(seeds[i]))
        pw.pw_server_drain(srv, 3600 * 1000)
        burst_s = time.perf_counter() - t0
        _, _, st, lat = pw.pw_server_collect(srv, 4 * n)
        assert np.all(st == 0)
        cap = nb / burst_s
        out["burst"] = {"queries": nb, "queries_per_s": cap, "p50_ms": float(np.percentile(lat, 50)),
                        "p99_ms": float(np.percentile(lat, 99))}
        loads = []
        for frac in (float(x) for x in args.loads.split(",")):
            rate = frac * cap
            arr = poisson_arrivals(n, rate, 4242 + int(100 * frac))
            sampler = ClockSampler(local)
            sampler.start()
            t0 = time.perf_counter()
            for i in range(n):
                d = arr[i] - (time.perf_counter() - t0)
                if d > 0:
                    time.sleep(d)
                pw.pw_server_submit(srv, int(s[i]), int(t[i]), float(eps[i]), L, int(seeds[i]))
            pw.pw_server_drain(srv, 3600 * 1000)
            wall = time.perf_counter() - t0
            clocks = sampler.stop()
            _, _, st, lat = pw.pw_server_collect(srv, 4 * n)
            assert np.all(st == 0)
            loads.append({"offered_frac_of_capacity": frac, "offered_qps": rate, "achieved_qps": n / wall,
                          "queries": n, "p50_ms": float(np.percentile(lat, 50)),
                          "p99_ms": float(np.percentile(lat, 99)), "p999_ms": float(np.percentile(lat, 99.9)),
                          "wall_s": wall, "clocks": clocks})
        out["poisson"] = loads
    finally:
        pw.pw_server_destroy(srv)
    line = {"metric": "serving: queries/s and p50/p99 latency of Poisson streams (continuous batching)",
            "unit": "queries/s", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}; {n} uniform pairs per stream; L={L}; "
                                   f"eps={wl['eps']}; PILOT budget c_B=0.5; 8 GiB accumulator pool"},
            "server": out}
    print(json.dumps(line), flush=True)
    g.close()


def run_scale_batch(args, wl, world, rank, local):
    """One batch of --queries queries (default 10,000) through
    pw_query_batch_device: an untimed batch of the same size first (it sizes
    the scratch and warms the kernels), then --steps timed batches with CUDA
    events on the launch stream; reports queries/s, walk steps/s, the walk
    kernels' share and the scratch the batch needed (Q_R and per-probe
    accumulators: nothing per replica)."""
    import torch

    from paper_2512_05460_gb300 import build as pwbuild
    from pw_inputs import query_seeds, uniform_pairs, workload_graph

    pwbuild.build()
    from paper_2512_05460_gb300 import probewalk as pw

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.queries or 10000
    host = workload_graph(wl["graph"])
    s, t = uniform_pairs(host.n, n, wl["pair_seed"] + 7919 * rank)
    seeds = query_seeds(n, wl["seed_seed"] + 7919 * rank)
    eps = workload_eps(wl, n, rank)
    L = np.full(n, wl["L"], np.int32)
    g = pw.Graph(host.row_ptr, host.col_idx, device=local)
    params = pw.make_params(c_B=args.c_B)
    tune = None
    if not args.no_autotune:
        k = min(n, args.tune_sample)
        tune = pw.pw_autotune(g.handle, s[:k], t[:k], eps[:k], L[:k], seeds[:k], params)
    d = [torch.from_numpy(a).to(dev) for a in (s, t, eps, L, seeds.view(np.int64))]
    beta = torch.empty(n, dtype=torch.float64, device=dev)
    status = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    mem0 = torch.cuda.mem_get_info(dev)[0]
    pw.pw_query_batch_device(g.handle, n, *d, beta, status, params, stream=stream)
    stream.synchronize()
    scratch = mem0 - torch.cuda.mem_get_info(dev)[0]
    assert int(status.abs().sum()) == 0
    sampler = ClockSampler(local)
    pw.pw_profile(g.handle, enable=True, reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler.start()
    for a, b in ev:
        a.record(stream)
        pw.pw_query_batch_device(g.handle, n, *d, beta, status, params, stream=stream)
        b.record(stream)
    stream.synchronize()
    clocks = sampler.stop()
    prof = pw.pw_profile(g.handle, enable=False, reset=True)
    assert int(status.abs().sum()) == 0 and bool(torch.isfinite(beta).all())
    ms = sum(a.elapsed_time(b) for a, b in ev)
    hbm_peak, peak_kind = load_peaks()
    gathers = 1 if prof["layout"] == 1 else 2
    walk_s = prof["walk_ms"] / 1000.0
    line = {"metric": "queries/s of one large batch (persistent walk kernels, per-query kernel choice)",
            "value": n * args.steps / (ms / 1000.0), "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": 1, "ms_per_step": ms / args.steps, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}; {n} uniform pairs in one batch; L={wl['L']}; "
                                   f"eps={wl['eps']}; PILOT budget c_B={args.c_B or 0.5}",
                       "inputs": "device-resident (pw_query_batch_device)"},
            "walk_steps_per_s": (prof["transitions"] + prof["pilot_transitions"]) / (ms / 1000.0),
            "walk_share": prof["walk_ms"] / ms,
            "walk_kernels": {1: "per-visit", 2: "table", 3: "both (chosen per query)"}.get(prof["walk_mode"]),
            "roofline": {"bound": "hbm", "achieved": prof["transitions"] * 32 * gathers / walk_s / 1e9,
                         "peak": hbm_peak, "unit": "GB/s", "peak_kind": peak_kind,
                         "frac": prof["transitions"] * 32 * gathers / walk_s / 1e9 / hbm_peak,
                         "bytes_model": f"{32 * gathers} B per walk transition"},
            "scratch_bytes": int(scratch), "autotune": tune, "clocks": clocks}
    print(json.dumps(line), flush=True)
    g.close()


def run_stabilized(args, wl, world, rank, local):
    """Section 4.3: L chosen per query by doubling from L = 1 until the estimate
    stabilises (cap L_max = 256, the paper's reference length); reports
    queries/s, the distribution of L_stop and the proxy relative error
    |beta(L_stop) - beta(L_max)| / |beta(L_max)| of Fig. 3."""
    import torch

    from paper_2512_05460_gb300 import build as pwbuild

    pwbuild.build()
    from paper_2512_05460_gb300 import probewalk as pw

    torch.cuda.set_device(local)
    host, s, t, seeds = workload_inputs(wl, rank)
    n = args.queries or 200
    s, t, seeds = s[:n], t[:n], seeds[:n]
    eps = workload_eps(wl, n, rank)
    g = pw.Graph(host.row_ptr, host.col_idx, device=local)
    L_max = 256
    pw.pw_query_stabilized(g.handle, s[:8], t[:8], eps[:8], L_max, seeds[:8])  # warm-up
    pw.pw_launch_count(reset=True)
    t0 = time.perf_counter()
    beta, L_stop, st = pw.pw_query_stabilized(g.handle, s, t, eps, L_max, seeds)
    wall = time.perf_counter() - t0
    launches = pw.pw_launch_count(reset=True)
    assert np.all(st == 0)
    ref_seeds = np.array([pw.pw_level_seed(int(x), L_max) for x in seeds], np.uint64)
    ref, _ = pw.pw_query_batch(g.handle, s, t, eps, np.full(n, L_max, np.int32), ref_seeds)
    proxy = np.abs(beta - ref) / np.abs(ref)
    hist = {int(L): int((L_stop == L).sum()) for L in np.unique(L_stop)}
    line = {"metric": "queries/s with L chosen by the stabilization rule (Section 4.3), L_max=256",
            "value": n / wall, "unit": "queries/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}; {n} uniform pairs; eps={wl['eps']}; "
                                   f"L_max={L_max}; PILOT budget c_B=0.5"},
            "L_stop_histogram": hist, "proxy_rel_error": {"median": float(np.median(proxy)),
                                                          "p95": float(np.percentile(proxy, 95)),
                                                          "frac_within_eps": float(np.mean(proxy <= eps))},
            "gpu_launches": launches, "wall_s": wall}
    print(json.dumps(line), flush=True)
    g.close()


def run_eps_sweep(args, wl, world, rank, local):
    """Fig. 2's protocol on the synthetic workload: for eps in {0.02, 0.04,
    0.06, 0.1, 0.2}, mean runtime per query (one batch of the queries, CUDA
    events) and mean relative error against the oracle's series beta^(L)."""
    import torch

    from oracle import exact
    from paper_2512_05460_gb300 import build as pwbuild

    pwbuild.build()
    from paper_2512_05460_gb300 import probewalk as pw

    torch.cuda.set_device(local)
    host, s, t, seeds = workload_inputs(wl, rank)
    n = args.queries or 32
    s, t, seeds = s[:n], t[:n], seeds[:n]
    L = wl["L"]
    ref = exact.series_beta_many(host.row_ptr, host.col_idx, host.n, s, t, L)
    g = pw.Graph(host.row_ptr, host.col_idx, device=local)
    pw.pw_query_batch(g.handle, s[:4], t[:4], 0.2, L, seeds[:4])
    rows = []
    for e in (0.02, 0.04, 0.06, 0.1, 0.2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        beta, st = pw.pw_query_batch(g.handle, s, t, e, L, seeds)
        wall = time.perf_counter() - t0
        assert np.all(st == 0)
        rel = np.abs(beta - ref) / ref
        rows.append({"eps": e, "ms_per_query": 1000 * wall / n, "mean_rel_error": float(rel.mean()),
                     "frac_within_eps": float(np.mean(rel <= e))})
    line = {"metric": "eps sweep (Fig. 2 protocol): mean runtime per query and mean relative error",
            "unit": "ms/query", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}; {n} uniform pairs; L={L}; batch of all queries; "
                                   "reference beta^(L) from the oracle's series"}, "rows": rows}
    print(json.dumps(line), flush=True)
    g.close()


def run_accuracy(args, wl, world, rank, local):
    """Problem 1's target on the workload: the fraction of queries whose
    estimate is within eps of beta^(L) (pw_series_batch, FP64-accurate to
    1e-9), at eps = 0.1 and 0.2 and each R_max of --r-max, with the walk
    transitions and the wall time each setting costs."""
    import torch

    from paper_2512_05460_gb300 import build as pwbuild

    pwbuild.build()
    from paper_2512_05460_gb300 import probewalk as pw

    torch.cuda.set_device(local)
    from pw_inputs import query_seeds, uniform_pairs, workload_graph

    n = args.queries or 256
    host = workload_graph(wl["graph"])
    s, t = uniform_pairs(host.n, n, wl["pair_seed"] + 7919 * rank)
    seeds = query_seeds(n, wl["seed_seed"] + 7919 * rank)
    L = wl["L"]
    g = pw.Graph(host.row_ptr, host.col_idx, device=local)
    ref = pw.pw_series_batch(g.handle, s, t, np.full(n, L, np.int32))
    rows = []
    budgets = {"pilot": pw.PW_BUDGET_PILOT, "adaptive": pw.PW_BUDGET_ADAPTIVE}
    settings = [(b, float(c), int(r), 0.0, 0.0) for b in args.budget_list.split(",") if b == "pilot"
                for c in args.c_B_list.split(",") for r in args.r_max.split(",")]
    settings += [("adaptive", float(c), int(r), float(z), float(cap)) for b in args.budget_list.split(",")
                 if b == "adaptive" for c in args.c_B_list.split(",") for r in args.r_max.split(",")
                 for z in args.z_list.split(",") for cap in args.cap_list.split(",")]
    for e in (0.1, 0.2):
        for bname, cb, rmax, z, cap in settings:
            params = pw.make_params(R_max=rmax, c_B=cb, budget_mode=budgets[bname], z=z, cap=cap)
            pw.pw_profile(g.handle, enable=True, reset=True)
            t0 = time.perf_counter()
            beta, st, KR, _ = pw.pw_debug_batch_probe_q(g.handle, s, t, e, L, seeds, [], [], params)
            wall = time.perf_counter() - t0
            prof = pw.pw_profile(g.handle, enable=False, reset=True)
            assert np.all(st == 0)
            rel = np.abs(beta - ref) / ref
            clamped = KR[:, 1] == rmax
            rows.append({"eps": e, "budget": bname, "c_B": cb, "R_max": rmax, "z": z or None, "cap": cap or None,
                         "frac_within_eps": float(np.mean(rel <= e)), "mean_B": float(KR[:, 0].mean()) / 37.0,
                         "frac_clamped": float(np.mean(clamped)),
                         "frac_within_eps_clamped": float(np.mean(rel[clamped] <= e)) if clamped.any() else None,
                         "frac_within_eps_unclamped": float(np.mean(rel[~clamped] <= e)) if (~clamped).any() else None,
                         "transitions": int(prof["transitions"]), "walk_s": prof["walk_ms"] / 1000.0, "wall_s": wall})
    line = {"metric": "fraction of queries within eps of beta^(L) (Problem 1) and its cost, by R_max",
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}; {n} uniform pairs; L={L}; PILOT budget; "
                                   "reference beta^(L) from pw_series_batch"}, "rows": rows}
    print(json.dumps(line), flush=True)
    g.close()


def run_series(args, wl, world, rank, local):
    """The deterministic truncated series beta^(L) (Lemma 2.3) on the GPU
    (pw_series_batch, double-float steps, 32 queries per pass): queries/s and
    the HBM roofline of its sparse steps, timed with CUDA events (pw_profile),
    next to the oracle's FP64 series on one host core."""
    import torch

    from oracle import exact
    from paper_2512_05460_gb300 import build as pwbuild

    pwbuild.build()
    from paper_2512_05460_gb300 import probewalk as pw

    torch.cuda.set_device(local)
    host, s, t, seeds = workload_inputs(wl, rank)
    nq = args.queries or 64
    s, t = s[:nq], t[:nq]
    L = wl["L"]
    g = pw.Graph(host.row_ptr, host.col_idx, device=local)
    for _ in range(args.warmup):
        pw.pw_series_batch(g.handle, s[:32], t[:32], L)
    pw.pw_profile(g.handle, enable=True, reset=True)
    pw.pw_launch_count(reset=True)
    sampler = ClockSampler(local)
    sampler.start()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        beta = pw.pw_series_batch(g.handle, s, t, L)
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    launches = pw.pw_launch_count(reset=True)
    prof = pw.pw_profile(g.handle, enable=False, reset=True)
    assert np.all(np.isfinite(beta))
    dev_s = prof["series_ms"] / 1000.0
    steps = prof["series_steps"]
    # requested bytes per sparse step: per node its x row (h += x), h read and
    # written, y written (4 x 256 B) and its 16-B record; per neighbour entry
    # the neighbour's x row (256 B) and its 16-B record
    step_bytes = host.n * (4 * 256 + 16) + host.nnz * (256 + 16)
    achieved = steps * step_bytes / dev_s / 1e9
    hbm_peak, peak_kind = load_peaks()
    # the steps run in double-float (FP32 pairs, about 20 FP32 operations per
    # addition), so they are bound by memory, not by GB300's FP64 rate
    # the oracle's series on one core: per-step time from two run lengths, 32 columns
    k = 1
    t_0 = time.perf_counter()
    exact.series_beta_many(host.row_ptr, host.col_idx, host.n, s[:32], t[:32], 0)
    t_base = time.perf_counter() - t_0
    while True:
        t_0 = time.perf_counter()
        exact.series_beta_many(host.row_ptr, host.col_idx, host.n, s[:32], t[:32], k)
        t_k = time.perf_counter() - t_0
        if t_k > 5.0 or k >= L:
            break
        k *= 2
    per_step = max(t_k - t_base, 1e-9) / k
    cpu_qps = 32 / (t_base + per_step * (L + 1))
    line = {"metric": "truncated series beta^(L) (Lemma 2.3) on the GPU: queries/s", "value": nq * args.steps / dev_s,
            "unit": "queries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f32x2", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}; {nq} uniform pairs; L={L}; "
                                   "32 queries per pass (n x 32 double-float rows)"},
            "series_steps_per_s": steps / dev_s, "wall_s": wall,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                         "bytes_model": "per step n (4 x 256 B + 16 B) + nnz (256 B + 16 B) requested; neighbour "
                                        "rows that hit L2 count as requested bytes",
                         "arithmetic": "double-float (hi + lo FP32 pairs, TwoSum / fused-multiply-add TwoProd); "
                                       "beta reduced in FP64"},
            "cpu_baseline": {"value": cpu_qps, "unit": "queries/s", "cores": 1, "kind": "oracle",
                             "sample": f"oracle series_beta_many on 32 queries: L=0 and L={k} timed, "
                                       f"per-step time scaled to L={L}"},
            "clocks": clocks, "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    g.close()


def batched_vs_plain(pw, name, device, params, reps=5):
    """One batch of the workload's queries (pw_query_batch) against the same
    queries one per call (pw_query), both host-array calls, host wall clock;
    each after two untimed calls, so both run as replayed CUDA graphs."""
    wl = WORKLOADS[name]
    host, s, t, seeds = workload_inputs(wl, 0)
    eps = workload_eps(wl, s.size)
    L = np.full(s.size, wl["L"], np.int32)
    with pw.Graph(host.row_ptr, host.col_idx, device=device) as g:
        for _ in range(2):
            pw.pw_query_batch(g.handle, s, t, eps, L, seeds, params)
        t0 = time.perf_counter()
        for _ in range(reps):
            beta, st = pw.pw_query_batch(g.handle, s, t, eps, L, seeds, params)
        batch_qps = reps * s.size / (time.perf_counter() - t0)
        assert np.all(st == 0)
        for i in range(2):
            pw.pw_query(g.handle, int(s[i]), int(t[i]), float(eps[i]), int(L[i]), int(seeds[i]), params)
        t0 = time.perf_counter()
        for i in range(s.size):
            b = pw.pw_query(g.handle, int(s[i]), int(t[i]), float(eps[i]), int(L[i]), int(seeds[i]), params)
            assert b == beta[i]
        plain_qps = s.size / (time.perf_counter() - t0)
    return {"workload": f"{name}: {wl['desc']}; {s.size} uniform pairs; L={wl['L']}; eps={wl['eps']}",
            "batch_queries_per_s": batch_qps, "plain_queries_per_s": plain_qps,
            "batched_over_plain": batch_qps / plain_qps,
            "timing": f"host wall clock, {reps} batches against one pass of single-query calls"}


def run_ours(args, wl, world, rank, local):
    import torch

    from paper_2512_05460_gb300 import build as pwbuild

    pwbuild.build()
    from paper_2512_05460_gb300 import probewalk as pw

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    host, s, t, seeds = workload_inputs(wl, rank)
    if args.queries:
        s, t, seeds = s[:args.queries], t[:args.queries], seeds[:args.queries]
    nq = s.size
    eps = workload_eps(wl, nq, rank)
    L = np.full(nq, wl["L"], np.int32)
    g = pw.Graph(host.row_ptr, host.col_idx, device=local, flags={0: 0, 1: pw.LOAD_FUSED, 2: pw.LOAD_SPLIT}[args.layout])
    params = pw.make_params(c_B=args.c_B, walk_mode=args.walk_mode)
    d_s = torch.from_numpy(s).to(dev)
    d_t = torch.from_numpy(t).to(dev)
    d_eps = torch.from_numpy(eps).to(dev)
    d_L = torch.from_numpy(L).to(dev)
    d_seed = torch.from_numpy(seeds.view(np.int64)).to(dev)
    d_beta = torch.empty(nq, dtype=torch.float64, device=dev)
    d_status = torch.empty(nq, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step():
        pw.pw_query_batch_device(g.handle, nq, d_s, d_t, d_eps, d_L, d_seed, d_beta, d_status, params, stream=stream)

    # walk-kernel cost model fitted on this graph (outside every timed region)
    tune = None
    if args.walk_mode == 0 and not args.no_autotune:
        k = min(nq, args.tune_sample)
        tune = pw.pw_autotune(g.handle, s[:k], t[:k], eps[:k], L[:k], seeds[:k], params)
        tune["sample"] = f"first {k} queries of the batch"
    if args.l2_window >= 0:
        pw.pw_graph_set_l2_window(g.handle, args.l2_window)
    l2_window = args.l2_window if args.l2_window >= 0 else (tune["l2_window"] if tune else 0)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            flush.fill_(i & 0xFF)
            step()
    stream.synchronize()
    assert int(d_status.abs().sum()) == 0, "query errors in warm-up"

    # ---- timed region: device-resident inputs --------------------------------
    sampler = ClockSampler(local)
    pw.pw_profile(g.handle, enable=True, reset=True)
    pw.pw_launch_count(reset=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_((i + 1) & 0xFF)
            starts[i].record(stream)
            step()
            ends[i].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    launches = pw.pw_launch_count(reset=True)
    prof = pw.pw_profile(g.handle, enable=False, reset=True)
    walk_mode = prof.get("walk_mode", 0)
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = max_over_ranks(world, sum(step_ms), dev)
    beta = d_beta.cpu().numpy()
    assert int(d_status.abs().sum()) == 0 and np.all(np.isfinite(beta))
    value = world * nq * args.steps / (total_ms / 1000.0)
    transitions_per_step = prof["transitions"] / max(1, args.steps)
    walk_ms_avg = prof["walk_ms"] / max(1, prof["walk_launches"])
    walk_steps_per_s = world * (prof["transitions"] + prof["pilot_transitions"]) / (total_ms / 1000.0)

    # ---- end to end through the host-array entry point -----------------------
    e2e_times = []
    for i in range(args.steps if not args.no_e2e else 0):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b2, st2 = pw.pw_query_batch(g.handle, s, t, eps, L, seeds, params)
        e2e_times.append(time.perf_counter() - t0)
        assert np.all(st2 == 0)
        assert np.array_equal(b2, beta), "host and device entry points disagree"
    e2e_value = None
    if e2e_times:
        e2e_total = max_over_ranks(world, sum(e2e_times), dev)
        e2e_value = world * nq * len(e2e_times) / e2e_total

    # ---- one query per launch (the plain form), on a prefix of the batch ------
    plain_n = min(args.plain, nq)
    lat = []
    for i in range(plain_n):
        t0 = time.perf_counter()
        pw.pw_query(g.handle, int(s[i]), int(t[i]), float(eps[i]), int(L[i]), int(seeds[i]), params)
        lat.append(time.perf_counter() - t0)
    plain_qps = plain_n / sum(lat) if lat else None
    # the same prefix as one batch through the same host-array entry point
    same = None
    if plain_n:
        sp, tp, ep, Lp, dp = s[:plain_n], t[:plain_n], eps[:plain_n], L[:plain_n], seeds[:plain_n]
        for _ in range(2):
            pw.pw_query_batch(g.handle, sp, tp, ep, Lp, dp, params)
        t0 = time.perf_counter()
        pw.pw_query_batch(g.handle, sp, tp, ep, Lp, dp, params)
        bq = plain_n / (time.perf_counter() - t0)
        same = {"queries": plain_n, "batch_queries_per_s": bq, "plain_queries_per_s": plain_qps,
                "batched_over_plain": bq / plain_qps}

    # ---- the regime where batching matters: the tiny graph (64 queries, eps = 0.2)
    tiny_regime = None
    if args.workload != "tiny-er200" and not args.no_tiny:
        tiny_regime = batched_vs_plain(pw, "tiny-er200", local, params)

    # ---- continuous-batching server: burst capacity, then Poisson arrivals ----
    server = None
    if not args.no_server:
        server = run_server(pw, g, s, t, eps, L, seeds, params, beta)

    # ---- roofline of the walk kernel -----------------------------------------
    # Algorithmic bytes per walk transition: one 32-byte sector per gather, one
    # gather (the 16-byte fused neighbour record) or two (a col_idx entry, then
    # the neighbour's 16-byte node record) by the graph's layout.  Arrays larger
    # than L2 are bound by HBM (MEASURED_PEAKS.json); L2-resident ones (this BA
    # graph: 16 MB of records) by L2 sector throughput, measured here by
    # dependent random gathers with the same access.
    hbm_peak, peak_kind = load_peaks()
    layout = prof.get("layout", 1)
    gathers = 1 if layout == 1 else 2
    walk_bytes = transitions_per_step * SECTOR_BYTES * gathers
    achieved = walk_bytes / (walk_ms_avg / 1000.0) / 1e9 if walk_ms_avg > 0 else 0.0
    record_bytes = 16 * host.nnz if layout == 1 else 4 * host.nnz + 16 * host.n
    if record_bytes < L2_BYTES // 2:
        l2_peak = pw.pw_debug_gather_peak(g.handle, 2048) * SECTOR_BYTES * gathers / 1e9
        roofline = {"bound": "l2", "achieved": achieved, "peak": l2_peak, "unit": "GB/s", "frac": achieved / l2_peak,
                    "peak_kind": "measured in this run: dependent random gathers with the walk's access over the "
                                 "same L2-resident arrays (pw_debug_gather_peak)",
                    "hbm_copy_peak": hbm_peak, "frac_of_hbm_copy_peak": achieved / hbm_peak,
                    "hbm_copy_peak_kind": peak_kind,
                    "note": "the arrays are L2-resident, so DRAM is idle; the headline fraction is against the "
                            "measured L2 gather ceiling, the copy-peak fraction is context"}
    else:
        # Context beside the copy peak: the ceiling of this access pattern
        # (dependent random 16-B gathers, uniform over the same records, which
        # is where a stationary walk's transitions land), measured in this run.
        gather = pw.pw_debug_gather_peak(g.handle, 512) * SECTOR_BYTES * gathers / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                    "gather_ceiling": gather, "frac_of_gather_ceiling": achieved / gather,
                    "gather_ceiling_kind": "measured in this run: dependent random 16-B gathers uniform over the "
                                           "same record array (pw_debug_gather_peak)"}
    tr = WALK_TRAFFIC.get((args.workload, walk_mode))
    roofline.update({"traffic": tr and tr["dram_per_launch"],
                     "l2_traffic": tr and tr["l2_per_transition"] * transitions_per_step,
                     "traffic_note": tr and tr["note"],
                     "kernel": WALK_KERNEL_NAME[walk_mode],
                     "algorithmic_bytes_per_launch": walk_bytes,
                     "layout": {1: "fused 16-B neighbour records", 2: "col_idx + 16-B node records"}[layout],
                     "bytes_model": ("32 B (one sector holding the 16 B neighbour record) per walk transition"
                                     if layout == 1 else "64 B per walk transition: the sector holding the 4 B "
                                                         "col_idx entry and the sector holding the 16 B node record"),
                     "walk_ms_per_launch": walk_ms_avg})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = args.cpu_threads or os.cpu_count()
        qps, dt, cnt, sps = cpu_oracle_sample(host, s, t, seeds, wl, threads, args.cpu_probes)
        cpu = {"value": qps, "unit": "queries/s", "cores": threads, "kind": "oracle",
               "sample": f"budget (pilot included) and the first {args.cpu_probes} probes of each of the first {cnt} "
                         f"queries, one host thread per query, {dt:.1f} s; queries/s = completed fraction / wall",
               "walk_steps_per_s": sps}

    if rank == 0:
        lat_ms = sorted(1000 * x for x in lat)

        def pct(p):
            return lat_ms[min(len(lat_ms) - 1, int(round(p / 100 * (len(lat_ms) - 1))))] if lat_ms else None

        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}; {nq} uniform pairs per GPU; L={wl['L']}; "
                                   f"eps={wl['eps']}; delta=0.01; PILOT budget c_B={args.c_B or 0.5}",
                       "queries_per_gpu": nq, "L": wl["L"], "eps": wl["eps"],
                       "l2": "flushed between timed steps (256 MiB write, outside the timed events)",
                       "parallelism": f"query sharding x{world}"},
            "walk_steps_per_s": walk_steps_per_s,
            "walk_kernel": {1: "per-visit probe evaluation", 2: "per-probe shared-memory table",
                            3: "both (chosen per query)"}.get(walk_mode, "?"),
            "autotune": tune,
            "l2_window": {0: "none", 1: "gathered array (persisting share = set-aside / array)",
                          2: "node records"}[l2_window],
            "transitions_per_step": transitions_per_step,
            "plain_queries_per_s": plain_qps, "plain_sample": plain_n,
            "batched_over_plain": (value / world) / plain_qps if plain_qps else None,
            "batched_over_plain_same_queries": same,
            "batched_over_plain_tiny": tiny_regime,
            "latency_ms": {"plain_p50": pct(50), "plain_p99": pct(99), "batch_step": total_ms / args.steps},
            "server": server,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": nq * 36,
                    "d2h_bytes_per_step": nq * 12},
            "gpu_launches": launches,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    g.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ba-1e5", choices=sorted(WORKLOADS))
    ap.add_argument("--plain", type=int, default=64, help="queries timed in the one-query-per-launch form")
    ap.add_argument("--c_B", type=float, default=0.0)
    ap.add_argument("--queries", type=int, default=0, help="use only the first N queries (small profiling runs)")
    ap.add_argument("--walk-mode", type=int, default=0,
                    help="0 auto (cost model fitted by pw_autotune on the first 8 queries), 1 per-visit, 2 probe table")
    ap.add_argument("--no-autotune", action="store_true", help="auto mode with the untuned default cost model")
    ap.add_argument("--cpu-threads", type=int, default=0)
    ap.add_argument("--cpu-probes", type=int, default=40, help="probes per sampled query in the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-server", action="store_true")
    ap.add_argument("--no-tiny", action="store_true", help="skip the tiny-graph batched-vs-plain comparison")
    ap.add_argument("--tune-sample", type=int, default=32,
                    help="queries of the pw_autotune sample (the first ones of the batch)")
    ap.add_argument("--l2-window", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="L2 access-policy window of the walks: -1 the autotuner's choice, 0 none, "
                         "1 the gathered array, 2 node records (split layout)")
    ap.add_argument("--layout", type=int, default=0, choices=[0, 1, 2],
                    help="walk layout: 0 by size, 1 fused records, 2 col_idx + node records")
    ap.add_argument("--stabilized", action="store_true", help="L by the stabilization rule (Section 4.3)")
    ap.add_argument("--eps-sweep", action="store_true", help="runtime and error over eps (Fig. 2 protocol)")
    ap.add_argument("--series", action="store_true", help="the GPU truncated series beta^(L) (Lemma 2.3)")
    ap.add_argument("--accuracy", action="store_true", help="fraction within eps of beta^(L), by R_max")
    ap.add_argument("--serving", action="store_true", help="server capacity and Poisson-stream latency")
    ap.add_argument("--scale-batch", action="store_true", help="one large batch (--queries, default 10000)")
    ap.add_argument("--burst", type=int, default=1000, help="queries of the --serving capacity burst")
    ap.add_argument("--loads", default="0.5,0.9", help="offered loads of --serving, as fractions of capacity")
    ap.add_argument("--r-max", default="4096,8192,16384", help="R_max values of --accuracy")
    ap.add_argument("--c-B-list", default="0.5", help="c_B values of --accuracy")
    ap.add_argument("--budget-list", default="pilot", help="budget modes of --accuracy: pilot, adaptive")
    ap.add_argument("--z-list", default="2.2", help="ADAPTIVE z values of --accuracy")
    ap.add_argument("--cap-list", default="1", help="ADAPTIVE caps (multiples of PILOT's B) of --accuracy")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    wl = WORKLOADS[args.workload]
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, wl, world, rank)
    elif args.stabilized:
        run_stabilized(args, wl, world, rank, local)
    elif args.series:
        run_series(args, wl, world, rank, local)
    elif args.accuracy:
        run_accuracy(args, wl, world, rank, local)
    elif args.serving:
        run_serving(args, wl, world, rank, local)
    elif args.scale_batch:
        run_scale_batch(args, wl, world, rank, local)
    elif args.eps_sweep:
        run_eps_sweep(args, wl, world, rank, local)
    else:
        run_ours(args, wl, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
