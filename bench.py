"""Benchmark: higher-order (k,h)-truss decomposition on one GB300 (or N replicas).

A step is one pass of the whole hot path over the workload with its inputs resident in
HBM: normalise + CSR/edge ids, every vertex's h-hop ball, every edge's h-support, and
level-synchronous peeling with recomputation limited to edges whose balls changed.
Default workload: R-MAT scale 18, edge factor 8, (a,b,c,d)=(0.57,0.19,0.19,0.05),
h = 2 (the paper's Amazon-TWEB-sized stand-in).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle instead.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import config_graph  # noqa: E402

WORKLOADS = {
    "rmat_s18_h2": ("rmat_s18", 2),
    "dcsbm_n200k_h2": ("dcsbm_n200k", 2),
    "dcsbm_n200k_h3": ("dcsbm_n200k", 3),
    "er_n2000_h2": ("er_n2000", 2),
    "rmat_s16_h2": ("rmat_s16", 2),
    "dcsbm_n50k_h3": ("dcsbm_n50k", 3),
}
# the other single-GPU workloads reported beside the headline (fewer steps each)
CONFIG_ENTRIES = ["er_n2000_h2", "dcsbm_n200k_h2", "dcsbm_n200k_h3"]
CONFIG_STEPS = {"dcsbm_n200k_h3": (1, 0)}  # (timed steps, warm-up steps); default (3, 1)
# batched form: 4,096 graphs, n ~ U[50, 5000], ER or BA, h ~ U{2,3}
BATCHED = {"count": 4096, "seed": 0x48545258, "steps": 1, "warmup": 1}
# served stream: Poisson arrivals at 200 requests/s over R-MAT and BA graphs, h in {2, 3}
# (the largest pool members are capped so that the stream finishes within the bench run)
SERVED = {"count": 120, "seed": 0x48545259, "rate": 200.0, "workers": 8,
          "rmat_scales": (10, 15), "ba_n": (1_000, 50_000)}
METRIC = "edges decomposed/sec"
UNIT = "edges/s"
L2_FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The largest value over all ranks (a replicated job takes as long as its slowest
    rank).  One all-reduce on the process group; with one rank, the value itself."""
    if world <= 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_replica: int, steps: int, t_max_ms: float, world: int) -> float:
    """Units all replicas processed per second of the slowest rank's time."""
    return world * units_per_replica * steps / (t_max_ms / 1e3)


def host_cpu():
    """Host core count and CPU model (the CPU baseline runs on these cores)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "model": model}


def oracle_sample(budget_s: float, h: int):
    """The CPU oracle, as it stands, on the 2,000-vertex Erdos-Renyi workload (G(2000,
    8000), the workload the oracle finishes in seconds), one thread: the median of up to
    three full decompositions within the budget.  Returns (edges/s, description, seconds
    of one decomposition)."""
    import oracle

    oracle.build()
    spec = config_graph("er_n2000")
    og = oracle.OracleGraph.from_raw(spec.n, spec.src, spec.dst)
    times = []
    while len(times) < 3 and (not times or sum(times) + times[-1] < budget_s):
        t0 = time.perf_counter()
        og.truss_decompose(h)
        times.append(time.perf_counter() - t0)
    dt = float(np.median(times))
    return (og.m / dt, f"oracle full decomposition of er_n2000 (G(2000,8000), m={og.m}, "
                       f"h={h}), single thread, median of {len(times)}", dt)


def run_reference(args, world, rank):
    if rank != 0:
        return
    h = WORKLOADS[args.workload][1]
    t_steps = []
    desc = None
    for _ in range(args.warmup + args.steps):
        v, desc, dt = oracle_sample(args.cpu_budget, h)
        t_steps.append((v, dt))
    vals = [v for v, _ in t_steps[args.warmup:]]
    value = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "ms_per_step": float(np.mean([dt for _, dt in t_steps[args.warmup:]]) * 1e3),
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "sample": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def round_bytes_host(n: int, eu: np.ndarray, ev: np.ndarray, stamp: np.ndarray, h: int):
    """Algorithmic bytes of the peel rounds, counted on the host from the graph and the round
    log (each edge's removal round), independently of the kernels' own counters.

    Per removed edge (a,b) of round s, with deg_s(x) the alive degree at the start of s:
      * selection: 8 B (the edge's bucket entry and its alive mark);
      * loss detection (h = 2): one candidate pair per old neighbour of either endpoint
        ({a,b}, {a, N(b)}, {b, N(a)}: deg_s(a) + deg_s(b) - 1 pairs; h = 1: the pair {a,b}),
        each 8 B: the adjacency slot that names it and one alive-adjacency word.
    Returns a dict of byte totals and counts for the whole peel."""
    m = eu.size
    if m == 0:
        return {"select": 0.0, "detect": 0.0, "pairs": 0, "frontier": 0}
    st = stamp.astype(np.int64)
    smax = int(st.max())
    x = np.concatenate([eu, ev]).astype(np.int64)
    s2 = np.concatenate([st, st])
    # alive degree of x at the start of round s = x's edges with stamp >= s
    key = x * (smax + 1) + (smax - s2)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    xs = x[order]
    block_start = np.searchsorted(xs, xs, side="left")
    run_end = np.searchsorted(ks, ks, side="right")
    deg_sorted = run_end - block_start
    deg = np.empty(2 * m, dtype=np.int64)
    deg[order] = deg_sorted
    da, db = deg[:m], deg[m:]
    pairs = (da + db - 1) if h >= 2 else np.ones(m, dtype=np.int64)
    return {"select": 8.0 * m, "detect": 8.0 * float(pairs.sum()), "pairs": int(pairs.sum()),
            "frontier": int(m)}


def _phase_classes(st, h):
    """Round kernels of a decomposition and their sampled device ms per timed slot."""
    timed = max(1, st["timed_slots"])
    if st["incremental"] and h == 3:
        return [("k_inc_select", st["ms_select"] / timed),
                ("k_loss_detect3 (radius-2 detection, radius-3 items)", st["ms_remove"] / timed),
                ("k_loss3_test", st["ms_find"] / timed),
                ("k_loss_delta", st["ms_update"] / timed),
                ("k_loss_apply_reduce", st["ms_minreduce"] / timed)]
    if st["incremental"]:
        return [("k_inc_select", st["ms_select"] / timed),
                ("k_loss_detect", st["ms_find"] / timed),
                ("k_loss_delta", st["ms_update"] / timed),
                ("k_loss_apply_reduce", st["ms_minreduce"] / timed)]
    return [("k_select", st["ms_select"] / timed),
            ("k_cand_*", st["ms_find"] / timed),
            ("k_remove", st["ms_remove"] / timed),
            ("k_ball (rebuild)", st["ms_ball"] / timed),
            ("k_make_items + k_hsup (rounds)", st["ms_update"] / timed),
            ("k_minreduce", st["ms_minreduce"] / timed)]


def measure_workload(htd, torch, lib, name, h, steps, warmup, flush, stream, dev, peaks,
                     profile=True, e2e=False):
    """Times `steps` steps (CSR build + decomposition, inputs in HBM, no timing flag) after
    `warmup` untimed ones, then runs one untimed profiling step with the phase events and
    stamps.  Returns the per-workload record (without the job-level keys)."""
    spec = config_graph(name)
    src_d = torch.from_numpy(spec.src).to(dev)
    dst_d = torch.from_numpy(spec.dst).to(dev)

    def step(flags, stamps=False):
        g = htd.htd_build_csr(spec.n, src_d, dst_d)
        t, stamp, st = htd.htd_truss_decompose(g, h, stamps=stamps, flags=flags)
        m = g.m
        eu, ev = htd.htd_edges(g) if stamps else (None, None)
        g.free()
        return m, st, (eu, ev, stamp)

    for _ in range(warmup):
        flush.zero_()
        step(0)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    stats, m = [], 0
    launches0 = lib.htd_kernel_launch_count()
    for i in range(steps):
        flush.zero_()  # untimed: evicts L2 between steps
        ev[i][0].record(stream)
        m, st, _ = step(0)
        ev[i][1].record(stream)
        stats.append(st)
    torch.cuda.synchronize()
    launches = (lib.htd_kernel_launch_count() - launches0) // max(1, steps)
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = float(np.mean(ms))
    s0 = stats[-1]
    rec = {"workload": f"{name}_h{h}", "n": spec.n, "m": m, "h": h, "steps": steps,
           "warmup": warmup, "ms_per_step": ms_step, "edges_per_sec": m / (ms_step / 1e3),
           "rounds": s0["rounds"], "levels": s0["levels"], "max_truss": s0["max_truss"],
           "incremental": s0["incremental"], "gpu_launches": int(launches),
           "kernel_counters": {"pairs_tested": s0["pairs_tested"], "pairs_lost": s0["pairs_lost"],
                               "pairs3_tested": s0["pairs3_tested"],
                               "pairs2_lost": s0["pairs2_lost"],
                               "rounds_rebuilt": s0["rounds_rebuilt"],
                               "member_tests": s0["member_tests"],
                               "edge_refreshes_per_endpoint": s0["hsup_evals"] - m,
                               "alg_bytes_detect": s0["alg_bytes_detect"],
                               "alg_bytes_update": s0["alg_bytes_update"],
                               "alg_bytes_ball": s0["alg_bytes_ball"],
                               "alg_bytes_hsup": s0["alg_bytes_hsup"]}}
    if not profile:
        return rec, ms, stats
    # profiling step (untimed): CSR build time, initial pass, sampled phase times, stamps
    flush.zero_()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    g = htd.htd_build_csr(spec.n, src_d, dst_d)
    c1.record(stream)
    t, stamp, stp = htd.htd_truss_decompose(g, h, stamps=True, flags=htd.HTD_OPT_TIMING)
    eu, evv = htd.htd_edges(g)
    g.free()
    torch.cuda.synchronize()
    ms_csr = c0.elapsed_time(c1)
    ms_init = stp["ms_initial_ball"] + stp["ms_initial_hsup"]
    # the untimed step's round time, split over the round kernels by their sampled shares
    rounds_ms = max(0.0, ms_step - ms_csr - ms_init)
    per_slot = _phase_classes(stp, h)
    tot = sum(v for _, v in per_slot) or 1.0
    slots = max(1, stp["slots"])
    phases = {"csr_build": {"ms": ms_csr, "launches": None},
              "k_ball (initial)": {"ms": stp["ms_initial_ball"], "launches": 1,
                                   # count and store passes count the same bytes
                                   # (h = 3 adds a radius-2 pass and the recovery rebuilds)
                                   "alg_bytes_kernel": (stp["alg_bytes_ball"] / 2
                                                        if stp["incremental"] and h <= 2 else None)},
              "k_hsup (initial)": {"ms": stp["ms_initial_hsup"], "launches": 1,
                                   "alg_bytes_kernel": stp["alg_bytes_hsup_initial"]}}
    for kname, v in per_slot:
        phases[kname] = {"ms": rounds_ms * v / tot, "launches": slots, "share_of_rounds": v / tot}
    hb = round_bytes_host(spec.n, host_np(eu), host_np(evv), host_np(stamp), h)
    if stp["incremental"] and h == 3:
        phases["k_inc_select"]["alg_bytes_host"] = hb["select"]
        phases["k_loss_detect3 (radius-2 detection, radius-3 items)"]["alg_bytes_host"] = hb["detect"]
        phases["k_loss3_test"]["alg_bytes_kernel"] = stp["alg_bytes_detect"]
        phases["k_loss_delta"]["alg_bytes_kernel"] = stp["alg_bytes_update"]
    elif stp["incremental"]:
        phases["k_inc_select"]["alg_bytes_host"] = hb["select"]
        phases["k_loss_detect"]["alg_bytes_host"] = hb["detect"]
        phases["k_loss_detect"]["alg_bytes_kernel"] = stp["alg_bytes_detect"]
        phases["k_loss_delta"]["alg_bytes_kernel"] = stp["alg_bytes_update"]
    else:
        phases["k_select"]["alg_bytes_host"] = hb["select"]
    rec["phases_ms_per_step"] = phases
    rec["phases_sum_over_step"] = sum(p["ms"] for p in phases.values()) / ms_step
    rec["host_round_counts"] = {"frontier_edges": hb["frontier"], "candidate_pairs": hb["pairs"]}
    # h-support evaluations: the initial pass computes every edge's h-support from scratch
    rec["hsup_evals_per_sec_initial"] = m / (ms_init / 1e3) if ms_init > 0 else None
    # dominant kernel and its roofline (host-counted bytes where defined)
    kern = max((k for k in phases if k != "csr_build"), key=lambda k: phases[k]["ms"])
    kp = phases[kern]
    byts = kp.get("alg_bytes_host", kp.get("alg_bytes_kernel"))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = (byts / (kp["ms"] / 1e3)) / 1e9 if (byts and kp["ms"] > 0) else None
    # the initial h-support pass streams every owned edge's other ball, reported beside the
    # (latency-bound) dominant kernel as a load rate: with dense balls each edge loads the
    # other endpoint's whole n-bit row, and the rows of hubs are re-read by many edges from
    # L2, so the rate is not DRAM traffic and is not set against the HBM copy peak
    hk = phases["k_hsup (initial)"]
    if hk["ms"] > 0 and hk.get("alg_bytes_kernel"):
        rec["initial_hsup_loads"] = {"kernel": "k_hsup (initial)",
                                     "bytes_loaded": hk["alg_bytes_kernel"],
                                     "load_rate_gbs": hk["alg_bytes_kernel"] / (hk["ms"] / 1e3) / 1e9,
                                     "ms": hk["ms"], "bytes_source": "kernel",
                                     "includes_l2_hits": True}
    rec["roofline"] = {"kernel": kern, "bound": "hbm", "achieved": achieved, "peak": hbm,
                       "unit": "GB/s", "frac": (achieved / hbm) if achieved else None,
                       "bytes_source": "host" if "alg_bytes_host" in kp else "kernel",
                       "alg_bytes_per_launch": (byts / kp["launches"]) if byts else None,
                       "launches_per_step": kp["launches"],
                       "ms_per_launch": kp["ms"] / kp["launches"] if kp["launches"] else None}
    return rec, ms, stats


def measure_served(htd, count: int, seed: int, rate: float, workers: int, rmat_scales, ba_n):
    """Served form: a Poisson request stream submitted on its arrival schedule to a server
    (continuous batching, admission by device memory); throughput and latency percentiles
    over the whole stream.  Graph generation happens before the stream starts."""
    from synth import served_requests

    reqs = served_requests(count, seed, rate, rmat_scales, ba_n)
    srv = htd.Server(workers=workers)
    try:
        ids = []
        t0 = time.perf_counter()
        for arr, n, s, d, h, _ in reqs:
            now = time.perf_counter() - t0
            if arr > now:
                time.sleep(arr - now)
            ids.append(srv.submit(n, s, d, h))
        infos = [srv.wait(rid, r[2].size)[3] for rid, r in zip(ids, reqs)]
        sinfo = srv.info()
    finally:
        srv.close()
    lat = np.array([i["done_s"] - i["submit_s"] for i in infos]) * 1e3
    wait = np.array([i["start_s"] - i["submit_s"] for i in infos]) * 1e3
    service = np.array([i["done_s"] - i["start_s"] for i in infos]) * 1e3
    span = max(i["done_s"] for i in infos) - min(i["submit_s"] for i in infos)
    edges = float(sum(i["m"] for i in infos))
    return {"workload": "served_poisson", "requests": count, "offered_rate_per_s": rate,
            "pool": {"rmat_scales": list(rmat_scales), "ba_n": list(ba_n), "h": [2, 3],
                     "seed": seed},
            "workers": workers, "edges": edges, "span_s": span,
            "edges_per_sec": edges / span, "requests_per_sec": count / span,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "queue_wait_ms": {"p50": float(np.percentile(wait, 50)),
                              "p99": float(np.percentile(wait, 99))},
            "service_ms": {"p50": float(np.percentile(service, 50)),
                           "p99": float(np.percentile(service, 99))},
            "offered_over_capacity": rate * float(np.mean(service)) / 1e3 / workers,
            "peak_running": sinfo["peak_running"], "budget_bytes": sinfo["budget_bytes"],
            "peak_reserved_bytes": sinfo["peak_reserved_bytes"],
            "retries": int(sum(i["retries"] for i in infos))}


_BATCH_CACHE = {}


def batch_workload(count: int, seed: int):
    """The batch's graphs, generated once per run in parallel processes."""
    if (count, seed) not in _BATCH_CACHE:
        import multiprocessing as mp

        from synth import batch_graphs

        with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
            _BATCH_CACHE[(count, seed)] = batch_graphs(count, seed, pool=pool)
    return _BATCH_CACHE[(count, seed)]


def measure_batched(htd, torch, count: int, seed: int, steps: int, warmup: int, stream, flush,
                    max_union_vertices: int = 0, flags: int = 0, table=None):
    """Batched form: `count` small graphs of mixed h decomposed by one call (or, with an
    autotuner table, one call per tuned setting), inputs resident on the device."""
    from paper_2411_06405_gb300 import autotune

    graphs = batch_workload(count, seed)
    if table is not None:
        prepared = autotune.prepare(graphs, table)
        run = lambda: autotune.run_prepared(prepared, count)
        sched = {"schedule": "autotuned", "settings": {f"{c}/{f}": len(i) for _, i, c, f in prepared}}
    else:
        b = htd.BatchInput(graphs)

        def run():
            res, st = htd.htd_truss_decompose_batched(b, flags=flags,
                                                      max_union_vertices=max_union_vertices)
            return res, st
        sched = {"schedule": "blocks" if flags & htd.HTD_OPT_BATCH_BLOCKS else "unions",
                 "max_union_vertices": max_union_vertices, "flags": flags}
    res, st = None, None
    for _ in range(warmup):
        res, st = run()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res, st = run()
        e.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(e))
    edges = float(sum(int(r.numel()) for r in res))
    mean = float(np.mean(ms))
    hs = np.array([g[3] for g in graphs])
    return dict({"workload": f"batched_{count}", "graphs": count, "seed": seed,
                 "vertices": int(sum(g[0] for g in graphs)),
                 "raw_pairs": int(sum(g[1].size for g in graphs)), "edges": edges,
                 "h_counts": {str(v): int((hs == v).sum()) for v in (2, 3)},
                 "steps": steps, "warmup": warmup, "ms_per_step": mean,
                 "edges_per_sec": edges / (mean / 1e3), "graphs_per_sec": count / (mean / 1e3),
                 "unions": st["unions"], "rounds_sum": st["rounds"],
                 "rounds_rebuilt": st["rounds_rebuilt"]}, **sched)


def measure_hindex(htd, torch, name: str, h: int, sweeps_list=(1, 8)):
    """The paper's H-index iteration (Sec. 4) on a workload: orders to the fixed point and
    device time, synchronous (Algorithm 2), with asynchronous updating by edge blocks, and
    synchronous with the Lemma 4 pruning (H^(n)(e) computed, summed over the orders); the
    fixed point + 2 is checked against the peel of the same graph."""
    spec = config_graph(name)
    g = htd.htd_build_csr(spec.n, torch.from_numpy(spec.src).cuda(), torch.from_numpy(spec.dst).cuda())
    t_peel, _, _ = htd.htd_truss_decompose(g, h)
    out = {"workload": f"{name}_h{h}_hindex", "m": g.m}
    runs = [(f"sweeps_{sw}", sw, False) for sw in sweeps_list] + [("sweeps_1_pruned", 1, True)]
    for label, sw, prune in runs:
        t, _, st = htd.htd_hindex_decompose(g, h, sweeps=sw, prune=prune)
        out[label] = {"orders": st["iterations"], "converged": st["converged"],
                      "ms": st["ms_total"], "edges_per_sec": g.m / (st["ms_total"] / 1e3),
                      "ball_entries": st["ball_entries"], "edge_evals": st["edge_evals"],
                      "vertex_evals": st["vertex_evals"],
                      "equals_peel": bool(torch.equal(t, t_peel))}
    g.free()
    return out


def ball_study(htd, torch):
    """Ball representation and hop threshold study: the same graphs decomposed with every
    ball dense (n-bit rows, one load per membership test) and in the compact form (sorted
    (word index, word) pairs; h = 3 then peels by rebuilds), and at h = 4 (rebuild rounds);
    device time and the ball storage of each."""
    out = []
    for name, h in (("rmat_s16", 2), ("dcsbm_n50k", 2), ("dcsbm_n50k", 3), ("dcsbm_n50k", 4),
                    ("er_n2000", 4), ("rmat_s16", 1)):
        spec = config_graph(name)
        src = torch.from_numpy(spec.src).cuda()
        dst = torch.from_numpy(spec.dst).cuda()
        for label, flags in (("dense", 0), ("compact", htd.HTD_OPT_COMPACT_BALLS)):
            if h >= 4 and label == "compact":
                continue  # h >= 4 always stores the smaller form
            g = htd.htd_build_csr(spec.n, src, dst)
            htd.htd_truss_decompose(g, h, flags=flags)  # warm (graph capture, allocation)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            _, _, st = htd.htd_truss_decompose(g, h, flags=flags)
            e.record()
            torch.cuda.synchronize()
            out.append({"graph": name, "n": spec.n, "m": g.m, "h": h, "balls": label,
                        "incremental": st["incremental"], "ms": a.elapsed_time(e),
                        "rounds": st["rounds"], "ball_pool_bytes": st["ball_pool_bytes"]})
            g.free()
    return out


def host_np(t):
    return t.cpu().numpy() if t is not None else None


def run_gpu(args, world, rank, local):
    import torch

    import paper_2411_06405_gb300 as htd
    from paper_2411_06405_gb300 import build as cuda_build

    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(htd.library_path()):
        cuda_build.build()
    if world > 1:
        torch.distributed.barrier()
    lib = htd._lib.load()
    name, h = WORKLOADS[args.workload]
    dev = torch.device("cuda", local)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    peaks, peak_kind = measured_peaks()

    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        rec, ms, stats = measure_workload(htd, torch, lib, name, h, args.steps, args.warmup,
                                          flush, stream, dev, peaks, profile=(rank == 0))
    m = rec["m"]
    t_max = max_over_ranks(float(np.sum(ms)), world, dev)
    ms_step = t_max / args.steps
    value = job_throughput(m, args.steps, t_max, world)

    # end to end through the host-buffer entry point (pinned buffers, copies inside)
    spec = config_graph(name)
    e2e_value, e2e_ms = None, []
    k = spec.src.size
    if not args.no_e2e:
        src_h = torch.from_numpy(spec.src).pin_memory()
        dst_h = torch.from_numpy(spec.dst).pin_memory()
        out = [torch.empty(k, dtype=torch.int32).pin_memory() for _ in range(3)]
        htd.htd_truss_decompose_host(spec.n, src_h, dst_h, h, *out)  # warm
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            htd.htd_truss_decompose_host(spec.n, src_h, dst_h, h, *out)
            b.record(stream)
            torch.cuda.synchronize()
            e2e_ms.append(a.elapsed_time(b))
        e2e_value = m / (float(np.mean(e2e_ms)) / 1e3)

    if rank != 0:
        return
    # the other single-GPU workloads, fewer steps each (their own records)
    configs = {}
    for wl in ([] if args.no_configs else [w for w in CONFIG_ENTRIES if w != args.workload]):
        cname, ch = WORKLOADS[wl]
        st_, wu_ = CONFIG_STEPS.get(wl, (3, 1))
        rc, _, _ = measure_workload(htd, torch, lib, cname, ch, st_, wu_, flush, stream, dev,
                                    peaks, profile=True)
        configs[wl] = rc
    if not args.no_hindex:
        for wl, sweeps in (("er_n2000_h2", (1, 8, 32)), ("dcsbm_n200k_h2", (1, 8))):
            cname, ch = WORKLOADS[wl]
            configs[wl + "_hindex"] = measure_hindex(htd, torch, cname, ch, sweeps)
    if not args.no_batched:
        # the batch as unions peeled round by round (one call), and with the autotuner's
        # schedule per group (one block per small graph in one persistent launch, unions of
        # tuned size and round variant for the rest)
        configs["batched_4096_unions"] = measure_batched(htd, torch, BATCHED["count"],
                                                         BATCHED["seed"], BATCHED["steps"],
                                                         BATCHED["warmup"], stream, flush)
        from paper_2411_06405_gb300 import autotune

        if os.path.exists(autotune.TABLE_PATH):
            configs["batched_4096_tuned"] = measure_batched(
                htd, torch, BATCHED["count"], BATCHED["seed"], BATCHED["steps"], BATCHED["warmup"],
                stream, flush, table=autotune.load(autotune.TABLE_PATH))
    if not args.no_served:
        configs["served_poisson"] = measure_served(htd, SERVED["count"], SERVED["seed"],
                                                   SERVED["rate"], SERVED["workers"],
                                                   SERVED["rmat_scales"], SERVED["ba_n"])
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, desc, dt = oracle_sample(args.cpu_budget, h)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
               "seconds_per_decomposition": dt, "host": host_cpu(),
               "workloads": {"er_n2000_h2": {"value": v, "unit": UNIT, "seconds": dt},
                             "rmat_s18_h2": "did not finish in budget (naive oracle; the "
                                            "initial pass alone is ~1e11 BFS steps)",
                             "dcsbm_n200k_h2": "did not finish in budget",
                             "dcsbm_n200k_h3": "did not finish in budget"}}
        if "er_n2000_h2" in configs:
            configs["er_n2000_h2"]["oracle_seconds"] = dt
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "graph": spec.recipe, "n": spec.n, "m": m, "h": h,
                   "parallelism": f"replicas{world}" if world > 1 else "single-gpu",
                   "l2": "256 MiB buffer written between timed steps (untimed)",
                   "timed_flags": "none (phase times come from one extra untimed step)"},
        "rounds": rec["rounds"], "levels": rec["levels"], "max_truss": rec["max_truss"],
        "hsup_evals_per_sec_initial": rec.get("hsup_evals_per_sec_initial"),
        "phases_ms_per_step": rec.get("phases_ms_per_step"),
        "phases_sum_over_step": rec.get("phases_sum_over_step"),
        "host_round_counts": rec.get("host_round_counts"),
        "kernel_counters": rec["kernel_counters"],
        "initial_hsup_loads": rec.get("initial_hsup_loads"),
        "roofline": dict(rec.get("roofline", {}), peak_source=peak_kind,
                         traffic=profile_traffic(args.workload, rec.get("roofline", {}).get("kernel"))),
        "e2e": None if e2e_value is None else {
            "value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(8 * k),
            "d2h_bytes_per_step": int(12 * m), "ms_per_step": float(np.mean(e2e_ms))},
        "gpu_launches": rec["gpu_launches"],
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "configs": configs,
    }
    print(json.dumps(line), flush=True)


def profile_traffic(workload, kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if any."""
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(prof) as f:
            ent = json.load(f).get(workload, {}).get(kernel)
        return ent.get("bytes_per_launch") if ent else None
    except (OSError, ValueError, AttributeError):
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat_s18_h2", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other single-GPU workloads' entries")
    ap.add_argument("--no-served", action="store_true", help="skip the served-stream entry")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched entry")
    ap.add_argument("--no-hindex", action="store_true", help="skip the H-index engine entries")
    ap.add_argument("--study", action="store_true",
                    help="ball representation / hop threshold study instead of the bench line")
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.study:
        import torch

        import paper_2411_06405_gb300 as htd
        from paper_2411_06405_gb300 import build as cuda_build

        torch.cuda.set_device(local)
        cuda_build.build()
        htd._lib.load()
        print(json.dumps({"study": "balls_and_h", "rows": ball_study(htd, torch)}), flush=True)
        return
    if world > 1:
        import torch

        backend = "nccl" if args.impl == "ours" else "gloo"
        torch.distributed.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        else:
            run_gpu(args, world, rank, local)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
