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

from synth import config_graph, rmat  # noqa: E402

WORKLOADS = {
    "rmat_s18_h2": ("rmat_s18", 2),
    "dcsbm_n200k_h2": ("dcsbm_n200k", 2),
    "dcsbm_n200k_h3": ("dcsbm_n200k", 3),
    "er_n2000_h2": ("er_n2000", 2),
    "rmat_s16_h2": ("rmat_s16", 2),
}
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


def oracle_sample(budget_s: float, h: int):
    """The CPU oracle, as it stands, on down-scaled R-MAT graphs with the workload's
    generator parameters: scales grow until the cumulative time passes the budget.
    Returns (edges/s of the largest completed scale, description, seconds)."""
    import oracle

    oracle.build()
    spent, best = 0.0, None
    for scale in range(8, 16):
        s, d = rmat(scale, 8, 0.57, 0.19, 0.19, 0x48545256)
        og = oracle.OracleGraph.from_raw(1 << scale, s, d)
        t0 = time.perf_counter()
        og.truss_decompose(h)
        dt = time.perf_counter() - t0
        spent += dt
        best = (og.m / dt, f"oracle full decomposition of R-MAT scale {scale} "
                           f"(m={og.m}, same a,b,c,d, h={h}), single thread", dt)
        if spent > budget_s or dt * 6 > budget_s:
            break
    return best


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


def run_gpu(args, world, rank, local):
    import torch

    import paper_2411_06405_gb300 as htd
    from paper_2411_06405_gb300 import build as cuda_build

    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(htd.library_path()):
        cuda_build.build()
    if world > 1:
        torch.distributed.barrier()
    htd._lib.load()
    lib = htd._lib.load()
    name, h = WORKLOADS[args.workload]
    spec = config_graph(name)
    dev = torch.device("cuda", local)
    src_d = torch.from_numpy(spec.src).to(dev)
    dst_d = torch.from_numpy(spec.dst).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step(flags):
        g = htd.htd_build_csr(spec.n, src_d, dst_d)
        t, _, st = htd.htd_truss_decompose(g, h, flags=flags)
        m = g.m
        g.free()
        return m, st

    for _ in range(args.warmup):
        flush.zero_()
        step(htd.HTD_OPT_TIMING)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats, m = [], 0
    launches0 = lib.htd_kernel_launch_count()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()  # untimed: evicts L2 between steps
            ev[i][0].record(stream)
            m, st = step(htd.HTD_OPT_TIMING)
            ev[i][1].record(stream)
            stats.append(st)
        torch.cuda.synchronize()
    launches = lib.htd_kernel_launch_count() - launches0
    ms = [a.elapsed_time(b) for a, b in ev]
    t_max = max_over_ranks(float(np.sum(ms)), world, dev)
    ms_step = t_max / args.steps
    value = job_throughput(m, args.steps, t_max, world)

    # end to end through the host-buffer entry point (pinned buffers, copies inside)
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
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    s0 = stats[-1]

    def mean(key):
        return float(np.mean([s[key] for s in stats]))

    slots = max(1, s0["slots"])
    timed = max(1, s0["timed_slots"])
    m_edges = float(m)
    # kernel classes of one step: (name, device ms per step, launches per step, alg bytes)
    if s0["round_kernel_launches"] > 0:  # persistent round kernel
        scan = 8.0 * m_edges * slots  # two passes over the supports per slot
        classes = [("k_rounds_persistent", mean("ms_round_kernel"), s0["round_kernel_launches"],
                     mean("alg_bytes_detect") + mean("alg_bytes_update") + scan)]
    elif s0["incremental"]:
        # phase times are sampled (every 16th batch); scale the per-slot mean to all slots
        per = slots / timed
        classes = [
            ("k_loss_detect", mean("ms_find") * per, slots, mean("alg_bytes_detect")),
            ("k_loss_delta", mean("ms_update") * per, slots, mean("alg_bytes_update")),
            ("k_inc_select", mean("ms_select") * per, slots, 4.0 * m_edges * slots),
            ("k_loss_apply_reduce", mean("ms_minreduce") * per, slots, 4.0 * m_edges * slots),
        ]
    else:
        per = slots / timed
        classes = [("k_ball (rebuild rounds)", mean("ms_ball") * per, slots, None),
                   ("k_hsup (rounds)", mean("ms_update") * per, slots, None)]
    classes += [
        ("k_ball (initial store)", mean("ms_initial_ball"), 1, mean("alg_bytes_ball") / 2),
        ("k_hsup (initial)", mean("ms_initial_hsup"), 1, mean("alg_bytes_hsup")),
    ]
    kern, k_ms, k_launches, k_bytes = max(classes, key=lambda c: c[1])
    achieved = (k_bytes / (k_ms / 1e3)) / 1e9 if (k_bytes and k_ms > 0) else None
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            with open(prof) as f:
                tj = json.load(f)
            ent = tj.get(args.workload, {}).get(kern)
            if ent:
                traffic = ent.get("bytes_per_launch")
        except (OSError, ValueError):
            traffic = None
    phases = {name: {"ms": ms, "launches": ln, "alg_bytes": b} for name, ms, ln, b in classes}
    hsup_rate = float(np.mean([s["hsup_evals"] for s in stats])) / (ms_step / 1e3)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, desc, dt = oracle_sample(args.cpu_budget, h)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "graph": spec.recipe, "n": spec.n, "m": m, "h": h,
                   "parallelism": f"replicas{world}" if world > 1 else "single-gpu",
                   "l2": "256 MiB buffer written between timed steps (untimed)"},
        "hsup_evals_per_sec": hsup_rate,
        "rounds": s0["rounds"], "levels": s0["levels"], "max_truss": s0["max_truss"],
        "hsup_evals": s0["hsup_evals"], "pairs_tested": s0["pairs_tested"],
        "pairs_lost": s0["pairs_lost"], "member_tests": s0["member_tests"],
        "phases_ms_per_step": phases,
        "roofline": {"kernel": kern, "bound": "hbm", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": (achieved / hbm) if achieved else None,
                     "traffic": traffic, "peak_source": peak_kind,
                     "alg_bytes_per_launch": (k_bytes / k_launches) if k_bytes else None,
                     "launches_per_step": k_launches, "ms_per_launch": k_ms / k_launches},
        "e2e": None if e2e_value is None else {
            "value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(8 * k),
            "d2h_bytes_per_step": int(12 * m), "ms_per_step": float(np.mean(e2e_ms))},
        "gpu_launches": int(launches // args.steps),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


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
    args = ap.parse_args()
    world, rank, local = dist_env()
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
