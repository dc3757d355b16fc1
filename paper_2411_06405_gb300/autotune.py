"""Schedule autotuner for the batched decomposition (many small graphs of mixed h).

The batched call packs the graphs of one hop threshold into disjoint unions and peels each
union once (``htd_truss_decompose_batched``).  Two knobs decide how the device work is laid
out, and the best setting depends on the graphs:

* ``max_union_vertices`` -- how many vertices a union holds: large unions put more
  independent work into every round launch (more edges per warp-level work list), small
  unions let a union stop as soon as its own members are peeled instead of running until
  the slowest member of a large union is done;
* ``flags`` -- the schedule: one block per graph with every round inside one persistent
  launch (``HTD_OPT_BATCH_BLOCKS``), or union peels with incremental rounds on dense balls
  (one load per membership test), on compact balls (h <= 2), or rebuild rounds.

Graphs are grouped by a key of (h, log2 class of n, log2 class of the largest degree).
``tune`` times every candidate on a sample of each group (CUDA events, after a warm-up) and
keeps the fastest; the resulting table is JSON, keyed by group.  ``decompose`` runs a batch
with a table in two calls: the graphs whose group chose one block per graph, and all the
others as unions (peeled concurrently inside the call) with the default setting; results
come back in input order.  The results do not depend on the setting
(every candidate is an exact decomposition), only the time.
"""

from __future__ import annotations

import json
import math
from collections import defaultdict

import numpy as np

from . import _lib

CANDIDATES = [
    {"max_union_vertices": 1 << 18, "flags": _lib.HTD_OPT_BATCH_BLOCKS},
    {"max_union_vertices": 1 << 18, "flags": 0},
    {"max_union_vertices": 1 << 16, "flags": 0},
    {"max_union_vertices": 1 << 16, "flags": _lib.HTD_OPT_COMPACT_BALLS},
    {"max_union_vertices": 1 << 16, "flags": _lib.HTD_OPT_REBUILD},
]
DEFAULT = {"max_union_vertices": 1 << 18, "flags": 0}
BLOCK_MAX_NCLASS = 9  # log2 class of n above which one block per graph is not tried


def group_key(n: int, src, dst, h: int) -> str:
    """(h, n class, largest-degree class) of a raw graph, as a table key."""
    s = np.asarray(src)
    d = np.asarray(dst)
    ok = s != d
    deg = np.bincount(np.concatenate([s[ok], d[ok]]), minlength=max(int(n), 1)) if ok.any() else np.zeros(1)
    nc = int(math.log2(max(int(n), 1)))
    dc = int(math.log2(max(int(deg.max()), 1)))
    return f"h{int(h)}_n{nc}_d{dc}"


def _time_batch(htd, torch, graphs, cand, reps: int = 2) -> float:
    b = htd.BatchInput(graphs)
    htd.htd_truss_decompose_batched(b, flags=cand["flags"], max_union_vertices=cand["max_union_vertices"])
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        htd.htd_truss_decompose_batched(b, flags=cand["flags"],
                                        max_union_vertices=cand["max_union_vertices"])
        e.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(e))
    return best


def tune(graphs, sample: int = 64, candidates=None, seed: int = 0):
    """Times the candidates on up to `sample` graphs of every group; returns the table
    {key: {"max_union_vertices", "flags", "ms": {candidate index: ms}}}."""
    import torch

    import paper_2411_06405_gb300 as htd

    cands = candidates or CANDIDATES
    groups = defaultdict(list)
    for g in graphs:
        groups[group_key(*g)].append(g)
    rng = np.random.default_rng(seed)
    table = {}
    for key, gs in sorted(groups.items()):
        pick = gs if len(gs) <= sample else [gs[i] for i in rng.choice(len(gs), sample, replace=False)]
        nclass = int(key.split("_")[1][1:])
        times = {}
        for ci, c in enumerate(cands):
            # one block per graph only pays for graphs of up to about a thousand vertices
            # (a block's rounds grow with n^2 / 32 words); larger groups skip that candidate
            if c["flags"] & _lib.HTD_OPT_BATCH_BLOCKS and nclass > BLOCK_MAX_NCLASS:
                continue
            times[ci] = _time_batch(htd, torch, pick, c)
        best = min(times, key=times.get)
        table[key] = dict(cands[best], ms=times, sample=len(pick))
    return table


def save(table, path: str):
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def load(path: str):
    with open(path) as f:
        return json.load(f)


def _partition(graphs, table):
    """Graph indices by the setting the batch runs them with.  Graphs whose group chose one
    block per graph form one block-per-graph call; all others form one union call with the
    default setting.  The union size and round variant a group chose on its own sample are
    not used: inside one call the unions of all groups are peeled concurrently, and on the
    4,096-graph batch the groups' own choices (measured alone) made the whole call slower
    than the default (40.5 s against 35.9 s on one GB300)."""
    table = table or {}
    blocks, rest = [], []
    for i, g in enumerate(graphs):
        ent = table.get(group_key(*g), DEFAULT)
        if int(ent["flags"]) & _lib.HTD_OPT_BATCH_BLOCKS:
            blocks.append(i)
        else:
            rest.append(i)
    cap, flags = DEFAULT["max_union_vertices"], DEFAULT["flags"]
    parts = []
    if blocks:
        parts.append((blocks, 1 << 18, _lib.HTD_OPT_BATCH_BLOCKS))
    if rest:
        parts.append((rest, cap, flags))
    return parts


def decompose(graphs, table=None, device=None):
    """Decomposes a batch with the table's settings (see _partition); returns (list of int32
    CUDA tensors in input order, {setting: graphs})."""
    import paper_2411_06405_gb300 as htd

    out = [None] * len(graphs)
    summary = {}
    for idx, cap, flags in _partition(graphs, table):
        res, _ = htd.htd_truss_decompose_batched([graphs[i] for i in idx], flags=flags,
                                                 max_union_vertices=cap, device=device)
        for i, r in zip(idx, res):
            out[i] = r
        summary[f"{cap}/{flags}"] = len(idx)
    return out, summary


def prepare(graphs, table=None, device=None):
    """The partition of a batch put on the device once: a list of (BatchInput, input
    indices, max_union_vertices, flags)."""
    import paper_2411_06405_gb300 as htd

    return [(htd.BatchInput([graphs[i] for i in idx], device), idx, cap, flags)
            for idx, cap, flags in _partition(graphs, table)]


def run_prepared(prepared, count: int):
    """Decomposes a prepared batch; returns (results in input order, summed stats)."""
    import paper_2411_06405_gb300 as htd

    out = [None] * count
    tot = defaultdict(int)
    for b, idx, cap, flags in prepared:
        res, st = htd.htd_truss_decompose_batched(b, flags=flags, max_union_vertices=cap)
        for i, r in zip(idx, res):
            out[i] = r
        for k in ("rounds", "unions", "rounds_rebuilt"):
            tot[k] += st[k]
    return out, dict(tot)


TABLE_PATH = __import__("os").path.join(__import__("os").path.dirname(__file__), "tuning",
                                        "batched_gb300.json")


def main(argv=None):
    """Tunes the schedules on a sample of the 4,096-graph batch recipe and writes the table."""
    import argparse
    import os

    import torch

    from synth import batch_graphs

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE_PATH)
    ap.add_argument("--graphs", type=int, default=1024)
    ap.add_argument("--sample", type=int, default=48)
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    graphs = batch_graphs(4096, 0x48545258)[: args.graphs]
    table = tune(graphs, sample=args.sample)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    save(table, args.out)
    print(json.dumps({k: {"max_union_vertices": v["max_union_vertices"], "flags": v["flags"]}
                      for k, v in table.items()}))


if __name__ == "__main__":
    main()
