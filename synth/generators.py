"""Random-graph models used as stand-ins for the paper's KONECT networks (Table 1).

Every generator is a pure function of its arguments and a seed (numpy PCG64), so the
same call returns the same arrays on x86 and on Arm.  Outputs are raw vertex-id pairs
as int32 numpy arrays; nothing here canonicalises, sorts or deduplicates unless the
model itself is defined over distinct pairs (G(n,M), DC-SBM with a distinct-edge target).

Workloads (sizes follow the paper's datasets, Table 1, by shape):

* ``er_n2000``    -- Erdos-Renyi G(n=2000, M=8000): small, the oracle finishes in seconds.
* ``rmat_s18``    -- R-MAT scale 18, edge factor 8, (a,b,c,d)=(0.57,0.19,0.19,0.05),
                     seeded vertex permutation; raw pairs (loops and duplicates kept).
                     Stands in for the Amazon TWEB graph (262,111 vertices).
* ``dcsbm_n200k`` -- degree-corrected SBM, 200 power-law blocks, mean degree 12,
                     10% inter-block edges.  Stands in for the Amazon MDS graph.
* ``batch_graphs`` -- many small ER / BA graphs with mixed h (the batched form; 4,096
                     graphs of 50..5,000 vertices at seed 0x48545258 for the benchmark).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Seed of workload i is CONFIG_SEED_BASE + i (0x48545255 = ASCII "HTRU").
CONFIG_SEED_BASE = 0x48545255


@dataclass(frozen=True)
class GraphSpec:
    name: str
    n: int
    src: np.ndarray  # int32 raw endpoints
    dst: np.ndarray  # int32 raw endpoints
    h: tuple  # hop thresholds this workload is decomposed at
    recipe: str


def _distinct_pairs(rng: np.random.Generator, draw, target: int, n: int):
    """Accumulate distinct unordered non-loop pairs from ``draw(batch)`` in draw order.

    Keeps the first occurrence of each pair so the result is a deterministic function
    of the seed.  Returns (src, dst) int32 with src < dst.
    """
    keys = np.empty(0, dtype=np.int64)
    order = np.empty(0, dtype=np.int64)
    drawn = 0
    batch = max(1024, int(target * 1.2))
    while keys.size < target:
        a, b = draw(batch)
        a = a.astype(np.int64)
        b = b.astype(np.int64)
        ok = a != b
        a, b = a[ok], b[ok]
        lo = np.minimum(a, b)
        hi = np.maximum(a, b)
        k = lo * n + hi
        allk = np.concatenate([keys, k])
        allo = np.concatenate([order, drawn + np.arange(k.size, dtype=np.int64)])
        drawn += k.size
        uk, first = np.unique(allk, return_index=True)
        keys = uk
        order = allo[first]
        batch = max(1024, int((target - keys.size) * 1.5) + 1024)
    sel = np.argsort(order, kind="stable")[:target]
    k = keys[sel]
    return (k // n).astype(np.int32), (k % n).astype(np.int32)


def erdos_renyi_gnm(n: int, m: int, seed: int):
    """G(n, M): M distinct unordered pairs drawn uniformly, no self-loops."""
    if m > n * (n - 1) // 2:
        raise ValueError("G(n,M) needs M <= n(n-1)/2")
    rng = np.random.default_rng(seed)

    def draw(b):
        return rng.integers(0, n, size=b), rng.integers(0, n, size=b)

    return _distinct_pairs(rng, draw, m, n)


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
         permute: bool = True):
    """Recursive-matrix (R-MAT) generator, Graph500 style, no noise.

    Draws ``edge_factor * 2**scale`` ordered pairs; at each of ``scale`` levels the
    quadrant is (0,0) w.p. a, (0,1) w.p. b, (1,0) w.p. c, (1,1) w.p. 1-a-b-c.
    A seeded permutation then relabels the vertices.  Loops and duplicates are kept.
    """
    n = 1 << scale
    m = edge_factor * n
    rng = np.random.default_rng(seed)
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    ab = a + b
    abc = a + b + c
    for lvl in range(scale):
        r = rng.random(m)
        sbit = r >= ab  # quadrants c, d
        dbit = ((r >= a) & (r < ab)) | (r >= abc)  # quadrants b, d
        src |= sbit.astype(np.int64) << lvl
        dst |= dbit.astype(np.int64) << lvl
    if permute:
        perm = rng.permutation(n)
        src = perm[src]
        dst = perm[dst]
    return src.astype(np.int32), dst.astype(np.int32)


def _largest_remainder(weights: np.ndarray, total: int) -> np.ndarray:
    q = weights / weights.sum() * total
    base = np.floor(q).astype(np.int64)
    rem = total - int(base.sum())
    if rem > 0:
        idx = np.argsort(-(q - base), kind="stable")[:rem]
        base[idx] += 1
    return base


def dcsbm(n: int, blocks: int, size_exponent: float, min_size: int,
          theta_exponent: float, m_target: int, inter_fraction: float, seed: int,
          max_block_fraction: float = 0.1):
    """Degree-corrected stochastic block model with power-law block sizes.

    * block sizes: discrete power law (exponent ``size_exponent``, minimum ``min_size``),
      each draw capped at ``max_block_fraction * n``, then scaled to sum to n by
      largest remainder;
    * degree propensities theta ~ Pareto(``theta_exponent``, min 1), capped at sqrt(n),
      normalised within each block;
    * ``m_target`` distinct edges: a share ``1 - inter_fraction`` inside one block
      (block chosen proportional to its size), the rest between two distinct blocks
      (each chosen proportional to size); endpoints drawn proportional to theta;
      loops and duplicates are rejected.
    """
    rng = np.random.default_rng(seed)
    u = rng.random(blocks)
    raw = np.floor(min_size * u ** (-1.0 / (size_exponent - 1.0)))
    raw = np.minimum(raw, max_block_fraction * n)
    sizes = _largest_remainder(raw, n)
    sizes = np.maximum(sizes, 1)
    # fix the total after the max(.,1) guard
    diff = n - int(sizes.sum())
    sizes[int(np.argmax(sizes))] += diff
    block_start = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    block_of = np.repeat(np.arange(blocks), sizes)

    theta = rng.random(n) ** (-1.0 / (theta_exponent - 1.0))
    theta = np.minimum(theta, np.sqrt(n))
    bsum = np.bincount(block_of, weights=theta, minlength=blocks)
    theta = theta / bsum[block_of]
    # per-block cumulative theta for inverse-CDF sampling
    cdf = np.empty(n)
    for bi in range(blocks):
        s, e = block_start[bi], block_start[bi] + sizes[bi]
        cdf[s:e] = np.cumsum(theta[s:e])
        cdf[e - 1] = 1.0
    bprob = sizes / sizes.sum()
    bcdf = np.cumsum(bprob)
    bcdf[-1] = 1.0

    def pick_vertex(blk):
        r = rng.random(blk.size)
        out = np.empty(blk.size, dtype=np.int64)
        for bi in np.unique(blk):
            sel = np.nonzero(blk == bi)[0]
            s, e = block_start[bi], block_start[bi] + sizes[bi]
            j = np.searchsorted(cdf[s:e], r[sel], side="right")
            out[sel] = s + np.minimum(j, e - s - 1)
        return out

    def pick_block(cnt):
        return np.minimum(np.searchsorted(bcdf, rng.random(cnt), side="right"), blocks - 1)

    def draw(b):
        n_inter = int(round(b * inter_fraction))
        n_intra = b - n_inter
        bi = pick_block(n_intra)
        a1 = pick_vertex(bi)
        a2 = pick_vertex(bi)
        b1 = pick_block(n_inter)
        b2 = pick_block(n_inter)
        same = b1 == b2
        while same.any():
            b2[same] = pick_block(int(same.sum()))
            same = b1 == b2
        c1 = pick_vertex(b1)
        c2 = pick_vertex(b2)
        return np.concatenate([a1, c1]), np.concatenate([a2, c2])

    return _distinct_pairs(rng, draw, m_target, n)


def barabasi_albert(n: int, m0: int, seed: int):
    """Preferential attachment: an m0-clique, then each new vertex attaches m0 edges
    to distinct existing vertices chosen with probability proportional to degree."""
    if n <= m0:
        raise ValueError("BA needs n > m0")
    rng = np.random.default_rng(seed)
    src, dst = [], []
    for i in range(m0):
        for j in range(i + 1, m0):
            src.append(i)
            dst.append(j)
    # endpoint multiset: each vertex appears deg times
    pool = np.empty(2 * (m0 * (m0 - 1) // 2 + (n - m0) * m0) + 2 * m0, dtype=np.int64)
    plen = 0
    for s, d in zip(src, dst):
        pool[plen] = s
        pool[plen + 1] = d
        plen += 2
    if plen == 0:  # m0 == 1: seed the pool with vertex 0
        pool[0] = 0
        plen = 1
    for v in range(m0, n):
        targets = set()
        while len(targets) < m0:
            for t in pool[rng.integers(0, plen, size=2 * m0)]:
                if len(targets) < m0:
                    targets.add(int(t))
        for t in sorted(targets):
            src.append(v)
            dst.append(t)
            pool[plen] = v
            pool[plen + 1] = t
            plen += 2
    return np.asarray(src, dtype=np.int32), np.asarray(dst, dtype=np.int32)


def config_graph(name: str) -> GraphSpec:
    """The named benchmark workloads (see module docstring)."""
    if name == "er_n2000":
        s, d = erdos_renyi_gnm(2000, 8000, CONFIG_SEED_BASE + 0)
        return GraphSpec(name, 2000, s, d, (2,),
                         "Erdos-Renyi G(n=2000, M=8000), distinct pairs, seed 0x48545255")
    if name == "rmat_s18":
        s, d = rmat(18, 8, 0.57, 0.19, 0.19, CONFIG_SEED_BASE + 1)
        return GraphSpec(name, 1 << 18, s, d, (2,),
                         "R-MAT scale 18, 2,097,152 raw pairs, (a,b,c,d)=(0.57,0.19,0.19,0.05), "
                         "seeded permutation, seed 0x48545256")
    if name == "dcsbm_n200k":
        s, d = dcsbm(200_000, 200, 2.1, 100, 2.5, 1_200_000, 0.10, CONFIG_SEED_BASE + 2)
        return GraphSpec(name, 200_000, s, d, (2, 3),
                         "DC-SBM n=200,000, 200 blocks (size exponent 2.1, min 100), theta "
                         "Pareto 2.5 capped at sqrt(n), 1,200,000 edges, 10% inter-block, "
                         "seed 0x48545257")
    if name == "dcsbm_n50k":
        # a quarter-size version of the DC-SBM workload (profiling runs)
        s, d = dcsbm(50_000, 50, 2.1, 100, 2.5, 300_000, 0.10, CONFIG_SEED_BASE + 2)
        return GraphSpec(name, 50_000, s, d, (2, 3),
                         "DC-SBM n=50,000, 50 blocks (size exponent 2.1, min 100), theta "
                         "Pareto 2.5 capped at sqrt(n), 300,000 edges, 10% inter-block, "
                         "seed 0x48545257")
    if name.startswith("rmat_s"):
        scale = int(name[len("rmat_s"):])
        s, d = rmat(scale, 8, 0.57, 0.19, 0.19, CONFIG_SEED_BASE + 1)
        return GraphSpec(name, 1 << scale, s, d, (2,),
                         f"R-MAT scale {scale}, edge factor 8, (0.57,0.19,0.19,0.05)")
    raise KeyError(name)


def batch_params(count: int, seed: int, n_lo: int = 50, n_hi: int = 5000):
    """Per-graph parameters of a batch, drawn in order from one seeded stream: a list of
    (sub_seed, n, h, kind, m0) with kind 0 = Erdos-Renyi (mean degree 8), 1 = BA."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        sub = seed ^ i
        n = int(rng.integers(n_lo, n_hi + 1))
        h = int(rng.integers(2, 4))
        if rng.random() < 0.5:
            out.append((sub, n, h, 0, 0))
        else:
            m0 = int(rng.integers(2, 9))
            out.append((sub, max(n, m0 + 1), h, 1, m0))
    return out


def batch_graph(param):
    """One graph of a batch from its batch_params entry: (n, src, dst, h)."""
    sub, n, h, kind, m0 = param
    if kind == 0:
        s, d = erdos_renyi_gnm(n, min(4 * n, n * (n - 1) // 2), sub)
    else:
        s, d = barabasi_albert(n, m0, sub)
    return n, s, d, h


def batch_graphs(count: int, seed: int, n_lo: int = 50, n_hi: int = 5000, pool=None):
    """A batch of small graphs: per graph n ~ U[n_lo, n_hi], either Erdos-Renyi with mean
    degree 8 (M = 4n distinct pairs) or Barabasi-Albert with m0 ~ U{2..8}, and a hop
    threshold h ~ U{2,3}.  Graph i draws its edges from sub-seed seed ^ i.  Returns a list
    of (n, src, dst, h).  `pool` (optional): a process pool whose map builds the graphs."""
    params = batch_params(count, seed, n_lo, n_hi)
    if pool is not None:
        return list(pool.map(batch_graph, params, chunksize=16))
    return [batch_graph(p) for p in params]


def served_requests(count: int, seed: int, rate: float = 200.0, rmat_scales=(10, 20),
                    ba_n=(1_000, 1_000_000)):
    """A Poisson request stream over a mixed pool: arrival times with exponential gaps of
    mean 1/rate seconds; each request is, with equal odds, an R-MAT graph (scale uniform in
    rmat_scales, edge factor 8, (0.57,0.19,0.19,0.05)) or a Barabasi-Albert graph (n
    log-uniform in ba_n, m0 ~ U{2..8}), with h ~ U{2,3}.  Request i draws its graph from
    sub-seed seed ^ i.  Returns a list of (arrival_s, n, src, dst, h, kind)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        sub = seed ^ i
        h = int(rng.integers(2, 4))
        if rng.random() < 0.5:
            sc = int(rng.integers(rmat_scales[0], rmat_scales[1] + 1))
            s, d = rmat(sc, 8, 0.57, 0.19, 0.19, sub)
            out.append((t, 1 << sc, s, d, h, f"rmat_s{sc}"))
        else:
            lo, hi = np.log(ba_n[0]), np.log(ba_n[1])
            n = int(round(np.exp(rng.uniform(lo, hi))))
            m0 = int(rng.integers(2, 9))
            s, d = barabasi_albert(max(n, m0 + 1), m0, sub)
            out.append((t, max(n, m0 + 1), s, d, h, f"ba_n{n}_m{m0}"))
    return out


def small_corpus(count: int, seed: int, max_n: int = 40):
    """Mixed small graphs (ER, BA, R-MAT) for bulk parity checks: yields (n, src, dst)."""
    rng = np.random.default_rng(seed)
    for i in range(count):
        kind = i % 3
        sub = int(rng.integers(0, 2**31))
        if kind == 0:
            n = int(rng.integers(2, max_n + 1))
            mmax = n * (n - 1) // 2
            m = int(rng.integers(1, max(2, min(mmax, 4 * n)) + 1))
            m = min(m, mmax)
            s, d = erdos_renyi_gnm(n, m, sub)
        elif kind == 1:
            m0 = int(rng.integers(1, 5))
            n = int(rng.integers(m0 + 1, max_n + 1))
            s, d = barabasi_albert(n, m0, sub)
        else:
            scale = int(rng.integers(2, max(3, int(np.log2(max_n))) + 1))
            n = 1 << scale
            s, d = rmat(scale, 4, 0.57, 0.19, 0.19, sub)
        yield n, s, d
