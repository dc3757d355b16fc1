"""Independent checks that pin the oracle to mathematics rather than to itself.

Nothing here calls or shares code with ``oracle/`` (a C library) or with the CUDA path:

* ``apsp``                -- all-pairs shortest paths by Floyd-Warshall (min-plus), a
                             different algorithm from the oracle's BFS.
* ``sup_from_distances``  -- Def. 2/3 read off a distance matrix.
* ``truss_by_definition`` -- Def. 4 by exhaustive enumeration of edge subsets: for every k,
                             the (k,h)-truss is the union of all subsets whose edges all
                             have h-support >= k-2 inside the subset; the union is checked
                             to satisfy the condition itself (so it is the unique maximal
                             one), and t(e,h) is the largest k whose truss holds e.
* ``classic_truss``       -- textbook triangle peeling (support decremented per lost
                             triangle), for the h = 1 special case.
* closed-form families    -- K_n, star, path, cycle, complete bipartite.
"""

from __future__ import annotations

import itertools

import numpy as np

INF = 1 << 20


def canonical(n, src, dst):
    """Set-based canonicalisation: sorted distinct (min,max) pairs without loops."""
    s = {(min(int(a), int(b)), max(int(a), int(b))) for a, b in zip(src, dst) if a != b}
    return sorted(s)


def apsp(n, edges, mask=None):
    """Floyd-Warshall over the edge subset ``mask`` (bool per edge; all edges if None)."""
    d = np.full((n, n), INF, dtype=np.int64)
    np.fill_diagonal(d, 0)
    for i, (u, v) in enumerate(edges):
        if mask is None or mask[i]:
            d[u, v] = 1
            d[v, u] = 1
    for k in range(n):
        d = np.minimum(d, d[:, k : k + 1] + d[k : k + 1, :])
    return d


def sup_from_distances(d, edges, h, mask=None):
    """sup(e,h) = #{w not in {u,v} : d(u,w) <= h and d(v,w) <= h} for edges in mask."""
    n = d.shape[0]
    out = np.full(len(edges), -1, dtype=np.int64)
    for i, (u, v) in enumerate(edges):
        if mask is not None and not mask[i]:
            continue
        near = (d[u] <= h) & (d[v] <= h)
        near[u] = False
        near[v] = False
        out[i] = int(near.sum()) if n else 0
    return out


def truss_by_definition(n, edges, h):
    """t(e,h) straight from Def. 4 by enumerating all 2^m edge subsets (m <= ~12)."""
    m = len(edges)
    if m == 0:
        return np.zeros(0, dtype=np.int64)
    # minimum h-support over each nonempty subset, sup measured inside the subset
    min_sup = {}
    for bits in range(1, 1 << m):
        mask = [(bits >> i) & 1 == 1 for i in range(m)]
        d = apsp(n, edges, mask)
        s = sup_from_distances(d, edges, h, mask)
        min_sup[bits] = int(min(s[i] for i in range(m) if mask[i]))
    t = np.zeros(m, dtype=np.int64)
    k = 2
    while True:
        union = 0
        for bits, ms in min_sup.items():
            if ms >= k - 2:
                union |= bits
        if union == 0:
            break
        # maximality / uniqueness: the union must itself be a (k,h)-truss
        assert min_sup[union] >= k - 2, "union of (k,h)-trusses is not a (k,h)-truss"
        for i in range(m):
            if (union >> i) & 1:
                t[i] = k
        k += 1
    return t


def classic_truss(n, edges):
    """Classic k-truss decomposition by triangle peeling (h = 1 special case)."""
    adj = [set() for _ in range(n)]
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    eid = {e: i for i, e in enumerate(edges)}
    sup = {i: len(adj[u] & adj[v]) for i, (u, v) in enumerate(edges)}
    t = np.zeros(len(edges), dtype=np.int64)
    alive = set(range(len(edges)))
    k = 2
    while alive:
        low = [i for i in alive if sup[i] <= k - 2]
        if not low:
            k += 1
            continue
        while low:
            i = low.pop()
            if i not in alive:
                continue
            u, v = edges[i]
            t[i] = k
            alive.discard(i)
            for w in adj[u] & adj[v]:
                for a, b in ((u, w), (v, w)):
                    j = eid[(min(a, b), max(a, b))]
                    if j in alive:
                        sup[j] -= 1
                        if sup[j] <= k - 2:
                            low.append(j)
            adj[u].discard(v)
            adj[v].discard(u)
    return t


def triangle_hindex_orders(n, edges, orders):
    """Classic H-index iteration for the k-truss (h = 1): order 0 is every edge's triangle
    count; order k+1 of e is the H-index of {min(H_k(e1), H_k(e2))} over the triangle edge
    pairs (e1, e2) of e.  Returns the value arrays of orders 0..orders."""
    adj = [set() for _ in range(n)]
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    eid = {e: i for i, e in enumerate(edges)}
    pairs = []
    for u, v in edges:
        pairs.append([(eid[(min(u, w), max(u, w))], eid[(min(v, w), max(v, w))])
                      for w in sorted(adj[u] & adj[v])])
    cur = np.array([len(p) for p in pairs], dtype=np.int64)
    out = [cur.copy()]
    for _ in range(orders):
        nxt = np.zeros_like(cur)
        for i, p in enumerate(pairs):
            vals = sorted((min(cur[a], cur[b]) for a, b in p), reverse=True)
            y = 0
            while y < len(vals) and vals[y] >= y + 1:
                y += 1
            nxt[i] = y
        cur = nxt
        out.append(cur.copy())
    return out


# ---- closed-form families -------------------------------------------------------------

def complete(n):
    return [(a, b) for a, b in itertools.combinations(range(n), 2)]


def star(s):
    return [(0, i) for i in range(1, s + 1)]


def path(p):
    return [(i, i + 1) for i in range(p - 1)]


def cycle(p):
    return sorted({(min(i, (i + 1) % p), max(i, (i + 1) % p)) for i in range(p)})


def complete_bipartite(a, b):
    return [(i, a + j) for i in range(a) for j in range(b)]


def closed_form_truss(family, size, h):
    """Expected h-trussness of every edge of a closed-form family (one value for all)."""
    if family == "complete":
        return size
    if family == "star":
        return 2 if h == 1 else size + 1
    if family == "path":
        return min(size, h + 1)
    if family == "cycle":
        return size if size <= 2 * h + 1 else 2 * h
    if family == "bipartite":
        a, b = size
        return 2 if h == 1 else a + b
    raise KeyError(family)
