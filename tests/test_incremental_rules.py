"""The exactness argument of the incremental rounds, checked on the CPU against the oracle.

The GPU rounds for h <= 2 never rebuild a ball: after a round removes the frontier F they
(1) list the vertex pairs that may have left each other's ball, (2) test each in the new
graph and (3) lower every alive edge's support by the members that left the intersection
of its endpoints' balls.  This module restates those three rules for any h, as plain set
arithmetic, and checks that peeling with them gives the oracle's trussness:

* candidates: a pair {x, y} can lose distance <= r only through an old path of at most r
  edges that uses a removed edge (a, b), so x lies within i hops of a and y within j hops
  of b with i + j <= r - 1, in the graph before the round;
* test: d_new(x, y) <= r iff y is within r - 1 hops of x or of a neighbour of x in the new
  graph, so radius r is tested with the already updated radius r - 1;
* support: for an alive edge (x, y) the intersection B(x) ∩ B(y) loses exactly
  |L(x) ∩ B_old(y)| + |L(y) ∩ B_new(x)| members, L(v) = B_old(v) \\ B_new(v) (a member
  leaves either B(x), or stays in B(x) and leaves B(y)).

h = 1 and h = 2 are the GPU's rules; h = 3 is the same cascade one radius further.
Nothing here is shared with the CUDA code.
"""

import numpy as np
import pytest

from synth import barabasi_albert, erdos_renyi_gnm, rmat, small_corpus


def closed_balls(n, adj, r):
    out = []
    for x in range(n):
        seen, frontier = {x}, [x]
        for _ in range(r):
            nxt = []
            for y in frontier:
                for z in adj[y]:
                    if z not in seen:
                        seen.add(z)
                        nxt.append(z)
            frontier = nxt
        out.append(seen)
    return out


def peel_incremental(n, eu, ev, h):
    """Level-synchronous peel whose balls and supports change only by the three rules."""
    m = len(eu)
    adj = [set() for _ in range(n)]
    for u, v in zip(eu, ev):
        adj[u].add(v)
        adj[v].add(u)
    # B[r][x] = closed ball of radius r (B[0][x] = {x})
    B = [closed_balls(n, adj, r) for r in range(h + 1)]
    sup = [len(B[h][u] & B[h][v]) - 2 for u, v in zip(eu, ev)]
    alive = [True] * m
    t = np.zeros(m, dtype=np.int64)
    k, remaining = 2, m
    while remaining:
        F = [e for e in range(m) if alive[e] and sup[e] <= k - 2]
        if not F:
            k = min(sup[e] for e in range(m) if alive[e]) + 2
            continue
        old = [[set(s) for s in Br] for Br in B]
        for e in F:
            t[e] = k
            alive[e] = False
            remaining -= 1
            adj[eu[e]].discard(ev[e])
            adj[ev[e]].discard(eu[e])
        B[1] = [adj[x] | {x} for x in range(n)]
        lost_h = set()
        for r in range(2, h + 1) if h >= 2 else ():
            cand = set()
            for e in F:
                for a, b in ((eu[e], ev[e]), (ev[e], eu[e])):
                    for i in range(r):
                        for j in range(r - i):
                            for x in old[i][a]:
                                for y in old[j][b]:
                                    if x != y:
                                        cand.add((min(x, y), max(x, y)))
            for x, y in cand:
                if y not in B[r][x]:
                    continue  # already out (the pair is listed twice, or lost earlier)
                if y in B[r - 1][x] or any(y in B[r - 1][z] for z in adj[x]):
                    continue
                B[r][x].discard(y)
                B[r][y].discard(x)
                if r == h:
                    lost_h.add((x, y))
        if h == 1:
            lost_h = {(min(eu[e], ev[e]), max(eu[e], ev[e])) for e in F}
        # the maintained balls are the balls of the new graph, every radius
        for r in range(1, h + 1):
            assert B[r] == closed_balls(n, adj, r), f"radius {r} ball missed a lost pair"

        L = {}
        for x, y in lost_h:
            L.setdefault(x, set()).add(y)
            L.setdefault(y, set()).add(x)
        for e in range(m):
            if not alive[e]:
                continue
            x, y = eu[e], ev[e]
            d = len(L.get(x, set()) & old[h][y]) + len(L.get(y, set()) & B[h][x])
            sup[e] -= d
            assert sup[e] == len(B[h][x] & B[h][y]) - 2
    return t


def cases():
    out = [(n, s, d) for n, s, d in small_corpus(40, 5, max_n=30)]
    for sc in (5, 6):
        s, d = rmat(sc, 6, 0.57, 0.19, 0.19, 11 + sc)
        out.append((1 << sc, s, d))
    s, d = erdos_renyi_gnm(60, 180, 60)
    out.append((60, s, d))
    s, d = barabasi_albert(80, 3, 9)
    out.append((80, s, d))
    return out


@pytest.mark.parametrize("h", [1, 2, 3])
def test_incremental_rules_give_the_trussness(oracle_mod, h):
    for n, s, d in cases():
        og = oracle_mod.OracleGraph.from_raw(n, s, d)
        ref = og.truss_decompose(h)[0]
        got = peel_incremental(n, og.eu.tolist(), og.ev.tolist(), h)
        np.testing.assert_array_equal(got, ref, err_msg=f"n={n} m={og.m} h={h}")
