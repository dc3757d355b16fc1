"""Pins for the CPU oracle: it must agree with mathematics, not only with itself.

Every check compares the C oracle with something independent of it: Floyd-Warshall
distances, exhaustive Def. 4 enumeration, closed forms, hand-worked examples, the
textbook h = 1 triangle peel, and invariants the paper's definitions imply.
"""

import os

import numpy as np
import pytest

import pins
from synth import barabasi_albert, erdos_renyi_gnm, rmat, small_corpus

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.txt")


def og(oracle_mod, n, edges):
    eu = np.array([u for u, _ in edges], dtype=np.int32)
    ev = np.array([v for _, v in edges], dtype=np.int32)
    return oracle_mod.OracleGraph(n, eu, ev)


def random_small(seed, n_max=8, m_max=12):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, n_max + 1))
    allp = [(a, b) for a in range(n) for b in range(a + 1, n)]
    m = int(rng.integers(1, min(m_max, len(allp)) + 1))
    pick = rng.choice(len(allp), size=m, replace=False)
    return n, sorted(allp[i] for i in pick)


# ---- normalisation -------------------------------------------------------------------

def test_normalise_matches_set_semantics(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(50):
        n = int(rng.integers(1, 30))
        k = int(rng.integers(0, 80))
        s = rng.integers(0, n, size=k).astype(np.int32)
        d = rng.integers(0, n, size=k).astype(np.int32)
        eu, ev = oracle_mod.normalise(n, s, d)
        assert list(zip(eu.tolist(), ev.tolist())) == pins.canonical(n, s, d)


def test_normalise_rejects_bad_ids(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.normalise(3, [0, 1], [1, 3])
    with pytest.raises(ValueError):
        oracle_mod.normalise(3, [-1], [1])


# ---- h-support against Floyd-Warshall --------------------------------------------------

@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_h_support_matches_floyd_warshall(oracle_mod, h):
    for seed in range(40):
        n, edges = random_small(1000 + seed, n_max=14, m_max=30)
        g = og(oracle_mod, n, edges)
        d = pins.apsp(n, edges)
        np.testing.assert_array_equal(g.h_support(h), pins.sup_from_distances(d, edges, h))


def test_h_support_on_subgraph_matches_floyd_warshall(oracle_mod):
    rng = np.random.default_rng(7)
    for seed in range(30):
        n, edges = random_small(2000 + seed, n_max=12, m_max=25)
        key = rng.integers(0, 4, size=len(edges)).astype(np.int32)
        thr = int(rng.integers(0, 4))
        mask = key >= thr
        g = og(oracle_mod, n, edges)
        for h in (1, 2, 3):
            d = pins.apsp(n, edges, mask)
            np.testing.assert_array_equal(
                g.h_support(h, key, thr), pins.sup_from_distances(d, edges, h, mask))


def test_h1_support_is_triangle_count(oracle_mod):
    for seed in range(20):
        n, edges = random_small(3000 + seed, n_max=20, m_max=60)
        g = og(oracle_mod, n, edges)
        adj = [set() for _ in range(n)]
        for u, v in edges:
            adj[u].add(v)
            adj[v].add(u)
        tri = [len(adj[u] & adj[v]) for u, v in edges]
        np.testing.assert_array_equal(g.h_support(1), tri)


# ---- decomposition against the definition ------------------------------------------------

@pytest.mark.parametrize("h", [1, 2, 3])
def test_decompose_matches_definition_bruteforce(oracle_mod, h):
    for seed in range(25):
        n, edges = random_small(4000 + 17 * h + seed, n_max=7, m_max=10)
        g = og(oracle_mod, n, edges)
        t, stamp, _ = g.truss_decompose(h)
        np.testing.assert_array_equal(t, pins.truss_by_definition(n, edges, h))


CLOSED = [("complete", s) for s in (2, 3, 4, 5, 7)] + \
         [("star", s) for s in (1, 2, 3, 6)] + \
         [("path", p) for p in (2, 3, 4, 5, 6, 9)] + \
         [("cycle", p) for p in (3, 4, 5, 6, 7, 8, 11)] + \
         [("bipartite", ab) for ab in ((1, 3), (2, 2), (2, 3), (3, 4))]


@pytest.mark.parametrize("family,size", CLOSED)
@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_closed_forms(oracle_mod, family, size, h):
    build = {"complete": pins.complete, "star": pins.star, "path": pins.path,
             "cycle": pins.cycle,
             "bipartite": lambda ab: pins.complete_bipartite(*ab)}[family]
    edges = sorted(build(size))
    n = 1 + max(max(e) for e in edges)
    g = og(oracle_mod, n, edges)
    t, _, _ = g.truss_decompose(h)
    assert set(t.tolist()) == {pins.closed_form_truss(family, size, h)}


def test_disjoint_union_decomposes_componentwise(oracle_mod):
    parts = [pins.complete(5), pins.cycle(9), pins.star(4), pins.path(6)]
    for h in (1, 2, 3):
        edges, off, expect = [], 0, []
        for p in parts:
            pn = 1 + max(max(e) for e in p)
            edges += [(u + off, v + off) for u, v in sorted(p)]
            expect += og(oracle_mod, pn, sorted(p)).truss_decompose(h)[0].tolist()
            off += pn
        t, _, _ = og(oracle_mod, off, edges).truss_decompose(h)
        assert t.tolist() == expect


def test_diameter_at_most_h_gives_component_size(oracle_mod):
    # a wheel (hub + cycle of 8) has diameter 2: every edge gets t = 9 at h = 2
    edges = sorted(pins.cycle(8)) + [(i, 8) for i in range(8)]
    edges = sorted((min(a, b), max(a, b)) for a, b in edges)
    t, _, _ = og(oracle_mod, 9, edges).truss_decompose(2)
    assert set(t.tolist()) == {9}


def test_hand_worked_examples(oracle_mod):
    seen = 0
    with open(GOLDEN) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            name, n, h, es, sup, t = [c.strip() for c in line.split("|")]
            edges = [tuple(int(x) for x in tok.split("-")) for tok in es.split()]
            g = og(oracle_mod, int(n), edges)
            assert g.h_support(int(h)).tolist() == [int(x) for x in sup.split()], name
            assert g.truss_decompose(int(h))[0].tolist() == [int(x) for x in t.split()], name
            seen += 1
    assert seen >= 6


def test_h1_equals_classic_truss(oracle_mod):
    for seed in range(12):
        n = 60
        s, d = erdos_renyi_gnm(n, 240, 5000 + seed)
        eu, ev = oracle_mod.normalise(n, s, d)
        edges = list(zip(eu.tolist(), ev.tolist()))
        t, _, _ = oracle_mod.OracleGraph(n, eu, ev).truss_decompose(1)
        np.testing.assert_array_equal(t, pins.classic_truss(n, edges))
    for seed in range(6):
        s, d = barabasi_albert(80, 4, 5100 + seed)
        eu, ev = oracle_mod.normalise(80, s, d)
        edges = list(zip(eu.tolist(), ev.tolist()))
        t, _, _ = oracle_mod.OracleGraph(80, eu, ev).truss_decompose(1)
        np.testing.assert_array_equal(t, pins.classic_truss(80, edges))


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_level_synchronous_equals_sequential_algorithm1(oracle_mod, h):
    for seed in range(8):
        n = 30
        s, d = erdos_renyi_gnm(n, 70, 6000 + 10 * h + seed)
        g = oracle_mod.OracleGraph.from_raw(n, s, d)
        np.testing.assert_array_equal(g.truss_decompose(h)[0], g.truss_sequential(h))
    s, d = barabasi_albert(40, 3, 6100 + h)
    g = oracle_mod.OracleGraph.from_raw(40, s, d)
    np.testing.assert_array_equal(g.truss_decompose(h)[0], g.truss_sequential(h))


def test_invariants_on_corpus(oracle_mod):
    for n, s, d in small_corpus(30, 77, max_n=40):
        g = oracle_mod.OracleGraph.from_raw(n, s, d)
        if g.m == 0:
            continue
        prev = None
        for h in (1, 2, 3, 4):
            t, stamp, _ = g.truss_decompose(h)
            sup = g.h_support(h)
            assert (t >= 2).all()
            assert (t <= sup + 2).all()  # t <= sup_G + 2
            # the edges of minimum h-support are peeled first, at k = min sup + 2
            assert t.min() == sup.min() + 2
            assert (t[sup == sup.min()] == sup.min() + 2).all()
            # validity: sup inside T_{t(e)} is at least t(e)-2 (Def. 4 (i))
            for e in range(g.m):
                assert g.edge_h_support(h, e, t, int(t[e])) >= t[e] - 2
            if prev is not None:
                assert (t >= prev).all()  # monotone non-decreasing in h
            prev = t


def test_relabelling_and_edge_order_invariance(oracle_mod):
    rng = np.random.default_rng(11)
    n = 50
    s, d = erdos_renyi_gnm(n, 160, 7000)
    base = oracle_mod.OracleGraph.from_raw(n, s, d)
    for h in (1, 2, 3):
        t0, _, _ = base.truss_decompose(h)
        ref = {(int(u), int(v)): int(x) for u, v, x in zip(base.eu, base.ev, t0)}
        perm = rng.permutation(n).astype(np.int32)
        order = rng.permutation(s.size)
        # relabel, shuffle, flip some pairs, add duplicates and self-loops
        s2 = perm[s][order]
        d2 = perm[d][order]
        flip = rng.random(s2.size) < 0.5
        s2[flip], d2[flip] = d2[flip], s2[flip].copy()
        s2 = np.concatenate([s2, s2[:20], np.arange(5, dtype=np.int32)])
        d2 = np.concatenate([d2, d2[:20], np.arange(5, dtype=np.int32)])
        g2 = oracle_mod.OracleGraph.from_raw(n, s2, d2)
        t2, _, _ = g2.truss_decompose(h)
        inv = np.argsort(perm)
        got = {(min(int(inv[u]), int(inv[v])), max(int(inv[u]), int(inv[v]))): int(x)
               for u, v, x in zip(g2.eu, g2.ev, t2)}
        assert got == ref


# ---- certificate --------------------------------------------------------------------------

def test_certificate_accepts_oracle_and_rejects_planted_errors(oracle_mod):
    rng = np.random.default_rng(5)
    for seed in range(6):
        s, d = rmat(6, 4, 0.57, 0.19, 0.19, 8000 + seed)
        g = oracle_mod.OracleGraph.from_raw(64, s, d)
        for h in (1, 2, 3):
            t, stamp, _ = g.truss_decompose(h)
            order_bad, bad, _ = g.certify(h, t, stamp)
            assert order_bad == 0 and bad.size == 0
            # planted error 1: one trussness raised by one -> validity or order fails
            e = int(rng.integers(0, g.m))
            t1 = t.copy()
            t1[e] += 1
            ob, b, _ = g.certify(h, t1, stamp)
            assert ob > 0 or b.size > 0
            # planted error 2: one trussness lowered by one -> removability or order fails
            t2 = t.copy()
            cand = np.nonzero(t2 > 2)[0]
            if cand.size:
                e = int(cand[rng.integers(0, cand.size)])
                t2[e] -= 1
                ob, b, _ = g.certify(h, t2, stamp)
                assert ob > 0 or b.size > 0
            # planted error 3: an edge stamped as removed later than it was
            st3 = stamp.copy()
            e = int(np.argmin(stamp))
            st3[e] = stamp.max() + 1
            ob, b, _ = g.certify(h, t, st3)
            if t[e] < t.max():
                assert ob > 0 or b.size > 0


def test_oracle_finishes_small_workload_quickly(oracle_mod):
    # a quarter-size version of the 2,000-vertex ER workload must finish in well under
    # a second; the full one is exercised by the GPU parity tests
    s, d = erdos_renyi_gnm(500, 2000, 9000)
    g = oracle_mod.OracleGraph.from_raw(500, s, d)
    t, stamp, rounds = g.truss_decompose(2)
    assert rounds > 0 and (t >= 2).all()


# ---- the H-index iteration of Sec. 4 (Theorems 3 and 4; asynchronous updating) -----------

@pytest.mark.parametrize("h", [1, 2, 3])
def test_hindex_converges_to_definition(oracle_mod, h):
    # Theorem 4: the fixed point plus 2 is t(e,h), here against Def. 4 by brute force
    for seed in range(20):
        n, edges = random_small(6000 + 13 * h + seed, n_max=7, m_max=10)
        g = og(oracle_mod, n, edges)
        ref = pins.truss_by_definition(n, edges, h)
        for asynchronous in (False, True):
            hv, _, converged = g.hindex(h, asynchronous=asynchronous)
            assert converged
            np.testing.assert_array_equal(hv + 2, ref)


@pytest.mark.parametrize("h", [1, 2, 3])
def test_hindex_fixed_point_equals_peeling_on_corpus(oracle_mod, h):
    for n, s, d in small_corpus(24, 900 + h, max_n=30):
        g = oracle_mod.OracleGraph.from_raw(n, s, d)
        t = g.truss_decompose(h)[0]
        for asynchronous in (False, True):
            hv, _, converged = g.hindex(h, asynchronous=asynchronous)
            assert converged
            np.testing.assert_array_equal(hv + 2, t)


def test_hindex_orders_monotone_and_bounded(oracle_mod):
    # order 0 is the h-support; orders never increase (Theorem 3) and never fall below
    # t(e,h) - 2 (Theorem 4 (i))
    for h in (1, 2, 3):
        for seed in range(4):
            s, d = erdos_renyi_gnm(25, 70, 7100 + 10 * h + seed)
            g = oracle_mod.OracleGraph.from_raw(25, s, d)
            t = g.truss_decompose(h)[0]
            _, final, _ = g.hindex(h)
            prev = None
            for k in range(final + 1):
                hv, _, _ = g.hindex(h, max_iter=k)
                if k == 0:
                    np.testing.assert_array_equal(hv, g.h_support(h))
                else:
                    assert np.all(hv <= prev)
                assert np.all(hv >= t - 2)
                prev = hv


def test_hindex_h1_is_the_triangle_hindex(oracle_mod):
    # h = 1: the only path of at most one edge is the edge itself, so each order is the
    # classic triangle-pair H-index, order by order
    for seed in range(6):
        s, d = erdos_renyi_gnm(30, 110, 7300 + seed)
        g = oracle_mod.OracleGraph.from_raw(30, s, d)
        edges = list(zip(g.eu.tolist(), g.ev.tolist()))
        ref = pins.triangle_hindex_orders(30, edges, 6)
        for k in range(7):
            hv, _, _ = g.hindex(1, max_iter=k)
            np.testing.assert_array_equal(hv, ref[k], err_msg=f"order {k}")


@pytest.mark.parametrize("h", [1, 2, 3])
def test_hindex_pruning_changes_no_order(oracle_mod, h):
    # Lemma 4: an edge whose neighbourhood had no value fall across its own H in the
    # previous order keeps its H.  The pruned iteration must equal the plain synchronous
    # one order by order (same values after every order, same number of orders) while
    # computing fewer H^(n)(e); the fixed point + 2 is still t(e,h)
    skipped = 0
    for seed in range(5):
        s, d = erdos_renyi_gnm(28, 90, 7500 + 10 * h + seed)
        g = oracle_mod.OracleGraph.from_raw(28, s, d)
        _, final, _ = g.hindex(h)
        for k in range(final + 1):
            ref, it_ref, conv_ref = g.hindex(h, max_iter=k)
            hv, it, conv, evals = g.hindex_pruned(h, max_iter=k)
            np.testing.assert_array_equal(hv, ref, err_msg=f"h={h} seed={seed} order {k}")
            assert (it, conv) == (it_ref, conv_ref)
            assert evals <= g.m * it
        hv, it, conv, evals = g.hindex_pruned(h)
        assert conv and it == final
        np.testing.assert_array_equal(hv + 2, g.truss_decompose(h)[0])
        skipped += g.m * it - evals
    assert skipped > 0


def test_hindex_pruning_is_not_vacuous(oracle_mod):
    # a planted mistake in the rule (pruning whenever the edge's own value did not change
    # in the previous order, ignoring its neighbourhood) must give a different result on
    # some graph, so the test above can tell a wrong rule from the right one
    differs = False
    for seed in range(12):
        s, d = erdos_renyi_gnm(24, 80, 7700 + seed)
        g = oracle_mod.OracleGraph.from_raw(24, s, d)
        ref, final, _ = g.hindex(2)
        prev = g.hindex(2, max_iter=0)[0]
        cur = g.hindex(2, max_iter=1)[0]
        wrong = cur.copy()
        for k in range(2, final + 1):
            nxt_full = g.hindex(2, max_iter=k)[0]
            nxt = np.where(cur == prev, cur, nxt_full)  # the planted rule
            prev, cur = cur, nxt
            wrong = nxt
        if not np.array_equal(wrong, ref):
            differs = True
            break
    assert differs


def _hull_rule_skips(n, eu, ev, h, old, cur, hops=None):
    """The GPU's form of the Lemma 4 test, restated on the host: per vertex the range of the
    values that fell at its edges (highest old, lowest new), widened h-1 hops over the
    graph; an edge is skipped when its endpoints' hull does not straddle its value."""
    hi = np.full(n, -1, dtype=np.int64)
    lo = np.full(n, np.iinfo(np.int64).max, dtype=np.int64)
    fell = old != cur
    for x in (eu[fell], ev[fell]):
        np.maximum.at(hi, x, old[fell])
        np.minimum.at(lo, x, cur[fell])
    for _ in range(h - 1 if hops is None else hops):
        hi2, lo2 = hi.copy(), lo.copy()
        for a, b in ((eu, ev), (ev, eu)):
            np.maximum.at(hi2, a, hi[b])
            np.minimum.at(lo2, a, lo[b])
        hi, lo = hi2, lo2
    l = np.minimum(lo[eu], lo[ev])
    hh = np.maximum(hi[eu], hi[ev])
    return ~((l < cur) & (cur <= hh))


@pytest.mark.parametrize("h", [1, 2, 3])
def test_hindex_range_hull_rule_never_skips_a_change(oracle_mod, h):
    # the rule the GPU engine uses must only skip edges whose value the next order keeps
    # (it may compute more than the lemma needs, never less); it must also skip something
    # (sparser graphs at h = 3, where two hops reach most of a dense small graph)
    n, m = (30, 100) if h < 3 else (90, 140)
    skipped = 0
    for seed in range(6):
        s, d = erdos_renyi_gnm(n, m, 7900 + 10 * h + seed)
        g = oracle_mod.OracleGraph.from_raw(n, s, d)
        _, final, _ = g.hindex(h)
        orders = [g.hindex(h, max_iter=k)[0].astype(np.int64) for k in range(final + 1)]
        for k in range(1, final):
            skip = _hull_rule_skips(n, g.eu, g.ev, h, orders[k - 1], orders[k])
            np.testing.assert_array_equal(orders[k + 1][skip], orders[k][skip],
                                          err_msg=f"h={h} seed={seed} order {k + 1}")
            skipped += int(skip.sum())
    assert skipped > 0


def test_hindex_range_hull_rule_with_one_hop_too_few_fails(oracle_mod):
    # planted mistake: widening the ranges h-2 hops instead of h-1 at h = 2 (only the
    # edges at the endpoints themselves) skips an edge that still changes on some graph
    wrong = False
    for seed in range(20):
        s, d = erdos_renyi_gnm(30, 100, 8100 + seed)
        g = oracle_mod.OracleGraph.from_raw(30, s, d)
        _, final, _ = g.hindex(2)
        orders = [g.hindex(2, max_iter=k)[0].astype(np.int64) for k in range(final + 1)]
        for k in range(1, final):
            skip = _hull_rule_skips(30, g.eu, g.ev, 2, orders[k - 1], orders[k], hops=0)
            if not np.array_equal(orders[k + 1][skip], orders[k][skip]):
                wrong = True
        if wrong:
            break
    assert wrong
