"""Pins of the all-edge peeling certificate (``oracle/htd_cert.c``), on the CPU.

The certificate proves a claimed (t, stamp) exact on every edge (order + validity +
removability, the induction over stamps of Sec. 3).  It obtains each h-support by
inserting edges in decreasing stamp order and growing closed balls; these tests pin that
machinery to Floyd-Warshall distances (``pins.apsp``, no shared code) and the verdicts to
the definition: every correct claim is accepted, every claim whose t differs from the true
trussness on some edge is rejected.
"""

import numpy as np
import pytest

import pins
from synth import erdos_renyi_gnm, rmat, small_corpus


def _fw_sup(n, edges, h, keep):
    d = pins.apsp(n, edges, keep)
    return pins.sup_from_distances(d, edges, h, keep)


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_supports_in_growing_subgraphs_match_floyd_warshall(oracle_mod, h):
    rng = np.random.default_rng(40 + h)
    for seed in range(8):
        n = 18
        s, d = erdos_renyi_gnm(n, 34, 7100 + 10 * h + seed)
        edges = pins.canonical(n, s, d)
        m = len(edges)
        eu = np.array([u for u, _ in edges], np.int32)
        ev = np.array([v for _, v in edges], np.int32)
        # arbitrary stamps with t constant per stamp and non-decreasing in it, so that both
        # supports are read (the claim itself is usually wrong; only the supports matter)
        stamp = rng.integers(0, 6, size=m).astype(np.int32)
        t = (stamp // 2 + 2).astype(np.int32)
        ob, _, _, sup_rem, sup_val = oracle_mod.certify_all(n, eu, ev, h, t, stamp, threads=2,
                                                             sups=True)
        assert ob == 0
        for e in range(m):
            keep = stamp >= stamp[e]
            assert sup_rem[e] == _fw_sup(n, edges, h, keep)[e], (seed, e)
            keep = t >= t[e]
            assert sup_val[e] == _fw_sup(n, edges, h, keep)[e], (seed, e)


@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_accepts_every_oracle_decomposition(oracle_mod, h):
    graphs = list(small_corpus(25, 300 + h, max_n=50))
    graphs += [(64, *rmat(6, 4, 0.57, 0.19, 0.19, 8100 + h)),
               (80, *erdos_renyi_gnm(80, 300, 8200 + h))]
    for n, s, d in graphs:
        g = oracle_mod.OracleGraph.from_raw(n, s, d)
        if g.m == 0:
            continue
        t, stamp, _ = g.truss_decompose(h)
        res = [oracle_mod.certify_all(n, g.eu, g.ev, h, t, stamp, threads=k, sups=True)
               for k in (1, 4)]
        for ob, bad, _, _, _ in res:
            assert ob == 0 and bad.size == 0
        # the supports do not depend on the thread count, and agree with the oracle's
        # per-edge BFS in the same subgraphs
        np.testing.assert_array_equal(res[0][3], res[1][3])
        np.testing.assert_array_equal(res[0][4], res[1][4])
        for e in range(0, g.m, max(1, g.m // 12)):
            assert res[0][3][e] == g.edge_h_support(h, e, key=stamp, thr=int(stamp[e]))
            assert res[0][4][e] == g.edge_h_support(h, e, key=t, thr=int(t[e]))


@pytest.mark.parametrize("h", [1, 2, 3])
def test_rejects_every_wrong_trussness(oracle_mod, h):
    # soundness: a claim that is accepted is exact, so any claim with a wrong t on some
    # edge must be rejected, whatever the stamps say
    rng = np.random.default_rng(90 + h)
    rejected = 0
    for seed in range(5):
        s, d = rmat(6, 5, 0.57, 0.19, 0.19, 8300 + 10 * h + seed)
        g = oracle_mod.OracleGraph.from_raw(64, s, d)
        t, stamp, _ = g.truss_decompose(h)
        for trial in range(30):
            t2, st2 = t.copy(), stamp.copy()
            kind = trial % 3
            e = int(rng.integers(0, g.m))
            if kind == 0:  # one edge moved by one level
                t2[e] += 1 if rng.random() < 0.5 or t2[e] == 2 else -1
            elif kind == 1:  # a whole round moved by one level, stamps kept
                grp = stamp == stamp[e]
                t2[grp] += 1 if rng.random() < 0.5 or t2[e] == 2 else -1
            else:  # a whole round moved, and its stamps moved to stay ordered
                grp = stamp == stamp[e]
                t2[grp] += 1
                st2[grp] = stamp.max() + 1
                st2[(stamp > stamp[e]) & (t2 > t2[e])] += 2
            if np.array_equal(t2, t):
                continue
            ob, bad, _ = oracle_mod.certify_all(64, g.eu, g.ev, h, t2, st2, threads=2)
            assert ob > 0 or bad.size > 0, (seed, trial)
            rejected += 1
    assert rejected > 50


def test_order_condition_and_arguments(oracle_mod):
    s, d = erdos_renyi_gnm(40, 120, 8400)
    g = oracle_mod.OracleGraph.from_raw(40, s, d)
    t, stamp, _ = g.truss_decompose(2)
    # two rounds of different levels swapped: the order condition fails
    lo, hi = np.argmin(t), np.argmax(t)
    st = stamp.copy()
    st[lo], st[hi] = stamp[hi], stamp[lo]
    ob, _, _ = oracle_mod.certify_all(40, g.eu, g.ev, 2, t, st)
    assert ob > 0
    with pytest.raises(ValueError):
        oracle_mod.certify_all(40, g.eu, g.ev, 0, t, stamp)
    with pytest.raises(ValueError):
        oracle_mod.certify_all(40, g.eu, g.ev, 2, t, np.full_like(stamp, -1))
    ob, bad, _ = oracle_mod.certify_all(5, np.zeros(0, np.int32), np.zeros(0, np.int32), 2,
                                        np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert ob == 0 and bad.size == 0
