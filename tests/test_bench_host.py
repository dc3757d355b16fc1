"""Host-side measurement logic of bench.py, on the CPU: the algorithmic byte count of the
peel rounds (from the graph and each edge's removal round) against a brute-force count."""

import os
import sys

import numpy as np

from synth import erdos_renyi_gnm, rmat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _brute_pairs(eu, ev, stamp, h):
    m = eu.size
    pairs = 0
    for e in range(m):
        if h < 2:
            pairs += 1
            continue
        alive = stamp >= stamp[e]
        da = int(((eu == eu[e]) | (ev == eu[e]))[alive].sum())
        db = int(((eu == ev[e]) | (ev == ev[e]))[alive].sum())
        pairs += da + db - 1
    return pairs


def test_round_bytes_match_brute_force(oracle_mod):
    sys.path.insert(0, ROOT)
    import bench

    for n, (s, d), h in ((256, rmat(8, 6, 0.57, 0.19, 0.19, 5), 2),
                         (120, erdos_renyi_gnm(120, 400, 6), 2),
                         (120, erdos_renyi_gnm(120, 400, 7), 1)):
        g = oracle_mod.OracleGraph.from_raw(n, s, d)
        _, stamp, _ = g.truss_decompose(h)
        hb = bench.round_bytes_host(n, g.eu, g.ev, stamp, h)
        p = _brute_pairs(g.eu, g.ev, stamp, h)
        assert hb["pairs"] == p and hb["detect"] == 8.0 * p
        assert hb["frontier"] == g.m and hb["select"] == 8.0 * g.m
    empty = bench.round_bytes_host(4, np.zeros(0, np.int32), np.zeros(0, np.int32),
                                   np.zeros(0, np.int32), 2)
    assert empty["detect"] == 0.0
