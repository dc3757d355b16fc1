"""The seeded input generators: shapes, ranges and determinism (no GPU)."""

import numpy as np

from synth import (CONFIG_SEED_BASE, barabasi_albert, batch_graphs, config_graph, dcsbm,
                   erdos_renyi_gnm, rmat)


def canon(s, d):
    return {(min(a, b), max(a, b)) for a, b in zip(s.tolist(), d.tolist())}


def test_er_draws_distinct_pairs():
    s, d = erdos_renyi_gnm(300, 1500, 5)
    assert s.dtype == np.int32 and d.dtype == np.int32 and s.size == d.size == 1500
    assert np.all(s != d) and s.min() >= 0 and max(s.max(), d.max()) < 300
    assert len(canon(s, d)) == 1500
    s2, d2 = erdos_renyi_gnm(300, 1500, 5)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)


def test_rmat_raw_pairs():
    s, d = rmat(10, 8, 0.57, 0.19, 0.19, 9)
    assert s.size == d.size == 8 * 1024
    assert s.min() >= 0 and max(s.max(), d.max()) < 1024
    # raw: loops and duplicates stay (normalisation is the library's job)
    assert np.any(s == d) or len(canon(s, d)) < s.size
    s2, _ = rmat(10, 8, 0.57, 0.19, 0.19, 9)
    assert np.array_equal(s, s2)
    # skewed: the busiest vertex has far more than the mean degree 16
    deg = np.bincount(np.concatenate([s, d]), minlength=1024)
    assert deg.max() > 8 * deg.mean()


def test_ba_edge_count_and_targets():
    for n, m0 in ((50, 2), (200, 5)):
        s, d = barabasi_albert(n, m0, 3)
        assert s.size == m0 * (m0 - 1) // 2 + (n - m0) * m0
        assert np.all(s != d) and len(canon(s, d)) == s.size
        # every new vertex attaches m0 edges to earlier vertices
        late = s >= m0
        assert np.all(d[late] < s[late])


def test_dcsbm_distinct_edges_and_inter_share():
    s, d = dcsbm(20_000, 50, 2.1, 100, 2.5, 60_000, 0.10, 11)
    assert s.size == 60_000 and len(canon(s, d)) == 60_000 and np.all(s != d)
    assert max(s.max(), d.max()) < 20_000


def test_named_workloads_are_seeded_as_documented():
    er = config_graph("er_n2000")
    s, d = erdos_renyi_gnm(2000, 8000, CONFIG_SEED_BASE + 0)
    assert er.n == 2000 and np.array_equal(er.src, s) and np.array_equal(er.dst, d)
    small = config_graph("rmat_s12")
    assert small.n == 4096 and small.src.size == 8 * 4096


def test_batch_graphs_shape():
    b = batch_graphs(40, 77, n_lo=50, n_hi=400)
    assert len(b) == 40
    for n, s, d, h in b:
        assert 50 <= n <= 400 + 8 and h in (2, 3)
        assert s.size == d.size and (s.size == 0 or max(s.max(), d.max()) < n)
    b2 = batch_graphs(40, 77, n_lo=50, n_hi=400)
    assert all(np.array_equal(x[1], y[1]) and x[3] == y[3] for x, y in zip(b, b2))
