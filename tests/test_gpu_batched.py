"""GPU parity of the batched entry point (htd_truss_decompose_batched) against the oracle.

A batch is decomposed as disjoint unions of its graphs; every graph's result must equal
the oracle's decomposition of that graph alone, element by element, whatever the packing
(one union per h, or many small unions), the round variant or the ball layout.
"""

import numpy as np
import pytest

from synth import barabasi_albert, batch_graphs, erdos_renyi_gnm, rmat

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def htd():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2411_06405_gb300 import build

    build.build()
    import paper_2411_06405_gb300 as mod

    mod._lib.load()
    torch.cuda.set_device(0)
    return mod


def mixed_batch():
    """Small graphs of every shape the normalisation and the peel meet, h in {1, 2, 3}."""
    g = []
    g.append((0, np.zeros(0, np.int32), np.zeros(0, np.int32), 2))          # no vertices
    g.append((5, np.zeros(0, np.int32), np.zeros(0, np.int32), 3))          # no edges
    g.append((2, np.array([0], np.int32), np.array([1], np.int32), 2))      # one edge
    g.append((3, np.array([0, 1, 2, 1, 2], np.int32),                       # triangle with a
             np.array([1, 2, 0, 0, 2], np.int32), 1))                       # reversed pair, a loop
    g.append((6, np.arange(6, dtype=np.int32), np.arange(6, dtype=np.int32), 2))  # loops only
    for i, (n, m) in enumerate([(40, 120), (80, 300), (150, 600), (220, 900)]):
        s, d = erdos_renyi_gnm(n, m, 100 + i)
        g.append((n, s, d, 1 + i % 3))
    for i, (n, m0) in enumerate([(60, 2), (120, 3), (200, 4), (90, 6)]):
        s, d = barabasi_albert(n, m0, 200 + i)
        g.append((n, s, d, 1 + (i + 1) % 3))
    for i, sc in enumerate([6, 7, 8]):
        s, d = rmat(sc, 6, 0.57, 0.19, 0.19, 300 + i)  # raw pairs: loops and duplicates
        g.append((1 << sc, s, d, 1 + (i + 2) % 3))
    return g


def oracle_truss(oracle_mod, n, s, d, h):
    og = oracle_mod.OracleGraph.from_raw(n, s, d)
    return og.truss_decompose(h)[0]


def check(res, graphs, expected):
    assert len(res) == len(graphs)
    for i, (t, ref) in enumerate(zip(res, expected)):
        np.testing.assert_array_equal(t.cpu().numpy(), ref, err_msg=f"graph {i}")


@pytest.fixture(scope="module")
def batch_and_truth(oracle_mod):
    graphs = mixed_batch()
    return graphs, [oracle_truss(oracle_mod, *gr) for gr in graphs]


def test_batched_matches_oracle_one_union_per_h(htd, batch_and_truth):
    graphs, truth = batch_and_truth
    res, st = htd.htd_truss_decompose_batched(graphs)
    check(res, graphs, truth)
    assert st["unions"] == 3  # h = 1, 2, 3
    assert st["frontier_edges"] == sum(len(t) for t in truth)


@pytest.mark.parametrize("cap", [1, 100, 300])
def test_batched_matches_oracle_many_unions(htd, batch_and_truth, cap):
    # small unions: graphs split over many peels (cap 1: every graph alone)
    graphs, truth = batch_and_truth
    res, st = htd.htd_truss_decompose_batched(graphs, max_union_vertices=cap)
    check(res, graphs, truth)
    assert st["unions"] > 3


@pytest.mark.parametrize("flags", ["REBUILD", "COMPACT_BALLS", "TINY_LOSS_TABLE", "NO_GRAPH"])
def test_batched_round_variants(htd, batch_and_truth, flags):
    graphs, truth = batch_and_truth
    res, _ = htd.htd_truss_decompose_batched(graphs, flags=getattr(htd, "HTD_OPT_" + flags))
    check(res, graphs, truth)


def test_batched_equals_single_graph_calls(htd):
    graphs = batch_graphs(12, 77, n_lo=50, n_hi=400)
    res, _ = htd.htd_truss_decompose_batched(graphs, max_union_vertices=1000)
    for i, (n, s, d, h) in enumerate(graphs):
        g = htd.htd_build_csr(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
        t, _, _ = htd.htd_truss_decompose(g, h)
        assert torch.equal(t, res[i]), f"graph {i}"
        g.free()


def test_batched_rejects_an_id_outside_its_graph(htd):
    ok = (4, np.array([0, 1], np.int32), np.array([1, 2], np.int32), 2)
    bad = (3, np.array([0, 3], np.int32), np.array([1, 0], np.int32), 2)  # 3 >= n = 3
    with pytest.raises(htd.HtdError) as e:
        htd.htd_truss_decompose_batched([ok, bad, ok])
    assert e.value.status == 1 and "graph 1" in str(e.value)


def test_every_autotuner_schedule_is_exact(htd, batch_and_truth):
    # every candidate schedule of the autotuner, and a tuned run, give the oracle's result
    from paper_2411_06405_gb300 import autotune

    graphs, expected = batch_and_truth
    for cand in autotune.CANDIDATES:
        res, _ = htd.htd_truss_decompose_batched(graphs, flags=cand["flags"],
                                                 max_union_vertices=cand["max_union_vertices"])
        check(res, graphs, expected)
    table = autotune.tune(graphs, sample=8)
    assert table and all(v["flags"] in [c["flags"] for c in autotune.CANDIDATES] for v in table.values())
    res, parts = autotune.decompose(graphs, table)
    check(res, graphs, expected)
    assert sum(parts.values()) == len(graphs)


def test_batch_of_the_benchmark_recipe_sampled(htd, oracle_mod):
    # 64 graphs of the 4,096-graph recipe (n in [50, 5000], ER or BA, h in {2, 3}): each
    # equals the oracle's decomposition of that graph alone
    graphs = batch_graphs(4096, 0x48545258)[:64]
    small = [i for i, g in enumerate(graphs) if g[0] <= 700][:12]
    res, st = htd.htd_truss_decompose_batched(graphs)
    assert len(res) == 64
    for i in small:
        np.testing.assert_array_equal(res[i].cpu().numpy(), oracle_truss(oracle_mod, *graphs[i]))
    # the rest against single-graph GPU calls (each certified by the oracle's certificate)
    for g, r in zip(graphs, res):
        n, s, d, h = g
        gg = htd.htd_build_csr(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
        t, stamp, _ = htd.htd_truss_decompose(gg, h, stamps=True)
        assert torch.equal(t, r)
        eu, ev = htd.htd_edges(gg)
        ob, bad, _ = oracle_mod.certify_all(n, eu.cpu().numpy(), ev.cpu().numpy(), h,
                                            t.cpu().numpy(), stamp.cpu().numpy())
        assert ob == 0 and bad.size == 0
