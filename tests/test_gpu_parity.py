"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit-exact.

Trussness and h-support are integers, so every comparison is exact equality.  Small and
medium graphs are compared element by element; the full-size workloads are checked on
every edge with the all-edge peeling certificate (stamp order, validity and removability,
which together prove each trussness exact) and on sampled edges with the oracle's
per-edge h-support.
"""

import numpy as np
import pytest

import pins
from synth import barabasi_albert, config_graph, erdos_renyi_gnm, rmat, small_corpus

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


def gpu_graph(htd, n, s, d):
    return htd.htd_build_csr(n, torch.from_numpy(np.asarray(s, dtype=np.int32)).cuda(),
                             torch.from_numpy(np.asarray(d, dtype=np.int32)).cuda())


def host(t):
    return t.cpu().numpy()


# ---- a1: normalisation, CSR and edge ids ----------------------------------------------------

def csr_cases():
    rng = np.random.default_rng(3)
    cases = []
    s, d = rmat(10, 16, 0.57, 0.19, 0.19, 31)  # loops + duplicates
    cases.append(("rmat10_raw", 1 << 10, s, d))
    # a hub above 4096 neighbours (shared-memory bit-set row sort), with duplicates
    hub = np.zeros(9000, dtype=np.int32)
    leaves = rng.integers(1, 6000, size=9000).astype(np.int32)
    cases.append(("hub9000", 6000, np.concatenate([hub, leaves]), np.concatenate([leaves, hub])))
    # rows of 33..4096 (block bitonic sort) and isolated vertices
    s = rng.integers(0, 200, size=20000).astype(np.int32)
    d = rng.integers(0, 200, size=20000).astype(np.int32)
    cases.append(("dense200_isolated", 500, s, d))
    cases.append(("empty_edges", 10, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    cases.append(("only_loops", 5, np.arange(5, dtype=np.int32), np.arange(5, dtype=np.int32)))
    cases.append(("single_edge", 2, np.array([1], np.int32), np.array([0], np.int32)))
    return cases


@pytest.mark.parametrize("case", csr_cases(), ids=lambda c: c[0])
def test_csr_and_edge_ids_match_oracle(htd, oracle_mod, case):
    _, n, s, d = case
    g = gpu_graph(htd, n, s, d)
    eu_ref, ev_ref = oracle_mod.normalise(n, s, d)
    assert g.m == eu_ref.size
    eu, ev = htd.htd_edges(g)
    np.testing.assert_array_equal(host(eu), eu_ref)
    np.testing.assert_array_equal(host(ev), ev_ref)
    row_ptr, col, slot_eid = (host(t) for t in htd.htd_csr(g))
    deg = np.bincount(np.concatenate([eu_ref, ev_ref]), minlength=n)
    np.testing.assert_array_equal(np.diff(row_ptr), deg)
    for x in range(n):
        r = col[row_ptr[x]:row_ptr[x + 1]]
        assert (np.diff(r) > 0).all()
    # slot -> edge id: the edge of slot (x, col) joins x and col
    xs = np.repeat(np.arange(n), np.diff(row_ptr))
    lo = np.minimum(xs, col)
    hi = np.maximum(xs, col)
    np.testing.assert_array_equal(eu_ref[slot_eid], lo)
    np.testing.assert_array_equal(ev_ref[slot_eid], hi)


def test_invalid_ids_rejected(htd):
    with pytest.raises(htd.HtdError) as ei:
        gpu_graph(htd, 4, [0, 1, 2], [1, 2, 4])
    assert ei.value.status == 1
    with pytest.raises(htd.HtdError):
        gpu_graph(htd, 4, [0, -1], [1, 2])


def test_invalid_h_rejected(htd):
    g = gpu_graph(htd, 3, [0, 1], [1, 2])
    for h in (0, 9, -1):
        with pytest.raises(htd.HtdError):
            htd.htd_h_support(g, h)
        with pytest.raises(htd.HtdError):
            htd.htd_truss_decompose(g, h)


# ---- a2/a3: h-support -------------------------------------------------------------------------

@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_h_support_corpus(htd, oracle_mod, h):
    for n, s, d in small_corpus(40, 100 + h, max_n=60):
        g = gpu_graph(htd, n, s, d)
        og = oracle_mod.OracleGraph.from_raw(n, s, d)
        np.testing.assert_array_equal(host(htd.htd_h_support(g, h)), og.h_support(h))


@pytest.mark.parametrize("h", [1, 2, 3])
def test_h_support_er_n2000(htd, oracle_mod, h):
    spec = config_graph("er_n2000")
    g = gpu_graph(htd, spec.n, spec.src, spec.dst)
    og = oracle_mod.OracleGraph.from_raw(spec.n, spec.src, spec.dst)
    np.testing.assert_array_equal(host(htd.htd_h_support(g, h)), og.h_support(h))


def test_h_support_against_floyd_warshall(htd):
    # independent of the oracle: distances by Floyd-Warshall
    for seed in range(10):
        n = 30
        s, d = erdos_renyi_gnm(n, 60, 900 + seed)
        edges = pins.canonical(n, s, d)
        g = gpu_graph(htd, n, s, d)
        dist = pins.apsp(n, edges)
        for h in (1, 2, 3, 5, 8):
            np.testing.assert_array_equal(host(htd.htd_h_support(g, h)),
                                          pins.sup_from_distances(dist, edges, h))


# ---- a4-a7: peeling -----------------------------------------------------------------------------

# incremental peels keep all balls dense when they fit; "compact" stores the smaller form
MODES = {"incremental": 0, "persistent": 16, "rebuild": 4, "compact": 32}


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_truss_corpus(htd, oracle_mod, h, mode):
    for n, s, d in small_corpus(40, 200 + h, max_n=60):
        g = gpu_graph(htd, n, s, d)
        og = oracle_mod.OracleGraph.from_raw(n, s, d)
        t, _, st = htd.htd_truss_decompose(g, h, flags=MODES[mode])
        np.testing.assert_array_equal(host(t), og.truss_decompose(h)[0])
        if g.m:
            # h = 3 rounds are incremental on dense balls only; h >= 4 rebuilds
            inc = (h <= 2 and mode != "rebuild") or (h == 3 and mode in ("incremental",
                                                                          "persistent"))
            assert st["incremental"] == (1 if inc else 0)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_truss_er_n2000_h2(htd, oracle_mod, mode):
    """The 2,000-vertex Erdos-Renyi workload at h=2, element by element."""
    spec = config_graph("er_n2000")
    g = gpu_graph(htd, spec.n, spec.src, spec.dst)
    og = oracle_mod.OracleGraph.from_raw(spec.n, spec.src, spec.dst)
    t_ref, _, _ = og.truss_decompose(2)
    t, stamp, stats = htd.htd_truss_decompose(g, 2, stamps=True, flags=MODES[mode])
    np.testing.assert_array_equal(host(t), t_ref)
    assert stats["frontier_edges"] == g.m
    assert stats["max_truss"] == t_ref.max()
    order_bad, bad, _ = og.certify(2, host(t), host(stamp))
    assert order_bad == 0 and bad.size == 0


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("h", [1, 3])
def test_truss_er_other_h(htd, oracle_mod, h, mode):
    n, m = (2000, 8000) if h == 1 else (600, 2400)
    s, d = erdos_renyi_gnm(n, m, 0x48545255)
    g = gpu_graph(htd, n, s, d)
    og = oracle_mod.OracleGraph.from_raw(n, s, d)
    np.testing.assert_array_equal(host(htd.htd_truss_decompose(g, h, flags=MODES[mode])[0]),
                                  og.truss_decompose(h)[0])


@pytest.mark.parametrize("mode", sorted(MODES))
def test_truss_ba_and_rmat(htd, oracle_mod, mode):
    for (n, (s, d)), h in (((400, barabasi_albert(400, 3, 41)), 2),
                           ((512, rmat(9, 8, 0.57, 0.19, 0.19, 42)), 2),
                           ((1024, rmat(10, 8, 0.57, 0.19, 0.19, 44)), 1),
                           ((256, rmat(8, 8, 0.57, 0.19, 0.19, 43)), 3)):
        g = gpu_graph(htd, n, s, d)
        og = oracle_mod.OracleGraph.from_raw(n, s, d)
        np.testing.assert_array_equal(
            host(htd.htd_truss_decompose(g, h, flags=MODES[mode])[0]), og.truss_decompose(h)[0])


@pytest.mark.parametrize("family,size", [("complete", 60), ("star", 5000), ("cycle", 1001),
                                         ("path", 700), ("bipartite", (40, 70))])
@pytest.mark.parametrize("h", [1, 2, 3])
def test_closed_forms_large(htd, family, size, h):
    build = {"complete": pins.complete, "star": pins.star, "path": pins.path,
             "cycle": pins.cycle, "bipartite": lambda ab: pins.complete_bipartite(*ab)}[family]
    edges = build(size)
    n = 1 + max(max(e) for e in edges)
    s = np.array([u for u, _ in edges], np.int32)
    d = np.array([v for _, v in edges], np.int32)
    g = gpu_graph(htd, n, s, d)
    t, _, _ = htd.htd_truss_decompose(g, h)
    assert set(host(t).tolist()) == {pins.closed_form_truss(family, size, h)}


def test_disjoint_union_and_isolated(htd, oracle_mod):
    parts = [(60, erdos_renyi_gnm(60, 200, 5)), (64, rmat(6, 6, 0.57, 0.19, 0.19, 6)),
             (30, barabasi_albert(30, 3, 7))]
    off = 0
    ss, dd, ref = [], [], []
    for n, (s, d) in parts:
        og = oracle_mod.OracleGraph.from_raw(n, s, d)
        ref.append(og.truss_decompose(2)[0])
        ss.append(s + off)
        dd.append(d + off)
        off += n + 5  # five isolated vertices between components
    g = gpu_graph(htd, off, np.concatenate(ss), np.concatenate(dd))
    np.testing.assert_array_equal(host(htd.htd_truss_decompose(g, 2)[0]), np.concatenate(ref))


def test_empty_graphs(htd):
    for n, s, d in ((0, [], []), (7, [], []), (3, [1, 2], [1, 2])):
        g = gpu_graph(htd, n, s, d)
        assert g.m == 0
        t, _, st = htd.htd_truss_decompose(g, 2)
        assert t.numel() == 0 and st["rounds"] == 0
        assert htd.htd_h_support(g, 3).numel() == 0


def test_graph_and_direct_launch_agree_and_repeat(htd, oracle_mod):
    s, d = rmat(11, 8, 0.57, 0.19, 0.19, 77)
    g = gpu_graph(htd, 1 << 11, s, d)
    t1, st1, s1 = htd.htd_truss_decompose(g, 2, stamps=True)
    t2, st2, s2 = htd.htd_truss_decompose(g, 2, stamps=True, flags=htd.HTD_OPT_NO_GRAPH)
    t3, _, s3 = htd.htd_truss_decompose(g, 2, flags=htd.HTD_OPT_TIMING)
    t5, st5, s5 = htd.htd_truss_decompose(g, 2, stamps=True,
                                          flags=htd.HTD_OPT_REBUILD | htd.HTD_OPT_TIMING)
    assert torch.equal(t1, t2) and torch.equal(t1, t3) and torch.equal(t1, t5)
    assert torch.equal(st1, st5)  # same level-synchronous schedule
    assert s1["rounds"] == s2["rounds"] == s3["rounds"] == s5["rounds"]
    assert 0 < s3["timed_slots"] <= s3["slots"] and s3["ms_find"] > 0 and s3["slots"] >= s3["rounds"]
    assert 0 < s5["timed_slots"] <= s5["slots"] and s5["ms_ball"] > 0
    assert s1["incremental"] == 1 and s5["incremental"] == 0
    # changing h on the same handle and coming back
    t_h3, _, _ = htd.htd_truss_decompose(g, 3)
    t4, _, _ = htd.htd_truss_decompose(g, 2)
    assert torch.equal(t1, t4)
    assert (t_h3 >= t1).all()  # monotone in h
    og = oracle_mod.OracleGraph.from_raw(1 << 11, s, d)
    ob, bad, _ = og.certify(2, host(t1), host(st1))
    assert ob == 0 and bad.size == 0


def test_host_entry_point(htd, oracle_mod):
    s, d = rmat(10, 8, 0.57, 0.19, 0.19, 88)
    n = 1 << 10
    eu, ev, t, stats = htd.htd_truss_decompose_host(n, s, d, 2)
    og = oracle_mod.OracleGraph.from_raw(n, s, d)
    np.testing.assert_array_equal(eu.numpy(), og.eu)
    np.testing.assert_array_equal(ev.numpy(), og.ev)
    np.testing.assert_array_equal(t.numpy(), og.truss_decompose(2)[0])


# ---- full-size workloads (the benchmark's launch configuration) ---------------------------------

def test_incremental_h3_matches_rebuild_on_hubby_graph(htd):
    # R-MAT scale 12 at h = 3: hub balls cover most of the graph; incremental rounds (with
    # and without forced rebuild finishes) and rebuild rounds must agree exactly, stamps too
    s, d = rmat(12, 8, 0.57, 0.19, 0.19, 98)
    g = gpu_graph(htd, 1 << 12, s, d)
    a, sa, st_a = htd.htd_truss_decompose(g, 3, stamps=True)
    b, sb, st_b = htd.htd_truss_decompose(g, 3, stamps=True, flags=htd.HTD_OPT_REBUILD)
    c, sc, st_c = htd.htd_truss_decompose(g, 3, stamps=True, flags=htd.HTD_OPT_TINY_LOSS_TABLE)
    assert st_a["incremental"] == 1 and st_b["incremental"] == 0 and st_c["incremental"] == 1
    assert st_a["pairs3_tested"] > 0 and st_c["rounds_rebuilt"] > 0
    assert torch.equal(a, b) and torch.equal(sa, sb)
    assert torch.equal(a, c) and torch.equal(sa, sc)


def test_incremental_matches_rebuild_on_hubby_graph(htd):
    # R-MAT scale 13: hubs, thousands of rounds; both round variants must agree exactly
    s, d = rmat(13, 8, 0.57, 0.19, 0.19, 99)
    g = gpu_graph(htd, 1 << 13, s, d)
    for h in (1, 2):
        a, sa, st_a = htd.htd_truss_decompose(g, h, stamps=True)
        b, sb, st_b = htd.htd_truss_decompose(g, h, stamps=True, flags=htd.HTD_OPT_REBUILD)
        c, sc, st_c = htd.htd_truss_decompose(g, h, stamps=True,
                                              flags=htd.HTD_OPT_PERSISTENT_ROUNDS)
        d, sd, st_d = htd.htd_truss_decompose(g, h, stamps=True, flags=htd.HTD_OPT_COMPACT_BALLS)
        assert st_a["incremental"] == 1 and st_b["incremental"] == 0 and st_c["incremental"] == 1
        assert st_a["round_kernel_launches"] == 0 and st_c["round_kernel_launches"] >= 1
        # all-dense storage takes n x W words; the compact form is smaller on this graph
        assert st_d["ball_pool_bytes"] < st_a["ball_pool_bytes"]
        assert torch.equal(a, b) and torch.equal(sa, sb)
        assert torch.equal(a, c) and torch.equal(sa, sc)
        assert torch.equal(a, d) and torch.equal(sa, sd)


def test_ball_layout_switch_on_one_handle(htd, oracle_mod):
    # the captured rounds address the balls by layout: alternating layouts on one handle
    # must recapture them
    n = 700
    s, d = erdos_renyi_gnm(n, 4200, 63)
    g = gpu_graph(htd, n, s, d)
    og = oracle_mod.OracleGraph.from_raw(n, s, d)
    for h in (2, 1):
        ref = og.truss_decompose(h)[0]
        for flags in (0, htd.HTD_OPT_COMPACT_BALLS, 0, htd.HTD_OPT_COMPACT_BALLS | htd.HTD_OPT_NO_GRAPH,
                      htd.HTD_OPT_TIMING, htd.HTD_OPT_COMPACT_BALLS | htd.HTD_OPT_TIMING):
            t, _, _ = htd.htd_truss_decompose(g, h, flags=flags)
            np.testing.assert_array_equal(host(t), ref, err_msg=f"h={h} flags={flags}")


@pytest.mark.parametrize("h", [1, 2, 3])
def test_batched_rounds_match_oracle(htd, oracle_mod, h):
    # a 128-slot lost-pair table splits most rounds into many batches
    for (n, (s, d)) in ((512, rmat(9, 8, 0.57, 0.19, 0.19, 61)),
                        (300, erdos_renyi_gnm(300, 1500, 62))):
        g = gpu_graph(htd, n, s, d)
        og = oracle_mod.OracleGraph.from_raw(n, s, d)
        t, stamp, st = htd.htd_truss_decompose(g, h, stamps=True,
                                               flags=htd.HTD_OPT_TINY_LOSS_TABLE)
        t2, stamp2, _ = htd.htd_truss_decompose(
            g, h, stamps=True, flags=htd.HTD_OPT_TINY_LOSS_TABLE | htd.HTD_OPT_PERSISTENT_ROUNDS)
        t3, stamp3, _ = htd.htd_truss_decompose(
            g, h, stamps=True, flags=htd.HTD_OPT_TINY_LOSS_TABLE | htd.HTD_OPT_COMPACT_BALLS)
        assert torch.equal(t, t2) and torch.equal(stamp, stamp2)
        assert torch.equal(t, t3) and torch.equal(stamp, stamp3)
        t_ref, stamp_ref, rounds = og.truss_decompose(h)
        np.testing.assert_array_equal(host(t), t_ref)
        np.testing.assert_array_equal(host(stamp), stamp_ref)  # same rounds as the oracle
        assert st["rounds"] == rounds and st["incremental"] == 1
        if h == 3:
            # 128-slot tables: most h = 3 rounds halt and are finished by rebuilds
            assert st["rounds_rebuilt"] > 0


@pytest.mark.slow
@pytest.mark.parametrize("name,h", [("rmat_s18", 2), ("dcsbm_n200k", 2), ("dcsbm_n200k", 3)])
def test_full_size_certificate(htd, oracle_mod, name, h):
    """Whole output of the full-size workloads: the all-edge peeling certificate on every
    edge (order, validity, removability: together they prove each t(e,h) exact), computed
    by the oracle side on all host cores from the GPU's t and stamps."""
    spec = config_graph(name)
    g = gpu_graph(htd, spec.n, spec.src, spec.dst)
    og = oracle_mod.OracleGraph.from_raw(spec.n, spec.src, spec.dst)
    eu, ev = htd.htd_edges(g)
    np.testing.assert_array_equal(host(eu), og.eu)
    np.testing.assert_array_equal(host(ev), og.ev)
    sup = host(htd.htd_h_support(g, h))
    t, stamp, stats = htd.htd_truss_decompose(g, h, stamps=True)
    t, stamp = host(t), host(stamp)
    assert stats["frontier_edges"] == g.m
    assert (t >= 2).all() and (t <= sup + 2).all()
    rng = np.random.default_rng(1234)
    # h-support on sampled edges, one BFS pair each in the oracle
    for e in rng.choice(g.m, size=60, replace=False):
        assert sup[e] == og.edge_h_support(h, int(e))
    order_bad, bad, codes = oracle_mod.certify_all(spec.n, og.eu, og.ev, h, t, stamp)
    assert order_bad == 0, f"stamps not ordered like t ({order_bad} stamps)"
    assert bad.size == 0, (f"certificate fails on {bad.size} of {g.m} edges, first {bad[:10]} "
                           f"codes {codes[:10]} at levels {np.unique(t[bad])[:10]}")
