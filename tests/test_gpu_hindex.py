"""The paper's own parallel method on the GPU: the H-index iteration of Sec. 4.

Pinned to the CPU oracle's iteration (``htdo_hindex``) and to the peel: the synchronous
orders (Algorithm 2) must give the oracle's H values order by order and the same number of
orders; at the fixed point H + 2 is the h-trussness (Theorem 4), so it must equal the
oracle's peel and the GPU peel bit for bit, synchronous or asynchronous.  Keys never
increase from order to order (Theorem 3).
"""

import numpy as np
import pytest

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


@pytest.mark.parametrize("h", [1, 2, 3])
def test_synchronous_orders_equal_the_oracle(htd, oracle_mod, h):
    for n, s, d in small_corpus(25, 400 + h, max_n=50):
        g = gpu_graph(htd, n, s, d)
        if g.m == 0:
            continue
        og = oracle_mod.OracleGraph.from_raw(n, s, d)
        ref_h, ref_it, ref_conv = og.hindex(h)
        t, hv, st = htd.htd_hindex_decompose(g, h)
        assert st["converged"] == 1 and ref_conv
        assert st["iterations"] == ref_it
        np.testing.assert_array_equal(hv.cpu().numpy(), ref_h)
        np.testing.assert_array_equal(t.cpu().numpy(), og.truss_decompose(h)[0])
        # order by order: the first orders' values and monotone keys (Theorem 3)
        prev = og.h_support(h)
        for k in (1, 2):
            _, hk, _ = htd.htd_hindex_decompose(g, h, max_iter=k)
            ok, _, _ = og.hindex(h, max_iter=k)
            np.testing.assert_array_equal(hk.cpu().numpy(), ok)
            assert (hk.cpu().numpy() <= prev).all()
            prev = hk.cpu().numpy()


@pytest.mark.parametrize("sweeps", [2, 8])
def test_asynchronous_fixed_point_equals_the_peel(htd, oracle_mod, sweeps):
    graphs = [(300, *erdos_renyi_gnm(300, 1200, 31)), (400, *barabasi_albert(400, 3, 32)),
              (512, *rmat(9, 8, 0.57, 0.19, 0.19, 33))]
    for n, s, d in graphs:
        g = gpu_graph(htd, n, s, d)
        og = oracle_mod.OracleGraph.from_raw(n, s, d)
        for h in (2, 3):
            ref = og.truss_decompose(h)[0]
            ta, _, sa = htd.htd_hindex_decompose(g, h, sweeps=sweeps)
            ts, _, ss = htd.htd_hindex_decompose(g, h)
            np.testing.assert_array_equal(ta.cpu().numpy(), ref)
            np.testing.assert_array_equal(ts.cpu().numpy(), ref)
            assert sa["converged"] == 1 and ss["converged"] == 1
            # the asynchronous sweeps use fresher keys: never more orders than synchronous
            assert sa["iterations"] <= ss["iterations"]


def test_small_workload_and_peel_agree(htd, oracle_mod):
    spec = config_graph("er_n2000")
    g = gpu_graph(htd, spec.n, spec.src, spec.dst)
    og = oracle_mod.OracleGraph.from_raw(spec.n, spec.src, spec.dst)
    ref = og.truss_decompose(2)[0]
    t_peel, _, _ = htd.htd_truss_decompose(g, 2)
    for sweeps in (1, 4):
        t, _, st = htd.htd_hindex_decompose(g, 2, sweeps=sweeps)
        np.testing.assert_array_equal(t.cpu().numpy(), ref)
        assert torch.equal(t, t_peel)


@pytest.mark.parametrize("h", [1, 2, 3])
def test_pruned_orders_equal_the_plain_orders(htd, oracle_mod, h):
    # Lemma 4 pruning changes no value of any order: after every order the pruned GPU
    # iteration equals the plain one (and the oracle's); the GPU's range test is a
    # conservative form of the oracle's per-edge test, so it computes at least as many
    # H^(n)(e) as the oracle's pruned iteration and at most m per order
    graphs = [(n, s, d) for n, s, d in small_corpus(8, 470 + h, max_n=40)]
    graphs += [(60, *erdos_renyi_gnm(60, 220, 480 + h)), (128, *rmat(7, 6, 0.57, 0.19, 0.19, 490 + h))]
    saved = 0
    for n, s, d in graphs:
        g = gpu_graph(htd, n, s, d)
        if g.m == 0:
            continue
        og = oracle_mod.OracleGraph.from_raw(n, s, d)
        tp, hp, sp = htd.htd_hindex_decompose(g, h, prune=True)
        t0, h0, s0 = htd.htd_hindex_decompose(g, h)
        assert sp["pruned"] == 1 and s0["pruned"] == 0
        assert sp["converged"] == 1 and sp["iterations"] == s0["iterations"]
        assert torch.equal(hp, h0) and torch.equal(tp, t0)
        np.testing.assert_array_equal(tp.cpu().numpy(), og.truss_decompose(h)[0])
        assert s0["edge_evals"] == g.m * s0["iterations"]
        assert sp["edge_evals"] <= s0["edge_evals"]
        _, o_it, _, o_evals = og.hindex_pruned(h)
        assert o_it == sp["iterations"] and sp["edge_evals"] >= o_evals
        for k in range(1, min(sp["iterations"], 4) + 1):
            _, hk, _ = htd.htd_hindex_decompose(g, h, max_iter=k, prune=True)
            ok, _, _ = og.hindex(h, max_iter=k)
            np.testing.assert_array_equal(hk.cpu().numpy(), ok, err_msg=f"order {k}")
        saved += s0["edge_evals"] - sp["edge_evals"]
    assert saved > 0


@pytest.mark.slow
def test_full_size_dcsbm_h2_equals_the_certified_peel(htd):
    # the GPU peel of this workload is certified on every edge by test_full_size_certificate
    spec = config_graph("dcsbm_n200k")
    g = gpu_graph(htd, spec.n, spec.src, spec.dst)
    t_peel, _, _ = htd.htd_truss_decompose(g, 2)
    t, _, st = htd.htd_hindex_decompose(g, 2, sweeps=1)
    assert st["converged"] == 1
    assert torch.equal(t, t_peel)
    tp, _, sp = htd.htd_hindex_decompose(g, 2, sweeps=1, prune=True)
    assert sp["iterations"] == st["iterations"] and torch.equal(tp, t_peel)
    assert sp["edge_evals"] < st["edge_evals"]


def test_bad_arguments(htd):
    g = gpu_graph(htd, 3, [0, 1], [1, 2])
    for h, sw in ((0, 1), (9, 1), (2, 0)):
        with pytest.raises(htd.HtdError):
            htd.htd_hindex_decompose(g, h, sweeps=sw)
    with pytest.raises(htd.HtdError):  # pruning is defined for synchronous orders only
        htd.htd_hindex_decompose(g, 2, sweeps=4, prune=True)
