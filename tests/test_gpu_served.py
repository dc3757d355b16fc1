"""Served decomposition (htd_server_*): a request loop with continuous batching.

Each request is an ordinary decomposition of its own graph (Def. 4; Sec. 3 peeling), so a
result must be the same alone and in the mix: these tests compare every served result with
the same graph decomposed alone (htd_truss_decompose_host) and with the CPU oracle, with
zero tolerance (trussness is an integer), under budgets that admit many requests at once,
one at a time, or none beside another.
"""

import numpy as np
import pytest

from synth import barabasi_albert, erdos_renyi_gnm, rmat

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


def requests():
    rng = np.random.default_rng(77)
    out = []
    for i in range(24):
        kind = i % 3
        h = int(rng.integers(1, 4))
        if kind == 0:
            n = int(rng.integers(200, 1500))
            s, d = erdos_renyi_gnm(n, 4 * n, 7000 + i)
        elif kind == 1:
            n = int(rng.integers(200, 1500))
            s, d = barabasi_albert(n, int(rng.integers(2, 6)), 7100 + i)
        else:
            sc = int(rng.integers(7, 11))
            n = 1 << sc
            s, d = rmat(sc, 8, 0.57, 0.19, 0.19, 7200 + i)
        out.append((n, s, d, h))
    return out


@pytest.fixture(scope="module")
def solo(htd):
    ref = []
    for n, s, d, h in requests():
        eu, ev, t, _ = htd.htd_truss_decompose_host(n, s, d, h)
        ref.append((eu.numpy().copy(), ev.numpy().copy(), t.numpy().copy()))
    return ref


def serve_all(htd, reqs, workers, budget, stagger=False):
    srv = htd.Server(workers=workers, budget_bytes=budget)
    try:
        ids = []
        res = {}
        for i, (n, s, d, h) in enumerate(reqs):
            ids.append(srv.submit(n, s, d, h))
            if stagger and i % 4 == 3:
                # later arrivals join while earlier ones run
                res[i - 3] = srv.wait(ids[i - 3], reqs[i - 3][1].size)
                ids[i - 3] = None
        for i, rid in enumerate(ids):
            if rid is not None:
                res[i] = srv.wait(rid, reqs[i][1].size)
        return res, srv.info()
    finally:
        srv.close()


def test_served_results_equal_solo_and_oracle(htd, solo, oracle_mod):
    reqs = requests()
    res, info = serve_all(htd, reqs, workers=4, budget=0)
    assert info["peak_running"] >= 2  # requests really ran side by side
    for i, (eu, ev, t, meta) in res.items():
        np.testing.assert_array_equal(eu, solo[i][0])
        np.testing.assert_array_equal(ev, solo[i][1])
        np.testing.assert_array_equal(t, solo[i][2], err_msg=f"request {i}")
        assert meta["status"] == 0 and meta["submit_s"] <= meta["admit_s"] <= meta["start_s"]
        assert meta["start_s"] <= meta["done_s"]
    for i in (0, 1, 2, 5):
        n, s, d, h = reqs[i]
        og = oracle_mod.OracleGraph.from_raw(n, s, d)
        np.testing.assert_array_equal(res[i][2], og.truss_decompose(h)[0])


def test_served_under_tight_budgets_and_staggered_arrivals(htd, solo):
    reqs = requests()[:12]
    est = max(htd.htd_footprint_estimate(n, s.size, h, 0) for n, s, _, h in reqs)
    for workers, budget, stagger in ((3, est + 1, True), (2, 1 << 20, False)):
        # est + 1: about one request at a time; 1 MiB: every request larger than the budget,
        # so each is admitted alone
        res, info = serve_all(htd, reqs, workers=workers, budget=budget, stagger=stagger)
        if budget == 1 << 20:
            assert info["peak_running"] == 1
        for i, (eu, ev, t, _) in res.items():
            np.testing.assert_array_equal(t, solo[i][2], err_msg=f"request {i}")


def test_served_errors_stay_with_their_request(htd, solo):
    reqs = requests()[:4]
    srv = htd.Server(workers=2)
    try:
        good = [srv.submit(n, s, d, h) for n, s, d, h in reqs[:2]]
        bad = srv.submit(5, np.array([0, 1], np.int32), np.array([1, 7], np.int32), 2)
        good += [srv.submit(n, s, d, h) for n, s, d, h in reqs[2:]]
        with pytest.raises(htd.HtdError) as ei:
            srv.wait(bad, 2)
        assert ei.value.status == 1
        for i, rid in enumerate(good):
            np.testing.assert_array_equal(srv.wait(rid, reqs[i][1].size)[2], solo[i][2])
        with pytest.raises(htd.HtdError):
            srv.poll(bad)  # collected: forgotten
    finally:
        srv.close()
