"""htd_h_support_static: h-support for callers that must not allocate device memory.

Code that runs inside an allocator or memory-pool callback, or under an external budget
that already owns all of the device's memory, cannot call cudaMalloc.  For them the
library offers one entry point whose scratch is a fixed static device array.  These tests
call it through the C ABI, twice in a row on different inputs (so that anything left in
the shared scratch by the first call would show), and compare each result with
htd_h_support, exactly (h-support is an integer).  The file name makes pytest collect it
after every other test file.
"""

import ctypes

import numpy as np
import pytest

from synth import erdos_renyi_gnm, rmat

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


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def static_h_support(htd, g, h):
    """Calls htd_h_support_static on the graph's CSR and edges (device tensors)."""
    row_ptr, col, _ = htd.htd_csr(g)
    eu, ev = htd.htd_edges(g)
    out = torch.full((g.m,), -7, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = htd._lib.load().htd_h_support_static(g.n, ptr(row_ptr), ptr(col), g.m, ptr(eu), ptr(ev),
                                              h, ptr(out), stream)
    htd._lib.check(st, "htd_h_support_static")
    torch.cuda.synchronize()
    return out


def test_static_entry_point_matches_h_support_on_consecutive_calls(htd, oracle_mod):
    # h = 1 (adjacency only), h = 2, and h = 3..5 (the level lists swap from depth 4 on);
    # the R-MAT graphs have hubs, so the deep levels are large.  Each result is compared
    # with htd_h_support and with the oracle's per-edge BFS.
    cases = [(1 << 9, rmat(9, 8, 0.57, 0.19, 0.19, 501), 2),
             (400, erdos_renyi_gnm(400, 1600, 502), 3),
             (1 << 9, rmat(9, 8, 0.57, 0.19, 0.19, 501), 2),
             (1 << 10, rmat(10, 8, 0.57, 0.19, 0.19, 503), 1),
             (600, erdos_renyi_gnm(600, 1500, 504), 4),
             (1 << 10, rmat(10, 4, 0.57, 0.19, 0.19, 505), 5),
             (1 << 10, rmat(10, 4, 0.57, 0.19, 0.19, 505), 4)]
    for n, (s, d), h in cases:
        g = htd.htd_build_csr(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
        ref = htd.htd_h_support(g, h)
        got = static_h_support(htd, g, h)
        again = static_h_support(htd, g, h)  # back to back on the shared scratch
        assert torch.equal(got, ref), (n, h)
        assert torch.equal(again, ref), (n, h)
        og = oracle_mod.OracleGraph.from_raw(n, s, d)
        np.testing.assert_array_equal(got.cpu().numpy(), og.h_support(h), err_msg=f"n={n} h={h}")
        g.free()


def test_static_entry_point_rejects_bad_arguments(htd):
    lib = htd._lib.load()
    null = ctypes.c_void_p(0)
    assert lib.htd_h_support_static(4, null, null, 1, null, null, 2, null, null) == 1
    assert lib.htd_h_support_static(htd._lib.HTD_STATIC_MAX_N + 1, ctypes.c_void_p(16), null, 0,
                                    null, null, 2, null, null) == 6
