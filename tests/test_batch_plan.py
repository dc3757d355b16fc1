"""Host logic of the batched call: the union packing (htd_batch_plan), no GPU needed."""

import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2411_06405_gb300 import _lib, build

    build.build()
    return _lib.load()


def plan(lib, n, h, counts, cap):
    n = np.asarray(n, dtype=np.int32)
    h = np.asarray(h, dtype=np.int32)
    off = np.concatenate([[0], np.cumsum(np.asarray(counts, dtype=np.int64))]).astype(np.int64)
    k = len(n)
    union_of = np.full(max(k, 1), -1, dtype=np.int32)
    voff = np.full(max(k, 1), -1, dtype=np.int32)
    nu = ctypes.c_int32(-1)
    vp = lambda a: ctypes.c_void_p(a.ctypes.data)
    st = lib.htd_batch_plan(k, vp(n), vp(h), vp(off), int(cap), vp(union_of), vp(voff), ctypes.byref(nu))
    return st, union_of[:k], voff[:k], nu.value


@pytest.mark.parametrize("seed", range(12))
def test_plan_packs_by_h_in_input_order(lib, seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 300))
    n = rng.integers(0, 5000, size=k)
    h = rng.integers(1, 4, size=k)
    counts = rng.integers(0, 20000, size=k)
    cap = int(rng.choice([0, 1, 3000, 20000, 100000]))
    st, union_of, voff, nu = plan(lib, n, h, counts, cap)
    assert st == 0
    limit = cap if cap > 0 else 262144
    order = [g for hh in (1, 2, 3) for g in range(k) if h[g] == hh]
    # unions are numbered along the order, each holds one h, members keep input order
    assert [union_of[g] for g in order] == sorted(union_of[g] for g in order)
    assert nu == len(set(union_of.tolist())) and sorted(set(union_of.tolist())) == list(range(nu))
    members = {}
    for g in order:
        members.setdefault(int(union_of[g]), []).append(g)
    for u, gs in members.items():
        assert len({int(h[g]) for g in gs}) == 1
        assert gs == sorted(gs)
        # ids shifted by the vertices of the earlier members
        assert [int(voff[g]) for g in gs] == [int(sum(n[x] for x in gs[:i])) for i in range(len(gs))]
        # within the vertex limit unless alone
        assert len(gs) == 1 or sum(int(n[g]) for g in gs) <= limit
    # greedy: a union is closed only when the next graph of the same h does not fit
    for a, b in zip(order, order[1:]):
        if union_of[b] != union_of[a] and h[a] == h[b]:
            gs = members[int(union_of[a])]
            assert sum(int(n[g]) for g in gs) + int(n[b]) > limit


def test_plan_rejects_what_the_batched_call_rejects(lib):
    assert plan(lib, [4], [0], [0], 0)[0] == 1
    assert plan(lib, [4], [9], [0], 0)[0] == 1
    assert plan(lib, [-1], [2], [0], 0)[0] == 1
    assert plan(lib, [2_000_000], [2], [0], 0)[0] == 6
    assert plan(lib, [4], [2], [1 << 31], 0)[0] == 5
    assert lib.htd_batch_plan(0, None, None, None, 0, None, None, None) == 0


def test_autotune_group_keys():
    from paper_2411_06405_gb300 import autotune

    s = np.array([0, 0, 0, 1], np.int32)
    d = np.array([1, 2, 3, 2], np.int32)
    assert autotune.group_key(4, s, d, 2) == "h2_n2_d1"   # n = 4, largest degree 3
    assert autotune.group_key(1000, s, d, 3).startswith("h3_n9_")
    # loops do not count towards degrees; an edgeless graph has class 0
    assert autotune.group_key(5, np.array([1, 1]), np.array([1, 1]), 2) == "h2_n2_d0"


def test_autotune_partition_sends_block_groups_to_one_call():
    # graphs whose group chose one block per graph form the block call; every other graph
    # (chosen union settings, or a group missing from the table) goes to one union call with
    # the default settings; every graph lands in exactly one call, in input order
    from paper_2411_06405_gb300 import _lib, autotune

    s = np.array([0, 1, 2], np.int32)
    d = np.array([1, 2, 0], np.int32)
    graphs = [(3, s, d, 2), (3, s, d, 3), (3, s, d, 2), (40, s, d, 2)]
    table = {autotune.group_key(3, s, d, 2): {"max_union_vertices": 1 << 18,
                                              "flags": _lib.HTD_OPT_BATCH_BLOCKS},
             autotune.group_key(3, s, d, 3): {"max_union_vertices": 1 << 16,
                                              "flags": _lib.HTD_OPT_REBUILD}}
    parts = autotune._partition(graphs, table)
    assert parts == [([0, 2], 1 << 18, _lib.HTD_OPT_BATCH_BLOCKS),
                     ([1, 3], autotune.DEFAULT["max_union_vertices"], autotune.DEFAULT["flags"])]
    assert autotune._partition(graphs, None) == [([0, 1, 2, 3], autotune.DEFAULT["max_union_vertices"],
                                                  autotune.DEFAULT["flags"])]
    assert autotune._partition([], table) == []
